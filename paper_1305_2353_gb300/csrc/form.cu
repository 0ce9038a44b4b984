// form.cu -- K6 (FP64): the Form task S = L21 D11 L21^T = W21 L21^T (Section 1
// task list), lower triangle only.
//
// W21 = L21 D11 is the Y produced by the Solve kernel.  The kernel walks only the
// tiles on or below the diagonal (a triangular tile index), stages 64 x 16
// slabs of W21 and L21 in shared memory, and gives each of 256 threads a 4 x 4
// block of S, rows strided by 16 along the lanes so that a warp's stores (or
// read-modify-writes) of S cover 16 consecutive rows of a column: coalesced,
// which matters when the inner dimension e is small and S traffic dominates.  The inner dimension e is read from device memory (it is only
// known after pivoting).  S is written as FP64 or FP32, full column-major or
// lower-packed by columns; strictly upper entries are never written.
#include "ctp_internal.cuh"

namespace ctp {

namespace {

constexpr int kTile = 64, kK = 16, kTh = 256;

template <typename OutT, bool kPacked, bool kSub = false>
__device__ __forceinline__ void form_tile(const double *__restrict__ L21, int64_t ldl,
                                          const double *__restrict__ W21, int64_t ldw, int64_t m,
                                          int e, OutT *__restrict__ S, int64_t lds, int64_t b) {
    __shared__ double sw[kK][kTile + 1];
    __shared__ double sl[kK][kTile + 1];
    // triangular tile index -> (ti, tj), ti >= tj
    int64_t ti = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= b) ti++;
    while (ti * (ti + 1) / 2 > b) ti--;
    const int64_t tj = b - ti * (ti + 1) / 2;
    const int64_t i0 = ti * kTile, j0 = tj * kTile;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < e; k0 += kK) {
        for (int idx = threadIdx.x; idx < kK * kTile; idx += kTh) {
            const int kk = idx / kTile, rr = idx % kTile;
            const int k = k0 + kk;
            const int64_t gi = i0 + rr, gj = j0 + rr;
            sw[kk][rr] = (k < e && gi < m) ? W21[(int64_t)k * ldw + gi] : 0.0;
            sl[kk][rr] = (k < e && gj < m) ? L21[(int64_t)k * ldl + gj] : 0.0;
        }
        __syncthreads();
        auto step = [&](int kk) {
            double a[4], bb[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                a[q] = sw[kk][tx + 16 * q];
                bb[q] = sl[kk][ty + 16 * q];
            }
#pragma unroll
            for (int q = 0; q < 4; q++)
#pragma unroll
                for (int s = 0; s < 4; s++) acc[q][s] += a[q] * bb[s];
        };
        if (k0 + kK <= e) {
#pragma unroll
            for (int kk = 0; kk < kK; kk++) step(kk);
        } else {
            // the last slab: only its e - k0 real terms (the FP64 pipe is the
            // bound, and small e -- a few dozen -- is common in batches)
            for (int kk = 0; kk < e - k0; kk++) step(kk);
        }
        __syncthreads();
    }
    // subtracting: every old value is loaded before any is stored, so that the
    // 16 loads are in flight together
    OutT old[4][4];
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const int64_t gi = i0 + tx + 16 * q, gj = j0 + ty + 16 * s;
            old[q][s] = (OutT)0;
            if (kSub && gi < m && gj < m && gi >= gj) old[q][s] = S[gj * lds + gi];
        }
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const int64_t gi = i0 + tx + 16 * q, gj = j0 + ty + 16 * s;
            if (gi < m && gj < m && gi >= gj) {
                const int64_t idx = kPacked ? gj * m - gj * (gj - 1) / 2 + (gi - gj) : gj * lds + gi;
                if (kSub)
                    S[idx] = old[q][s] - (OutT)acc[q][s];
                else
                    S[idx] = (OutT)acc[q][s];
            }
        }
}

template <typename OutT, bool kPacked, bool kSub = false>
__global__ void __launch_bounds__(kTh)
    k_form_fp64(const double *__restrict__ L21, int64_t ldl, const double *__restrict__ W21,
                int64_t ldw, int64_t m, const int32_t *__restrict__ nelim_p, OutT *__restrict__ S,
                int64_t lds) {
    form_tile<OutT, kPacked, kSub>(L21, ldl, W21, ldw, m, *nelim_p, S, lds, blockIdx.x);
}

// Batched: CTA b takes work item b = (front, triangular 64 x 64 tile of its S):
// S lower-packed per front, or (kSub) subtracted from the front's full
// column-major S (leading dimension lds).  The front is item_front[b], the tile
// item_tile[b] (or, without that list, the item's place among the front's
// consecutive items).
template <typename OutT, bool kSub = false>
__global__ void __launch_bounds__(kTh)
    k_form_fp64_batch(const ctp_front *__restrict__ fronts, const BFront *__restrict__ tab, char *ws,
                      const int *__restrict__ item_front, const int *__restrict__ item_tile, BatchOpts o) {
    const int f = item_front[blockIdx.x];
    const ctp_front fr = fronts[f];
    const BFront bt = tab[f];
    ctp_options oo;
    oo.pivot = o.pivot;
    oo.smode = o.smode;
    oo.prec = o.prec;
    const BSection sec = bsection(bt.n, bt.p, &oo);
    const double *W21 = reinterpret_cast<const double *>(ws + bt.ws + sec.W21);
    form_tile<OutT, !kSub, kSub>(fr.A + bt.p, fr.lda, W21, bt.m, bt.m, *fr.nelim, (OutT *)fr.S, fr.lds,
                                 item_tile != nullptr ? (int64_t)item_tile[blockIdx.x] : (int64_t)blockIdx.x - bt.f0);
}


}  // namespace

cudaError_t launch_form_fp64(const double *L21, int64_t ldl, const double *W21, int64_t ldw,
                             int64_t m, const int32_t *nelim, void *S, int64_t lds, int smode,
                             cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    const int64_t nt = (m + kTile - 1) / kTile;
    const int64_t ntiles = nt * (nt + 1) / 2;
    if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (smode == CTP_S_FP64)
        k_form_fp64<double, false><<<(unsigned)ntiles, kTh, 0, st>>>(L21, ldl, W21, ldw, m, nelim,
                                                                     (double *)S, lds);
    else if (smode == CTP_S_FP32)
        k_form_fp64<float, false><<<(unsigned)ntiles, kTh, 0, st>>>(L21, ldl, W21, ldw, m, nelim,
                                                                    (float *)S, lds);
    else if (smode == CTP_S_FP64_SUB)
        k_form_fp64<double, false, true><<<(unsigned)ntiles, kTh, 0, st>>>(L21, ldl, W21, ldw, m, nelim,
                                                                           (double *)S, lds);
    else if (smode == CTP_S_FP64_PACKED)
        k_form_fp64<double, true><<<(unsigned)ntiles, kTh, 0, st>>>(L21, ldl, W21, ldw, m, nelim,
                                                                    (double *)S, lds);
    else
        k_form_fp64<float, true><<<(unsigned)ntiles, kTh, 0, st>>>(L21, ldl, W21, ldw, m, nelim,
                                                                   (float *)S, lds);
    return cudaGetLastError();
}

cudaError_t launch_form_fp64_batch(const ctp_front *fronts, const BFront *tab, char *ws,
                                   const int *item_front, int64_t items, BatchOpts o,
                                   cudaStream_t st, const int *item_tile) {
    if (items == 0) return cudaSuccess;
    if (o.smode == CTP_S_FP64_SUB)
        k_form_fp64_batch<double, true>
            <<<(unsigned)items, kTh, 0, st>>>(fronts, tab, ws, item_front, item_tile, o);
    else if (o.smode == CTP_S_FP64_PACKED)
        k_form_fp64_batch<double><<<(unsigned)items, kTh, 0, st>>>(fronts, tab, ws, item_front, item_tile, o);
    else
        k_form_fp64_batch<float><<<(unsigned)items, kTh, 0, st>>>(fronts, tab, ws, item_front, item_tile, o);
    return cudaGetLastError();
}

int64_t form_fp64_tiles(int64_t m) {
    const int64_t nt = (m + kTile - 1) / kTile;
    return nt * (nt + 1) / 2;
}

}  // namespace ctp
