// solve.cu -- K5: the Solve task L21 = A21 P^T (D11 L11^T)^{-1} (Section 1 task
// list; Figure 4.1 (d),(e)) fused with the update of the delayed columns, in FP64.
//
// Every A21 row is independent: with x = A21(i, perm) the permuted row,
//   Y  = x_e L11^{-T}          (forward substitution, right-looking by column),
//   x_d <- x_d - Y L_d^T        (delayed columns: L_d are the delayed rows of L),
//   L21(i,:) = Y D11^{-1}       (1x1 and 2x2 blocks; zero pivots give 0).
// A CTA owns a tile of kRows consecutive rows; the tile is gathered through the
// permutation with coalesced loads into shared memory (padded [p][kRows+1]),
// eliminated in place, and written back in place (L21 in the first e columns,
// the updated delayed columns after them).  Y = L21 D11 is also written to the
// workspace when the Form step needs it.  Arithmetic is O(p^2) FP64 FMAs per row
// and the GB300 FP64 pipe is the bound: eight warps share each row tile (each
// updates every eighth column) so that every FP64 pipe of the SM has work.
#include <cuda_bf16.h>

#include "ctp_internal.cuh"

namespace ctp {

namespace {

constexpr int kRows = 32;   // rows per tile (one per lane)
constexpr int kWarps = 8;   // warps per CTA: warp w updates the columns k = w (mod 8)

// Entry k of row rr of L21 = Y D11^{-1}, from the rows of Y in xs ([k][kRows+1]):
// 1x1 and 2x2 blocks of D11^{-1}; zero pivots give 0.
__device__ __forceinline__ double l21_of(const double *xs, int k, int rr, const int32_t *__restrict__ piv,
                                         const double *__restrict__ Dinv) {
    constexpr int LDX = kRows + 1;
    const int kd = piv[k];
    const double y = xs[k * LDX + rr];
    if (kd == CTP_PIVKIND_1X1) return y * Dinv[2 * k];
    if (kd == CTP_PIVKIND_2X2_FIRST) return __fma_rn(xs[(k + 1) * LDX + rr], Dinv[2 * k + 1], y * Dinv[2 * k]);
    if (kd == CTP_PIVKIND_2X2_SECOND) return __fma_rn(y, Dinv[2 * k], xs[(k - 1) * LDX + rr] * Dinv[2 * k - 1]);
    return 0.0;
}

// The BF16 pieces of the first e columns of a tile's rows (rows of Y in xs, or
// with kL the rows of L21 computed from them) into the K-major operand copy B (row brow of B is the tile's first row), each
// piece rounding what the previous ones left (lo_off elements apart), and
// zeros from e to Kz.  Every thread of the CTA takes (row, column pair) items
// of the real columns, so that lanes do not idle on the zero tail (the
// conversions cost about a nanosecond per value per SM).
template <bool kL>
__device__ __forceinline__ void write_pieces(__nv_bfloat16 *__restrict__ B, int64_t brow, int rows, int Kp, int e,
                                             int Kz, int pieces, int64_t lo_off, const double *xs,
                                             const int32_t *__restrict__ piv, const double *__restrict__ Dinv) {
    constexpr int LDX = kRows + 1;
    const int eh = (e + 1) >> 1, zn = (Kz >> 1) - eh;
    for (int t = threadIdx.x; t < rows * eh; t += blockDim.x) {
        const int rr = t / eh, k = 2 * (t - rr * eh);
        __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(B + (brow + rr) * Kp) + (k >> 1);
        const double v0 = kL ? l21_of(xs, k, rr, piv, Dinv) : xs[k * LDX + rr];
        const double v1 = k + 1 < e ? (kL ? l21_of(xs, k + 1, rr, piv, Dinv) : xs[(k + 1) * LDX + rr]) : 0.0;
        __nv_bfloat162 b;
        b.x = __double2bfloat16(v0);
        b.y = __double2bfloat16(v1);
        dst[0] = b;
        double r0 = v0 - (double)__bfloat162float(b.x);
        double r1 = v1 - (double)__bfloat162float(b.y);
        for (int pc = 1; pc < pieces; pc++) {
            __nv_bfloat162 l;
            l.x = __double2bfloat16(r0);
            l.y = __double2bfloat16(r1);
            dst[pc * (lo_off / 2)] = l;
            r0 -= (double)__bfloat162float(l.x);
            r1 -= (double)__bfloat162float(l.y);
        }
    }
    if (zn <= 0) return;
    const __nv_bfloat162 z = __floats2bfloat162_rn(0.0f, 0.0f);
    for (int t = threadIdx.x; t < rows * zn; t += blockDim.x) {
        const int rr = t / zn, k2 = eh + (t - rr * zn);
        __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(B + (brow + rr) * Kp) + k2;
        for (int pc = 0; pc < pieces; pc++) dst[pc * (lo_off / 2)] = z;
    }
}

// Right-looking substitution over a tile of 32 rows: for each eliminated
// position j, every warp reads y_j of its lane's row and updates its share of
// the later columns (four independent updates in flight per warp); a CTA
// barrier separates consecutive pivots.  The outputs are computed from the
// rows of Y in shared memory without a register copy, so that a CTA needs few
// registers and as many CTAs fit on an SM as its shared memory allows (three at
// p = 256, more for narrower fronts): enough warps for all four FP64 pipes.
// One 32-row tile.  brow0: row of this front's first A21 row in the BF16
// operand copies (0 for a single supernode; the stacked offset in a batch).
// pieces > 1: also write the further BF16 pieces of the split operands (piece
// k rounds what pieces 0..k-1 left), lo_off elements apart.
__device__ __forceinline__ void solve_tile(double *__restrict__ A, int64_t n, int p, int64_t lda,
                                           const int32_t *__restrict__ perm,
                                           const int32_t *__restrict__ piv,
                                           const double *__restrict__ Dinv, int e,
                                           double *__restrict__ W21, int64_t ldw,
                                           __nv_bfloat16 *__restrict__ Wb,
                                           __nv_bfloat16 *__restrict__ Lb, int Kp, int64_t brow0,
                                           int64_t lo_off, int pieces, int64_t tile, double *xs) {
    constexpr int LDX = kRows + 1;
    const int64_t m = n - p;
    const int64_t row0 = tile * kRows;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t row = row0 + lane;
    const bool valid = row < m;
    double *A21 = A + p;

    // gather x = A21(rows, perm): each warp reads 32 consecutive rows of a column
    for (int k = w; k < p; k += kWarps) {
        const int c = perm[k];
        xs[k * LDX + lane] = valid ? A21[(int64_t)c * lda + row] : 0.0;
    }
    __syncthreads();

    for (int j = 0; j < e;) {
        const int kd = piv[j];
        if (kd == CTP_PIVKIND_2X2_FIRST) {
            const double y0 = xs[j * LDX + lane], y1 = xs[(j + 1) * LDX + lane];
            const double *l0 = A + (int64_t)j * lda, *l1 = A + (int64_t)(j + 1) * lda;
#pragma unroll 4
            for (int k = j + 2 + w; k < p; k += kWarps)
                xs[k * LDX + lane] -= y0 * __ldg(l0 + k) + y1 * __ldg(l1 + k);
            j += 2;
        } else {
            if (kd == CTP_PIVKIND_1X1) {
                const double y0 = xs[j * LDX + lane];
                const double *l0 = A + (int64_t)j * lda;
#pragma unroll 4
                for (int k = j + 1 + w; k < p; k += kWarps) xs[k * LDX + lane] -= y0 * __ldg(l0 + k);
            }
            j += 1;  // zero pivots have an all-zero L column
        }
        __syncthreads();
    }

    // BF16 copy of Y = W21 for the tensor-core Form: row-major, K contiguous,
    // zero from e to the end of e's last 64-wide K block (the Form reads no
    // further; a batch's rows are 256 wide whatever the front's p)
    const int Kz = min(Kp, (e + 63) / 64 * 64);
    const int tile_rows = m - row0 < kRows ? (int)(m - row0) : kRows;
    if (Wb != nullptr) write_pieces<false>(Wb, brow0 + row0, tile_rows, Kp, e, Kz, pieces, lo_off, xs, piv, Dinv);
    // W21 = Y (= L21 D11) for the FP64 Form step, L21 = Y D11^{-1} in place, the
    // delayed columns as they are.  xs is only read from here on.
    for (int k = w; k < p; k += kWarps) {
        if (!valid) break;
        double out;
        if (k >= e) {
            out = xs[k * LDX + lane];
        } else {
            if (W21 != nullptr) W21[(int64_t)k * ldw + row] = xs[k * LDX + lane];
            out = l21_of(xs, k, lane, piv, Dinv);
        }
        A21[(int64_t)k * lda + row] = out;
    }
    // BF16 copy of L21 for the tensor-core Form
    if (Lb != nullptr) write_pieces<true>(Lb, brow0 + row0, tile_rows, Kp, e, Kz, pieces, lo_off, xs, piv, Dinv);
}

__global__ void __launch_bounds__(kRows * kWarps)
    k_solve_fp64(double *__restrict__ A, int64_t n, int p, int64_t lda,
                 const int32_t *__restrict__ perm, const int32_t *__restrict__ piv,
                 const double *__restrict__ Dinv, const int32_t *__restrict__ nelim_p,
                 double *__restrict__ W21, int64_t ldw, __nv_bfloat16 *__restrict__ Wb,
                 __nv_bfloat16 *__restrict__ Lb, int Kp, int64_t lo_off, int pieces) {
    extern __shared__ __align__(16) double xs[];  // [p][kRows+1]
    solve_tile(A, n, p, lda, perm, piv, Dinv, *nelim_p, W21, ldw, Wb, Lb, Kp, 0, lo_off, pieces, blockIdx.x, xs);
}

// Batched: CTA b takes work item b = (front, 32-row tile of its A21): the
// front is item_front[b], the tile item_tile[b] (or, without that list, the
// item's place among the front's consecutive items).
__global__ void __launch_bounds__(kRows * kWarps)
    k_solve_batch(const ctp_front *__restrict__ fronts, const BFront *__restrict__ tab, char *ws,
                  const int *__restrict__ item_front, const int *__restrict__ item_tile, BatchOpts o,
                  __nv_bfloat16 *__restrict__ Wb, __nv_bfloat16 *__restrict__ Lb) {
    extern __shared__ __align__(16) double xs[];
    const int f = item_front[blockIdx.x];
    const ctp_front fr = fronts[f];
    const BFront bt = tab[f];
    ctp_options oo;
    oo.pivot = o.pivot;
    oo.smode = o.smode;
    oo.prec = o.prec;
    const BSection sec = bsection(bt.n, bt.p, &oo);
    char *base = ws + bt.ws;
    const bool w64 = o.smode != CTP_S_NONE && o.prec == CTP_FP64;
    solve_tile(fr.A, bt.n, bt.p, fr.lda, fr.perm, fr.piv, reinterpret_cast<const double *>(base + sec.Dinv),
               *fr.nelim, w64 ? reinterpret_cast<double *>(base + sec.W21) : nullptr, bt.m, Wb, Lb,
               kBatchKp, bt.row0, o.lo_off, o.pieces,
               item_tile != nullptr ? (int64_t)item_tile[blockIdx.x] : (int64_t)blockIdx.x - bt.s0, xs);
}


}  // namespace

cudaError_t launch_solve_fp64(double *A, int64_t n, int p, int64_t lda, const int32_t *perm,
                              const int32_t *piv, const double *Dinv, const int32_t *nelim,
                              double *W21, int64_t ldw, void *Wb, void *Lb, int Kp, int64_t lo_off,
                              int pieces, cudaStream_t st) {
    const int64_t m = n - p;
    if (m <= 0) return cudaSuccess;
    size_t smem = sizeof(double) * (size_t)p * (kRows + 1);
    cudaError_t err =
        smem_at_least((const void *)k_solve_fp64, smem);
    if (err != cudaSuccess) return err;
    int64_t grid = (m + kRows - 1) / kRows;
    k_solve_fp64<<<(unsigned)grid, kRows * kWarps, smem, st>>>(
        A, n, p, lda, perm, piv, Dinv, nelim, W21, ldw, (__nv_bfloat16 *)Wb, (__nv_bfloat16 *)Lb, Kp,
        lo_off, pieces);
    return cudaGetLastError();
}

cudaError_t launch_solve_batch(const ctp_front *fronts, const BFront *tab, char *ws,
                               const int *item_front, int64_t items, BatchOpts o, void *Wb, void *Lb,
                               int pmax, cudaStream_t st, const int *item_tile) {
    if (items == 0) return cudaSuccess;
    const size_t smem = sizeof(double) * (size_t)pmax * (kRows + 1);
    cudaError_t err =
        smem_at_least((const void *)k_solve_batch, smem);
    if (err != cudaSuccess) return err;
    k_solve_batch<<<(unsigned)items, kRows * kWarps, smem, st>>>(
        fronts, tab, ws, item_front, item_tile, o, (__nv_bfloat16 *)Wb, (__nv_bfloat16 *)Lb);
    return cudaGetLastError();
}

int solve_rows_per_tile() { return kRows; }

}  // namespace ctp
