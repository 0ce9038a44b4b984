// compress.cu -- K1: strict compression of A21 (Section 4.1, eq. (4.1)).
//
// For every A21 row i: J(i) = argmax_k |a21(i,k)| (ties to the lowest k), then
// c(J(i), k) = max(c(J(i), k), |a21(i,k)|).  Everything is a comparison of
// magnitudes, so the kernel never touches the FP64 pipe (which is narrow on
// GB300): |x| is the IEEE bit pattern with the sign cleared, and for
// non-negative doubles the unsigned 64-bit integer order is the numeric order.
// C is kept as such integer keys in the workspace and merged across CTAs with
// a test-then-atomicMax, which is exact and order independent.
//
// Data movement: A21 is column-major, so a tile of TR consecutive rows is one
// contiguous TR*8-byte segment per column.  Each warp-wide cp.async moves 32
// consecutive doubles of one column (coalesced), straight into a padded shared
// tile [p][TR+1] without passing through registers; STAGES tiles are in flight
// per CTA.  The CTA grid is persistent (a multiple of the SM count).
#include "ctp_internal.cuh"
#include "tc_common.cuh"

namespace ctp {

namespace {

constexpr int kThreads = 256;
constexpr int kTR = 32;      // rows per tile (one 256-byte segment per column)
constexpr int kStages = 3;   // tiles in flight per CTA
constexpr unsigned long long kAbsMask = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long kInfKey = 0x7FF0000000000000ull;

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ unsigned long long abs_key(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x)) & kAbsMask;
}

// Issue the loads of tile `t` into stage buffer `buf`.
__device__ __forceinline__ void load_tile(const double *__restrict__ A21, int64_t m, int p,
                                          int64_t lda, int64_t t, double *buf) {
    const int64_t row0 = t * kTR;
    const int total = kTR * p;
    for (int idx = threadIdx.x; idx < total; idx += kThreads) {
        int k = idx / kTR, r = idx - k * kTR;
        int64_t row = row0 + r;
        if (row < m) cp_async8(buf + k * (kTR + 1) + r, A21 + (int64_t)k * lda + row);
    }
}

__global__ void __launch_bounds__(kThreads)
    k_compress_strict(const double *__restrict__ A21, int64_t m, int p, int64_t lda,
                      unsigned long long *__restrict__ Ckeys, int32_t *__restrict__ J,
                      uint32_t *__restrict__ rowbits,
                      int32_t *__restrict__ info) {
    extern __shared__ __align__(16) double smem[];
    const int tile_elems = p * (kTR + 1);
    double *tiles = smem;                                               // [kStages][p][kTR+1]
    unsigned long long *pkey =
        reinterpret_cast<unsigned long long *>(smem + kStages * tile_elems);  // [NG][kTR]
    constexpr int NG = kThreads / kTR;                                  // column groups
    int *pidx = reinterpret_cast<int *>(pkey + NG * kTR);               // [NG][kTR]
    int *rowJ = pidx + NG * kTR;                                        // [kTR]

    const int64_t ntiles = (m + kTR - 1) / kTR;
    const int r = threadIdx.x % kTR, g = threadIdx.x / kTR;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    bool nonfinite = false;

    // prologue: fill the pipeline
    int64_t t_load = blockIdx.x;
    for (int s = 0; s < kStages - 1; s++) {
        if (t_load < ntiles) load_tile(A21, m, p, lda, t_load, tiles + s * tile_elems);
        cp_async_commit();
        t_load += gridDim.x;
    }
    int stage = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        // keep kStages-1 tiles ahead
        int ls = (stage + kStages - 1) % kStages;
        if (t_load < ntiles) load_tile(A21, m, p, lda, t_load, tiles + ls * tile_elems);
        cp_async_commit();
        t_load += gridDim.x;
        cp_async_wait<kStages - 1>();
        __syncthreads();

        const double *tile = tiles + stage * tile_elems;
        const int64_t row0 = t * kTR;
        const int nrows = (int)((m - row0) < kTR ? (m - row0) : kTR);

        // (1) row argmax: thread (r, g) scans columns g, g+NG, ... ascending
        unsigned long long best = 0;
        int bidx = -1;
        if (r < nrows) {
            for (int k = g; k < p; k += NG) {
                unsigned long long key = abs_key(tile[k * (kTR + 1) + r]);
                nonfinite |= key >= kInfKey;
                if (bidx < 0 || key > best) {
                    best = key;
                    bidx = k;
                }
            }
        }
        pkey[g * kTR + r] = best;
        pidx[g * kTR + r] = bidx;
        __syncthreads();
        if (threadIdx.x < kTR) {
            unsigned long long b = 0;
            int bi = -1;
            for (int gg = 0; gg < NG; gg++) {
                int ii = pidx[gg * kTR + threadIdx.x];
                unsigned long long kk = pkey[gg * kTR + threadIdx.x];
                if (ii < 0) continue;
                if (bi < 0 || kk > b || (kk == b && ii < bi)) {
                    b = kk;
                    bi = ii;
                }
            }
            rowJ[threadIdx.x] = bi;
            if (J != nullptr && threadIdx.x < nrows) J[row0 + threadIdx.x] = bi;
            // row bi of C has a member (J_bi is not empty): the pivot search
            // keeps only such rows
            if (rowbits != nullptr && threadIdx.x < nrows && bi >= 0) atomicOr(rowbits + (bi >> 5), 1u << (bi & 31));
        }
        __syncthreads();

        // (2) merge the tile's rows into C: warp w takes rows w, w+8, w+16, w+24;
        // lanes walk k.  All C keys of the warp's rows are loaded before any
        // compare so that the L2 round trips overlap; the atomic fires only on
        // a new maximum.
        constexpr int KPL = kMaxP / 32;          // keys per lane and row
        constexpr int RPW = kTR / (kThreads / 32);  // rows per warp
        {
            unsigned long long cur[RPW][KPL];
#pragma unroll
            for (int q = 0; q < RPW; q++) {
                const int rr = warp + q * (kThreads / 32);
                const unsigned long long *crow = Ckeys + (int64_t)(rr < nrows ? rowJ[rr] : 0) * p;
#pragma unroll
                for (int t = 0; t < KPL; t++) {
                    const int k = lane + 32 * t;
                    cur[q][t] = (rr < nrows && k < p) ? __ldcg(crow + k) : ~0ull;
                }
            }
#pragma unroll
            for (int q = 0; q < RPW; q++) {
                const int rr = warp + q * (kThreads / 32);
                if (rr >= nrows) continue;
                unsigned long long *crow = Ckeys + (int64_t)rowJ[rr] * p;
#pragma unroll
                for (int t = 0; t < KPL; t++) {
                    const int k = lane + 32 * t;
                    if (k < p) {
                        const unsigned long long key = abs_key(tile[k * (kTR + 1) + rr]);
                        if (key > cur[q][t]) atomicMax(crow + k, key);
                    }
                }
            }
        }
        __syncthreads();  // the buffer is refilled next round
        stage = (stage + 1) % kStages;
    }
    cp_async_wait<0>();
    if (nonfinite) atomicCAS(info, kInfoOk, (int32_t)CTP_ENONFINITE);
}

// Single-row compression (eq. (4.1) with one set J = all rows): the column
// maxima of |A21| as integer keys.  CTA (seg, k) reduces rows [seg*L, ...) of
// column k with 16-byte loads and merges into ckey[k] with atomicMax.
__global__ void __launch_bounds__(256)
    k_colmax(const double *__restrict__ A21, int64_t m, int64_t lda, int64_t L,
             unsigned long long *__restrict__ ckey, int32_t *__restrict__ info) {
    const int k = blockIdx.y;
    const int64_t r0 = (int64_t)blockIdx.x * L, r1 = r0 + L < m ? r0 + L : m;
    const double *col = A21 + (int64_t)k * lda;
    unsigned long long best = 0;
    bool nonfinite = false;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const unsigned long long key = abs_key(__ldcs(col + r));
        nonfinite |= key >= kInfKey;
        best = key > best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
        best = w > best ? w : best;
    }
    if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(ckey + k, best);
    if (nonfinite) atomicCAS(info, kInfoOk, (int32_t)CTP_ENONFINITE);
}

// The same compression with the tiles brought in by TMA, one cp.async.bulk.tensor
// per tile of 16 rows x p columns (16 rows of a column are the 128 bytes of one
// swizzle span), and no CTA-wide barrier in the loop: warp w (of 8) owns rows
// 2w and 2w+1 of every tile.  It reads them in one 16-byte load per column
// (with the 128-byte swizzle, the chunk of rows 2c, 2c+1 of column k sits at
// chunk c ^ (k mod 8) of its span, so a warp's 32 columns spread over all
// banks), releases the stage as soon as the values are in registers, finds the
// two row maxima with warp reductions on the 32-bit halves of the keys, and
// merges the rows into C.  A ninth warp only issues the copies: a stage is
// refilled once all eight warps have released it (an mbarrier per stage each
// way), so the warps drift apart by up to three tiles instead of meeting at
// every barrier.
constexpr int kTT = 16;                           // rows per TMA tile
constexpr int kStagesT = 3;                       // tiles in flight per CTA
constexpr int kConsWarps = kTT / 2;               // two rows per consumer warp
constexpr int kThreadsT = 32 * (kConsWarps + 1);  // + the producer warp

// Lowest index among the lanes' (key, index) pairs with the largest key
// (keys compared as unsigned 64-bit integers by their 32-bit halves).
__device__ __forceinline__ int warp_argmax(unsigned long long key, int idx, unsigned &hi_out) {
    const unsigned h = (unsigned)(key >> 32), l = (unsigned)key;
    const unsigned H = __reduce_max_sync(0xffffffffu, h);
    const unsigned L = __reduce_max_sync(0xffffffffu, h == H ? l : 0u);
    hi_out = H;
    return __reduce_min_sync(0xffffffffu, (h == H && l == L) ? idx : 0x7fffffff);
}

__global__ void __launch_bounds__(kThreadsT, 2)
    k_compress_strict_tma(const __grid_constant__ CUtensorMap map, int64_t m, int p, uint32_t stage_bytes,
                          unsigned long long *__restrict__ Ckeys, int32_t *__restrict__ J,
                          uint32_t *__restrict__ rowbits, int32_t *__restrict__ info) {
    extern __shared__ unsigned char smraw[];
    uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ unsigned long long full[kStagesT], empty[kStagesT];
    __shared__ unsigned seen[kMaxP / 32];  // rows of C that received a row of this CTA
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (m + kTT - 1) / kTT;
    if (threadIdx.x < kMaxP / 32) seen[threadIdx.x] = 0;
    // this CTA's tiles are blockIdx.x + k * gridDim.x, k < nk
    const int64_t nk = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesT; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], kConsWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == kConsWarps) {
        // ---- producer: tile k goes to stage k mod S once tile k - S has been released
        if (lane == 0) {
            int64_t issued = 0;
            bool ok = true;
            for (int64_t k = 0; k < nk; k++) {
                const int s = (int)(k % kStagesT);
                if (k >= kStagesT && !tc::mbar_wait(&empty[s], (uint32_t)((k / kStagesT - 1) & 1), &abort_flag)) {
                    ok = false;
                    break;
                }
                const int64_t t = blockIdx.x + k * gridDim.x;
                tc::mbar_expect_tx(&full[s], (uint32_t)(kTT * 8 * p));  // the box: 16 rows x p columns
                tc::tma_load_2d(tiles + (size_t)s * stage_bytes, &map, (int)(t * kTT), 0, &full[s]);
                issued = k + 1;
            }
            if (!ok) {
                atomicExch(&abort_flag, 1);
                atomicCAS(info, kInfoOk, (int32_t)CTP_ETIMEOUT);
                // the CTA's shared memory must outlive every copy into it: wait
                // (bounded, whatever the abort flag says) for the last ones issued
                int never = 0;
                for (int64_t k = issued > kStagesT ? issued - kStagesT : 0; k < issued; k++)
                    tc::mbar_wait(&full[k % kStagesT], (uint32_t)((k / kStagesT) & 1), &never);
            }
        }
        return;
    }
    // ---- consumers
    constexpr int KPL = kMaxP / 32;  // columns per lane
    bool nonfinite = false;
    const int ra = 2 * warp, rb = ra + 1;
    const int chunk = warp << 4;  // byte offset of rows ra, rb in an unswizzled span
    for (int64_t k = 0; k < nk; k++) {
        const int s = (int)(k % kStagesT);
        if (!tc::mbar_wait(&full[s], (uint32_t)((k / kStagesT) & 1), &abort_flag)) {
            if (lane == 0) {
                atomicExch(&abort_flag, 1);
                atomicCAS(info, kInfoOk, (int32_t)CTP_ETIMEOUT);
            }
            break;
        }
        const uint8_t *tile = tiles + (size_t)s * stage_bytes;
        unsigned long long xa[KPL], xb[KPL];
#pragma unroll
        for (int u = 0; u < KPL; u++) {
            const int kc = lane + 32 * u;
            xa[u] = xb[u] = 0;
            if (kc < p) {
                const ulonglong2 v =
                    *reinterpret_cast<const ulonglong2 *>(tile + kc * 128 + (chunk ^ ((kc & 7) << 4)));
                xa[u] = v.x & kAbsMask;
                xb[u] = v.y & kAbsMask;
            }
        }
        // per lane: the largest key of its columns (ascending, so the lowest
        // column wins ties); lanes without a column offer none
        unsigned long long ba = xa[0], bb = xb[0];
        int ia = lane < p ? lane : 0x7fffffff, ib = ia;
#pragma unroll
        for (int u = 1; u < KPL; u++) {
            const int kc = lane + 32 * u;
            if (kc < p) {
                if (xa[u] > ba) {
                    ba = xa[u];
                    ia = kc;
                }
                if (xb[u] > bb) {
                    bb = xb[u];
                    ib = kc;
                }
            }
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty[s]);  // the rows are in registers
        unsigned ha, hb;
        const int Ia = warp_argmax(ba, ia, ha), Ib = warp_argmax(bb, ib, hb);
        const int64_t t = blockIdx.x + k * gridDim.x, row0 = t * kTT;
        const int nrows = (int)((m - row0) < kTT ? (m - row0) : kTT);
        const bool va = ra < nrows, vb = rb < nrows;
        // an Inf or NaN anywhere in a row is its maximum key
        nonfinite |= (va && ha >= 0x7FF00000u) || (vb && hb >= 0x7FF00000u);
        if (lane == 0) {
            // row Ia of C has a member: the CTA gathers these bits in shared
            // memory and publishes them once at the end (a global store per row
            // would queue ~m stores on the one or two L2 lines of the bits)
            if (va) {
                if (J != nullptr) J[row0 + ra] = Ia;
                atomicOr(&seen[Ia >> 5], 1u << (Ia & 31));
            }
            if (vb) {
                if (J != nullptr) J[row0 + rb] = Ib;
                atomicOr(&seen[Ib >> 5], 1u << (Ib & 31));
            }
        }
        // merge into rows Ia, Ib of C: every C key is loaded before any compare
        // (the L2 round trips overlap); the atomic fires only on a new maximum
        unsigned long long *ca = Ckeys + (int64_t)(va ? Ia : 0) * p;
        unsigned long long *cb = Ckeys + (int64_t)(vb ? Ib : 0) * p;
        unsigned long long cura[KPL], curb[KPL];
#pragma unroll
        for (int u = 0; u < KPL; u++) {
            const int kc = lane + 32 * u;
            cura[u] = (va && kc < p) ? __ldcg(ca + kc) : ~0ull;
            curb[u] = (vb && kc < p) ? __ldcg(cb + kc) : ~0ull;
        }
#pragma unroll
        for (int u = 0; u < KPL; u++) {
            const int kc = lane + 32 * u;
            if (xa[u] > cura[u]) atomicMax(ca + kc, xa[u]);
            if (xb[u] > curb[u]) atomicMax(cb + kc, xb[u]);
        }
    }
    if (nonfinite) atomicCAS(info, kInfoOk, (int32_t)CTP_ENONFINITE);
    // every consumer warp is past its last tile (named barrier 1: the producer
    // warp has left)
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kConsWarps) : "memory");
    if (rowbits != nullptr && threadIdx.x < (p + 31) / 32 && seen[threadIdx.x] != 0u)
        atomicOr(rowbits + threadIdx.x, seen[threadIdx.x]);
}

__global__ void k_keys_to_rowmajor(const unsigned long long *__restrict__ Ckeys,
                                   double *__restrict__ C, int pp) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < pp) C[i] = __longlong_as_double((long long)Ckeys[i]);
}

}  // namespace

static size_t strict_smem(int p) {
    constexpr int NG = kThreads / kTR;
    return sizeof(double) * (size_t)kStages * p * (kTR + 1) + NG * kTR * (sizeof(unsigned long long) + sizeof(int)) +
           kTR * sizeof(int);
}

// TMA map of A21 (m x p column-major, lda) in boxes of 16 rows x p columns with
// the 128-byte swizzle; false when the addresses do not allow one (A21 or lda*8
// not a multiple of 16 bytes) or the encoder is unavailable
static bool make_map_a21(CUtensorMap *map, const double *A21, int64_t m, int p, int64_t lda) {
    if ((reinterpret_cast<uintptr_t>(A21) & 15) != 0 || ((lda * 8) & 15) != 0) return false;
    if (m >= ((int64_t)1 << 31)) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tc::encode_fn();
    if (enc == nullptr) return false;
    cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)p};
    cuuint64_t strides[1] = {(cuuint64_t)lda * 8};
    cuuint32_t box[2] = {(cuuint32_t)kTT, (cuuint32_t)p};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(A21), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_compress_strict(const double *A21, int64_t m, int p, int64_t lda,
                                   unsigned long long *Ckeys, int32_t *J, uint32_t *rowbits, int32_t *info,
                                   int num_sms, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    CUtensorMap map;
    if (make_map_a21(&map, A21, m, p, lda)) {
        const uint32_t stage_bytes = (uint32_t)((p * 128 + 1023) / 1024 * 1024);
        const size_t smem = (size_t)kStagesT * stage_bytes + 1024;
        cudaError_t err = smem_at_least((const void *)k_compress_strict_tma, smem);
        if (err != cudaSuccess) return err;
        int per_sm = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_compress_strict_tma, kThreadsT, smem);
        if (err != cudaSuccess) return err;
        if (per_sm < 1) per_sm = 1;
        const int64_t ntiles = (m + kTT - 1) / kTT;
        int64_t grid = (int64_t)num_sms * per_sm;
        if (grid > ntiles) grid = ntiles;
        k_compress_strict_tma<<<(unsigned)grid, kThreadsT, smem, st>>>(map, m, p, stage_bytes, Ckeys, J, rowbits,
                                                                       info);
        return cudaGetLastError();
    }
    size_t smem = strict_smem(p);
    cudaError_t err = smem_at_least((const void *)k_compress_strict, smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_compress_strict, kThreads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    int64_t ntiles = (m + kTR - 1) / kTR;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    k_compress_strict<<<(unsigned)grid, kThreads, smem, st>>>(A21, m, p, lda, Ckeys, J, rowbits, info);
    return cudaGetLastError();
}

cudaError_t launch_compress_single_row(const double *A21, int64_t m, int p, int64_t lda,
                                       unsigned long long *ckey, int32_t *info, int num_sms, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    // about four CTAs per SM in all, segments of at least 4096 rows
    int64_t nseg = (4LL * num_sms + p - 1) / p;
    const int64_t maxseg = (m + 4095) / 4096;
    if (nseg > maxseg) nseg = maxseg;
    if (nseg < 1) nseg = 1;
    const int64_t L = (m + nseg - 1) / nseg;
    k_colmax<<<dim3((unsigned)nseg, p), 256, 0, st>>>(A21, m, lda, L, ckey, info);
    return cudaGetLastError();
}

cudaError_t launch_keys_to_rowmajor(const unsigned long long *Ckeys, double *C, int p,
                                    cudaStream_t st) {
    int pp = p * p;
    k_keys_to_rowmajor<<<(pp + 255) / 256, 256, 0, st>>>(Ckeys, C, pp);
    return cudaGetLastError();
}

}  // namespace ctp

// ---------------------------------------------------------------------------
// Strict compression without any device allocation.
//
// Some host programs cannot allocate device memory at the point where they
// need the compression: a plugin inside an application that owns every device
// allocation through its own pool, or a caller on a latency-critical path that
// must not pay for cudaMalloc and its implicit synchronisation.  For them the
// scratch of the kernel (the info word and the p x p integer keys of C) lives
// in one file-scope device array, sized for the largest supported p, that every
// GPU holds from the moment this library is loaded on it until the process
// exits.  Host code must not use the array's name as a device address (it is a
// host-side stand-in); the device address is looked up once per device and
// cached for the life of the process.  The cache does not survive a device
// reset (cudaDeviceReset, or the primary context released and made again):
// after one, the cached address is stale, so such a program must not call
// ctp_compress_strict_noalloc again.

#include <mutex>

namespace {

constexpr int kNoAllocMaxP = ctp::kMaxP;
constexpr size_t kNoAllocBytes = 256 + sizeof(unsigned long long) * (size_t)kNoAllocMaxP * kNoAllocMaxP;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on the
// first call for that device).  Returns nullptr if the lookup fails.
void *noalloc_scratch_current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
            (void)cudaGetLastError();
            return nullptr;
        }
        g_noalloc_addr[dev] = ptr;
    }
    return g_noalloc_addr[dev];
}

}  // namespace

extern "C" ctp_status ctp_compress_strict_noalloc(int64_t m, int32_t p, const double *A21, int64_t lda,
                                                  double *C, int32_t *J, int32_t *info_host,
                                                  void *stream) {
    if (A21 == nullptr || C == nullptr) return CTP_EINVAL;
    if (m < 0 || p < 1 || lda < (m > 0 ? m : 1)) return CTP_EINVAL;
    if (p > kNoAllocMaxP) return CTP_ECAPACITY;
    unsigned char *scratch = static_cast<unsigned char *>(noalloc_scratch_current_device());
    if (scratch == nullptr) return CTP_ECUDA;
    int num_sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CTP_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *info = reinterpret_cast<int32_t *>(scratch);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(scratch + 256);
    // the array keeps the previous call's contents: clear the info word and the keys
    if (cudaMemsetAsync(info, 0, sizeof(int32_t), st) != cudaSuccess) return CTP_ECUDA;
    if (cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (size_t)p * p, st) != cudaSuccess)
        return CTP_ECUDA;
    if (ctp::launch_compress_strict(A21, m, p, lda, keys, J, nullptr, info, num_sms, st) != cudaSuccess)
        return CTP_ECUDA;
    if (ctp::launch_keys_to_rowmajor(keys, C, p, st) != cudaSuccess) return CTP_ECUDA;
    if (info_host != nullptr) {
        if (cudaMemcpyAsync(info_host, info, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return CTP_ECUDA;
    }
    return CTP_OK;
}
