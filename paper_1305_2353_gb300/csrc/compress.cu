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
                      int32_t *__restrict__ rowflags,
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
            if (rowflags != nullptr && threadIdx.x < nrows && bi >= 0) rowflags[bi] = 1;
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

// The same compression with the tiles brought in by TMA: one
// cp.async.bulk.tensor per tile of 16 rows x p columns (16 rows of a column are
// the 128 bytes of one swizzle span), three stages per CTA, two CTAs per SM.  With the 128-byte swizzle, the 16-byte chunk c of column k sits at
// chunk c ^ (k mod 8) of its 128-byte row, so both the row-per-lane reads of
// the argmax and the column-per-lane reads of the merge into C meet few bank
// conflicts.  Each tile costs one instruction to load instead of one per
// element, which is what kept the per-element kernel above at a quarter of HBM.
constexpr int kTT = 16;         // rows per TMA tile
constexpr int kStagesT = 3;     // tiles per CTA: one in use, two in flight
__global__ void __launch_bounds__(kThreads, 2)
    k_compress_strict_tma(const __grid_constant__ CUtensorMap map, int64_t m, int p, uint32_t stage_bytes,
                          unsigned long long *__restrict__ Ckeys, int32_t *__restrict__ J,
                          int32_t *__restrict__ rowflags, int32_t *__restrict__ info) {
    extern __shared__ unsigned char smraw[];
    uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ unsigned long long full[kStagesT];
    __shared__ unsigned long long pkey[kThreads / 32][kTT];  // per warp: best key of each row
    __shared__ int pidx[kThreads / 32][kTT];
    __shared__ int rowJ[kTT];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (m + kTT - 1) / kTT;
    if (tid == 0) {
        for (int s = 0; s < kStagesT; s++) tc::mbar_init(&full[s], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int64_t k) {  // the k-th tile of this CTA into its stage
        const int64_t t = blockIdx.x + k * gridDim.x;
        if (t >= ntiles) return;
        const int s = (int)(k % kStagesT);
        tc::mbar_expect_tx(&full[s], (uint32_t)(kTT * 8 * p));  // the box: 16 rows x p columns
        tc::tma_load_2d(tiles + (size_t)s * stage_bytes, &map, (int)(t * kTT), 0, &full[s]);
    };
    if (tid == 0)
        for (int k = 0; k < kStagesT - 1; k++) issue(k);
    bool nonfinite = false;
    // phase 1 mapping: thread (rp, g) takes rows 2rp, 2rp+1 (one 16-byte chunk)
    // of columns g, g + 32, ...; a warp covers four column groups
    const int rp = tid & 7, g = tid >> 3;
    for (int64_t k = 0;; k++) {
        const int64_t t = blockIdx.x + k * gridDim.x;
        if (t >= ntiles) break;
        if (tid == 0) issue(k + kStagesT - 1);  // that stage was released at the end of round k-1
        const int s = (int)(k % kStagesT);
        // one warp waits for the tile; the others wait at the barrier (issuing
        // nothing), which then orders the tile's shared memory for all of them
        bool ok = true;
        if (warp == 0) ok = tc::mbar_wait(&full[s], (uint32_t)((k / kStagesT) & 1), &abort_flag);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicCAS(info, kInfoOk, (int32_t)CTP_ETIMEOUT);
                // wait (bounded) for the copies still in flight into this CTA's stages
                for (int64_t k2 = k + 1; k2 < k + kStagesT; k2++)
                    if (blockIdx.x + k2 * gridDim.x < ntiles)
                        tc::mbar_wait(&full[k2 % kStagesT], (uint32_t)((k2 / kStagesT) & 1), &abort_flag);
            }
            break;
        }
        const uint8_t *tile = tiles + (size_t)s * stage_bytes;
        const int64_t row0 = t * kTT;
        const int nrows = (int)((m - row0) < kTT ? (m - row0) : kTT);
        // (1) row argmax, two rows per 16-byte load; columns ascend per thread,
        // so a strict > keeps the lowest column on ties
        unsigned long long b0 = 0, b1 = 0;
        int i0 = -1, i1 = -1;
        for (int kc = g; kc < p; kc += 32) {
            const ulonglong2 v =
                *reinterpret_cast<const ulonglong2 *>(tile + kc * 128 + (((rp ^ (kc & 7)) & 7) << 4));
            const unsigned long long x = v.x & kAbsMask, y = v.y & kAbsMask;
            if (i0 < 0 || x > b0) {
                b0 = x;
                i0 = kc;
            }
            if (i1 < 0 || y > b1) {
                b1 = y;
                i1 = kc;
            }
        }
        // the four column groups of this warp (lanes 8 apart), lowest column on ties
#pragma unroll
        for (int o = 8; o < 32; o <<= 1) {
            const unsigned long long ob0 = __shfl_xor_sync(0xffffffffu, b0, o), ob1 = __shfl_xor_sync(0xffffffffu, b1, o);
            const int oi0 = __shfl_xor_sync(0xffffffffu, i0, o), oi1 = __shfl_xor_sync(0xffffffffu, i1, o);
            if (oi0 >= 0 && (i0 < 0 || ob0 > b0 || (ob0 == b0 && oi0 < i0))) {
                b0 = ob0;
                i0 = oi0;
            }
            if (oi1 >= 0 && (i1 < 0 || ob1 > b1 || (ob1 == b1 && oi1 < i1))) {
                b1 = ob1;
                i1 = oi1;
            }
        }
        if (lane < 8) {
            pkey[warp][2 * rp] = b0;
            pidx[warp][2 * rp] = i0;
            pkey[warp][2 * rp + 1] = b1;
            pidx[warp][2 * rp + 1] = i1;
        }
        __syncthreads();
        if (tid < kTT) {
            unsigned long long b = 0;
            int bi = -1;
            for (int ww = 0; ww < kThreads / 32; ww++) {
                const int ii = pidx[ww][tid];
                const unsigned long long kk = pkey[ww][tid];
                if (ii < 0) continue;
                if (bi < 0 || kk > b || (kk == b && ii < bi)) {
                    b = kk;
                    bi = ii;
                }
            }
            rowJ[tid] = bi;
            // an Inf or NaN anywhere in a row is its maximum key
            if (tid < nrows && b >= kInfKey) nonfinite = true;
            if (J != nullptr && tid < nrows) J[row0 + tid] = bi;
            if (rowflags != nullptr && tid < nrows && bi >= 0) rowflags[bi] = 1;
        }
        __syncthreads();
        // (2) merge rows 2w, 2w+1 into C (warp w), lanes walk k with one 16-byte
        // load per two entries; every C key is loaded before any compare (the
        // L2 round trips overlap), the atomic fires only on a new maximum
        constexpr int KPL = kMaxP / 32;
        const int ra = 2 * warp, rb = ra + 1;
        const bool va = ra < nrows, vb = rb < nrows;
        const unsigned long long *ca = Ckeys + (int64_t)(va ? rowJ[ra] : 0) * p;
        const unsigned long long *cb = Ckeys + (int64_t)(vb ? rowJ[rb] : 0) * p;
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
            if (kc < p) {
                const ulonglong2 v =
                    *reinterpret_cast<const ulonglong2 *>(tile + kc * 128 + (((warp ^ (kc & 7)) & 7) << 4));
                const unsigned long long x = v.x & kAbsMask, y = v.y & kAbsMask;
                if (x > cura[u]) atomicMax(const_cast<unsigned long long *>(ca) + kc, x);
                if (y > curb[u]) atomicMax(const_cast<unsigned long long *>(cb) + kc, y);
            }
        }
        __syncthreads();  // this stage is refilled next round
    }
    if (nonfinite) atomicCAS(info, kInfoOk, (int32_t)CTP_ENONFINITE);
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
                                   unsigned long long *Ckeys, int32_t *J, int32_t *rowflags, int32_t *info,
                                   int num_sms, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    CUtensorMap map;
    if (make_map_a21(&map, A21, m, p, lda)) {
        const uint32_t stage_bytes = (uint32_t)((p * 128 + 1023) / 1024 * 1024);
        const size_t smem = (size_t)kStagesT * stage_bytes + 1024;
        cudaError_t err = smem_at_least((const void *)k_compress_strict_tma, smem);
        if (err != cudaSuccess) return err;
        int per_sm = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_compress_strict_tma, kThreads, smem);
        if (err != cudaSuccess) return err;
        if (per_sm < 1) per_sm = 1;
        const int64_t ntiles = (m + kTT - 1) / kTT;
        int64_t grid = (int64_t)num_sms * per_sm;
        if (grid > ntiles) grid = ntiles;
        k_compress_strict_tma<<<(unsigned)grid, kThreads, smem, st>>>(map, m, p, stage_bytes, Ckeys, J, rowflags,
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
    k_compress_strict<<<(unsigned)grid, kThreads, smem, st>>>(A21, m, p, lda, Ckeys, J, rowflags, info);
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
