// form_tc.cu -- K6 (tensor cores): the Form task S = L21 D11 L21^T = W21 L21^T
// (Section 1 task list), lower triangle, with BF16 operands and FP32
// accumulation on the 5th-generation tensor cores (tcgen05), S stored as FP32:
// full column-major, lower-packed by columns, or in contiguous 128 x 128 blocks
// (the layout HBM absorbs at full write speed: each block is written front to
// back, where the column layouts scatter 512-byte pieces over 256 columns).
//
// Layout: W21 and L21 are BF16 copies written by the Solve kernel, row-major
// m x Kp (K = pivot position contiguous, Kp = p rounded up to 64, zero beyond
// e).  Both GEMM operands are therefore K-major, which is what the tensor core
// reads directly: S(i,j) = sum_k W21(i,k) L21(j,k).
//
// Kernel: persistent, one CTA per SM, walking the tiles of the lower triangle
// (128 rows of S by 256 columns).  Warp roles:
//   warp 0     TMA producer: 128B-swizzled K-blocks (64 BF16 = 128 bytes per
//              row).  The L21 block of a column block of S (256 rows, all of K)
//              stays resident in shared memory while consecutive tiles of this
//              CTA share it; W21 blocks (128 rows) stream through a 6-stage
//              ring.  Warp 0 also allocates and frees the tensor memory.
//   warp 1     MMA issuer: one thread issues tcgen05.mma (M=128, N=256, K=16)
//              into one of two FP32 accumulators of 256 TMEM columns each and
//              commits stage releases and accumulator completion to mbarriers.
//   warps 2-9  epilogue: tcgen05.ld of a 32-lane x 32-column slice, coalesced
//              stores of column-major S (lanes are consecutive rows), masking
//              the strict upper triangle; the accumulator is handed back as
//              soon as it has been read, so MMA of the next tile overlaps the
//              stores of this one.
// Every mbarrier wait is bounded; on timeout the kernel records CTP_ETIMEOUT in
// the info word, stops issuing work, waits for nothing further, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "ctp_internal.cuh"

namespace ctp {

namespace {

constexpr int kBM = 128, kBN = 256, kBK = 64, kStages = 6;
constexpr int kMaxKB = 4;  // K blocks of 64 (p <= 256)
constexpr int kUmmaK = 16;
constexpr int kEpiWarps = 8;
constexpr int kThreadsTC = 32 * (2 + kEpiWarps);
constexpr uint32_t kStageA = kBM * kBK * 2;  // 16 KB
constexpr uint32_t kStageB = kBN * kBK * 2;  // 32 KB
constexpr uint32_t kTmemCols = 512;          // two 256-column FP32 accumulators
constexpr long kSpinLimit = 1L << 22;

struct Bars {
    unsigned long long full[kStages], empty[kStages], acc_full[2], acc_empty[2], bfull, bempty;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `bar` with the given parity; false on timeout
// or when another role has already aborted.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, Bars *b) {
    for (long it = 0; it < kSpinLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255 && *(volatile int *)&b->abort) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor for a K-major operand in the canonical
// 128-byte-swizzle layout written by TMA: rows of 128 bytes, groups of 8 rows
// 1024 bytes apart (stride byte offset), version bits 46-47 = 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D = FP32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// Tiles of the lower triangle, walked column block by column block: column
// block b (256 columns) meets row blocks 2b..nM-1 (128 rows), so
// T(b) = b*nM - b(b-1) tiles precede column block b.  Consecutive tiles --
// which run at the same time on neighbouring SMs -- are vertically adjacent,
// so their stores into a column of S land next to each other in HBM.
__host__ __device__ inline int64_t tiles_before_col(int64_t b, int64_t nM) { return b * nM - b * (b - 1); }
__host__ __device__ inline int64_t tile_count(int64_t nM) {
    const int64_t nN = (nM + 1) / 2;  // column blocks that meet the triangle
    return tiles_before_col(nN, nM);
}
__device__ __forceinline__ void decode_tile(int64_t t, int nM, int &ti, int &tj) {
    int lo = 0, hi = (nM + 1) / 2;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tiles_before_col(mid, nM) <= t)
            lo = mid;
        else
            hi = mid;
    }
    tj = lo;
    ti = 2 * lo + (int)(t - tiles_before_col(lo, nM));
}

// Everything the roles need to know about one tile of work.
struct TileInfo {
    int ti, tj, KB, key;  // key: identifies the resident L21 block (front and column block)
    int64_t arow, brow;   // first rows of the W21 / L21 boxes in the operand buffers
    int64_t m, nb, lds;
    float *S;
    int layout;
};

struct BatchTab {
    const ctp_front *fronts;
    const BFront *tab;
    const int *item_front;
};

template <bool kBatch>
__device__ __forceinline__ TileInfo tile_info(int64_t t, int nM, int KB, int64_t m, float *S,
                                              int64_t lds, int layout, const BatchTab &bt) {
    TileInfo x;
    if (!kBatch) {
        decode_tile(t, nM, x.ti, x.tj);
        x.KB = KB;
        x.key = x.tj;
        x.arow = (int64_t)x.ti * kBM;
        x.brow = (int64_t)x.tj * kBN;
        x.m = m;
        x.nb = nM;
        x.S = S;
        x.lds = lds;
        x.layout = layout;
    } else {
        const int f = bt.item_front[t];
        const BFront b = bt.tab[f];
        decode_tile(t - b.f0, b.nM, x.ti, x.tj);
        const int e = *bt.fronts[f].nelim;
        x.KB = (e + kBK - 1) / kBK;
        x.key = f * 65536 + x.tj;
        x.arow = b.row0 + (int64_t)x.ti * kBM;
        x.brow = b.row0 + (int64_t)x.tj * kBN;
        x.m = b.m;
        x.nb = b.nM;
        x.S = reinterpret_cast<float *>(bt.fronts[f].S);
        x.lds = 0;
        x.layout = 2;
    }
    return x;
}

template <bool kBatch>
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_form_tc(const __grid_constant__ CUtensorMap mapW, const __grid_constant__ CUtensorMap mapL,
              int64_t m_single, const int32_t *__restrict__ nelim_p, float *__restrict__ S_single,
              int64_t lds_single, int layout_single, int32_t *__restrict__ info, int64_t ntiles_batch,
              BatchTab btab) {
    extern __shared__ unsigned char smraw[];
    __shared__ Bars bars;
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    uint8_t *sB = smem;                                 // [kMaxKB][kStageB]: resident L21 block
    uint8_t *sA = smem + (size_t)kMaxKB * kStageB;     // [kStages][kStageA]: W21 ring
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int KB1 = kBatch ? 0 : (*nelim_p + kBK - 1) / kBK;
    const int nM1 = kBatch ? 0 : (int)((m_single + kBM - 1) / kBM);
    const int64_t ntiles = kBatch ? ntiles_batch : tile_count(nM1);
#define TILE(t) tile_info<kBatch>((t), nM1, KB1, m_single, S_single, lds_single, layout_single, btab)

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&bars.full[s], 1);
            mbar_init(&bars.empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bars.acc_full[b], 1);
            mbar_init(&bars.acc_empty[b], kEpiWarps);
        }
        mbar_init(&bars.bfull, 1);
        mbar_init(&bars.bempty, 1);
        bars.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&bars.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars.tmem_base;
    const uint32_t idesc = idesc_bf16(kBM, kBN);

    if (warp == 0) {
        // ---------------- TMA producer: the L21 block of the current column block
        // stays resident while consecutive tiles share it; W21 blocks stream
        if (lane == 0) {
            int stage = 0, cur_key = -1;
            uint32_t phase = 0, bphase = 0;
            for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
                const TileInfo x = TILE(t);
                if (x.KB == 0) continue;
                bool ok = true;
                if (x.key != cur_key) {
                    if (!mbar_wait(&bars.bempty, bphase ^ 1u, &bars)) {
                        atomicExch(&bars.abort, 1);
                        break;
                    }
                    mbar_expect_tx(&bars.bfull, (uint32_t)x.KB * kStageB);
                    for (int kb = 0; kb < x.KB; kb++)
                        tma_load_2d(sB + (size_t)kb * kStageB, &mapL, kb * kBK, (int)x.brow, &bars.bfull);
                    bphase ^= 1u;
                    cur_key = x.key;
                }
                for (int kb = 0; kb < x.KB; kb++) {
                    if (!mbar_wait(&bars.empty[stage], phase ^ 1u, &bars)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&bars.full[stage], kStageA);
                    tma_load_2d(sA + (size_t)stage * kStageA, &mapW, kb * kBK, (int)x.arow, &bars.full[stage]);
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) {
                    atomicExch(&bars.abort, 1);
                    break;
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int stage = 0, acc = 0, cur_key = -1;
            uint32_t phase = 0, accphase = 0, bphase = 0;
            for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
                const TileInfo x = TILE(t);
                if (!mbar_wait(&bars.acc_empty[acc], accphase ^ 1u, &bars)) {
                    atomicExch(&bars.abort, 1);
                    break;
                }
                tc_fence_after();
                bool ok = true;
                if (x.KB > 0 && x.key != cur_key) {
                    if (!mbar_wait(&bars.bfull, bphase, &bars)) {
                        atomicExch(&bars.abort, 1);
                        break;
                    }
                    tc_fence_after();
                    bphase ^= 1u;
                    cur_key = x.key;
                }
                const uint32_t dt = tmem + (uint32_t)(acc * kBN);
                for (int kb = 0; kb < x.KB; kb++) {
                    if (!mbar_wait(&bars.full[stage], phase, &bars)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + (size_t)stage * kStageA);
                    const uint32_t b0 = smem_u32(sB + (size_t)kb * kStageB);
#pragma unroll
                    for (int k = 0; k < kBK / kUmmaK; k++) {
                        // advance 16 BF16 = 32 bytes along K inside the swizzled rows
                        umma_bf16(dt, sdesc(a0 + k * 32), sdesc(b0 + k * 32), idesc,
                                  (kb > 0 || k > 0) ? 1u : 0u);
                    }
                    umma_commit(&bars.empty[stage]);  // W21 stage free once these MMAs finish
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) {
                    atomicExch(&bars.abort, 1);
                    break;
                }
                umma_commit(&bars.acc_full[acc]);  // accumulator ready
                // release the resident L21 block when the next tile with work needs another
                if (x.KB > 0) {
                    int next_key = -2;
                    for (int64_t tn = t + gridDim.x; tn < ntiles; tn += gridDim.x) {
                        const TileInfo y = TILE(tn);
                        if (y.KB > 0) {
                            next_key = y.key;
                            break;
                        }
                    }
                    if (next_key != x.key) umma_commit(&bars.bempty);
                }
                if (++acc == 2) {
                    acc = 0;
                    accphase ^= 1u;
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..9
        const int q = warp & 3;             // TMEM lane quarter this warp may access
        const int half = (warp - 2) >> 2;   // 128-column half of the 256-column tile
        int acc = 0;
        uint32_t accphase = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const TileInfo x = TILE(t);
            const int ti = x.ti, tj = x.tj, KB = x.KB, layout = x.layout;
            const int64_t m = x.m, nb = x.nb, lds = x.lds;
            float *S = x.S;
            if (!mbar_wait(&bars.acc_full[acc], accphase, &bars)) {
                if (lane == 0) atomicExch(&bars.abort, 1);
                break;
            }
            tc_fence_after();
            const int64_t i = (int64_t)ti * kBM + q * 32 + lane;
            const int64_t jbase = (int64_t)tj * kBN + half * 128;
            // tiles strictly below the diagonal and inside S need no masking
            const bool interior = (jbase + 127 < (int64_t)ti * kBM) && ((int64_t)ti * kBM + kBM <= m);
            // block layout: this half of the tile is block (ti, 2 tj + half) of S;
            // blocks above the block diagonal are not part of S
            const int64_t bj = 2 * (int64_t)tj + half;
            const bool tiled = layout == 2;
            if (tiled && bj > ti) goto next_tile_half;
#pragma unroll 1
            for (int c = 0; c < 4; c += 2) {
                uint32_t r[64];
                const uint32_t taddr =
                    tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kBN + half * 128 + c * 32);
                tmem_ld32_nowait(taddr, *reinterpret_cast<uint32_t(*)[32]>(&r[0]));
                tmem_ld32_nowait(taddr + 32, *reinterpret_cast<uint32_t(*)[32]>(&r[32]));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (KB == 0) {
#pragma unroll
                    for (int x = 0; x < 64; x++) r[x] = 0u;
                }
                const int64_t j0 = jbase + c * 32;
                if (tiled) {
                    // whole blocks, front to back: column c of the block is the
                    // 512 bytes written by the four lane quarters
                    float *blk = S + (int64_t)16384 * (bj * nb - bj * (bj - 1) / 2 + (ti - bj));
                    float *ptr = blk + (int64_t)(c * 32) * 128 + q * 32 + lane;
#pragma unroll
                    for (int x = 0; x < 64; x++) ptr[x * 128] = __uint_as_float(r[x]);
                    continue;
                }
                // S(i, j) lives at S + col(j) + i, with col(j) = j*lds (full) or
                // j*m - j(j+1)/2 (packed; consecutive columns are m-1-j apart)
                const bool packed = layout == 1;
                float *ptr = S + (packed ? j0 * m - j0 * (j0 + 1) / 2 : j0 * lds) + i;
                if (interior) {
                    if (packed) {
                        int d = (int)(m - 1 - j0);
#pragma unroll
                        for (int x = 0; x < 64; x++) {
                            *ptr = __uint_as_float(r[x]);
                            ptr += d;
                            --d;
                        }
                    } else {
#pragma unroll
                        for (int x = 0; x < 64; x++) {
                            *ptr = __uint_as_float(r[x]);
                            ptr += lds;
                        }
                    }
                } else {
                    int64_t j = j0;
#pragma unroll
                    for (int x = 0; x < 64; x++) {
                        if (i < m && j <= i) *ptr = __uint_as_float(r[x]);
                        ptr += packed ? (m - 1 - j) : lds;
                        ++j;
                    }
                }
            }
        next_tile_half:
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.acc_empty[acc]);
            if (++acc == 2) {
                acc = 0;
                accphase ^= 1u;
            }
        }
    }
#undef TILE
    __syncthreads();
    if (threadIdx.x == 0 && bars.abort) atomicCAS(info, kInfoOk, (int32_t)CTP_ETIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn == nullptr) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap *map, const void *base, int64_t rows, int Kp, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (enc == nullptr) return false;
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

int form_tc_kpad(int p) { return (p + kBK - 1) / kBK * kBK; }

cudaError_t launch_form_tc(const void *Wb, const void *Lb, int64_t m, int Kp, const int32_t *nelim,
                           float *S, int64_t lds, int layout, int32_t *info, int num_sms,
                           cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    if ((((uintptr_t)Wb) | ((uintptr_t)Lb)) & 15) return cudaErrorMisalignedAddress;
    CUtensorMap mW, mL;
    if (!make_map(&mW, Wb, m, Kp, kBM) || !make_map(&mL, Lb, m, Kp, kBN)) return cudaErrorInvalidValue;
    const size_t smem = (size_t)kMaxKB * kStageB + (size_t)kStages * kStageA + 1024;
    cudaError_t err =
        cudaFuncSetAttribute(k_form_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int nM = (int)((m + kBM - 1) / kBM);
    const int64_t ntiles = tile_count(nM);
    const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
    BatchTab none = {nullptr, nullptr, nullptr};
    k_form_tc<false><<<grid, kThreadsTC, smem, st>>>(mW, mL, m, nelim, S, lds, layout, info, 0, none);
    return cudaGetLastError();
}

int64_t form_tc_tiles(int64_t m) { return m > 0 ? tile_count((m + kBM - 1) / kBM) : 0; }

cudaError_t launch_form_tc_batch(const ctp_front *fronts, const BFront *tab, const int *item_front,
                                 int64_t items, int64_t total_rows, const void *Wb, const void *Lb,
                                 int32_t *info, int num_sms, cudaStream_t st) {
    if (items == 0) return cudaSuccess;
    if ((((uintptr_t)Wb) | ((uintptr_t)Lb)) & 15) return cudaErrorMisalignedAddress;
    CUtensorMap mW, mL;
    if (!make_map(&mW, Wb, total_rows, kBatchKp, kBM) || !make_map(&mL, Lb, total_rows, kBatchKp, kBN))
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)kMaxKB * kStageB + (size_t)kStages * kStageA + 1024;
    cudaError_t err =
        cudaFuncSetAttribute(k_form_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int grid = (int)(items < num_sms ? items : num_sms);
    BatchTab bt = {fronts, tab, item_front};
    k_form_tc<true><<<grid, kThreadsTC, smem, st>>>(mW, mL, 0, nullptr, nullptr, 0, 2, info, items, bt);
    return cudaGetLastError();
}

}  // namespace ctp
