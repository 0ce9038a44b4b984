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
#include "ctp_internal.cuh"
#include "tc_common.cuh"

namespace ctp {

using namespace tc;

namespace {

constexpr int kBM = 128, kBN = 256, kStages = 6;
constexpr int kMaxKB = 4;  // K blocks of 64 (p <= 256)
constexpr int kEpiWarps = 8;
constexpr int kThreadsTC = 32 * (2 + kEpiWarps);
constexpr uint32_t kStageA = kBM * kBK * 2;  // 16 KB
constexpr uint32_t kStageB = kBN * kBK * 2;  // 32 KB
constexpr uint32_t kTmemCols = 512;          // two 256-column FP32 accumulators
struct Bars {
    unsigned long long full[kStages], empty[kStages], acc_full[2], acc_empty[2], bfull, bempty;
    uint32_t tmem_base;
    int abort;
};


// Tile shapes and operand pieces.  Plain BF16 (P = 1): tiles of 128 rows x
// 256 columns.  Split BF16: every operand x is held as P BF16 pieces -- P = 2:
// hi = bf16(x), lo = bf16(x - hi); P = 3: hi, mid = bf16(x - hi), lo =
// bf16(x - hi - mid) -- and the accumulator receives the products of pieces
// whose orders sum to at most P - 1 (P = 2: hi*hi + hi*lo + lo*hi; P = 3: the
// six products hi*hi, hi*mid, mid*hi, hi*lo, lo*hi, mid*mid), the splitting
// scheme of Henry, Tang and Heinecke ("Leveraging the bfloat16 artificial
// intelligence datatype for higher-precision computations", 2019): P = 2
// gives products close to 2^-17 relative accuracy, P = 3 close to FP32's.  Split
// tiles are 128 x 128.  For P <= 2 the L21 block of a column block stays
// resident in shared memory (K blocks of 32 KB) beside a 96 KB ring of W21
// blocks; for P = 3 both operands stream through a 2-stage ring of 96 KB.
template <int P>
struct Cfg {
    static constexpr int BN = P == 1 ? 256 : 128;
    static constexpr int R = BN / kBM;                        // column blocks are R row blocks wide
    static constexpr bool kResident = P < 3;
    static constexpr int Stages = P == 1 ? 6 : (P == 2 ? 3 : 2);
    static constexpr uint32_t PieceA = kBM * kBK * 2;        // one 128 x 64 BF16 block
    static constexpr uint32_t PieceB = BN * kBK * 2;
    static constexpr uint32_t StageA = PieceA * P + (kResident ? 0 : PieceB * P);
    static constexpr uint32_t StageB = PieceB * P;           // resident block, per K block
    static constexpr size_t ResidentBytes = kResident ? (size_t)kMaxKB * StageB : 0;
    // Split forms: one MMA of N = 256 takes the hi and next pieces of L21 together
    // (they are contiguous), so a tile's accumulator is 256 columns wide and the
    // epilogue adds its two 128-column halves.
    static constexpr int AccN = 256;
    static constexpr uint32_t TmemCols = 2 * AccN;           // two FP32 accumulators
};
constexpr size_t kSmemBody = (size_t)kMaxKB * kStageB + (size_t)kStages * kStageA;
static_assert(Cfg<1>::ResidentBytes + Cfg<1>::Stages * Cfg<1>::StageA <= kSmemBody, "smem P=1");
static_assert(Cfg<2>::ResidentBytes + Cfg<2>::Stages * Cfg<2>::StageA <= kSmemBody, "smem P=2");
static_assert(Cfg<3>::ResidentBytes + Cfg<3>::Stages * Cfg<3>::StageA <= kSmemBody, "smem P=3");

// Tiles of the lower triangle, walked column block by column block: column
// block b meets row blocks R*b..nM-1, so T(b) = b*nM - R*b(b-1)/2 tiles
// precede it.  Consecutive tiles -- which run at the same time on
// neighbouring SMs in the round-robin walk -- are vertically adjacent.
__host__ __device__ inline int64_t tiles_before_col(int64_t b, int64_t nM, int R) {
    return b * nM - R * (b * (b - 1) / 2);
}
__host__ __device__ inline int64_t col_blocks(int64_t nM, int R) { return (nM + R - 1) / R; }
__host__ __device__ inline int64_t tile_count(int64_t nM, int R) {
    return tiles_before_col(col_blocks(nM, R), nM, R);
}
__device__ __forceinline__ void decode_tile(int64_t t, int nM, int R, int &ti, int &tj) {
    int lo = 0, hi = (int)col_blocks(nM, R);
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tiles_before_col(mid, nM, R) <= t)
            lo = mid;
        else
            hi = mid;
    }
    tj = lo;
    ti = R * lo + (int)(t - tiles_before_col(lo, nM, R));
}

// Everything the roles need to know about one tile of work.
struct TileInfo {
    int ti, tj, KB, key;  // key: identifies the resident L21 block (front and column block)
    int klast;            // 16-wide K-steps of the last K block that hold columns below e
    int64_t arow, brow;   // first rows of the W21 / L21 boxes in the operand buffers
    int64_t m, nb, lds;
    float *S;
    int layout;
};

struct BatchTab {
    const ctp_front *fronts;
    const BFront *tab;
    const int *item_front;
    int layout;  // 2: S in 128 x 128 blocks; 3: subtracted from the front's full FP64 S (lds)
    const int *item_tile;  // each item's tile of its front (nullptr: items of a front are consecutive from f0)
};

// Which tiles a CTA takes.  mode 0: round robin over the column-block-major
// tile list (all CTAs work down the same column block).  mode 2 (chunks): CTA
// c takes the c-th of G equal contiguous runs of that list, so consecutive
// tiles of a CTA share their column block and its resident L21 block (the walk
// for operands that fit in L2).  mode 1 (panels):
// the column blocks are taken G at a time; CTA c owns one column block of
// each panel (c, or G-1-c in odd panels, which evens out the work) and walks
// it from the diagonal down, keeping its L21 block resident.  All CTAs then
// move down the rows together, so each W21 block is fetched from HBM about
// once per panel and served to the other CTAs from L2 -- what keeps the
// operand traffic small when the operands do not fit in L2.
struct Sched {
    int mode, nM, G, c;
    int64_t ntiles, nN;
    int64_t t0, t1;  // mode 2: this CTA's run [t0, t1)
};

template <bool kBatch, int R>
__device__ __forceinline__ bool tile_k(int64_t k, const Sched &s, int e1, int64_t m1, float *S1,
                                       int64_t lds1, int layout1, const BatchTab &bt, TileInfo &x) {
    int ti, tj;
    if (kBatch) {
        const int64_t t = s.mode == 2 ? s.t0 + k : s.c + k * s.G;
        if (t >= (s.mode == 2 ? s.t1 : s.ntiles)) return false;
        const int f = bt.item_front[t];
        const BFront b = bt.tab[f];
        decode_tile(bt.item_tile != nullptr ? (int64_t)bt.item_tile[t] : t - b.f0, b.nM, R, ti, tj);
        const int e = *bt.fronts[f].nelim;
        x.ti = ti;
        x.tj = tj;
        x.KB = (e + kBK - 1) / kBK;
        x.klast = (e - (x.KB - 1) * kBK + kUmmaK - 1) / kUmmaK;
        x.key = f * 65536 + tj;
        x.arow = b.row0 + (int64_t)ti * kBM;
        x.brow = b.row0 + (int64_t)tj * R * kBM;
        x.m = b.m;
        x.nb = b.nM;
        x.S = reinterpret_cast<float *>(bt.fronts[f].S);
        x.lds = bt.fronts[f].lds;
        x.layout = bt.layout;
        return true;
    }
    if (s.mode != 1) {
        const int64_t t = s.mode == 2 ? s.t0 + k : s.c + k * s.G;
        if (t >= (s.mode == 2 ? s.t1 : s.ntiles)) return false;
        decode_tile(t, s.nM, R, ti, tj);
    } else {
        int64_t rem = k;
        bool found = false;
        for (int64_t P = 0; P * s.G < s.nN; P++) {
            const int64_t j = P * s.G + ((P & 1) ? (s.G - 1 - s.c) : s.c);
            if (j >= s.nN) continue;
            const int64_t cnt = s.nM - R * j;
            if (rem < cnt) {
                tj = (int)j;
                ti = (int)(R * j + rem);
                found = true;
                break;
            }
            rem -= cnt;
        }
        if (!found) return false;
    }
    x.ti = ti;
    x.tj = tj;
    x.KB = (e1 + kBK - 1) / kBK;
    x.klast = (e1 - (x.KB - 1) * kBK + kUmmaK - 1) / kUmmaK;
    x.key = tj;
    x.arow = (int64_t)ti * kBM;
    x.brow = (int64_t)tj * R * kBM;
    x.m = m1;
    x.nb = s.nM;
    x.S = S1;
    x.lds = lds1;
    x.layout = layout1;
    return true;
}

// Store 64 consecutive columns j0..j0+63 of row i of S (FP32 values in r) in
// the layout of S: 0 full column-major (lds), 1 lower-packed by columns, 2 in
// 128 x 128 blocks (this row's block row bi, block column bj, from column boffc
// of the block on; quarter q and lane name the row inside the block), 3
// subtracted from a full column-major FP64 matrix (lds).  Entries above the
// diagonal or below row m are skipped unless `interior` says there are none.
__device__ __forceinline__ void store64(const uint32_t (&r)[64], int layout, float *S, int64_t m, int64_t lds,
                                        int64_t nb, int64_t i, int64_t j0, bool interior, int64_t bi, int64_t bj,
                                        int boffc, int q, int lane) {
    if (layout == 3) {
        // subtract into a full column-major FP64 matrix (lower
        // triangle): 16 old values loaded before any is stored, so
        // that the loads are in flight together
        double *dp = reinterpret_cast<double *>(S) + j0 * lds + i;
#pragma unroll
        for (int h = 0; h < 64; h += 16) {
            double old[16];
#pragma unroll
            for (int xx = 0; xx < 16; xx++) {
                old[xx] = 0.0;
                if (interior || (i < m && j0 + h + xx <= i)) old[xx] = dp[(int64_t)(h + xx) * lds];
            }
#pragma unroll
            for (int xx = 0; xx < 16; xx++)
                if (interior || (i < m && j0 + h + xx <= i))
                    dp[(int64_t)(h + xx) * lds] = old[xx] - (double)__uint_as_float(r[h + xx]);
        }
        return;
    }
    if (layout == 2) {
        // whole blocks, front to back: column c of the block is the
        // 512 bytes written by the four lane quarters
        float *blk = S + (int64_t)16384 * (bj * nb - bj * (bj - 1) / 2 + (bi - bj));
        float *ptr = blk + (int64_t)boffc * 128 + q * 32 + lane;
#pragma unroll
        for (int xx = 0; xx < 64; xx++) __stcs(ptr + xx * 128, __uint_as_float(r[xx]));
        return;
    }
    // S(i, j) lives at S + col(j) + i, with col(j) = j*lds (full) or
    // j*m - j(j+1)/2 (packed; consecutive columns are m-1-j apart)
    const bool packed = layout == 1;
    float *ptr = S + (packed ? j0 * m - j0 * (j0 + 1) / 2 : j0 * lds) + i;
    if (interior) {
        if (packed) {
            int d = (int)(m - 1 - j0);
#pragma unroll
            for (int xx = 0; xx < 64; xx++) {
                __stcs(ptr, __uint_as_float(r[xx]));
                ptr += d;
                --d;
            }
        } else {
#pragma unroll
            for (int xx = 0; xx < 64; xx++) {
                __stcs(ptr, __uint_as_float(r[xx]));
                ptr += lds;
            }
        }
    } else {
        int64_t j = j0;
#pragma unroll
        for (int xx = 0; xx < 64; xx++) {
            if (i < m && j <= i) __stcs(ptr, __uint_as_float(r[xx]));
            ptr += packed ? (m - 1 - j) : lds;
            ++j;
        }
    }
}

// Maps: pieces 1..3 of W21 (mW1..3) and of L21 (mL1..3); pieces beyond P unused.
template <bool kBatch, int P>
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_form_tc(const __grid_constant__ CUtensorMap mW1, const __grid_constant__ CUtensorMap mL1,
              const __grid_constant__ CUtensorMap mW2, const __grid_constant__ CUtensorMap mL2,
              const __grid_constant__ CUtensorMap mW3, const __grid_constant__ CUtensorMap mL3,
              int64_t m_single, const int32_t *__restrict__ nelim_p, float *__restrict__ S_single,
              int64_t lds_single, int layout_single, int32_t *__restrict__ info, int64_t ntiles_batch,
              BatchTab btab, int sched_mode) {
    using C = Cfg<P>;
    constexpr int BN = C::BN, R = C::R, NS = C::Stages;
    const CUtensorMap *mapW[3] = {&mW1, &mW2, &mW3};
    const CUtensorMap *mapL[3] = {&mL1, &mL2, &mL3};
    extern __shared__ unsigned char smraw[];
    __shared__ Bars bars;
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    uint8_t *sB = smem;                       // [kMaxKB][StageB]: resident L21 block (P <= 2)
    uint8_t *sA = smem + C::ResidentBytes;    // [NS][StageA]: W21 ring (and L21 for P = 3)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e1 = kBatch ? 0 : *nelim_p;
    Sched sc;
    sc.mode = sched_mode;
    sc.nM = kBatch ? 0 : (int)((m_single + kBM - 1) / kBM);
    sc.nN = kBatch ? 0 : col_blocks(sc.nM, R);
    sc.ntiles = kBatch ? ntiles_batch : tile_count(sc.nM, R);
    sc.G = gridDim.x;
    sc.c = blockIdx.x;
    sc.t0 = sc.ntiles * sc.c / sc.G;
    sc.t1 = sc.ntiles * (sc.c + 1) / sc.G;
#define TILE_K(k, x) tile_k<kBatch, R>((k), sc, e1, m_single, S_single, lds_single, layout_single, btab, (x))

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++) {
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
        tmem_alloc(&bars.tmem_base, C::TmemCols);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars.tmem_base;
    const uint32_t idesc = idesc_bf16(kBM, BN);
    const uint32_t idesc_w = idesc_bf16(kBM, 256);

    if (warp == 0) {
        // ---------------- TMA producer: the L21 block of the current column block
        // stays resident while consecutive tiles share it; W21 blocks stream
        if (lane == 0) {
            int stage = 0, cur_key = -1;
            uint32_t phase = 0, bphase = 0;
            TileInfo x;
            for (int64_t k = 0; TILE_K(k, x); k++) {
                if (x.KB == 0) continue;
                bool ok = true;
                if (C::kResident && x.key != cur_key) {
                    if (!mbar_wait(&bars.bempty, bphase ^ 1u, &bars.abort)) {
                        atomicExch(&bars.abort, 1);
                        break;
                    }
                    mbar_expect_tx(&bars.bfull, (uint32_t)x.KB * C::StageB);
                    for (int kb = 0; kb < x.KB; kb++) {
                        uint8_t *dst = sB + (size_t)kb * C::StageB;
#pragma unroll
                        for (int pc = 0; pc < P; pc++)
                            tma_load_2d(dst + pc * C::PieceB, mapL[pc], kb * kBK, (int)x.brow, &bars.bfull);
                    }
                    bphase ^= 1u;
                    cur_key = x.key;
                }
                for (int kb = 0; kb < x.KB; kb++) {
                    if (!mbar_wait(&bars.empty[stage], phase ^ 1u, &bars.abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&bars.full[stage], C::StageA);
                    uint8_t *dst = sA + (size_t)stage * C::StageA;
#pragma unroll
                    for (int pc = 0; pc < P; pc++)
                        tma_load_2d(dst + pc * C::PieceA, mapW[pc], kb * kBK, (int)x.arow, &bars.full[stage]);
                    if (!C::kResident) {
#pragma unroll
                        for (int pc = 0; pc < P; pc++)
                            tma_load_2d(dst + P * C::PieceA + pc * C::PieceB, mapL[pc], kb * kBK, (int)x.brow,
                                        &bars.full[stage]);
                    }
                    if (++stage == NS) {
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
            TileInfo x;
            for (int64_t k = 0; TILE_K(k, x); k++) {
                if (!mbar_wait(&bars.acc_empty[acc], accphase ^ 1u, &bars.abort)) {
                    atomicExch(&bars.abort, 1);
                    break;
                }
                tc_fence_after();
                bool ok = true;
                if (C::kResident && x.KB > 0 && x.key != cur_key) {
                    if (!mbar_wait(&bars.bfull, bphase, &bars.abort)) {
                        atomicExch(&bars.abort, 1);
                        break;
                    }
                    tc_fence_after();
                    bphase ^= 1u;
                    cur_key = x.key;
                }
                const uint32_t dt = tmem + (uint32_t)(acc * C::AccN);
                for (int kb = 0; kb < x.KB; kb++) {
                    if (!mbar_wait(&bars.full[stage], phase, &bars.abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + (size_t)stage * C::StageA);
                    const uint32_t b0 = C::kResident ? smem_u32(sB + (size_t)kb * C::StageB)
                                                     : a0 + P * C::PieceA;
                    // the operands are zero past column e: the last block runs only
                    // the K-steps that reach below e
                    const int nkk = kb == x.KB - 1 ? x.klast : kBK / kUmmaK;
#pragma unroll
                    for (int kk = 0; kk < kBK / kUmmaK; kk++) {
                        if (kk >= nkk) break;
                        // advance 16 BF16 = 32 bytes along K inside the swizzled rows;
                        // products of pieces i, j with i + j <= P - 1.  Split forms:
                        // B pieces 0 and 1 side by side as one N = 256 operand, so
                        //   P = 2: [hi*hi | hi*lo] + lo*hi into the first half;
                        //   P = 3: [hi*hi | hi*mid] + [mid*hi | mid*mid], then
                        //          hi*lo and lo*hi into the first half.
                        const uint64_t a1 = sdesc(a0 + kk * 32), b1 = sdesc(b0 + kk * 32);
                        const uint32_t first = (kb > 0 || kk > 0) ? 1u : 0u;
                        if (P == 1) {
                            umma_bf16(dt, a1, b1, idesc, first);
                        } else {
                            const uint64_t a2 = sdesc(a0 + C::PieceA + kk * 32);
                            umma_bf16(dt, a1, b1, idesc_w, first);
                            if (P == 2) {
                                umma_bf16(dt, a2, b1, idesc, 1u);
                            } else {
                                umma_bf16(dt, a2, b1, idesc_w, 1u);
                                umma_bf16(dt, a1, sdesc(b0 + 2 * C::PieceB + kk * 32), idesc, 1u);
                                umma_bf16(dt, sdesc(a0 + 2 * C::PieceA + kk * 32), b1, idesc, 1u);
                            }
                        }
                    }
                    umma_commit(&bars.empty[stage]);  // W21 stage free once these MMAs finish
                    if (++stage == NS) {
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
                if (C::kResident && x.KB > 0) {
                    int next_key = -2;
                    TileInfo y;
                    for (int64_t kn = k + 1; TILE_K(kn, y); kn++) {
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
        const int half = (warp - 2) >> 2;   // which half of the tile's columns
        int acc = 0;
        uint32_t accphase = 0;
        TileInfo x;
        for (int64_t k = 0; TILE_K(k, x); k++) {
            const int ti = x.ti, tj = x.tj, KB = x.KB, layout = x.layout;
            const int64_t m = x.m, nb = x.nb, lds = x.lds;
            float *S = x.S;
            if (!mbar_wait(&bars.acc_full[acc], accphase, &bars.abort)) {
                if (lane == 0) atomicExch(&bars.abort, 1);
                break;
            }
            tc_fence_after();
            const int64_t i = (int64_t)ti * kBM + q * 32 + lane;
            const int64_t jbase = (int64_t)tj * BN + half * (BN / 2);
            // tiles strictly below the diagonal and inside S need no masking
            const bool interior = (jbase + BN / 2 - 1 < (int64_t)ti * kBM) && ((int64_t)ti * kBM + kBM <= m);
            // block layout: these columns belong to block (ti, bj) of S, from
            // column boff of the block on; blocks above the diagonal are not part of S
            const int64_t bj = jbase / 128;
            const int boff = (int)(jbase % 128);
            const bool tiled = layout == 2;
            if (tiled && bj > ti) goto next_tile_half;
#pragma unroll 1
            for (int c = 0; c < BN / 64; c += 2) {
                uint32_t r[64];
                const uint32_t taddr =
                    tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * C::AccN + half * (BN / 2) + c * 32);
                tmem_ld32_nowait(taddr, *reinterpret_cast<uint32_t(*)[32]>(&r[0]));
                tmem_ld32_nowait(taddr + 32, *reinterpret_cast<uint32_t(*)[32]>(&r[32]));
                tmem_wait_ld();
                if (P > 1) {  // the accumulator's second half holds the other products
#pragma unroll
                    for (int hh = 0; hh < 64; hh += 32) {
                        uint32_t t2[32];
                        tmem_ld32_nowait(taddr + 128 + hh, t2);
                        tmem_wait_ld();
#pragma unroll
                        for (int xx = 0; xx < 32; xx++)
                            r[hh + xx] = __float_as_uint(__uint_as_float(r[hh + xx]) + __uint_as_float(t2[xx]));
                    }
                }
                if (KB == 0) {
#pragma unroll
                    for (int xx = 0; xx < 64; xx++) r[xx] = 0u;
                }
                const int64_t j0 = jbase + c * 32;
                store64(r, layout, S, m, lds, nb, i, j0, interior, ti, bj, boff + c * 32, q, lane);
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
#undef TILE_K
    __syncthreads();
    if (threadIdx.x == 0 && bars.abort) atomicCAS(info, kInfoOk, (int32_t)CTP_ETIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TmemCols);
    }
}

// ---------------------------------------------------------------------------
// Split BF16 with two pieces (hi, lo) on pairs of SMs (cta_group::2): each
// pair computes 256 x 256 tiles of S.  CTA r of the pair holds the W21 rows
// and the L21 rows (the A and the B half of the MMA) of its 128 rows and its
// 128 of the tile's 256 columns; one thread of CTA 0 issues M=256, N=256,
// K=16 MMAs, hi*hi, hi*lo and lo*hi into one accumulator, and each CTA's
// tensor memory receives its 128 rows of the tile.  Against the one-SM kernel
// every SM reads half of B per product and the W21 tile it streams serves 256
// columns instead of 128, so the operands' shared-memory and L2 traffic per
// product halves.
// Protocol: CTA 1's copies complete on its own barriers and a relay thread
// (warp 1 of CTA 1) passes each completion on to CTA 0's barrier (2 arrivals);
// MMA completions are multicast to both CTAs' barriers; CTA 1's epilogue warps
// arrive on CTA 0's accumulator barriers remotely.  Every wait is bounded; a
// timeout raises the abort flag of both CTAs.
struct PairBars {
    unsigned long long full[Cfg<2>::Stages], empty[Cfg<2>::Stages], acc_full[2], acc_empty[2], bfull, bempty, drain;
    uint32_t tmem_base;
    int abort;
};

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreadsTC, 1)
    k_form_tc_pair(const __grid_constant__ CUtensorMap mW1, const __grid_constant__ CUtensorMap mL1,
                   const __grid_constant__ CUtensorMap mW2, const __grid_constant__ CUtensorMap mL2, int64_t m,
                   const int32_t *__restrict__ nelim_p, float *__restrict__ S, int64_t lds, int layout,
                   int32_t *__restrict__ info, int sched_mode) {
    using C = Cfg<2>;
    constexpr int NS = C::Stages;
    constexpr uint32_t kAccCols = 256;
    const CUtensorMap *mapW[2] = {&mW1, &mW2};
    const CUtensorMap *mapL[2] = {&mL1, &mL2};
    extern __shared__ unsigned char smraw[];
    __shared__ PairBars bars;
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    uint8_t *sB = smem;                     // [kMaxKB][StageB]: this CTA's 128 L21 rows, hi and lo
    uint8_t *sA = smem + C::ResidentBytes;  // [NS][StageA]: this CTA's 128 W21 rows, hi and lo
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int e1 = *nelim_p;
    const int nM2 = (int)((m + 255) / 256);  // 256-row blocks
    const int64_t nb128 = (m + kBM - 1) / kBM;
    Sched sc;
    sc.mode = sched_mode;
    sc.nM = nM2;
    sc.nN = nM2;
    sc.ntiles = tile_count(nM2, 1);
    sc.G = gridDim.x >> 1;
    sc.c = blockIdx.x >> 1;
    sc.t0 = sc.ntiles * sc.c / sc.G;
    sc.t1 = sc.ntiles * (sc.c + 1) / sc.G;
    const BatchTab none = {nullptr, nullptr, nullptr, 0, nullptr};
#define TILE_P(k, x) tile_k<false, 1>((k), sc, e1, m, S, lds, layout, none, (x))
    auto raise_abort = [&]() {
        atomicExch(&bars.abort, 1);
        st_remote_u32(peer_addr(&bars.abort, rank ^ 1u), 1u);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(&bars.full[s], rank == 0 ? 2 : 1);  // CTA 0: its copies + CTA 1's relay
            mbar_init(&bars.empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bars.acc_full[b], 1);
            mbar_init(&bars.acc_empty[b], 2 * kEpiWarps);  // both CTAs' epilogue warps (used in CTA 0)
        }
        mbar_init(&bars.bfull, rank == 0 ? 2 : 1);
        mbar_init(&bars.bempty, 1);
        mbar_init(&bars.drain, 1);
        bars.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    cluster_sync_all();  // both CTAs' barriers exist before any remote arrival
    if (warp == 0) tmem_alloc_pair(&bars.tmem_base, 2 * kAccCols);
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = bars.tmem_base;

    if (warp == 0) {
        // ---------------- TMA producer (both CTAs): this CTA's L21 half of the
        // column block stays resident; its W21 rows stream through the ring
        if (lane == 0) {
            int stage = 0, cur_key = -1;
            uint32_t phase = 0, bphase = 0;
            TileInfo x;
            for (int64_t k = 0; TILE_P(k, x); k++) {
                if (x.KB == 0) continue;
                const int arow = x.ti * 256 + 128 * (int)rank, brow = x.tj * 256 + 128 * (int)rank;
                if (x.key != cur_key) {
                    if (!mbar_wait(&bars.bempty, bphase ^ 1u, &bars.abort)) {
                        raise_abort();
                        break;
                    }
                    mbar_expect_tx(&bars.bfull, (uint32_t)x.KB * C::StageB);
                    for (int kb = 0; kb < x.KB; kb++)
#pragma unroll
                        for (int pc = 0; pc < 2; pc++)
                            tma_load_2d(sB + (size_t)kb * C::StageB + pc * C::PieceB, mapL[pc], kb * kBK, brow,
                                        &bars.bfull);
                    bphase ^= 1u;
                    cur_key = x.key;
                }
                bool ok = true;
                for (int kb = 0; kb < x.KB; kb++) {
                    if (!mbar_wait(&bars.empty[stage], phase ^ 1u, &bars.abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&bars.full[stage], C::StageA);
#pragma unroll
                    for (int pc = 0; pc < 2; pc++)
                        tma_load_2d(sA + (size_t)stage * C::StageA + pc * C::PieceA, mapW[pc], kb * kBK, arow,
                                    &bars.full[stage]);
                    if (++stage == NS) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) {
                    raise_abort();
                    break;
                }
            }
        }
    } else if (warp == 1 && rank == 1) {
        // ---------------- relay (CTA 1): pass each of this CTA's completed
        // copies on to CTA 0's barrier, in the MMA's order
        if (lane == 0) {
            int stage = 0, cur_key = -1;
            uint32_t phase = 0, bphase = 0;
            const uint32_t rb = peer_addr(&bars.bfull, 0);
            TileInfo x;
            for (int64_t k = 0; TILE_P(k, x); k++) {
                if (x.KB == 0) continue;
                bool ok = true;
                if (x.key != cur_key) {
                    if (!mbar_wait(&bars.bfull, bphase, &bars.abort)) {
                        raise_abort();
                        break;
                    }
                    mbar_arrive_remote(rb);
                    bphase ^= 1u;
                    cur_key = x.key;
                }
                for (int kb = 0; kb < x.KB; kb++) {
                    if (!mbar_wait(&bars.full[stage], phase, &bars.abort)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_remote(peer_addr(&bars.full[stage], 0));
                    if (++stage == NS) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) {
                    raise_abort();
                    break;
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (CTA 0)
        if (lane == 0) {
            int stage = 0, acc = 0, cur_key = -1;
            uint32_t phase = 0, accphase = 0, bphase = 0;
            const uint32_t idesc = idesc_bf16(256, 256);
            TileInfo x;
            for (int64_t k = 0; TILE_P(k, x); k++) {
                if (!mbar_wait_cl(&bars.acc_empty[acc], accphase ^ 1u, &bars.abort)) {
                    raise_abort();
                    break;
                }
                tc_fence_after();
                if (x.KB > 0 && x.key != cur_key) {
                    if (!mbar_wait_cl(&bars.bfull, bphase, &bars.abort)) {
                        raise_abort();
                        break;
                    }
                    tc_fence_after();
                    bphase ^= 1u;
                    cur_key = x.key;
                }
                const uint32_t dt = tmem + (uint32_t)(acc * kAccCols);
                bool ok = true;
                for (int kb = 0; kb < x.KB; kb++) {
                    if (!mbar_wait_cl(&bars.full[stage], phase, &bars.abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + (size_t)stage * C::StageA);
                    const uint32_t b0 = smem_u32(sB + (size_t)kb * C::StageB);
                    const int nkk = kb == x.KB - 1 ? x.klast : kBK / kUmmaK;  // zero past column e
#pragma unroll
                    for (int kk = 0; kk < kBK / kUmmaK; kk++) {
                        if (kk >= nkk) break;
                        const uint64_t ah = sdesc(a0 + kk * 32), al = sdesc(a0 + C::PieceA + kk * 32);
                        const uint64_t bh = sdesc(b0 + kk * 32), bl = sdesc(b0 + C::PieceB + kk * 32);
                        umma_bf16_pair(dt, ah, bh, idesc, (kb > 0 || kk > 0) ? 1u : 0u);  // hi*hi
                        umma_bf16_pair(dt, ah, bl, idesc, 1u);                            // hi*lo
                        umma_bf16_pair(dt, al, bh, idesc, 1u);                            // lo*hi
                    }
                    umma_commit_pair(&bars.empty[stage], (uint16_t)0x3);  // both CTAs' stage free
                    if (++stage == NS) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) {
                    raise_abort();
                    break;
                }
                umma_commit_pair(&bars.acc_full[acc], (uint16_t)0x3);  // both halves of the tile ready
                if (x.KB > 0) {
                    int next_key = -2;
                    TileInfo y;
                    for (int64_t kn = k + 1; TILE_P(kn, y); kn++) {
                        if (y.KB > 0) {
                            next_key = y.key;
                            break;
                        }
                    }
                    if (next_key != x.key) umma_commit_pair(&bars.bempty, (uint16_t)0x3);
                }
                if (++acc == 2) {
                    acc = 0;
                    accphase ^= 1u;
                }
            }
            // every MMA issued has completed before the pair tears down
            umma_commit_pair(&bars.drain, (uint16_t)0x1);
            int never = 0;
            mbar_wait(&bars.drain, 0, &never);
        }
    } else {
        // ---------------- epilogue: warps 2..9 of both CTAs, this CTA's 128 rows
        const int q = warp & 3;            // TMEM lane quarter this warp may access
        const int half = (warp - 2) >> 2;  // which 128 of the tile's 256 columns
        const uint32_t ae0 = peer_addr(&bars.acc_empty[0], 0), ae1 = peer_addr(&bars.acc_empty[1], 0);
        int acc = 0;
        uint32_t accphase = 0;
        TileInfo x;
        for (int64_t k = 0; TILE_P(k, x); k++) {
            if (!mbar_wait_cl(&bars.acc_full[acc], accphase, &bars.abort)) {
                if (lane == 0) raise_abort();
                break;
            }
            tc_fence_after();
            const int64_t rbase = (int64_t)x.ti * 256 + 128 * rank;  // this CTA's first row
            const int64_t i = rbase + q * 32 + lane;
            const int64_t jbase = (int64_t)x.tj * 256 + half * 128;
            const bool interior = (jbase + 127 < rbase) && (rbase + kBM <= m);
            const int64_t bi = rbase / 128, bj = jbase / 128;
            if (!(layout == 2 && bj > bi) && rbase < m) {
#pragma unroll 1
                for (int c = 0; c < 4; c += 2) {
                    uint32_t r[64];
                    const uint32_t taddr =
                        tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kAccCols + half * 128 + c * 32);
                    tmem_ld32_nowait(taddr, *reinterpret_cast<uint32_t(*)[32]>(&r[0]));
                    tmem_ld32_nowait(taddr + 32, *reinterpret_cast<uint32_t(*)[32]>(&r[32]));
                    tmem_wait_ld();
                    if (x.KB == 0) {
#pragma unroll
                        for (int xx = 0; xx < 64; xx++) r[xx] = 0u;
                    }
                    store64(r, layout, S, m, lds, nb128, i, jbase + c * 32, interior, bi, bj, c * 32, q, lane);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (rank == 0)
                    mbar_arrive(&bars.acc_empty[acc]);
                else
                    mbar_arrive_remote(acc == 0 ? ae0 : ae1);
            }
            if (++acc == 2) {
                acc = 0;
                accphase ^= 1u;
            }
        }
    }
#undef TILE_P
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // no remote access into either CTA from here on
    if (threadIdx.x == 0 && bars.abort) atomicCAS(info, kInfoOk, (int32_t)CTP_ETIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 2 * kAccCols);
    }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tc::encode_fn() {
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

bool tc::make_map_bf16(CUtensorMap *map, const void *base, int64_t rows, int Kp, int box_rows) {
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

int form_tc_kpad(int p) { return (p + kBK - 1) / kBK * kBK; }

namespace {
template <bool kBatch, int P>
cudaError_t set_smem(size_t smem) {
    return smem_at_least((const void *)k_form_tc<kBatch, P>, smem);
}
constexpr size_t kSmemTC = kSmemBody + 1024;

int bn_of(int P) { return P == 1 ? Cfg<1>::BN : (P == 2 ? Cfg<2>::BN : Cfg<3>::BN); }

// Tensor maps of the P pieces of both operands (pieces `off` elements apart).
bool make_maps(CUtensorMap (&mW)[3], CUtensorMap (&mL)[3], const void *Wb, const void *Lb, int64_t off, int P,
               int64_t rows, int Kp) {
    for (int pc = 0; pc < 3; pc++) {
        const int q = pc < P ? pc : 0;  // unused pieces: valid copies of the first
        const char *w = (const char *)Wb + 2 * off * q, *l = (const char *)Lb + 2 * off * q;
        if ((((uintptr_t)w) | ((uintptr_t)l)) & 15) return false;
        if (!make_map_bf16(&mW[pc], w, rows, Kp, kBM) || !make_map_bf16(&mL[pc], l, rows, Kp, bn_of(P))) return false;
    }
    return true;
}

template <bool kBatch, int P>
cudaError_t launch_p(int grid, const CUtensorMap (&mW)[3], const CUtensorMap (&mL)[3], int64_t m,
                     const int32_t *nelim, float *S, int64_t lds, int layout, int32_t *info, int64_t items,
                     const BatchTab &bt, int mode, cudaStream_t st) {
    cudaError_t err = set_smem<kBatch, P>(kSmemTC);
    if (err != cudaSuccess) return err;
    k_form_tc<kBatch, P><<<grid, kThreadsTC, kSmemTC, st>>>(mW[0], mL[0], mW[1], mL[1], mW[2], mL[2], m, nelim, S,
                                                             lds, layout, info, items, bt, mode);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_form_tc(const void *Wb, const void *Lb, int64_t piece_off, int pieces, int64_t m, int Kp,
                           const int32_t *nelim, float *S, int64_t lds, int layout, int32_t *info,
                           int num_sms, int walk, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    if (pieces < 1 || pieces > 3) return cudaErrorInvalidValue;
    CUtensorMap mW[3], mL[3];
    if (!make_maps(mW, mL, Wb, Lb, piece_off, pieces, m, Kp)) return cudaErrorInvalidValue;
    const int R = bn_of(pieces) / kBM;
    const int nM = (int)((m + kBM - 1) / kBM);
    const int64_t ntiles = tile_count(nM, R), nN = col_blocks(nM, R);
    // walk: CTP_WALK_AUTO picks panels when the split operands (two or three
    // times the bytes) need the L2-friendly walk, contiguous runs otherwise
    int mode;
    if (walk == CTP_WALK_ROUND_ROBIN)
        mode = 0;
    else if (walk == CTP_WALK_CHUNKS)
        mode = 2;
    else if (walk == CTP_WALK_PANELS)
        mode = nN >= (int64_t)num_sms ? 1 : 2;
    else
        mode = (pieces > 1 && nN >= 2 * (int64_t)num_sms) ? 1 : 2;
    if (pieces == 2 && m > kBM && num_sms >= 2) {
        // two pieces: 256 x 256 tiles on pairs of SMs
        const int nM2 = (int)((m + 255) / 256);
        const int64_t nt2 = tile_count(nM2, 1);
        int64_t pairs = num_sms / 2;
        if (pairs > nt2) pairs = nt2;
        int mode2 = mode;
        if (mode2 == 1 && nM2 < pairs) mode2 = 2;  // panels need a column block per pair
        cudaError_t err = smem_at_least((const void *)k_form_tc_pair, kSmemTC);
        if (err != cudaSuccess) return err;
        k_form_tc_pair<<<(unsigned)(2 * pairs), kThreadsTC, kSmemTC, st>>>(mW[0], mL[0], mW[1], mL[1], m, nelim, S,
                                                                          lds, layout, info, mode2);
        return cudaGetLastError();
    }
    const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
    BatchTab none = {nullptr, nullptr, nullptr, 0, nullptr};
    if (pieces == 1) return launch_p<false, 1>(grid, mW, mL, m, nelim, S, lds, layout, info, 0, none, mode, st);
    if (pieces == 2) return launch_p<false, 2>(grid, mW, mL, m, nelim, S, lds, layout, info, 0, none, mode, st);
    return launch_p<false, 3>(grid, mW, mL, m, nelim, S, lds, layout, info, 0, none, mode, st);
}

int64_t form_tc_tiles(int64_t m, int pieces) {
    const int R = bn_of(pieces) / kBM;
    return m > 0 ? tile_count((m + kBM - 1) / kBM, R) : 0;
}

cudaError_t launch_form_tc_batch(const ctp_front *fronts, const BFront *tab, const int *item_front,
                                 int64_t items, int64_t total_rows, const void *Wb, const void *Lb,
                                 int pieces, int layout, int32_t *info, int num_sms, cudaStream_t st,
                                 const int *item_tile) {
    if (items == 0) return cudaSuccess;
    if (pieces < 1 || pieces > 3) return cudaErrorInvalidValue;
    CUtensorMap mW[3], mL[3];
    if (!make_maps(mW, mL, Wb, Lb, total_rows * kBatchKp, pieces, total_rows, kBatchKp))
        return cudaErrorInvalidValue;
    const int grid = (int)(items < num_sms ? items : num_sms);
    BatchTab bt = {fronts, tab, item_front, layout, item_tile};
    if (pieces == 1) return launch_p<true, 1>(grid, mW, mL, 0, nullptr, nullptr, 0, 2, info, items, bt, 2, st);
    if (pieces == 2) return launch_p<true, 2>(grid, mW, mL, 0, nullptr, nullptr, 0, 2, info, items, bt, 2, st);
    return launch_p<true, 3>(grid, mW, mL, 0, nullptr, nullptr, 0, 2, info, items, bt, 2, st);
}

}  // namespace ctp
