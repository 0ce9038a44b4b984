// solve_tc.cu -- K5 on the tensor cores: the Solve task L21 = A21 P^T (D11 L11^T)^{-1}
// (Section 1 task list; Figure 4.1 (d),(e)) and the update of the delayed
// columns, as one GEMM per supernode with split-BF16 operands and FP32
// accumulation (tcgen05), for the mixed-precision factorizations.
//
// With x = A21(i, perm) the permuted row of A21, x_e its e eliminated and x_d its
// d = p - e delayed positions, the FP64 Solve computes
//   Y = x_e U,  U = L11^{-T}  (unit upper),   L21 = Y D11^{-1},   x_d' = x_d - Y L_d^T,
// all of which are linear in x_e.  So one product x_e Z gives every output:
//   Z = [ U D11^{-1} | U | -U L_d^T ]        (e x (e + e + d))
// -- L21 (written to A21 in FP64 and as the Form's BF16 operand pieces), Y = W21
// (the Form's other operand) and the correction added to x_d.  The three
// blocks start at output columns 0, E and 2E with E = e rounded up to 32 (the
// columns between are zero), so a 32-column slice of the accumulator lies in
// one block and its BF16 pieces go out as 16-byte stores.  Z is the
// substitution applied to the identity rows e_k, k < e: the prep kernel runs
// exactly the FP64 Solve's recurrence on them.
//
// Kernels:
//   k_stc_prep    Z^T in BF16 pieces (K-major: row o of the operand is output
//                 column o; 640 rows, zero past 2E + d), from the factored
//                 A11 block in FP64;
//   k_stc_gather  per 32-row tile: x gathered through the permutation, x_e
//                 written as BF16 pieces (row-major, K contiguous, zero past
//                 e), x_d written back in place in FP64 at the delayed
//                 positions (all reads of a tile precede its writes; tiles own
//                 disjoint rows), and the Form operands' tails past e zeroed;
//   k_solve_tc<PS> persistent GEMM x_e Z: 128-row blocks of x_e times
//                 128-column windows of Z, K = e.  Warp 0: TMA of 128B-swizzled
//                 K-blocks of both operands through a ring; warp 1: tcgen05.mma
//                 of the split products (PS pieces: products of total order
//                 <= PS - 1) into two TMEM accumulators; warps 2-9: epilogue
//                 (L21 in FP64 into A21 and its BF16 pieces, Y's BF16 pieces,
//                 x_d += correction in FP64).
// The products carry the split's error (PS = 2: about 2^-16 relative to
// |x_e||Z|; PS = 3, what the library uses: close to FP32), which FP64
// iterative refinement on the complete system removes; pivots are unaffected
// (they are chosen before).
// Every mbarrier wait is bounded; on timeout the kernel records CTP_ETIMEOUT,
// stops, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "ctp_internal.cuh"
#include "tc_common.cuh"

namespace ctp {

using namespace tc;

namespace {

constexpr int kRowsG = 32;  // rows per gather / prep tile (one per lane)
constexpr int kWarpsG = 8;
constexpr int kBM = 128, kBN = 128;  // GEMM tile: 128 rows of x_e by 128 output columns
constexpr int kZRows = 640;          // rows of the Z^T operand (2 E + d <= p + e + 62 < 640)
constexpr int kEpiWarps = 8;
constexpr int kThreadsTC = 32 * (2 + kEpiWarps);
constexpr uint32_t kPiece = kBM * kBK * 2;  // one 128 x 64 BF16 block (16 KB), both operands
constexpr size_t kSmemRing = 192 * 1024;

// BF16 pieces of v: piece k is the BF16 rounding (through FP32) of what pieces
// 0..k-1 left, and that remainder is kept exactly in FP64 (v minus a BF16 value
// within 2^-8 of it is exact), so three pieces hold v to about 2^-26.  (Rounding
// v to FP32 first would cost 2^-24, which the Solve's cancellation amplifies:
// measured as slower refinement.)
// A BF16 value as a double, built from its bits (no FP64 operation) when it is
// normal; zero, subnormal, Inf and NaN take the conversion.
__device__ __forceinline__ double bf16_as_double(__nv_bfloat16 b) {
    const unsigned int h = __bfloat16_as_ushort(b);
    const unsigned int ex = (h >> 7) & 0xFFu;
    if (ex == 0u || ex == 0xFFu) return (double)__bfloat162float(b);
    const unsigned long long bits = ((unsigned long long)(h >> 15) << 63) |
                                    ((unsigned long long)(ex - 127u + 1023u) << 52) |
                                    ((unsigned long long)(h & 0x7Fu) << 45);
    return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ void put_pieces(__nv_bfloat16 *dst, int64_t piece_off, int pieces, double v) {
    double r = v;
    for (int pc = 0; pc < pieces; pc++) {
        const __nv_bfloat16 b = __float2bfloat16_rn((float)r);
        dst[pc * piece_off] = b;
        if (pc + 1 < pieces) r -= bf16_as_double(b);
    }
}

// 32 consecutive FP32 values of one row as BF16 pieces (16-byte stores; dst
// 16-byte aligned), each piece rounding what the earlier ones left (exact in
// FP32: a float minus its BF16 rounding is a float).
__device__ __forceinline__ void put_pieces32(__nv_bfloat16 *dst, int64_t piece_off, int pieces, const uint32_t (&r)[32]) {
    float cur[32];
#pragma unroll
    for (int x = 0; x < 32; x++) cur[x] = __uint_as_float(r[x]);
    for (int pc = 0; pc < pieces; pc++) {
        uint32_t pk[16];
#pragma unroll
        for (int x = 0; x < 16; x++) {
            const __nv_bfloat16 b0 = __float2bfloat16_rn(cur[2 * x]), b1 = __float2bfloat16_rn(cur[2 * x + 1]);
            cur[2 * x] -= __bfloat162float(b0);
            cur[2 * x + 1] -= __bfloat162float(b1);
            pk[x] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
        }
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + pc * piece_off);
#pragma unroll
        for (int x = 0; x < 4; x++) d4[x] = make_uint4(pk[4 * x], pk[4 * x + 1], pk[4 * x + 2], pk[4 * x + 3]);
    }
}

// L21 entry at position o of a row y (positions contiguous) from its Y entries
// (D11^{-1} by blocks).
__device__ __forceinline__ double l21_of(const double *y, int o, const int32_t *piv,
                                         const double *__restrict__ Dinv) {
    const int kd = piv[o];
    if (kd == CTP_PIVKIND_1X1) return y[o] * Dinv[2 * o];
    if (kd == CTP_PIVKIND_2X2_FIRST) return y[o] * Dinv[2 * o] + y[o + 1] * Dinv[2 * o + 1];
    if (kd == CTP_PIVKIND_2X2_SECOND) return y[o - 1] * Dinv[2 * (o - 1) + 1] + y[o] * Dinv[2 * o];
    return 0.0;  // zero pivot
}

constexpr int kPrepRows = 1;  // identity rows (warps) per CTA: one, so the rows spread over the SMs' FP64 pipes

// Z^T pieces: Zt[o * Kp + k] for output column o < kZRows, K index k < Kp.
// One warp per identity row k (a CTA per row): the row lives in shared memory, each
// position updated by one lane, and the warp runs the FP64 Solve's recurrence
// with only warp barriers (row k is zero before position k, so its pivots
// start at k's block).  The CTA then writes the Z^T column of its row.
__global__ void __launch_bounds__(32 * kPrepRows)
    k_stc_prep(const double *__restrict__ A, int p, int64_t lda, const int32_t *__restrict__ piv,
               const double *__restrict__ Dinv, const int32_t *__restrict__ nelim_p, __nv_bfloat16 *__restrict__ Zt,
               int Kp, int64_t zoff, int pieces) {
    __shared__ double rows[kPrepRows][kMaxP];
    const int e = *nelim_p;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k0 = blockIdx.x * kPrepRows, k = k0 + w;
    __shared__ int spiv[kMaxP];
    double *x = rows[w];  // this warp's row; position q is updated by lane q % 32 only
    for (int q = threadIdx.x; q < p; q += blockDim.x) spiv[q] = piv[q];
    for (int q = lane; q < kMaxP; q += 32) x[q] = (q == k && k < e) ? 1.0 : 0.0;
    __syncthreads();
    if (k < e) {
        int j = (k > 0 && spiv[k] == CTP_PIVKIND_2X2_SECOND) ? k - 1 : k;
        while (j < e) {
            const int kd = spiv[j];
            const double y0 = x[j];
            // all of a lane's positions at once (predicated), so that the loads
            // of the L column(s) are in flight together
            if (kd == CTP_PIVKIND_2X2_FIRST) {
                const double y1 = x[j + 1];
                const double *l0 = A + (int64_t)j * lda, *l1 = A + (int64_t)(j + 1) * lda;
#pragma unroll
                for (int s2 = 0; s2 < kMaxP / 32; s2++) {
                    const int q = lane + 32 * s2;
                    if (q >= j + 2 && q < p) x[q] -= y0 * __ldg(l0 + q) + y1 * __ldg(l1 + q);
                }
                j += 2;
            } else {
                if (kd == CTP_PIVKIND_1X1) {
                    const double *l0 = A + (int64_t)j * lda;
#pragma unroll
                    for (int s2 = 0; s2 < kMaxP / 32; s2++) {
                        const int q = lane + 32 * s2;
                        if (q > j && q < p) x[q] -= y0 * __ldg(l0 + q);
                    }
                }
                j += 1;  // zero pivots have an all-zero L column
            }
            __syncwarp();  // the next pivot's y is written by another lane
        }
    }
    __syncthreads();
    // Z^T columns of these rows: thread (o, r) writes Zt[o * Kp + k0 + r]
    const int d = p - e, E = (e + 31) & ~31;
    for (int idx = threadIdx.x; idx < kZRows * kPrepRows; idx += blockDim.x) {
        const int o = idx / kPrepRows, r = idx % kPrepRows, kr = k0 + r;
        if (kr >= Kp) continue;
        const double *y = rows[r];
        double v = 0.0;
        if (kr < e) {
            if (o < e)
                v = l21_of(y, o, spiv, Dinv);
            else if (o >= E && o < E + e)
                v = y[o - E];
            else if (o >= 2 * E && o < 2 * E + d)
                v = y[e + o - 2 * E];  // -(U L_d^T)[k, o - 2E]
        }
        put_pieces(Zt + (int64_t)o * Kp + kr, zoff, pieces, v);
    }
}

// Gather of x through perm; x_e to BF16 pieces, x_d back in place (FP64), and
// the zero tails (K >= e) of the Form's operand pieces.
__global__ void __launch_bounds__(kRowsG * kWarpsG)
    k_stc_gather(double *__restrict__ A, int64_t n, int p, int64_t lda, const int32_t *__restrict__ perm,
                 const int32_t *__restrict__ nelim_p, __nv_bfloat16 *__restrict__ Xb, int64_t xoff, int xpieces,
                 __nv_bfloat16 *__restrict__ Wb, __nv_bfloat16 *__restrict__ Lb, int64_t foff, int fpieces,
                 int Kp) {
    extern __shared__ __align__(16) double xs[];  // [p][kRowsG + 1]
    constexpr int LDX = kRowsG + 1;
    const int e = *nelim_p;
    const int64_t m = n - p;
    const int64_t row0 = (int64_t)blockIdx.x * kRowsG;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t row = row0 + lane;
    const bool valid = row < m;
    double *A21 = A + p;
    for (int k = w; k < p; k += kWarpsG) {
        const int c = perm[k];
        xs[k * LDX + lane] = valid ? A21[(int64_t)c * lda + row] : 0.0;
    }
    __syncthreads();
    // x_e pieces and the Form operands' zero tails: a warp writes one row at a time
    for (int rr = w; rr < kRowsG; rr += kWarpsG) {
        const int64_t rw = row0 + rr;
        if (rw >= m) break;
        for (int k = lane; k < Kp; k += 32) {
            const double v = k < e ? xs[k * LDX + rr] : 0.0;
            put_pieces(Xb + rw * Kp + k, xoff, xpieces, v);
            if (k >= e && Lb != nullptr) {
                put_pieces(Lb + rw * Kp + k, foff, fpieces, 0.0);
                put_pieces(Wb + rw * Kp + k, foff, fpieces, 0.0);
            }
        }
    }
    // x_d at the delayed positions, in place (this tile's rows only)
    if (valid)
        for (int k = e + w; k < p; k += kWarpsG) A21[(int64_t)k * lda + row] = xs[k * LDX + lane];
}

// ---- batched forms: x_e and Z^T of every front in 128 x 64 BF16 tiles (the
// K blocks of a 128-row block, or of a 128-column window, are consecutive
// tiles), three pieces per tile array.
constexpr int64_t kTileElems = (int64_t)kBM * kBK;

// One CTA per group of 8 identity rows of a front (a warp each; the groups of
// a front run in parallel), written to the front's Z^T tiles as 16-byte pieces
// of 8 consecutive K.
__global__ void __launch_bounds__(256)
    k_stc_prep_batch(const ctp_front *__restrict__ fronts, const BFront *__restrict__ tab, char *ws,
                     const int *__restrict__ item_front, BatchOpts o, __nv_bfloat16 *__restrict__ Zt) {
    __shared__ double rows[8][kMaxP];
    __shared__ int spiv[kMaxP];
    const int f = item_front[blockIdx.x];
    const BFront b = tab[f];
    const ctp_front fr = fronts[f];
    if (b.m <= 0) return;
    ctp_options oo;
    oo.pivot = o.pivot;
    oo.smode = o.smode;
    oo.prec = o.prec;
    const double *Dinv = reinterpret_cast<const double *>(ws + b.ws + bsection(b.n, b.p, &oo).Dinv);
    const int p = b.p, e = *fr.nelim;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int d = p - e, E = (e + 31) & ~31;
    const int KZ = (e + kBK - 1) / kBK * kBK;  // K columns the GEMM reads
    const int nW = (2 * E + d + kBN - 1) / kBN;
    for (int q = threadIdx.x; q < p; q += blockDim.x) spiv[q] = fr.piv[q];
    __syncthreads();
    {
        const int k0 = (int)((int64_t)blockIdx.x - b.r0) * 8;
        if (k0 >= KZ) return;
        const int k = k0 + w;
        double *x = rows[w];
        for (int q = lane; q < kMaxP; q += 32) x[q] = (q == k && k < e) ? 1.0 : 0.0;
        __syncwarp();
        if (k < e) {
            int j = (k > 0 && spiv[k] == CTP_PIVKIND_2X2_SECOND) ? k - 1 : k;
            while (j < e) {
                const int kd = spiv[j];
                const double y0 = x[j];
                if (kd == CTP_PIVKIND_2X2_FIRST) {
                    const double y1 = x[j + 1];
                    const double *l0 = fr.A + (int64_t)j * fr.lda, *l1 = fr.A + (int64_t)(j + 1) * fr.lda;
#pragma unroll
                    for (int s2 = 0; s2 < kMaxP / 32; s2++) {
                        const int q = lane + 32 * s2;
                        if (q >= j + 2 && q < p) x[q] -= y0 * __ldg(l0 + q) + y1 * __ldg(l1 + q);
                    }
                    j += 2;
                } else {
                    if (kd == CTP_PIVKIND_1X1) {
                        const double *l0 = fr.A + (int64_t)j * fr.lda;
#pragma unroll
                        for (int s2 = 0; s2 < kMaxP / 32; s2++) {
                            const int q = lane + 32 * s2;
                            if (q > j && q < p) x[q] -= y0 * __ldg(l0 + q);
                        }
                    }
                    j += 1;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // Z^T rows oc of the windows this front uses, K columns k0..k0+7
        for (int oc = threadIdx.x; oc < nW * kBN; oc += blockDim.x) {
            uint32_t pk[3][4];
            for (int h = 0; h < 4; h++) {
                double v2[2];
                for (int r = 0; r < 2; r++) {
                    const int kr = k0 + 2 * h + r;
                    const double *y = rows[2 * h + r];
                    double v = 0.0;
                    if (kr < e) {
                        if (oc < e)
                            v = l21_of(y, oc, spiv, Dinv);
                        else if (oc >= E && oc < E + e)
                            v = y[oc - E];
                        else if (oc >= 2 * E && oc < 2 * E + d)
                            v = y[e + oc - 2 * E];
                    }
                    v2[r] = v;
                }
                // three pieces of the pair, each rounding what the earlier left
                double r0 = v2[0], r1 = v2[1];
                for (int pc = 0; pc < 3; pc++) {
                    const __nv_bfloat16 b0 = __float2bfloat16_rn((float)r0), b1 = __float2bfloat16_rn((float)r1);
                    pk[pc][h] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
                    r0 -= bf16_as_double(b0);
                    r1 -= bf16_as_double(b1);
                }
            }
            const int64_t tile = b.zt0 + (int64_t)(oc / kBN) * b.kbx + k0 / kBK;
            const int64_t el = tile * kTileElems + (int64_t)(oc % kBN) * kBK + (k0 % kBK);
#pragma unroll
            for (int pc = 0; pc < 3; pc++)
                *reinterpret_cast<uint4 *>(Zt + el + pc * o.zoff) = make_uint4(pk[pc][0], pk[pc][1], pk[pc][2], pk[pc][3]);
        }
        __syncthreads();
    }
}

// One CTA per (front, 32-row tile): x gathered through the permutation, x_e
// into the front's x_e tiles (K < e's last 64-wide block), x_d back in place,
// and the Form operands' zero tails from e to that block's end.
__global__ void __launch_bounds__(kRowsG * kWarpsG)
    k_stc_gather_batch(const ctp_front *__restrict__ fronts, const BFront *__restrict__ tab,
                       const int *__restrict__ item_front, BatchOpts o, __nv_bfloat16 *__restrict__ Xt,
                       __nv_bfloat16 *__restrict__ Wb, __nv_bfloat16 *__restrict__ Lb) {
    extern __shared__ __align__(16) double xs[];  // [p][kRowsG + 1]
    constexpr int LDX = kRowsG + 1;
    const int f = item_front[blockIdx.x];
    const BFront b = tab[f];
    const ctp_front fr = fronts[f];
    const int p = b.p, e = *fr.nelim;
    const int64_t m = b.m;
    const int64_t row0 = ((int64_t)blockIdx.x - b.s0) * kRowsG;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t row = row0 + lane;
    const bool valid = row < m;
    double *A21 = fr.A + p;
    for (int k = w; k < p; k += kWarpsG) {
        const int c = fr.perm[k];
        xs[k * LDX + lane] = valid ? A21[(int64_t)c * fr.lda + row] : 0.0;
    }
    __syncthreads();
    const int KZ = (e + kBK - 1) / kBK * kBK;
    for (int rr = w; rr < kRowsG; rr += kWarpsG) {
        const int64_t rw = row0 + rr;
        if (rw >= m) break;
        const int64_t tbase = (b.xt0 + (rw / kBM) * b.kbx) * kTileElems + (rw % kBM) * kBK;
        for (int k = lane; k < KZ; k += 32) {
            const double v = k < e ? xs[k * LDX + rr] : 0.0;
            put_pieces(Xt + tbase + (int64_t)(k / kBK) * kTileElems + (k % kBK), o.xoff, 3, v);
            if (k >= e) {
                put_pieces(Lb + (b.row0 + rw) * kBatchKp + k, o.lo_off, o.pieces, 0.0);
                put_pieces(Wb + (b.row0 + rw) * kBatchKp + k, o.lo_off, o.pieces, 0.0);
            }
        }
    }
    if (valid)
        for (int k = e + w; k < p; k += kWarpsG) A21[(int64_t)k * fr.lda + row] = xs[k * LDX + lane];
}

struct Bars {
    unsigned long long full[6], empty[6], acc_full[2], acc_empty[2];
    uint32_t tmem_base;
    int abort;
};

template <int PS>
struct SCfg {
    static constexpr uint32_t Stage = 2 * PS * kPiece;  // PS pieces of x_e, then PS of Z^T
    static constexpr int Stages = (int)(kSmemRing / Stage) < 6 ? (int)(kSmemRing / Stage) : 6;
};

// What the roles of the GEMM need to know about one tile (128 rows of x_e by
// one 128-column window of Z^T): its front, the TMA rows/columns of its K
// blocks, and where the epilogue writes.
struct STile {
    double *A21;
    int64_t lda, m, i0;  // i0: first row of the tile within the front
    int p, e, E, KB, o0;  // o0: first output column of the window
    __nv_bfloat16 *Lb, *Wb;
    int64_t lrow0;  // the front's first row in the Form's operand buffers
    int Kst;        // their K stride
    int xk, xy, zk, zy, kstep_x, kstep_y;  // TMA coordinates of K block 0, and per K block
};

// Kernel arguments of the single-supernode and the batched GEMM.
struct SArgs {
    // single supernode
    double *A21;
    int64_t m, lda;
    int p;
    const int32_t *nelim;
    int Kp;
    // batch
    const ctp_front *fronts;
    const BFront *tab;
    const int *qitem;
    int64_t q_items;
    // both
    __nv_bfloat16 *Wb, *Lb;
    int64_t foff;
    int fpieces;
    int32_t *info;
};

// Output windows of a front of width p, at most over its possible e.
int windows_for(int p) {
    int w = 1;
    for (int e = 1; e <= p; e++) {
        const int we = (2 * ((e + 31) & ~31) + p - e + kBN - 1) / kBN;
        w = we > w ? we : w;
    }
    return w;
}

// Tiles of this launch: the single supernode's from its e (read on the
// device), the batch's from the plan's item table.
template <bool kBatch>
__device__ __forceinline__ int64_t tile_count(const SArgs &g) {
    if (kBatch) return g.q_items;
    const int e = *g.nelim;
    const int KB = (e + kBK - 1) / kBK;
    const int E = (e + 31) & ~31;
    const int nW = (2 * E + g.p - e + kBN - 1) / kBN;
    return KB > 0 ? ((g.m + kBM - 1) / kBM) * nW : 0;
}

// Tile t, or false when it has no work (a batch window past its front's
// outputs, or a front that eliminated nothing); every role decodes alike.
template <bool kBatch>
__device__ __forceinline__ bool tile_at(int64_t t, const SArgs &g, STile &s) {
    if (!kBatch) {
        const int e = *g.nelim;
        const int E = (e + 31) & ~31;
        const int nW = (2 * E + g.p - e + kBN - 1) / kBN;
        const int rb = (int)(t / nW), w = (int)(t % nW);
        s.A21 = g.A21, s.lda = g.lda, s.m = g.m, s.p = g.p, s.e = e, s.E = E;
        s.KB = (e + kBK - 1) / kBK;
        s.i0 = (int64_t)rb * kBM, s.o0 = w * kBN;
        s.Lb = g.Lb, s.Wb = g.Wb, s.lrow0 = 0, s.Kst = g.Kp;
        s.xk = 0, s.xy = rb * kBM, s.zk = 0, s.zy = w * kBN, s.kstep_x = kBK, s.kstep_y = 0;
        return true;
    }
    const int f = g.qitem[t];
    const BFront b = g.tab[f];
    const ctp_front fr = g.fronts[f];
    const int e = *fr.nelim;
    const int64_t local = t - b.q0;
    const int rb = (int)(local / b.nwz), w = (int)(local % b.nwz);
    const int E = (e + 31) & ~31;
    const int nW = (2 * E + b.p - e + kBN - 1) / kBN;
    if (e <= 0 || w >= nW) return false;
    s.A21 = fr.A + b.p, s.lda = fr.lda, s.m = b.m, s.p = b.p, s.e = e, s.E = E;
    s.KB = (e + kBK - 1) / kBK;
    s.i0 = (int64_t)rb * kBM, s.o0 = w * kBN;
    s.Lb = g.Lb, s.Wb = g.Wb, s.lrow0 = b.row0, s.Kst = kBatchKp;
    // tiles of 128 x 64: K blocks of a row block (or window) are consecutive tiles
    s.xk = 0, s.xy = (int)((b.xt0 + (int64_t)rb * b.kbx) * kBM);
    s.zk = 0, s.zy = (int)((b.zt0 + (int64_t)w * b.kbx) * kBN);
    s.kstep_x = 0, s.kstep_y = kBM;
    return true;
}

template <int PS, bool kBatch>
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_solve_tc(const __grid_constant__ CUtensorMap mX1, const __grid_constant__ CUtensorMap mX2,
               const __grid_constant__ CUtensorMap mX3, const __grid_constant__ CUtensorMap mZ1,
               const __grid_constant__ CUtensorMap mZ2, const __grid_constant__ CUtensorMap mZ3,
               const SArgs g) {
    using C = SCfg<PS>;
    constexpr int NS = C::Stages;
    const CUtensorMap *mapX[3] = {&mX1, &mX2, &mX3};
    const CUtensorMap *mapZ[3] = {&mZ1, &mZ2, &mZ3};
    extern __shared__ unsigned char smraw[];
    __shared__ Bars bars;
    uint8_t *ring = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = tile_count<kBatch>(g);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(&bars.full[s], 1);
            mbar_init(&bars.empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bars.acc_full[b], 1);
            mbar_init(&bars.acc_empty[b], kEpiWarps);
        }
        bars.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&bars.tmem_base, 2 * kBN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars.tmem_base;
    const uint32_t idesc = idesc_bf16(kBM, kBN);

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                STile s;
                if (!tile_at<kBatch>(t, g, s)) continue;
                for (int kb = 0; kb < s.KB; kb++) {
                    if (!mbar_wait(&bars.empty[stage], phase ^ 1u, &bars.abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&bars.full[stage], C::Stage);
                    uint8_t *dst = ring + (size_t)stage * C::Stage;
                    const int dx = kb * s.kstep_x, dy = kb * s.kstep_y;
#pragma unroll
                    for (int pc = 0; pc < PS; pc++) {
                        tma_load_2d(dst + pc * kPiece, mapX[pc], s.xk + dx, s.xy + dy, &bars.full[stage]);
                        tma_load_2d(dst + (PS + pc) * kPiece, mapZ[pc], s.zk + dx, s.zy + dy, &bars.full[stage]);
                    }
                    if (++stage == NS) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) atomicExch(&bars.abort, 1);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int stage = 0, acc = 0;
            uint32_t phase = 0, accphase = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                STile s;
                if (!tile_at<kBatch>(t, g, s)) continue;
                if (!mbar_wait(&bars.acc_empty[acc], accphase ^ 1u, &bars.abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(acc * kBN);
                for (int kb = 0; kb < s.KB; kb++) {
                    if (!mbar_wait(&bars.full[stage], phase, &bars.abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t x0 = smem_u32(ring + (size_t)stage * C::Stage);
                    const uint32_t z0 = x0 + PS * kPiece;
#pragma unroll
                    for (int kk = 0; kk < kBK / kUmmaK; kk++) {
                        // pieces i of x_e and j of Z^T with i + j <= PS - 1
                        const uint64_t a1 = sdesc(x0 + kk * 32), b1 = sdesc(z0 + kk * 32);
                        umma_bf16(dt, a1, b1, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                        const uint64_t a2 = sdesc(x0 + kPiece + kk * 32), b2 = sdesc(z0 + kPiece + kk * 32);
                        umma_bf16(dt, a1, b2, idesc, 1u);
                        umma_bf16(dt, a2, b1, idesc, 1u);
                        if (PS >= 3) {
                            umma_bf16(dt, a1, sdesc(z0 + 2 * kPiece + kk * 32), idesc, 1u);
                            umma_bf16(dt, sdesc(x0 + 2 * kPiece + kk * 32), b1, idesc, 1u);
                            umma_bf16(dt, a2, b2, idesc, 1u);
                        }
                    }
                    umma_commit(&bars.empty[stage]);
                    if (++stage == NS) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                umma_commit(&bars.acc_full[acc]);
                if (++acc == 2) {
                    acc = 0;
                    accphase ^= 1u;
                }
            }
            if (!ok) atomicExch(&bars.abort, 1);
        }
    } else {
        // ---------------- epilogue: warps 2..9
        const int q = warp & 3;            // TMEM lane quarter this warp may access
        const int half = (warp - 2) >> 2;  // which 64 columns of the window
        int acc = 0;
        uint32_t accphase = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            STile s;
            if (!tile_at<kBatch>(t, g, s)) continue;
            if (!mbar_wait(&bars.acc_full[acc], accphase, &bars.abort)) {
                if (lane == 0) atomicExch(&bars.abort, 1);
                break;
            }
            tc_fence_after();
            const int64_t i = s.i0 + q * 32 + lane;
            const int e = s.e, E = s.E, d = s.p - e;
#pragma unroll 1
            for (int c = 0; c < 64; c += 32) {
                uint32_t r[32];
                tmem_ld32_nowait(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kBN + half * 64 + c), r);
                tmem_wait_ld();
                if (i >= s.m) continue;
                const int o0 = s.o0 + half * 64 + c;  // a multiple of 32: one block of Z
                if (o0 < E) {
                    // L21: FP64 at positions < e; pieces over the whole slice (zero past e)
                    double *dst = s.A21 + (int64_t)o0 * s.lda + i;
#pragma unroll
                    for (int x = 0; x < 32; x++)
                        if (o0 + x < e) dst[(int64_t)x * s.lda] = (double)__uint_as_float(r[x]);
                    put_pieces32(s.Lb + (s.lrow0 + i) * s.Kst + o0, g.foff, g.fpieces, r);
                } else if (o0 < 2 * E) {
                    put_pieces32(s.Wb + (s.lrow0 + i) * s.Kst + (o0 - E), g.foff, g.fpieces, r);  // Y = W21
                } else {
                    // x_d += correction at delayed position e + (o - 2E)
                    const int j0 = o0 - 2 * E;
                    double *dst = s.A21 + (int64_t)(e + j0) * s.lda + i;
#pragma unroll
                    for (int x = 0; x < 32; x++)
                        if (j0 + x < d) dst[(int64_t)x * s.lda] += (double)__uint_as_float(r[x]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.acc_empty[acc]);
            if (++acc == 2) {
                acc = 0;
                accphase ^= 1u;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && bars.abort) atomicCAS(g.info, kInfoOk, (int32_t)CTP_ETIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * kBN);
    }
}

template <int PS, bool kBatch>
cudaError_t launch_gemm(int grid, const CUtensorMap (&mX)[3], const CUtensorMap (&mZ)[3], const SArgs &g,
                        cudaStream_t st) {
    const size_t smem = kSmemRing + 1024;
    cudaError_t err =
        smem_at_least((const void *)k_solve_tc<PS, kBatch>, smem);
    if (err != cudaSuccess) return err;
    k_solve_tc<PS, kBatch><<<grid, kThreadsTC, smem, st>>>(mX[0], mX[1], mX[2], mZ[0], mZ[1], mZ[2], g);
    return cudaGetLastError();
}

}  // namespace

size_t solve_tc_tile_elems() { return (size_t)kTileElems; }
int solve_tc_windows(int p) { return windows_for(p); }

cudaError_t launch_solve_tc_batch(const ctp_front *fronts, const BFront *tab, char *ws, const int *sitem,
                                  int64_t s_items, const int *qitem, int64_t q_items, const int *ritem,
                                  int64_t r_items, BatchOpts o,
                                  void *Xt, void *Zt, int64_t nxt, int64_t nzt, void *Wb, void *Lb,
                                  int32_t *ginfo, int num_sms, cudaStream_t st) {
    if (q_items == 0 || s_items == 0 || r_items == 0) return cudaSuccess;
    k_stc_prep_batch<<<(unsigned)r_items, 256, 0, st>>>(fronts, tab, ws, ritem, o, (__nv_bfloat16 *)Zt);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const size_t smem = sizeof(double) * (size_t)kMaxP * (kRowsG + 1);
    err = smem_at_least((const void *)k_stc_gather_batch, smem);
    if (err != cudaSuccess) return err;
    k_stc_gather_batch<<<(unsigned)s_items, kRowsG * kWarpsG, smem, st>>>(
        fronts, tab, sitem, o, (__nv_bfloat16 *)Xt, (__nv_bfloat16 *)Wb, (__nv_bfloat16 *)Lb);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    CUtensorMap mX[3], mZ[3];
    for (int pc = 0; pc < 3; pc++)
        if (!make_map_bf16(&mX[pc], (__nv_bfloat16 *)Xt + pc * o.xoff, nxt * kBM, kBK, kBM) ||
            !make_map_bf16(&mZ[pc], (__nv_bfloat16 *)Zt + pc * o.zoff, nzt * kBN, kBK, kBN))
            return cudaErrorInvalidValue;
    SArgs g = {};
    g.fronts = fronts, g.tab = tab, g.qitem = qitem, g.q_items = q_items;
    g.Wb = (__nv_bfloat16 *)Wb, g.Lb = (__nv_bfloat16 *)Lb, g.foff = o.lo_off, g.fpieces = o.pieces, g.info = ginfo;
    const int grid = (int)(q_items < num_sms ? q_items : num_sms);
    return launch_gemm<3, true>(grid, mX, mZ, g, st);
}

size_t solve_tc_ws_bytes(int64_t m, int p, int spieces) {
    const int Kp = form_tc_kpad(p);
    return align256(2 * (size_t)m * Kp * spieces) + align256(2 * (size_t)kZRows * Kp * spieces);
}

cudaError_t launch_solve_tc(double *A, int64_t n, int p, int64_t lda, const int32_t *perm, const int32_t *piv,
                            const double *Dinv, const int32_t *nelim, void *ws, int spieces, void *Wb, void *Lb,
                            int64_t foff, int fpieces, int32_t *info, int num_sms, cudaStream_t st) {
    const int64_t m = n - p;
    if (m <= 0) return cudaSuccess;
    if ((spieces != 2 && spieces != 3) || p < 1 || p > kMaxP) return cudaErrorInvalidValue;
    const int Kp = form_tc_kpad(p);
    __nv_bfloat16 *Xb = (__nv_bfloat16 *)ws;
    __nv_bfloat16 *Zt = (__nv_bfloat16 *)((char *)ws + align256(2 * (size_t)m * Kp * spieces));
    const int64_t xoff = m * Kp, zoff = (int64_t)kZRows * Kp;
    const size_t smem = sizeof(double) * (size_t)p * (kRowsG + 1);
    cudaError_t err = smem_at_least((const void *)k_stc_gather, smem);
    if (err != cudaSuccess) return err;
    k_stc_prep<<<Kp / kPrepRows, 32 * kPrepRows, 0, st>>>(A, p, lda, piv, Dinv, nelim, Zt, Kp, zoff, spieces);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_stc_gather<<<(unsigned)((m + kRowsG - 1) / kRowsG), kRowsG * kWarpsG, smem, st>>>(
        A, n, p, lda, perm, nelim, Xb, xoff, spieces, (__nv_bfloat16 *)Wb, (__nv_bfloat16 *)Lb, foff, fpieces, Kp);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    CUtensorMap mX[3], mZ[3];
    for (int pc = 0; pc < 3; pc++) {
        const int q = pc < spieces ? pc : 0;  // unused pieces: valid copies of the first
        if (!make_map_bf16(&mX[pc], Xb + q * xoff, m, Kp, kBM) ||
            !make_map_bf16(&mZ[pc], Zt + q * zoff, kZRows, Kp, kBN))
            return cudaErrorInvalidValue;
    }
    const int64_t tiles_max = ((m + kBM - 1) / kBM) * (kZRows / kBN);
    const int grid = (int)(tiles_max < num_sms ? tiles_max : num_sms);
    SArgs g = {};
    g.A21 = A + p, g.m = m, g.lda = lda, g.p = p, g.nelim = nelim, g.Kp = Kp;
    g.Wb = (__nv_bfloat16 *)Wb, g.Lb = (__nv_bfloat16 *)Lb, g.foff = foff, g.fpieces = fpieces, g.info = info;
    if (spieces == 2) return launch_gemm<2, false>(grid, mX, mZ, g, st);
    return launch_gemm<3, false>(grid, mX, mZ, g, st);
}

}  // namespace ctp
