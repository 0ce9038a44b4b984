// factor.cu -- K3: pivot selection on [A11; C] by Listing 1 (Section 2) in FP64,
// with the worst-case update of the strict compressed matrix (eq. (4.3); the
// 2x2 form follows the proof of Theorem 5.2).
//
// GB300 design.  The working matrix [A11; C] (A11 held in full symmetric form so
// that every column carries all of its entries, C the R outer rows that can be
// nonzero) is (p + R) x p doubles.  Three kernels share one set of rules:
//
//  * a team of G CTAs (a thread-block cluster, G >= 2) when it is larger than
//    one SM's shared memory -- 1 MB at p = 256: column c lives in the shared
//    memory of CTA (c mod G); other CTAs' columns are read through distributed
//    shared memory (DSMEM);
//  * one CTA, no cluster, when it fits (plain shared memory and __syncthreads);
//  * one warp per front for the small fronts of a batch (p <= 32 and at most 64
//    rows): no barrier at all, only warp-synchronous steps.
//
// Listing 1 is sequential, but a rejected candidate leaves the matrix unchanged,
// so every candidate tested between two acceptances sees the same matrix.  The
// CTA and cluster kernels therefore test a window of candidates at once (one
// warp per candidate, every CTA its own columns) and accept the lowest-index
// candidate that passes; all candidates before it in the window were rejected by
// Listing 1 as well.  A round costs one team barrier, plus one for the update
// when a pivot is accepted, instead of one barrier per test:
//   test round   each warp runs the zero test, the 2x2 test with its partner t
//                (largest |a(m, j)| over live j < m) and the 1x1 test for one
//                candidate; a passing warp pushes (candidate, warp) into every
//                CTA's slot with a DSMEM atomicMin, so after the barrier each
//                CTA finds the winner in its own shared memory;
//   update       every CTA copies the pivot column(s), takes the per-column
//                scalars from them and applies the 1x1 or 2x2 update to its own
//                live columns (one CTA barrier, then the team barrier).
// The warp kernel runs the same tests one candidate at a time.
// Columns are never moved: accepted pivots leave the live set, and because the
// paper's stable shift never reorders the remaining columns, the candidate
// order is simply the original column order of the live columns.  The final
// pivot order (accepted pivots in acceptance order, then the delayed columns in
// original order) is applied only when the factor is written back.
//
// Determinism: every CTA holds the same replicated control state (live flags,
// nelim, m) and executes the same sequence of barriers.  Tests use explicitly
// rounded operations (no FMA contraction) and updates one fused multiply-add
// per term, in the order of a plain sequential implementation of the listing.
#include <cooperative_groups.h>

#include "ctp_internal.cuh"

namespace cg = cooperative_groups;

namespace ctp {

namespace {

// threads per CTA (CTA and cluster kernels): 16 warps, one CTA per SM.  Eight
// warps with up to three CTAs per SM were slower: a front's FP64 update then
// has half the warps of its SM to issue from (the pipe is about 70 cycles per
// warp instruction), while small fronts sharing an SM gained nothing measurable
constexpr int kT = 512;
constexpr int kNW = kT / 32;
constexpr int kWarpFronts = 4;  // fronts (warps) per CTA of the warp kernel
constexpr int kNoKey = 0x7fffffff;

enum { DEC_REJECT = 0, DEC_1X1 = 1, DEC_2X2 = 2, DEC_ZERO = -1 };

struct Decision {
    int kind, t, m, pad;
    double d0, d1, d2;  // 1x1: d0 = d; 2x2: a_tt, a_tm, a_mm
    double i0, i1, i2;  // 1x1: i0 = 1/d; 2x2: D^-1 entries (t,t), (m,t), (m,m)
};
static_assert(sizeof(Decision) == 64, "Decision is copied as eight 8-byte words");

struct Shared {
    Decision res[2][kNW];  // per warp's candidate, double-buffered by round
    Decision cur;
    int cmin[2];           // lowest (candidate * kNW + warp) that passed, pushed by every CTA
    unsigned char live[kMaxP];
    int order[kMaxP];
    int kind[kMaxP];
    int pos_of[kMaxP];
    double sD[2 * kMaxP + 2];
    double sInv[2 * kMaxP + 2];
    int cand[kNW];
    int cstar;
    int rowmap[kMaxP];  // nonzero outer rows
    int nz_count;
    unsigned char nzflag[kMaxP];
    unsigned short lrow[kMaxP];  // the live A11 rows, ascending (rebuilt before each update)
    unsigned short lpos[kMaxP];  // lpos[i]: how many live rows lie above row i
    int nlive;
};

// The team that owns one front: a cluster of G CTAs, or one CTA.
template <bool kSingle>
struct Team;
template <>
struct Team<true> {
    __device__ __forceinline__ int rank() const { return 0; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    template <typename T>
    __device__ __forceinline__ T *at(T *ptr, int) const { return ptr; }
};
template <>
struct Team<false> {
    cg::cluster_group cl;
    __device__ __forceinline__ Team() : cl(cg::this_cluster()) {}
    __device__ __forceinline__ int rank() const { return (int)cl.block_rank(); }
    __device__ __forceinline__ void sync() const { cl.sync(); }
    template <typename T>
    __device__ __forceinline__ T *at(T *ptr, int r) const { return cl.map_shared_rank(ptr, r); }
};

__device__ __forceinline__ unsigned long long akey(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
// Largest key of the warp: two single-instruction reductions on the 32-bit
// halves (the high halves, then the low halves of the lanes that hold the
// highest) instead of five shuffle steps on the 64-bit value.
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
    const unsigned h = (unsigned)(v >> 32);
    const unsigned H = __reduce_max_sync(0xffffffffu, h);
    const unsigned L = __reduce_max_sync(0xffffffffu, h == H ? (unsigned)v : 0u);
    return ((unsigned long long)H << 32) | L;
}
__device__ __forceinline__ double key_val(unsigned long long k) {
    return __longlong_as_double((long long)k);
}
// x is Inf or NaN: all exponent bits set (an integer test)
__device__ __forceinline__ bool nonfinite_bits(double x) { return akey(x) >= 0x7FF0000000000000ull; }
// x != 0 (either sign)
__device__ __forceinline__ bool nonzero_bits(double x) { return akey(x) != 0ull; }
// |x| and -x on the sign bit (integer instructions, never the FP64 pipe)
__device__ __forceinline__ double abs_bits(double x) { return key_val(akey(x)); }
__device__ __forceinline__ double neg_bits(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// GB300's FP64 pipe takes about 70 cycles per warp instruction whatever the
// number of active lanes, while integer instructions cost one.  So the tests
// below do every comparison, maximum and absolute value of non-negative
// doubles on their IEEE bit patterns (for x, y >= 0, x < y as doubles iff
// bits(x) < bits(y) as unsigned integers), and keep FP64 arithmetic for the
// products, sums and reciprocals whose rounding the test defines.

// FP32 filters in front of the FP64 tests.  Most candidates of a strict front
// fail their tests, and a failing test's FP64 instructions (a reciprocal and a
// dozen products) are most of its latency.  Where FP32 arithmetic with wide
// error margins already proves the outcome the FP64 test would reach, the
// FP64 test is skipped; every other case runs it unchanged, so the decisions
// are exactly those of the FP64 test.
//
// key_f32: binary32 value of a magnitude key whose binary exponent lies in
// [-32, 32] (or 0): same exponent, the top 23 mantissa bits (truncated, so
// 0 <= |x| - f < 2^-23 |x|).  Integer instructions only; false out of range.
__device__ __forceinline__ bool key_f32(unsigned long long k, float &f) {
    if (k == 0ull) {
        f = 0.0f;
        return true;
    }
    const unsigned e = (unsigned)(k >> 52);
    if (e < 1023u - 32u || e > 1023u + 32u) return false;
    f = __uint_as_float((unsigned)((k >> 29) - (896ull << 23)));
    return true;
}

// true when the 2x2 test below surely rejects (t, m).  With inputs truncated
// by < 2^-23 and a handful of FP32 roundings (2^-24 each), every FP32 product
// here is within 2^-20 of the FP64 value the test computes (whose own
// roundings are 2^-53), so:
//   |detpiv - det| <= 2^-20 (|d0| + |d1|) + 2^-24 |det| < err = 2^-16 (p0 + p1 + |det|),
//   glow = (1 - 2^-16) max(p0, p1) / 2 <= max(|d0|, |d1|) / 2 <= guard,
// and |det| + err < glow proves |detpiv| <= guard.  Likewise the growth test
// fails for sure when (1 - 2^-16) gt_f exceeds an upper bound of
// lim = |detpiv| / u, which the FP64 test only evaluates when the column
// maxima reach `small` (the same integer condition here).
__device__ __forceinline__ bool reject_2x2_f32(double a_tt, double a_tm, double a_mm, unsigned long long ktt,
                                               unsigned long long ktm, unsigned long long kmm,
                                               unsigned long long kmax, unsigned long long maxt,
                                               unsigned long long maxm, double rcp_u, unsigned long long small_k) {
    float ftt, ftm, fmm, fmax;
    if (kmax == 0ull || !key_f32(ktt, ftt) || !key_f32(ktm, ftm) || !key_f32(kmm, fmm) || !key_f32(kmax, fmax))
        return false;
    const float ds = 1.0f / fmax;
    const float p0 = (fmm * ds) * ftt;  // |detpiv0| = |a_mm| |a_tt| / amax
    const float p1 = (ftm * ds) * ftm;  // detpiv1 = a_tm^2 / amax >= 0
    const bool neg0 = (__double_as_longlong(a_mm) ^ __double_as_longlong(a_tt)) < 0;
    const float adet = fabsf((neg0 ? -p0 : p0) - p1);
    const float err = 0x1p-16f * (p0 + p1 + adet);
    const float glow = 0.5f * fmaxf(p0, p1) * (1.0f - 0x1p-16f);
    if (adet + err < glow) return true;
    if ((maxm > maxt ? maxm : maxt) < small_k) return false;  // the FP64 test accepts without growth test
    float fvt, fvm, fru;
    if (!key_f32(maxt, fvt) || !key_f32(maxm, fvm) || !key_f32(akey(rcp_u), fru) || fru > 0x1p20f) return false;
    const float lim_up = (adet + err) * (fru * (1.0f + 0x1p-21f)) * (1.0f + 0x1p-16f);
    const float gt = (fmm * fvt + ftm * fvm) * ds;
    const float gm = (ftm * fvt + ftt * fvm) * ds;
    return gt * (1.0f - 0x1p-16f) > lim_up || gm * (1.0f - 0x1p-16f) > lim_up;
}

// The 1x1 test |a_mm| >= u * maxm1 (rounded in FP64) decided in FP32 when the
// margin is wide: 1 accept, 0 reject, -1 undecided (run the FP64 test).
__device__ __forceinline__ int test_1x1_f32(unsigned long long kmm, unsigned long long maxm1, double u) {
    float fmm, fmx, fu;
    if (!key_f32(kmm, fmm) || !key_f32(maxm1, fmx) || !key_f32(akey(u), fu)) return -1;
    const float lim = fu * fmx;  // u maxm1 (1 - 2^-22) <= lim <= u maxm1 (1 + 2^-24)
    if (fmm * (1.0f + 0x1p-16f) < lim * (1.0f - 0x1p-16f)) return 0;
    if (fmm * (1.0f - 0x1p-16f) > lim * (1.0f + 0x1p-16f)) return 1;
    return -1;
}

// |x| / 2 as a key: an exponent decrement, exact for normal x above the
// smallest binade; the rare others take the FP64 product.
__device__ __forceinline__ unsigned long long half_key(unsigned long long k) {
    return (k >> 52) > 1 ? k - (1ull << 52) : akey(0.5 * key_val(k));
}

// Listing 1's test_2x2 with the nonsingularity/cancellation guard and the growth
// test of eq. (2.2), |D^-1| (maxt, maxm)^T <= 1/u, on keys maxt, maxm of the
// column maxima.  rcp_u = 1/u rounded, small_k = key of `small`.  Fills d on
// acceptance.
__device__ __forceinline__ bool test_2x2(double a_tt, double a_tm, double a_mm, unsigned long long maxt,
                                         unsigned long long maxm, double rcp_u, unsigned long long small_k,
                                         Decision &d) {
    const unsigned long long ktt = akey(a_tt), ktm = akey(a_tm), kmm = akey(a_mm);
    unsigned long long kmax = ktt > ktm ? ktt : ktm;
    kmax = kmm > kmax ? kmm : kmax;
    if (kmax < small_k) return false;
    if (reject_2x2_f32(a_tt, a_tm, a_mm, ktt, ktm, kmm, kmax, maxt, maxm, rcp_u, small_k)) return false;
    // 1/amax correctly rounded: the same value as the division 1.0/amax
    const double detscale = __drcp_rn(key_val(kmax));
    const double detpiv1 = __dmul_rn(__dmul_rn(a_tm, detscale), a_tm);
    const double detpiv0 = __dmul_rn(__dmul_rn(a_mm, detscale), a_tt);
    const double detpiv = __dsub_rn(detpiv0, detpiv1);
    unsigned long long guard = half_key(akey(detpiv0));
    const unsigned long long g1 = half_key(akey(detpiv1));
    guard = g1 > guard ? g1 : guard;
    guard = small_k > guard ? small_k : guard;
    const unsigned long long kdet = akey(detpiv);
    if (kdet <= guard) return false;
    bool ok;
    if ((maxm > maxt ? maxm : maxt) < small_k) {
        ok = true;
    } else {
        // |D^-1| (maxt, maxm)^T <= 1/u, each row compared as num*detscale <= |detpiv|/u
        // (the quotient form of the test, without FP64 divisions)
        const double vt = key_val(maxt), vm = key_val(maxm);
        const unsigned long long lim = akey(__dmul_rn(key_val(kdet), rcp_u));
        const unsigned long long gt = akey(
            __dmul_rn(__dadd_rn(__dmul_rn(key_val(kmm), vt), __dmul_rn(key_val(ktm), vm)), detscale));
        ok = gt <= lim;
        if (ok) {
            const unsigned long long gm = akey(
                __dmul_rn(__dadd_rn(__dmul_rn(key_val(ktm), vt), __dmul_rn(key_val(ktt), vm)), detscale));
            ok = gm <= lim;
        }
    }
    if (ok) {
        // D^-1 = (detscale / detpiv) [[a_mm, -a_tm], [-a_tm, a_tt]], each entry
        // scaled first and then divided, as the update's multipliers expect
        d.d0 = a_tt;
        d.d1 = a_tm;
        d.d2 = a_mm;
        d.i0 = __ddiv_rn(__dmul_rn(a_mm, detscale), detpiv);
        d.i1 = __ddiv_rn(__dmul_rn(-a_tm, detscale), detpiv);
        d.i2 = __ddiv_rn(__dmul_rn(a_tt, detscale), detpiv);
    }
    return ok;
}

// live flags of the warp kernel: one bit per column (p <= 32)
struct BitLive {
    unsigned bits;
    __device__ __forceinline__ bool operator[](int i) const { return (bits >> i) & 1u; }
};

// The tests of Listing 1 for candidate c (one warp): zero test, 2x2 with the
// partner t, 1x1, from two scans of the column (the partner, then the maxima).
// cm is the candidate's column (rows 0..p-1 A11, then outer).
// Column maxima of |a| are taken on the IEEE bit patterns with the sign cleared
// (integer order = magnitude order), which keeps the scans off the FP64 pipe.
// The maxima scan keeps four loads per lane in flight: the partner's column
// may sit in another CTA's shared memory.
template <typename ColPtr, typename Live>
__device__ __forceinline__ Decision test_candidate(int c, const double *cm, ColPtr colptr,
                                                   const Live &live, int p, int LD, double u,
                                                   double rcp_u, unsigned long long small_k) {
    const int lane = threadIdx.x & 31;
    Decision d;
    d.kind = DEC_REJECT;
    d.t = -1;
    d.m = c;
    d.pad = 0;
    d.d0 = d.d1 = d.d2 = d.i0 = d.i1 = d.i2 = 0.0;
    // partner t: largest |a(c, j)| over live j < c, lowest j on ties
    // (four rows per lane per step, their loads issued together; each lane
    // visits its rows in ascending order, so it keeps the lowest on ties)
    unsigned long long bv = 0;
    int bi = -1;
    constexpr int UP = 4;
    for (int j0 = lane; j0 < c; j0 += 32 * UP) {
        unsigned long long kq[UP];
        bool lq[UP];
#pragma unroll
        for (int q = 0; q < UP; q++) {
            const int j = j0 + 32 * q;
            lq[q] = j < c && live[j];
            kq[q] = j < c ? akey(cm[j]) : 0ull;
        }
#pragma unroll
        for (int q = 0; q < UP; q++)
            if (lq[q] && (bi < 0 || kq[q] > bv)) {
                bv = kq[q];
                bi = j0 + 32 * q;
            }
    }
    // the warp's largest key among the lanes that have a candidate (lanes
    // without one offer key 0, which never beats a candidate's key, and are
    // left out of the index), then the lowest column holding it
    const unsigned bh = bi >= 0 ? (unsigned)(bv >> 32) : 0u, bl = bi >= 0 ? (unsigned)bv : 0u;
    const unsigned BH = __reduce_max_sync(0xffffffffu, bh);
    const unsigned BL = __reduce_max_sync(0xffffffffu, bh == BH ? bl : 0u);
    const int t0 = __reduce_min_sync(0xffffffffu, (bi >= 0 && bh == BH && bl == BL) ? bi : 0x7fffffff);
    const int t = t0 == 0x7fffffff ? -1 : t0;
    // one pass over the live rows but t and c: the column maximum of c (and of
    // the partner's column); the zero test's maximum over every live row of c
    // adds rows t and c back
    const double *ct = t >= 0 ? colptr(t) : cm;
    unsigned long long vm = 0, vt = 0;
    constexpr int U = 4;
    for (int i0 = lane; i0 < LD; i0 += 32 * U) {
        double xm[U], xt[U];
        bool lq[U];
#pragma unroll
        for (int q = 0; q < U; q++) {
            const int i = i0 + 32 * q;
            xm[q] = i < LD ? cm[i] : 0.0;
            xt[q] = i < LD ? ct[i] : 0.0;
            lq[q] = i < LD && (i >= p || (i != t && i != c && live[i]));
        }
#pragma unroll
        for (int q = 0; q < U; q++) {
            if (lq[q]) {
                const unsigned long long km = akey(xm[q]), kt = akey(xt[q]);
                vm = km > vm ? km : vm;
                vt = kt > vt ? kt : vt;
            }
        }
    }
    vm = warp_max_key(vm);
    const double amm = cm[c];
    const unsigned long long kmm = akey(amm), ktm = t >= 0 ? akey(cm[t]) : 0ull;
    unsigned long long vall = vm > kmm ? vm : kmm;
    vall = ktm > vall ? ktm : vall;
    if (vall < small_k) {
        d.kind = DEC_ZERO;
        return d;
    }
    unsigned long long maxm1 = vm;  // the live rows but c (and t, added back for the 1x1 test)
    if (t >= 0) {
        if (test_2x2(ct[t], cm[t], amm, warp_max_key(vt), vm, rcp_u, small_k, d)) {
            d.kind = DEC_2X2;
            d.t = t;
            return d;
        }
        maxm1 = ktm > vm ? ktm : vm;
    }
    const int f1 = test_1x1_f32(kmm, maxm1, u);
    if (f1 == 1 || (f1 < 0 && kmm >= akey(__dmul_rn(u, key_val(maxm1))))) {
        d.kind = DEC_1X1;
        d.d0 = amm;
        d.i0 = __drcp_rn(amm);
    }
    return d;
}

template <bool kSingle>
__device__ __forceinline__ void factor_body(const FactorArgs &a, int G) {
    Team<kSingle> team;
    extern __shared__ __align__(16) double dsm[];
    __shared__ Shared sh;

    const int p = a.p;
    const int rank = team.rank();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // Outer rows: rows of C that are identically zero (a strict C row whose set
    // J_j is empty, or a relaxed row past the last A21 row) stay zero under the
    // updates and never change a column maximum, so only the nonzero rows are
    // kept: R <= min(p, m).  Every CTA builds the same list.
    // (All per-entry loops below run over flattened (column, row) indices so
    // that every thread has work whatever the front's size: a loop over
    // columns with the rows spread over the threads leaves most of them idle
    // when the columns are short, and its steps add up.)
    // With the compression's flags (which rows of C received an A21 row) no
    // scan is needed.  Otherwise a row whose first entry is nonzero is nonzero
    // (almost every row of a front with many A21 rows); only the others are
    // scanned in full, all of them together over (row, column) pairs.
    if (a.rowbits != nullptr) {
        for (int j = tid; j < a.R; j += kT) sh.nzflag[j] = (a.rowbits[j >> 5] >> (j & 31)) & 1u;
        if (tid == 0) sh.nz_count = 0;
    } else if (warp == 0) {
        int r = 0;
        for (int j0 = 0; j0 < a.R; j0 += 32) {
            const int j = j0 + lane;
            const bool first = j < a.R && nonzero_bits(a.C[(int64_t)j * p]);
            if (j < a.R) sh.nzflag[j] = first ? 1 : 0;
            const bool scan = j < a.R && !first;
            const unsigned int bal = __ballot_sync(0xffffffffu, scan);
            if (scan) sh.rowmap[r + __popc(bal & ((1u << lane) - 1u))] = j;  // rows still to scan
            r += __popc(bal);
        }
        if (lane == 0) sh.nz_count = r;
    }
    __syncthreads();
    {
        const int ns = sh.nz_count;
        for (int idx = tid; idx < ns * p; idx += kT) {
            const int q = idx / p, k = idx - q * p;
            const int j = sh.rowmap[q];
            if (nonzero_bits(a.C[(int64_t)j * p + k])) sh.nzflag[j] = 1;
        }
    }
    __syncthreads();
    if (warp == 0) {  // compaction of the nonzero rows, 32 at a time
        int r = 0;
        for (int j0 = 0; j0 < a.R; j0 += 32) {
            const int j = j0 + lane;
            const bool nz = j < a.R && sh.nzflag[j];
            const unsigned int bal = __ballot_sync(0xffffffffu, nz);
            if (nz) sh.rowmap[r + __popc(bal & ((1u << lane) - 1u))] = j;
            r += __popc(bal);
        }
        if (lane == 0) sh.nz_count = r;
    }
    __syncthreads();
    const int R = sh.nz_count, LD = p + R;
    const int gs = __ffs(G) - 1, gm = G - 1;  // G is a power of two: column c is slot c >> gs of CTA c & gm
    const int ncl = (p + gm) >> gs;
    double *cols = dsm;                    // [ncl][LD]
    double *pc0 = dsm + (size_t)ncl * LD;  // pivot column copies
    double *pc1 = pc0 + LD;
    double *rl0 = pc1 + LD, *rl1 = rl0 + LD;  // row multipliers of the pivot, signed
    double *apc0 = rl1 + LD, *apc1 = apc0 + p;  // |pivot column| on the A11 rows
    auto colptr = [&](int c) -> const double * { return team.at(cols, c & gm) + (size_t)(c >> gs) * LD; };

    // ---- load: own columns of A11 (full symmetric) and of the nonzero outer rows
    bool nonfinite = false;
    // flattened (column, row) loops step their indices by kT without divisions
    const int dl = kT / LD, di = kT - dl * LD;
    for (int idx = tid, lc = tid / LD, i = tid - (tid / LD) * LD; idx < ncl * LD; idx += kT) {
        const int c = (lc << gs) + rank;
        const int ii = i;
        i += di;
        lc += dl;
        if (i >= LD) {
            i -= LD;
            lc++;
        }
        if (c >= p) continue;
        const int i0 = ii;
        double v;
        if (i0 < p)
            v = (i0 >= c) ? a.A[(int64_t)c * a.lda + i0] : a.A[(int64_t)i0 * a.lda + c];
        else
            v = a.C[(int64_t)sh.rowmap[i0 - p] * p + c];
        nonfinite |= nonfinite_bits(v);
        cols[idx] = v;
    }
    for (int i = tid; i < p; i += kT) {
        sh.live[i] = 1;
        sh.lrow[i] = (unsigned short)i;
        sh.lpos[i] = (unsigned short)i;
    }
    if (tid == 0) sh.nlive = p;
    if (tid < 2) sh.cmin[tid] = kNoKey;
    if (nonfinite) atomicCAS(a.info, kInfoOk, (int32_t)CTP_ENONFINITE);
    team.sync();

    const double u = a.u, rcp_u = __drcp_rn(a.u);
    const unsigned long long small_k = akey(a.small);
    int nelim = 0, m = (p >= 2) ? 1 : 0, accepted = 0, round = 0;
    int win = 1;                  // candidates tested in the next round
    const int win_max = kNW * G;  // no CTA owns more than kNW of them
    int m0 = m;                   // where the search for the next pivot began
    for (;;) {
        if (nelim >= p) break;
        while (m < p && !sh.live[m]) m++;
        if (m >= p) {
            if (!accepted) break;  // a whole sweep without a pivot: stop
            accepted = 0;
            m = 0;  // new sweep from the first live column
            m0 = 0;
            continue;
        }
        const int buf = round & 1;
        round++;
        // ---------------- test round: the live candidates in [m, m + win)
        // (team-wide order); each CTA tests the ones it owns, one per warp.
        // The window is 1 after an acceptance and grows fourfold after a round
        // with no pass, so accepted-first candidates cost a single test and runs
        // of rejections are tested in parallel (a rejection is cheap: most are
        // settled by the FP32 filters).
        const int hi = min(p, m + win);  // the same on every CTA
        if (warp == 0) {
            // this CTA's live columns in [m, hi), in order, go to its warps
            // (win <= kNW * G, so no CTA owns more than kNW of them)
            const int j0 = m > rank ? (m - rank + gm) >> gs : 0;
            const int c = rank + G * (j0 + lane);
            const bool ok = c < hi && sh.live[c];
            const unsigned int bal = __ballot_sync(0xffffffffu, ok);
            if (ok) sh.cand[__popc(bal & ((1u << lane) - 1u))] = c;
            if (lane >= __popc(bal) && lane < kNW) sh.cand[lane] = -1;
        }
        __syncthreads();
        {
            const int c = sh.cand[warp];
            if (c >= 0) {
                Decision d = test_candidate(c, cols + (size_t)(c >> gs) * LD, colptr, sh.live, p, LD, u, rcp_u,
                                            small_k);
                if (d.kind != DEC_REJECT) {
                    // publish: the decision stays here, (candidate, warp) goes to
                    // every CTA's slot for this round
                    if (lane == 0) sh.res[buf][warp] = d;
                    const int key = c * kNW + warp;
                    if (lane < G) atomicMin(team.at(&sh.cmin[buf], lane), key);
                }
            }
        }
        team.sync();
        // the lowest passing candidate: read the own slot (and clear it for the
        // round after next), fetch the winner's decision from its CTA
        if (warp == 0) {
            int key = 0;
            if (lane == 0) {
                key = sh.cmin[buf];
                sh.cmin[buf] = kNoKey;
            }
            key = __shfl_sync(0xffffffffu, key, 0);
            const int cs = key == kNoKey ? p : key / kNW;
            if (cs < p && lane < 8) {
                const Decision *src = team.at(&sh.res[buf][key % kNW], cs & gm);
                reinterpret_cast<double *>(&sh.cur)[lane] = reinterpret_cast<const double *>(src)[lane];
            }
            if (lane == 0) sh.cstar = cs;
        }
        __syncthreads();
        const int cstar = sh.cstar;
        if (cstar >= hi) {
            // every tested candidate before the window's end failed: the sweep
            // continues there, with a wider window
            m = hi;
            win = win * 4 < win_max ? win * 4 : win_max;
            continue;
        }
        // the next search starts with a window of twice the distance this one
        // covered (1 when the first candidate passed): all-accepting runs test
        // one candidate per round, runs of rejections start wide
        {
            const int gap = cstar - m0;
            win = 1;
            while (win < 2 * gap && win < win_max) win *= 2;
            if (win > win_max) win = win_max;
            m0 = cstar + 1;
        }
        const Decision dv = sh.cur;
        if (dv.kind == DEC_ZERO) {
            // the live-row list without cstar (every thread reads its own rows'
            // old positions only)
            for (int i = tid; i < p; i += kT) {
                const int np = sh.lpos[i] - (cstar < i ? 1 : 0);
                sh.lpos[i] = (unsigned short)np;
                if (sh.live[i] && i != cstar) sh.lrow[np] = (unsigned short)i;
            }
            if (tid == 0) {
                sh.nlive--;
                sh.live[cstar] = 0;
                sh.order[nelim] = cstar;
                sh.kind[nelim] = CTP_PIVKIND_ZERO;
                sh.sD[2 * nelim] = sh.sD[2 * nelim + 1] = 0.0;
                sh.sInv[2 * nelim] = sh.sInv[2 * nelim + 1] = 0.0;
            }
            __syncthreads();
            nelim++;
            accepted = 1;
            m = cstar + 1;
            // no update; the next round writes the other buffers, and the round
            // after that comes behind the next team barrier
            continue;
        }
        // ---------------- update: apply the pivot to the own live columns with
        // the rounding of a plain right-looking update: row multipliers
        // l(i) = a(i,q)/d (1x1) or [a(i,t) a(i,m)] D^-1 (2x2; abs rows of strict
        // C with |d|, |D^-1|), rounded per operation, then
        // a(i,c) = fma(-l(i), a(c,q), a(i,c)) (and the m term after the t term):
        // one rounding per term; entries above the diagonal take their mirror's
        // operands, so the full symmetric copy stays exactly symmetric.  Equal
        // inputs then give bit-identical working matrices on any team shape,
        // and exact ties between entries (Listing 1's partner choice) are broken
        // identically.
        const int q0 = (dv.kind == DEC_2X2) ? dv.t : dv.m;
        const int q1 = (dv.kind == DEC_2X2) ? dv.m : -1;
        const bool abs_rows = a.abs_update != 0;
        {
            // copies of the pivot column(s), every row's multipliers, and the
            // bookkeeping of the pivot, in one phase (the pivot columns are not
            // written in this round; live[] is read nowhere in this phase)
            // multipliers are stored with the sign of their term (-l on normal
            // rows, +l on abs rows) and the A11 pivot entries also as |.|, so
            // that the update loop needs no FP64 sign or abs operation
            const double *s0 = colptr(q0);
            const double *s1 = q1 >= 0 ? colptr(q1) : s0;
            const double ad0 = abs_bits(dv.d0), ai0 = abs_bits(dv.i0), ai1 = abs_bits(dv.i1), ai2 = abs_bits(dv.i2);
            for (int i = tid; i < LD; i += kT) {
                if (i < p) {
                    // the live-row list without the pivot rows: the rank of a
                    // row drops by the pivots above it (the pivots' own flags
                    // are cleared in this phase, so they are named explicitly)
                    const int np = sh.lpos[i] - (q0 < i ? 1 : 0) - (q1 >= 0 && q1 < i ? 1 : 0);
                    sh.lpos[i] = (unsigned short)np;
                    if (sh.live[i] && i != q0 && i != q1) sh.lrow[np] = (unsigned short)i;
                }
                const double x = s0[i];
                pc0[i] = x;
                const bool ab = abs_rows && i >= p;
                if (i < p) apc0[i] = abs_bits(x);
                if (q1 < 0) {
                    const double l = __ddiv_rn(x, ab ? ad0 : dv.d0);
                    rl0[i] = ab ? l : neg_bits(l);
                } else {
                    const double y = s1[i];
                    pc1[i] = y;
                    if (i < p) apc1[i] = abs_bits(y);
                    const double i11 = ab ? ai0 : dv.i0, i21 = ab ? ai1 : dv.i1, i22 = ab ? ai2 : dv.i2;
                    const double l0 = __dadd_rn(__dmul_rn(x, i11), __dmul_rn(y, i21));
                    const double l1 = __dadd_rn(__dmul_rn(x, i21), __dmul_rn(y, i22));
                    rl0[i] = ab ? l0 : neg_bits(l0);
                    rl1[i] = ab ? l1 : neg_bits(l1);
                }
            }
            if (tid == 0) {
                sh.nlive -= q1 < 0 ? 1 : 2;
                if (q1 < 0) {
                    sh.live[q0] = 0;
                    sh.order[nelim] = q0;
                    sh.kind[nelim] = CTP_PIVKIND_1X1;
                    sh.sD[2 * nelim] = dv.d0;
                    sh.sD[2 * nelim + 1] = 0.0;
                    sh.sInv[2 * nelim] = dv.i0;
                    sh.sInv[2 * nelim + 1] = 0.0;
                } else {
                    sh.live[q0] = 0;
                    sh.live[q1] = 0;
                    sh.order[nelim] = q0;
                    sh.order[nelim + 1] = q1;
                    sh.kind[nelim] = CTP_PIVKIND_2X2_FIRST;
                    sh.kind[nelim + 1] = CTP_PIVKIND_2X2_SECOND;
                    sh.sD[2 * nelim] = dv.d0;
                    sh.sD[2 * nelim + 1] = dv.d1;
                    sh.sD[2 * nelim + 2] = dv.d2;
                    sh.sD[2 * nelim + 3] = 0.0;
                    sh.sInv[2 * nelim] = dv.i0;
                    sh.sInv[2 * nelim + 1] = dv.i1;
                    sh.sInv[2 * nelim + 2] = dv.i2;
                    sh.sInv[2 * nelim + 3] = 0.0;
                }
            }
        }
        __syncthreads();
        // the update: warp w takes the own live columns w, w + kNW, ...; column
        // c gets its live A11 rows from the diagonal down and the R outer rows,
        // one fused multiply-add per pivot column: -l(i) a(c,q), or +l(i)
        // |a(c,q)| on the abs rows (eq. (4.3)).  The entry (c, i) above the
        // diagonal, in row i's column, is the same product (row i's multiplier,
        // row c's pivot entry) on the same old value (the working matrix is
        // symmetric), so column c's owner stores the result there too (in
        // another CTA's shared memory when column i lives there): the upper half
        // costs a store instead of a second FP64 update, and both halves stay
        // bit-identical.  Only live rows are visited, so no lane of an FP64
        // instruction idles on a retired row.
        {
            const int nl = sh.nlive;
            for (int lc = warp; lc < ncl; lc += kNW) {
                const int c = (lc << gs) + rank;
                if (c >= p || !sh.live[c]) continue;  // warp-uniform
                const int a0 = sh.lpos[c], lenA = nl - a0, len = lenA + R;
                double *col = cols + (size_t)lc * LD;
                const double q0c = pc0[c], aq0c = apc0[c];
                const double q1c = q1 >= 0 ? pc1[c] : 0.0, aq1c = q1 >= 0 ? apc1[c] : 0.0;
                for (int j = lane; j < len; j += 32) {
                    const int i = j < lenA ? (int)sh.lrow[a0 + j] : p + (j - lenA);
                    const bool ab = abs_rows && i >= p;
                    double v = fma(rl0[i], ab ? aq0c : q0c, col[i]);
                    if (q1 >= 0) v = fma(rl1[i], ab ? aq1c : q1c, v);
                    col[i] = v;
                    if (i < p && i != c) team.at(cols, i & gm)[(size_t)(i >> gs) * LD + c] = v;
                }
            }
        }
        nelim += (q1 < 0) ? 1 : 2;
        accepted = 1;
        m = cstar + 1;
        team.sync();  // every update done before the next tests read columns
    }

    // ---- final order: accepted pivots, then the delayed columns in original order
    const int e = nelim;
    if (tid == 0) {
        int k = e;
        for (int c = 0; c < p; c++)
            if (sh.live[c]) {
                sh.order[k] = c;
                sh.kind[k] = CTP_PIVKIND_DELAYED;
                sh.sD[2 * k] = sh.sD[2 * k + 1] = 0.0;
                sh.sInv[2 * k] = sh.sInv[2 * k + 1] = 0.0;
                k++;
            }
    }
    __syncthreads();
    for (int k = tid; k < p; k += kT) sh.pos_of[sh.order[k]] = k;
    __syncthreads();

    // ---- write back the A11 block in pivot order (lower triangle), over
    // (column, row) pairs of the own columns
    const int dlp = kT / p, dip = kT - dlp * p;
    for (int idx = tid, lc2 = tid / p, i2 = tid - (tid / p) * p; idx < ncl * p; idx += kT) {
        const int lc = lc2, i = i2;
        i2 += dip;
        lc2 += dlp;
        if (i2 >= p) {
            i2 -= p;
            lc2++;
        }
        const int c = (lc << gs) + rank;
        if (c >= p) continue;
        const double *col = cols + (size_t)lc * LD;
        const int pos = sh.pos_of[c];
        const int kd = sh.kind[pos];
        double *out = a.A + (int64_t)pos * a.lda;
        const int pi = sh.pos_of[i];
        if (kd == CTP_PIVKIND_DELAYED) {
            if (pi >= pos) out[pi] = col[i];
        } else if (kd == CTP_PIVKIND_ZERO) {
            if (pi >= pos) out[pi] = 0.0;
        } else if (kd == CTP_PIVKIND_1X1) {
            if (pi > pos) out[pi] = col[i] * sh.sInv[2 * pos];
            if (i == 0) out[pos] = sh.sD[2 * pos];
        } else if (kd == CTP_PIVKIND_2X2_FIRST) {
            const int mo = sh.order[pos + 1];
            if (pi > pos + 1) out[pi] = col[i] * sh.sInv[2 * pos] + colptr(mo)[i] * sh.sInv[2 * pos + 1];
            if (i == 0) {
                out[pos] = sh.sD[2 * pos];
                out[pos + 1] = sh.sD[2 * pos + 1];
            }
        } else {  // second column of a 2x2
            const int to = sh.order[pos - 1];
            if (pi > pos) out[pi] = colptr(to)[i] * sh.sInv[2 * (pos - 1) + 1] + col[i] * sh.sInv[2 * (pos - 1) + 2];
            if (i == 0) out[pos] = sh.sD[2 * pos];
        }
    }
    if (rank == 0) {
        for (int k = tid; k < p; k += kT) {
            a.perm[k] = sh.order[k];
            a.piv[k] = sh.kind[k];
            a.D[2 * k] = sh.sD[2 * k];
            a.D[2 * k + 1] = sh.sD[2 * k + 1];
            a.Dinv[2 * k] = sh.sInv[2 * k];
            a.Dinv[2 * k + 1] = sh.sInv[2 * k + 1];
        }
        if (tid == 0) *a.nelim = e;
    }
    team.sync();  // no CTA leaves while its shared memory may still be read
}

__global__ void __launch_bounds__(kT, 1) k_factor_cluster(FactorArgs a, int G) { factor_body<false>(a, G); }
__global__ void __launch_bounds__(kT, 1) k_factor_cta(FactorArgs a) { factor_body<true>(a, 1); }

// The arguments of front f of a batch, from its descriptor and its workspace
// section.
__device__ __forceinline__ FactorArgs batch_args(const ctp_front *__restrict__ fronts,
                                                 const BFront *__restrict__ tab, char *ws, int f,
                                                 const BatchOpts &o) {
    const ctp_front fr = fronts[f];
    const BFront bt = tab[f];
    ctp_options oo;
    oo.pivot = o.pivot;
    oo.smode = o.smode;
    oo.prec = o.prec;
    const BSection sec = bsection(bt.n, bt.p, &oo);
    char *base = ws + bt.ws;
    FactorArgs a;
    a.A = fr.A;
    a.lda = fr.lda;
    a.p = bt.p;
    a.R = o.pivot == CTP_PIV_STRICT ? bt.p : 0;
    a.abs_update = o.pivot == CTP_PIV_STRICT ? 1 : 0;
    a.C = reinterpret_cast<const double *>(base + sec.C);
    a.u = o.u;
    a.small = o.small;
    a.perm = fr.perm;
    a.piv = fr.piv;
    a.nelim = fr.nelim;
    a.D = fr.D;
    a.Dinv = reinterpret_cast<double *>(base + sec.Dinv);
    a.info = reinterpret_cast<int32_t *>(base + sec.info);
    a.rowbits = o.pivot == CTP_PIV_STRICT ? reinterpret_cast<const uint32_t *>(base + sec.nz) : nullptr;
    return a;
}

// Batched: cluster c (or CTA c) factors front list[c].
__global__ void __launch_bounds__(kT, 1)
    k_factor_cluster_batch(const ctp_front *__restrict__ fronts, const BFront *__restrict__ tab,
                           char *ws, const int *__restrict__ list, BatchOpts o, int G) {
    factor_body<false>(batch_args(fronts, tab, ws, list[blockIdx.x / G], o), G);
}
__global__ void __launch_bounds__(kT, 1)
    k_factor_cta_batch(const ctp_front *__restrict__ fronts, const BFront *__restrict__ tab, char *ws,
                       const int *__restrict__ list, BatchOpts o) {
    factor_body<true>(batch_args(fronts, tab, ws, list[blockIdx.x], o), 1);
}

// ---------------------------------------------------------------------------
// One warp per front (p <= 32, at most 64 rows of [A11; C]): Listing 1 one
// candidate at a time, lanes over rows, no barrier beyond the warp.  Lane k < p
// keeps the record of pivot position k (column, kind, D, D^-1).
__global__ void __launch_bounds__(32 * kWarpFronts)
    k_factor_warp_batch(const ctp_front *__restrict__ fronts, const BFront *__restrict__ tab, char *ws,
                        const int *__restrict__ list, int count, BatchOpts o, int pcap, int ldcap) {
    extern __shared__ __align__(16) double wsm[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * kWarpFronts + w;
    if (item >= count) return;  // the whole warp; nothing below waits on other warps
    const unsigned full = 0xffffffffu;
    const FactorArgs a = batch_args(fronts, tab, ws, list[item], o);
    const int p = a.p;
    double *cols = wsm + (size_t)w * pcap * ldcap;
    // nonzero outer rows, in order (a.R <= p <= 32: one row per lane); lane k
    // holds the C row of outer row k
    bool nz = false;
    if (lane < a.R) {
        if (a.rowbits != nullptr) {
            nz = (a.rowbits[0] >> lane) & 1u;
        } else {
            for (int k = 0; k < p && !nz; k++) nz = nonzero_bits(a.C[(int64_t)lane * p + k]);
        }
    }
    const unsigned nzbits = __ballot_sync(full, nz);
    const int R = __popc(nzbits);
    int myrow = 0;
    {
        unsigned b = nzbits;
        for (int s = 0; s < lane && b; s++) b &= b - 1;
        if (b) myrow = __ffs(b) - 1;
    }
    const int LD = p + R;
    bool nonfinite = false;
    for (int c = 0; c < p; c++)
        for (int i0 = 0; i0 < LD; i0 += 32) {  // the same trip count on every lane
            const int i = i0 + lane;
            const int r = __shfl_sync(full, myrow, (i - p) & 31);
            if (i < LD) {
                const double v = (i < p) ? ((i >= c) ? a.A[(int64_t)c * a.lda + i] : a.A[(int64_t)i * a.lda + c])
                                         : a.C[(int64_t)r * p + c];
                nonfinite |= nonfinite_bits(v);
                cols[(size_t)c * LD + i] = v;
            }
        }
    if (__any_sync(full, nonfinite) && lane == 0) atomicCAS(a.info, kInfoOk, (int32_t)CTP_ENONFINITE);
    __syncwarp();

    const double u = a.u, rcp_u = __drcp_rn(a.u);
    const unsigned long long small_k = akey(a.small);
    const bool abs_rows = a.abs_update != 0;
    BitLive live;
    live.bits = p >= 32 ? full : ((1u << p) - 1u);
    // record of pivot position `lane`
    int r_order = 0, r_kind = CTP_PIVKIND_DELAYED;
    double r_d0 = 0.0, r_d1 = 0.0, r_i0 = 0.0, r_i1 = 0.0;
    int nelim = 0, m = (p >= 2) ? 1 : 0, accepted = 0;
    auto colptr = [&](int c) -> const double * { return cols + (size_t)c * LD; };
    for (;;) {
        if (nelim >= p) break;
        while (m < p && !live[m]) m++;
        if (m >= p) {
            if (!accepted) break;  // a whole sweep without a pivot: stop
            accepted = 0;
            m = 0;
            continue;
        }
        const Decision dv = test_candidate(m, colptr(m), colptr, live, p, LD, u, rcp_u, small_k);
        if (dv.kind == DEC_REJECT) {
            m++;
            continue;
        }
        if (dv.kind == DEC_ZERO) {
            if (lane == nelim) {
                r_order = m;
                r_kind = CTP_PIVKIND_ZERO;
            }
            live.bits &= ~(1u << m);
            nelim++;
            accepted = 1;
            m++;
            continue;
        }
        const int q0 = (dv.kind == DEC_2X2) ? dv.t : dv.m;
        const int q1 = (dv.kind == DEC_2X2) ? dv.m : -1;
        const double *p0 = colptr(q0);
        const double *p1 = q1 >= 0 ? colptr(q1) : p0;
        unsigned upd_cols = live.bits & ~(1u << q0);
        if (q1 >= 0) upd_cols &= ~(1u << q1);
        const unsigned rows_live = upd_cols;  // the live A11 rows after this pivot
        // row multipliers of this lane's rows (the same arithmetic as factor_body)
        double l0[2] = {0.0, 0.0}, l1[2] = {0.0, 0.0};  // signed: -l normal rows, +l abs rows
        const double ad0 = abs_bits(dv.d0), ai0 = abs_bits(dv.i0), ai1 = abs_bits(dv.i1), ai2 = abs_bits(dv.i2);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int i = lane + 32 * h;
            if (i < LD) {
                const bool ab = abs_rows && i >= p;
                const double x = p0[i];
                if (q1 < 0) {
                    const double l = __ddiv_rn(x, ab ? ad0 : dv.d0);
                    l0[h] = ab ? l : neg_bits(l);
                } else {
                    const double y = p1[i];
                    const double i11 = ab ? ai0 : dv.i0, i21 = ab ? ai1 : dv.i1, i22 = ab ? ai2 : dv.i2;
                    const double a0 = __dadd_rn(__dmul_rn(x, i11), __dmul_rn(y, i21));
                    const double a1 = __dadd_rn(__dmul_rn(x, i21), __dmul_rn(y, i22));
                    l0[h] = ab ? a0 : neg_bits(a0);
                    l1[h] = ab ? a1 : neg_bits(a1);
                }
            }
        }
        // |pivot entry| of A11 row `lane` (p <= 32)
        const double ap0 = lane < p ? abs_bits(p0[lane]) : 0.0, ap1 = lane < p ? abs_bits(p1[lane]) : 0.0;
        // the update, column by column, lanes over rows (the pivot columns are
        // only read); above the diagonal from the mirror's operands (row c's
        // multipliers, row i's pivot entries), as in factor_body
        while (upd_cols) {
            const int c = __ffs(upd_cols) - 1;
            upd_cols &= upd_cols - 1;
            double *col = cols + (size_t)c * LD;
            const double lc0 = __shfl_sync(full, l0[0], c), lc1 = __shfl_sync(full, l1[0], c);  // row c's
            const double ac0 = __shfl_sync(full, ap0, c), ac1 = __shfl_sync(full, ap1, c);   // |a(c, q)|
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int i = lane + 32 * h;
                if (i >= LD || (i < p && !((rows_live >> i) & 1u))) continue;
                const bool up = i < c, ab = abs_rows && i >= p;  // eq. (4.3) for abs rows
                const double m0 = up ? lc0 : l0[h], m1 = up ? lc1 : l1[h];
                const double b0 = up ? p0[i] : (ab ? ac0 : p0[c]), b1 = up ? p1[i] : (ab ? ac1 : p1[c]);
                double v = fma(m0, b0, col[i]);
                if (q1 >= 0) v = fma(m1, b1, v);
                col[i] = v;
            }
        }
        __syncwarp();
        if (q1 < 0) {
            if (lane == nelim) {
                r_order = q0;
                r_kind = CTP_PIVKIND_1X1;
                r_d0 = dv.d0;
                r_i0 = dv.i0;
            }
            live.bits &= ~(1u << q0);
            nelim++;
        } else {
            if (lane == nelim) {
                r_order = q0;
                r_kind = CTP_PIVKIND_2X2_FIRST;
                r_d0 = dv.d0;
                r_d1 = dv.d1;
                r_i0 = dv.i0;
                r_i1 = dv.i1;
            }
            if (lane == nelim + 1) {
                r_order = q1;
                r_kind = CTP_PIVKIND_2X2_SECOND;
                r_d0 = dv.d2;
                r_i0 = dv.i2;
            }
            live.bits &= ~((1u << q0) | (1u << q1));
            nelim += 2;
        }
        accepted = 1;
        m = dv.m + 1;
    }
    // the delayed columns after the pivots, in original order
    {
        const unsigned rest = live.bits;
        const int k = lane - nelim;  // this lane's rank among the delayed positions
        if (k >= 0 && k < __popc(rest)) {
            unsigned b = rest;
            for (int s = 0; s < k; s++) b &= b - 1;
            r_order = __ffs(b) - 1;
            r_kind = CTP_PIVKIND_DELAYED;
        }
    }
    // output position of column `lane`
    int pos_c = 0;
    for (int k = 0; k < p; k++)
        if (__shfl_sync(full, r_order, k) == lane) pos_c = k;
    // write back the A11 block in pivot order (lower triangle): lane i takes
    // source row i, which goes to output row pos_c
    for (int pos = 0; pos < p; pos++) {
        const int c = __shfl_sync(full, r_order, pos);
        const int kd = __shfl_sync(full, r_kind, pos);
        const double sd0 = __shfl_sync(full, r_d0, pos), sd1 = __shfl_sync(full, r_d1, pos);
        const double si0 = __shfl_sync(full, r_i0, pos), si1 = __shfl_sync(full, r_i1, pos);
        const int cnext = __shfl_sync(full, r_order, pos + 1 < p ? pos + 1 : pos);
        const int cprev = __shfl_sync(full, r_order, pos > 0 ? pos - 1 : 0);
        const double prev_i1 = __shfl_sync(full, r_i1, pos > 0 ? pos - 1 : 0);
        const double *col = colptr(c);
        double *out = a.A + (int64_t)pos * a.lda;
        const int i = lane, pi = pos_c;
        if (i < p) {
            if (kd == CTP_PIVKIND_DELAYED) {
                if (pi >= pos) out[pi] = col[i];
            } else if (kd == CTP_PIVKIND_ZERO) {
                if (pi >= pos) out[pi] = 0.0;
            } else if (kd == CTP_PIVKIND_1X1) {
                if (pi > pos) out[pi] = col[i] * si0;
                if (i == 0) out[pos] = sd0;
            } else if (kd == CTP_PIVKIND_2X2_FIRST) {
                if (pi > pos + 1) out[pi] = col[i] * si0 + colptr(cnext)[i] * si1;
                if (i == 0) {
                    out[pos] = sd0;
                    out[pos + 1] = sd1;
                }
            } else {  // second column of a 2x2: D^-1 entries (m,t) and (m,m)
                if (pi > pos) out[pi] = colptr(cprev)[i] * prev_i1 + col[i] * si0;
                if (i == 0) out[pos] = sd0;
            }
        }
    }
    if (lane < p) {
        a.perm[lane] = r_order;
        a.piv[lane] = r_kind;
        // D: (k,k) and, for the first of a 2x2, (k+1,k); D^-1 in the same slots
        const bool first2 = r_kind == CTP_PIVKIND_2X2_FIRST;
        const bool pivot = r_kind == CTP_PIVKIND_1X1 || first2 || r_kind == CTP_PIVKIND_2X2_SECOND;
        a.D[2 * lane] = pivot ? r_d0 : 0.0;
        a.D[2 * lane + 1] = first2 ? r_d1 : 0.0;
        a.Dinv[2 * lane] = pivot ? r_i0 : 0.0;
        a.Dinv[2 * lane + 1] = first2 ? r_i1 : 0.0;
    }
    if (lane == 0) *a.nelim = nelim;
}

}  // namespace

static size_t factor_smem(int p, int R, int G) {
    int ncl = (p + G - 1) / G;
    return sizeof(double) * ((size_t)ncl * (p + R) + 4 * (size_t)(p + R) + 2 * (size_t)p);
}
size_t factor_smem_bytes(int p, int R, int G) { return factor_smem(p, R, G); }
size_t factor_warp_smem_bytes(int pcap, int ldcap) {
    return sizeof(double) * (size_t)kWarpFronts * pcap * ldcap;
}

static cudaError_t launch_factor_cta(const FactorArgs &a, cudaStream_t st) {
    const size_t smem = factor_smem(a.p, a.R, 1);
    cudaError_t err = smem_at_least((const void *)k_factor_cta, smem);
    if (err != cudaSuccess) return err;
    k_factor_cta<<<1, kT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_factor_cluster(const FactorArgs &a, int G_req, cudaStream_t st) {
    // preferred cluster width by p (unless the caller asks for one): more CTAs
    // give more FP64 lanes to the right-looking update, fewer make the cluster
    // barriers cheaper; widen further if the columns do not fit on chip
    int G = G_req > 0 ? G_req : (a.p > 128 ? 16 : (a.p > 64 ? 8 : (a.p > 16 ? 4 : 1)));
    while (factor_smem(a.p, a.R, G) > 160 * 1024 && G < 16) G <<= 1;
    if (G == 1) return launch_factor_cta(a, st);  // one CTA: no cluster
    cudaError_t err;
    if (G > 8) {
        err = cudaFuncSetAttribute(k_factor_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (err != cudaSuccess) return err;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kT, 1, 1);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // fall back to narrower clusters if this one cannot be scheduled
    for (;;) {
        const size_t smem = factor_smem(a.p, a.R, G);
        cfg.gridDim = dim3(G, 1, 1);
        cfg.dynamicSmemBytes = smem;
        attr[0].val.clusterDim.x = G;
        int nclusters = 0;
        err = smem_at_least((const void *)k_factor_cluster, smem);
        if (err == cudaSuccess) err = cudaOccupancyMaxActiveClusters(&nclusters, k_factor_cluster, &cfg);
        if (err == cudaSuccess && nclusters > 0) break;
        (void)cudaGetLastError();
        if (G <= 1 || factor_smem(a.p, a.R, G >> 1) > 160 * 1024)
            return err != cudaSuccess ? err : cudaErrorLaunchOutOfResources;
        G >>= 1;
        if (G == 1) return launch_factor_cta(a, st);
    }
    return cudaLaunchKernelEx(&cfg, k_factor_cluster, a, G);
}

size_t factor_batch_max_dynamic_smem() {
    // per-CTA opt-in limit minus what the batched CTA and cluster kernels hold
    // statically
    static size_t cached = 0;
    if (cached == 0) {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa, fb;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, k_factor_cluster_batch) != cudaSuccess ||
            cudaFuncGetAttributes(&fb, k_factor_cta_batch) != cudaSuccess) {
            (void)cudaGetLastError();
            return 100 * 1024;
        }
        const size_t st = fa.sharedSizeBytes > fb.sharedSizeBytes ? fa.sharedSizeBytes : fb.sharedSizeBytes;
        cached = (size_t)optin > st ? (size_t)optin - st : 0;
    }
    return cached;
}

cudaError_t launch_factor_batch(const ctp_front *fronts, const BFront *tab, char *ws, const int *list,
                                int count, int kind, int G, size_t smem, int pcap, int ldcap, BatchOpts o,
                                cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    cudaError_t err;
    if (kind == kFactorWarp) {
        err = smem_at_least((const void *)k_factor_warp_batch, smem);
        if (err != cudaSuccess) return err;
        const unsigned grid = (unsigned)((count + kWarpFronts - 1) / kWarpFronts);
        k_factor_warp_batch<<<grid, 32 * kWarpFronts, smem, st>>>(fronts, tab, ws, list, count, o, pcap, ldcap);
        return cudaGetLastError();
    }
    if (kind == kFactorCta) {
        err = smem_at_least((const void *)k_factor_cta_batch, smem);
        if (err != cudaSuccess) return err;
        k_factor_cta_batch<<<(unsigned)count, kT, smem, st>>>(fronts, tab, ws, list, o);
        return cudaGetLastError();
    }
    err = smem_at_least((const void *)k_factor_cluster_batch, smem);
    if (err != cudaSuccess) return err;
    if (G > 8) {
        err = cudaFuncSetAttribute(k_factor_cluster_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (err != cudaSuccess) return err;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(count * G), 1, 1);
    cfg.blockDim = dim3(kT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_factor_cluster_batch, fronts, tab, ws, list, o, G);
}

}  // namespace ctp
