// factor.cu -- K3: pivot selection on [A11; C] by Listing 1 (Section 2) in FP64,
// with the worst-case update of the strict compressed matrix (eq. (4.3); the
// 2x2 form follows the proof of Theorem 5.2).
//
// GB300 design.  The working matrix [A11; C] (A11 held in full symmetric form so
// that every column carries all of its entries, C the R = p outer rows) is
// 2p x p doubles -- 1 MB at p = 256, far beyond one SM -- and GB300's FP64 pipe
// is narrow, so the right-looking updates must be spread over many SMs.  One
// thread-block cluster of G CTAs owns the matrix: column c lives in the shared
// memory of CTA (c mod G); partner columns are read through distributed shared
// memory (DSMEM).
//
// Listing 1 is sequential, but a rejected candidate leaves the matrix unchanged,
// so every candidate tested between two acceptances sees the same matrix.  The
// kernel therefore tests a window of candidates at once (one warp per candidate,
// every CTA its own columns) and accepts the lowest-index candidate that passes;
// all candidates before it in the window were rejected by Listing 1 as well.
// A round costs one cluster barrier, plus one for the update when a pivot is
// accepted, instead of one barrier per test:
//   test round   each warp runs the zero test, the 2x2 test with its partner t
//                (largest |a(m, j)| over live j < m) and the 1x1 test for one
//                candidate; results are published as a bit mask per CTA;
//   update       every CTA copies the pivot column(s) over DSMEM and applies the
//                1x1 or 2x2 update to its own live columns.
// Columns are never moved: accepted pivots leave the live set, and because the
// paper's stable shift never reorders the remaining columns, the candidate
// order is simply the original column order of the live columns.  The final
// pivot order (accepted pivots in acceptance order, then the delayed columns in
// original order) is applied only when the factor is written back.
//
// Determinism: every CTA holds the same replicated control state (live flags,
// nelim, m) and executes the same sequence of barriers.  The test arithmetic
// uses explicitly rounded operations (no FMA contraction) so that it matches
// the plain-CPU formulas up to the rounding of the inputs.
#include <cooperative_groups.h>

#include "ctp_internal.cuh"

namespace cg = cooperative_groups;

namespace ctp {

namespace {

constexpr int kT = 256;  // threads per CTA
constexpr int kNW = kT / 32;

enum { DEC_REJECT = 0, DEC_1X1 = 1, DEC_2X2 = 2, DEC_ZERO = -1 };

struct Decision {
    int kind, t, m, pad;
    double d0, d1, d2;  // 1x1: d0 = d; 2x2: a_tt, a_tm, a_mm
    double i0, i1, i2;  // 1x1: i0 = 1/d; 2x2: D^-1 entries (t,t), (m,t), (m,m)
};

struct Shared {
    Decision res[2][kMaxP];  // per own column slot (ncl <= kMaxP), double-buffered
    Decision cur;
    unsigned int mask[2][kMaxP / 32];  // passing candidates, by global column index
    int hi[2];                         // first own candidate not tested this round
    unsigned char live[kMaxP];
    int order[kMaxP];
    int kind[kMaxP];
    int pos_of[kMaxP];
    double sD[2 * kMaxP + 2];
    double sInv[2 * kMaxP + 2];
    int cand[kNW];
    int cstar, hiall;
    int rowmap[kMaxP];  // nonzero outer rows
    int nz_count;
    unsigned char nzflag[kMaxP];
};

// Listing 1's test_2x2 with the nonsingularity/cancellation guard and the growth
// test of eq. (2.2), |D^-1| (maxt, maxm)^T <= 1/u.  Fills d on acceptance.
__device__ __forceinline__ bool test_2x2(double a_tt, double a_tm, double a_mm, double maxt,
                                         double maxm, double u, double small, Decision &d) {
    double amax = fmax(fabs(a_tt), fmax(fabs(a_tm), fabs(a_mm)));
    if (amax < small) return false;
    double detscale = __ddiv_rn(1.0, amax);
    double detpiv1 = __dmul_rn(__dmul_rn(a_tm, detscale), a_tm);
    double detpiv0 = __dmul_rn(__dmul_rn(a_mm, detscale), a_tt);
    double detpiv = __dsub_rn(detpiv0, detpiv1);
    double guard = fmax(small, fmax(0.5 * fabs(detpiv0), 0.5 * fabs(detpiv1)));
    if (fabs(detpiv) <= guard) return false;
    bool ok;
    if (fmax(maxm, maxt) < small) {
        ok = true;
    } else {
        // |D^-1| (maxt, maxm)^T <= 1/u, each row compared as num*detscale <= |detpiv|/u
        // (the quotient form of the test, without FP64 divisions)
        const double lim = __dmul_rn(fabs(detpiv), __drcp_rn(u));
        const double gt = __dmul_rn(__dadd_rn(__dmul_rn(fabs(a_mm), maxt), __dmul_rn(fabs(a_tm), maxm)), detscale);
        const double gm = __dmul_rn(__dadd_rn(__dmul_rn(fabs(a_tm), maxt), __dmul_rn(fabs(a_tt), maxm)), detscale);
        ok = (gt <= lim) && (gm <= lim);
    }
    if (ok) {
        const double rdet = __ddiv_rn(detscale, detpiv);
        d.d0 = a_tt;
        d.d1 = a_tm;
        d.d2 = a_mm;
        d.i0 = __dmul_rn(a_mm, rdet);
        d.i1 = __dmul_rn(-a_tm, rdet);
        d.i2 = __dmul_rn(a_tt, rdet);
    }
    return ok;
}

__device__ __forceinline__ unsigned long long akey(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}
__device__ __forceinline__ double key_val(unsigned long long k) {
    return __longlong_as_double((long long)k);
}

// The tests of Listing 1 for candidate c (one warp): zero test, 2x2 with the
// partner t, 1x1, from two scans of the column (the partner, then the maxima).
// cm is the candidate's column (rows 0..p-1 A11, then outer).
// Column maxima of |a| are taken on the IEEE bit patterns with the sign cleared
// (integer order = magnitude order), which keeps the scans off the FP64 pipe.
template <typename ColPtr>
__device__ __forceinline__ Decision test_candidate(int c, const double *cm, ColPtr colptr,
                                                   const unsigned char *live, int p, int LD,
                                                   double u, double small) {
    const int lane = threadIdx.x & 31;
    Decision d;
    d.kind = DEC_REJECT;
    d.t = -1;
    d.m = c;
    d.pad = 0;
    d.d0 = d.d1 = d.d2 = d.i0 = d.i1 = d.i2 = 0.0;
    // partner t: largest |a(c, j)| over live j < c, lowest j on ties
    unsigned long long bv = 0;
    int bi = -1;
    for (int j = lane; j < c; j += 32)
        if (live[j]) {
            const unsigned long long k = akey(cm[j]);
            if (bi < 0 || k > bv) {
                bv = k;
                bi = j;
            }
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) {
            bv = ov;
            bi = oi;
        }
    }
    const int t = bi;
    // one pass over the live rows but t and c: the column maximum of c (and of
    // the partner's column); the zero test's maximum over every live row of c
    // adds rows t and c back
    const double *ct = t >= 0 ? colptr(t) : cm;
    unsigned long long vm = 0, vt = 0;
    for (int i = lane; i < LD; i += 32)
        if (i >= p || (live[i] && i != t && i != c)) {
            const unsigned long long km = akey(cm[i]);
            vm = km > vm ? km : vm;
            if (t >= 0) {
                const unsigned long long kt = akey(ct[i]);
                vt = kt > vt ? kt : vt;
            }
        }
    vm = warp_max_key(vm);
    unsigned long long vall = vm > akey(cm[c]) ? vm : akey(cm[c]);
    if (t >= 0 && akey(cm[t]) > vall) vall = akey(cm[t]);
    if (key_val(vall) < small) {
        d.kind = DEC_ZERO;
        return d;
    }
    double maxm1;
    if (t >= 0) {
        const double maxm2 = key_val(vm);
        const double maxt = key_val(warp_max_key(vt));
        if (test_2x2(ct[t], cm[t], cm[c], maxt, maxm2, u, small, d)) {
            d.kind = DEC_2X2;
            d.t = t;
            return d;
        }
        maxm1 = fmax(maxm2, fabs(cm[t]));
    } else {
        maxm1 = key_val(vm);  // the live rows but c
    }
    const double amm = cm[c];
    if (fabs(amm) >= __dmul_rn(u, maxm1)) {
        d.kind = DEC_1X1;
        d.d0 = amm;
        d.i0 = __ddiv_rn(1.0, amm);
    }
    return d;
}

__device__ __forceinline__ void factor_cluster_body(const FactorArgs &a, int G) {
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) double dsm[];
    __shared__ Shared sh;

    const int p = a.p;
    const int rank = (int)cluster.block_rank();
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
    if (a.rowflags != nullptr) {
        for (int j = tid; j < a.R; j += kT) sh.nzflag[j] = a.rowflags[j] != 0 ? 1 : 0;
        if (tid == 0) sh.nz_count = 0;
    } else if (warp == 0) {
        int r = 0;
        for (int j0 = 0; j0 < a.R; j0 += 32) {
            const int j = j0 + lane;
            const bool first = j < a.R && a.C[(int64_t)j * p] != 0.0;
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
            if (a.C[(int64_t)j * p + k] != 0.0) sh.nzflag[j] = 1;
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
    const int ncl = (p + G - 1) / G;
    double *cols = dsm;                    // [ncl][LD]
    double *pc0 = dsm + (size_t)ncl * LD;  // pivot column copies
    double *pc1 = pc0 + LD;
    double *cs0 = pc1 + LD, *cs1 = cs0 + ncl, *cas0 = cs1 + ncl, *cas1 = cas0 + ncl;  // update scalars
    const int nmask = (p + 31) / 32;
    auto colptr = [&](int c) -> const double * {
        return cluster.map_shared_rank(cols, c % G) + (size_t)(c / G) * LD;
    };

    // ---- load: own columns of A11 (full symmetric) and of the nonzero outer rows
    bool nonfinite = false;
    // flattened (column, row) loops step their indices by kT without divisions
    const int dl = kT / LD, di = kT - dl * LD;
    for (int idx = tid, lc = tid / LD, i = tid - (tid / LD) * LD; idx < ncl * LD; idx += kT) {
        const int c = lc * G + rank;
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
        nonfinite |= !isfinite(v);
        cols[idx] = v;
    }
    for (int i = tid; i < p; i += kT) sh.live[i] = 1;
    if (nonfinite) atomicCAS(a.info, kInfoOk, (int32_t)CTP_ENONFINITE);
    cluster.sync();

    const double u = a.u, small = a.small;
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
        // (cluster-wide order); each CTA tests the ones it owns, one per warp.
        // The window is 1 after an acceptance and doubles after a round with no
        // pass, so accepted-first candidates cost a single test and runs of
        // rejections are tested in parallel.
        if (tid < nmask) sh.mask[buf][tid] = 0u;
        if (warp == 0) {
            // the window is the index range [m, m + win) (win <= kNW * G, so no
            // CTA owns more than kNW of its columns); this CTA's live columns in
            // it, in order, go to its warps (one ballot over its column slots)
            const int hi = min(p, m + win);
            const int j0 = m > rank ? (m - rank + G - 1) / G : 0;
            const int c = rank + G * (j0 + lane);
            const bool ok = c < hi && sh.live[c];
            const unsigned int bal = __ballot_sync(0xffffffffu, ok);
            if (ok) sh.cand[__popc(bal & ((1u << lane) - 1u))] = c;
            if (lane >= __popc(bal) && lane < kNW) sh.cand[lane] = -1;
            if (lane == 0) sh.hi[buf] = hi;
        }
        __syncthreads();
        {
            const int c = sh.cand[warp];
            if (c >= 0) {
                Decision d = test_candidate(c, cols + (size_t)(c / G) * LD, colptr, sh.live, p, LD,
                                            u, small);
                if (lane == 0) {
                    sh.res[buf][c / G] = d;
                    if (d.kind != DEC_REJECT) atomicOr(&sh.mask[buf][c >> 5], 1u << (c & 31));
                }
            }
        }
        cluster.sync();
        // lowest passing candidate over the cluster, and the end of the tested
        // window: lane r of warp 0 reads CTA r's mask and window end over DSMEM
        if (warp == 0) {
            int cs = p, h = p;
            if (lane < G) {
                h = *cluster.map_shared_rank(&sh.hi[buf], lane);
                const unsigned int *mk = cluster.map_shared_rank(&sh.mask[buf][0], lane);
                for (int w = 0; w < nmask; w++) {
                    const unsigned int bits = mk[w];
                    if (bits) {
                        cs = w * 32 + __ffs(bits) - 1;
                        break;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                cs = min(cs, __shfl_xor_sync(0xffffffffu, cs, o));
                h = min(h, __shfl_xor_sync(0xffffffffu, h, o));
            }
            if (lane == 0) {
                sh.cstar = cs;
                sh.hiall = h;
                if (cs < h) sh.cur = *cluster.map_shared_rank(&sh.res[buf][cs / G], cs % G);
            }
        }
        __syncthreads();
        const int cstar = sh.cstar;
        if (cstar >= sh.hiall) {
            // every tested candidate before the window's end failed: the sweep
            // continues there, with a wider window
            m = sh.hiall;
            win = win * 2 < win_max ? win * 2 : win_max;
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
            if (tid == 0) {
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
            // after that comes behind the next cluster barrier
            continue;
        }
        // ---------------- update: apply the pivot to the own live columns
        const int q0 = (dv.kind == DEC_2X2) ? dv.t : dv.m;
        const int q1 = (dv.kind == DEC_2X2) ? dv.m : -1;
        {
            const double *s0 = colptr(q0);
            for (int i = tid; i < LD; i += kT) pc0[i] = s0[i];
            if (q1 >= 0) {
                const double *s1 = colptr(q1);
                for (int i = tid; i < LD; i += kT) pc1[i] = s1[i];
            }
        }
        __syncthreads();
        const bool abs_rows = a.abs_update != 0;
        // per own live column: the update's scalars (a column that is not live,
        // or is a pivot column, gets none and is skipped)
        for (int lc = tid; lc < ncl; lc += kT) {
            const int c = lc * G + rank;
            const bool upd = c < p && sh.live[c] && c != q0 && c != q1;
            double s0 = 0.0, s1 = 0.0, as0 = 0.0, as1 = 0.0;
            if (upd && q1 < 0) {
                s0 = pc0[c] * dv.i0;
                as0 = fabs(pc0[c]) * fabs(dv.i0);
            } else if (upd) {
                const double i11 = dv.i0, i21 = dv.i1, i22 = dv.i2;
                const double b0 = pc0[c], b1 = pc1[c];
                s0 = i11 * b0 + i21 * b1;
                s1 = i21 * b0 + i22 * b1;
                const double ab0 = fabs(b0), ab1 = fabs(b1);
                as0 = fabs(i11) * ab0 + fabs(i21) * ab1;
                as1 = fabs(i21) * ab0 + fabs(i22) * ab1;
            }
            cs0[lc] = s0, cs1[lc] = s1, cas0[lc] = as0, cas1[lc] = as1;
            sh.nzflag[lc] = upd ? 1 : 0;
        }
        __syncthreads();
        // the update over (column, row) pairs
        for (int idx = tid, lc2 = tid / LD, i2 = tid - (tid / LD) * LD; idx < ncl * LD; idx += kT) {
            const int lc = lc2, i = i2;
            i2 += di;
            lc2 += dl;
            if (i2 >= LD) {
                i2 -= LD;
                lc2++;
            }
            if (!sh.nzflag[lc]) continue;
            if (i < p && (!sh.live[i] || i == q0 || i == q1)) continue;
            double *e = cols + idx;
            if (q1 < 0) {
                // 1x1: a(i,c) -= a(i,q) (a(c,q) / d); C rows (strict): c += chat |a(c,q)|
                if (i < p || !abs_rows)
                    *e -= pc0[i] * cs0[lc];
                else
                    *e += pc0[i] * cas0[lc];  // eq. (4.3)
            } else {
                // 2x2: a(i,c) -= [a(i,t) a(i,m)] (D^-1 [a(c,t) a(c,m)]^T)
                const double x0 = pc0[i], x1 = pc1[i];
                if (i < p || !abs_rows)
                    *e -= x0 * cs0[lc] + x1 * cs1[lc];
                else
                    *e += x0 * cas0[lc] + x1 * cas1[lc];
            }
        }
        __syncthreads();
        if (tid == 0) {
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
        __syncthreads();
        nelim += (q1 < 0) ? 1 : 2;
        accepted = 1;
        m = cstar + 1;
        cluster.sync();  // every update done before the next tests read columns
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
        const int c = lc * G + rank;
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
            if (pi > pos + 1) {
                const double *cmo = cluster.map_shared_rank(cols, mo % G) + (size_t)(mo / G) * LD;
                out[pi] = col[i] * sh.sInv[2 * pos] + cmo[i] * sh.sInv[2 * pos + 1];
            }
            if (i == 0) {
                out[pos] = sh.sD[2 * pos];
                out[pos + 1] = sh.sD[2 * pos + 1];
            }
        } else {  // second column of a 2x2
            const int to = sh.order[pos - 1];
            if (pi > pos) {
                const double *cto = cluster.map_shared_rank(cols, to % G) + (size_t)(to / G) * LD;
                out[pi] = cto[i] * sh.sInv[2 * (pos - 1) + 1] + col[i] * sh.sInv[2 * (pos - 1) + 2];
            }
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
    cluster.sync();  // no CTA leaves while its shared memory may still be read
}

__global__ void __launch_bounds__(kT, 3) k_factor_cluster(FactorArgs a, int G) { factor_cluster_body(a, G); }

// Batched: cluster c factors front list[c]; its arguments come from the
// front's descriptor and its workspace section.
__global__ void __launch_bounds__(kT, 3)
    k_factor_cluster_batch(const ctp_front *__restrict__ fronts, const BFront *__restrict__ tab,
                           char *ws, const int *__restrict__ list, BatchOpts o, int G) {
    const int f = list[blockIdx.x / G];
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
    a.rowflags = o.pivot == CTP_PIV_STRICT ? reinterpret_cast<const int32_t *>(base + sec.nz) : nullptr;
    factor_cluster_body(a, G);
}

}  // namespace

static size_t factor_smem(int p, int R, int G) {
    int ncl = (p + G - 1) / G;
    return sizeof(double) * ((size_t)ncl * (p + R) + 2 * (size_t)(p + R) + 4 * (size_t)ncl);
}
size_t factor_smem_bytes(int p, int R, int G) { return factor_smem(p, R, G); }

cudaError_t launch_factor_cluster(const FactorArgs &a, int G_req, cudaStream_t st) {
    // preferred cluster width by p (unless the caller asks for one): more CTAs
    // give more FP64 lanes to the right-looking update, fewer make the cluster
    // barriers cheaper; widen further if the columns do not fit on chip
    int G = G_req > 0 ? G_req : (a.p > 128 ? 16 : (a.p > 64 ? 8 : (a.p > 16 ? 4 : 1)));
    while (factor_smem(a.p, a.R, G) > 160 * 1024 && G < 16) G <<= 1;
    size_t smem = factor_smem(a.p, a.R, G);
    cudaError_t err = smem_at_least((const void *)k_factor_cluster, smem);
    if (err != cudaSuccess) return err;
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
        smem = factor_smem(a.p, a.R, G);
        cfg.gridDim = dim3(G, 1, 1);
        cfg.dynamicSmemBytes = smem;
        attr[0].val.clusterDim.x = G;
        int nclusters = 0;
        err = smem_at_least((const void *)k_factor_cluster, smem);
        if (err == cudaSuccess) err = cudaOccupancyMaxActiveClusters(&nclusters, k_factor_cluster, &cfg);
        if (err == cudaSuccess && nclusters > 0) break;
        (void)cudaGetLastError();
        if (G <= 1 || factor_smem(a.p, a.R, G >> 1) > 160 * 1024) return err != cudaSuccess ? err : cudaErrorLaunchOutOfResources;
        G >>= 1;
    }
    return cudaLaunchKernelEx(&cfg, k_factor_cluster, a, G);
}

size_t factor_batch_max_dynamic_smem() {
    // per-CTA opt-in limit minus what the kernel holds statically
    static size_t cached = 0;
    if (cached == 0) {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, k_factor_cluster_batch) != cudaSuccess) {
            (void)cudaGetLastError();
            return 100 * 1024;
        }
        cached = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    }
    return cached;
}

cudaError_t launch_factor_batch(const ctp_front *fronts, const BFront *tab, char *ws,
                                const int *list, int count, int G, int pmax, BatchOpts o,
                                cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const int R = o.pivot == CTP_PIV_STRICT ? pmax : 0;
    const size_t smem = factor_smem(pmax, R, G);
    cudaError_t err = smem_at_least((const void *)k_factor_cluster_batch, smem);
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
