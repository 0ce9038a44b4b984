// tpp.cu -- K4: threshold partial pivoting on the whole supernode (Listing 1,
// Section 2), i.e. without compression: every test takes its column maxima over
// all n rows, which must be up to date.  This is the comparator of the
// compressed path.
//
// GB300 design.  One cooperative, persistent launch (all CTAs co-resident) with
// a software grid barrier whose spin is bounded.  Per accepted pivot:
//   decide  CTA 0 runs the tests of Listing 1 on a full symmetric copy of A11
//           (W11, p x p in the workspace) and on the column maxima of the
//           trailing A21 (integer keys of |a|, one per column); rejected
//           candidates change nothing, so it tests windows of 8 candidates (one
//           warp each) and loops until it accepts a pivot or the sweep ends;
//   update  every CTA applies that pivot to its share of all n rows (W11 rows
//           and A21 rows, coalesced along the rows of each column), writes the
//           L21 entries of the pivot column(s), and takes the new column maxima
//           of A21 in the same pass.
// So each accepted pivot costs one pass over the trailing A21 -- the traffic
// the paper's compressed pivoting avoids (Section 6).  At the end the A21
// columns are permuted into pivot order through shared memory and L11 / D /
// the delayed block are written from W11, in the same layout as the compressed
// path.  All grid barriers give up after a bounded number of polls; a timeout
// sets CTP_ETIMEOUT in the info word and every CTA leaves the main loop.
#include "ctp_internal.cuh"

namespace ctp {

namespace {

constexpr int kT = 256;
constexpr int kNW = kT / 32;
constexpr long kBarSpin = 1L << 24;  // default polls of ~100 ns: about a second and a half
constexpr int kTilesPerWarp = 4;     // 32-row tiles a warp keeps pivot values for

enum { D_STOP = -2, D_ZERO = -1, D_REJECT = 0, D_1X1 = 1, D_2X2 = 2 };

struct Dec {
    int kind, t, m, pad;
    double d0, d1, d2, i0, i1, i2;
};

struct Ctl {
    unsigned bar_count, bar_gen;
    int abort, pad0;
    Dec dec;
};

struct TppArgs {
    double *A;
    int64_t lda, n;
    int p;
    double u, small;
    double *W11;                 // p x p, column c at W11 + c*p
    unsigned long long *M21;     // [2][p] column-maximum keys of the trailing A21
    int *live_g;                 // [p] live flags published by CTA 0
    Ctl *ctl;
    int32_t *perm, *piv, *nelim;
    double *D, *Dinv;
    int32_t *info;
    long spin;                   // polls a grid barrier waits before it gives up
};

__device__ __forceinline__ unsigned long long akey(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ double key_val(unsigned long long k) { return __longlong_as_double((long long)k); }
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// software grid barrier for a cooperative launch; false on timeout (more than
// `spin` polls) or when another CTA gave up
__device__ bool grid_sync(Ctl *ctl, int *s_ok, long spin) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *genp = &ctl->bar_gen;
        const unsigned gen = *genp;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
        int ok = 1;
        if (arrived == gridDim.x) {
            ctl->bar_count = 0;
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            long it = 0;
            while (*genp == gen) {
                if (++it > spin) {
                    ok = 0;
                    atomicExch(&ctl->abort, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *s_ok = ok && (*(volatile int *)&ctl->abort == 0);
    }
    __syncthreads();
    return *s_ok != 0;
}

// Listing 1's test_2x2 (readings Q3-Q5), explicitly rounded.
__device__ __forceinline__ bool test_2x2(double a_tt, double a_tm, double a_mm, double maxt,
                                         double maxm, double u, double small, Dec &d) {
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
        double ad = fabs(detpiv);
        double gt = __ddiv_rn(__dmul_rn(__dadd_rn(__dmul_rn(fabs(a_mm), maxt), __dmul_rn(fabs(a_tm), maxm)), detscale), ad);
        double gm = __ddiv_rn(__dmul_rn(__dadd_rn(__dmul_rn(fabs(a_tm), maxt), __dmul_rn(fabs(a_tt), maxm)), detscale), ad);
        double iu = __ddiv_rn(1.0, u);
        ok = (gt <= iu) && (gm <= iu);
    }
    if (ok) {
        d.d0 = a_tt;
        d.d1 = a_tm;
        d.d2 = a_mm;
        d.i0 = __ddiv_rn(__dmul_rn(a_mm, detscale), detpiv);
        d.i1 = __ddiv_rn(__dmul_rn(-a_tm, detscale), detpiv);
        d.i2 = __ddiv_rn(__dmul_rn(a_tt, detscale), detpiv);
    }
    return ok;
}

// Tests of Listing 1 for candidate c (one warp): the A11 part of every column
// maximum comes from W11, the A21 part is the precomputed key M[c].
__device__ Dec test_candidate(int c, const double *W11, const unsigned long long *M,
                              const unsigned char *live, int p, double u, double small) {
    const int lane = threadIdx.x & 31;
    const double *cm = W11 + (size_t)c * p;
    Dec d;
    d.kind = D_REJECT;
    d.t = -1;
    d.m = c;
    d.pad = 0;
    d.d0 = d.d1 = d.d2 = d.i0 = d.i1 = d.i2 = 0.0;
    unsigned long long v = 0;
    for (int i = lane; i < p; i += 32)
        if (live[i]) {
            const unsigned long long k = akey(__ldcg(cm + i));
            v = k > v ? k : v;
        }
    v = warp_max_key(v);
    const unsigned long long mc = M[c];
    if (key_val(v > mc ? v : mc) < small) {
        d.kind = D_ZERO;
        return d;
    }
    unsigned long long bv = 0;
    int bi = -1;
    for (int j = lane; j < c; j += 32)
        if (live[j]) {
            const unsigned long long k = akey(__ldcg(cm + j));
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
    double maxm2 = 0.0;
    if (t >= 0) {
        const double *ct = W11 + (size_t)t * p;
        unsigned long long vm = 0, vt = 0;
        for (int i = lane; i < p; i += 32)
            if (live[i] && i != t && i != c) {
                const unsigned long long km = akey(__ldcg(cm + i)), kt = akey(__ldcg(ct + i));
                vm = km > vm ? km : vm;
                vt = kt > vt ? kt : vt;
            }
        vm = warp_max_key(vm);
        vt = warp_max_key(vt);
        vm = vm > mc ? vm : mc;
        vt = vt > M[t] ? vt : M[t];
        maxm2 = key_val(vm);
        if (test_2x2(__ldcg(ct + t), __ldcg(cm + t), __ldcg(cm + c), key_val(vt), maxm2, u, small, d)) {
            d.kind = D_2X2;
            d.t = t;
            return d;
        }
    }
    double maxm1;
    if (t >= 0) {
        maxm1 = fmax(maxm2, fabs(__ldcg(cm + t)));
    } else {
        unsigned long long w = 0;
        for (int i = lane; i < p; i += 32)
            if (live[i] && i != c) {
                const unsigned long long k = akey(__ldcg(cm + i));
                w = k > w ? k : w;
            }
        w = warp_max_key(w);
        maxm1 = key_val(w > mc ? w : mc);
    }
    const double amm = __ldcg(cm + c);
    if (fabs(amm) >= __dmul_rn(u, maxm1)) {
        d.kind = D_1X1;
        d.d0 = amm;
        d.i0 = __ddiv_rn(1.0, amm);
    }
    return d;
}

struct Cta0 {  // decision state, kept by CTA 0 across rounds
    unsigned char live[kMaxP];
    int order[kMaxP], kind[kMaxP];
    double sD[2 * kMaxP + 2], sInv[2 * kMaxP + 2];
    unsigned long long M[kMaxP];
    int cand[kNW];
    Dec res[kNW];
    int nelim, m, accepted, hi, cstar;
};

__global__ void __launch_bounds__(kT) k_tpp(TppArgs a) {
    extern __shared__ __align__(16) double dsm[];
    __shared__ Cta0 st;
    __shared__ int s_ok;
    __shared__ Dec s_dec;
    const int p = a.p;
    const int64_t n = a.n, m = n - p, lda = a.lda;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned long long *ckey = reinterpret_cast<unsigned long long *>(dsm);  // [p] column maxima
    double *s0 = dsm + p, *s1 = s0 + p;                                       // [p] folded pivot row
    unsigned char *live = reinterpret_cast<unsigned char *>(s1 + p);         // [p]
    Ctl *ctl = a.ctl;

    // ---- phase 0: W11 (full symmetric) and the initial column maxima of A21
    for (int64_t idx = (int64_t)blockIdx.x * kT + tid; idx < (int64_t)p * p; idx += (int64_t)gridDim.x * kT) {
        const int c = (int)(idx / p), i = (int)(idx % p);
        a.W11[idx] = (i >= c) ? a.A[(int64_t)c * lda + i] : a.A[(int64_t)i * lda + c];
    }
    for (int k = tid; k < p; k += kT) ckey[k] = 0;
    __syncthreads();
    bool nonfinite = false;
    {
        const int64_t ntiles = (m + 31) / 32;
        const int64_t gw = (int64_t)blockIdx.x * kNW + warp, nw = (int64_t)gridDim.x * kNW;
        for (int k = 0; k < p; k++) {
            unsigned long long mx = 0;
            for (int64_t tl = gw; tl < ntiles; tl += nw) {
                const int64_t r = tl * 32 + lane;
                if (r < m) {
                    const unsigned long long kk = akey(a.A[(int64_t)k * lda + p + r]);
                    nonfinite |= kk >= 0x7FF0000000000000ull;
                    mx = kk > mx ? kk : mx;
                }
            }
            mx = warp_max_key(mx);
            if (lane == 0 && mx) atomicMax(&ckey[k], mx);
        }
    }
    __syncthreads();
    for (int k = tid; k < p; k += kT)
        if (ckey[k]) atomicMax(&a.M21[k], ckey[k]);
    if (nonfinite) atomicCAS(a.info, kInfoOk, (int32_t)CTP_ENONFINITE);
    if (blockIdx.x == 0) {
        for (int i = tid; i < p; i += kT) {
            st.live[i] = 1;
            a.live_g[i] = 1;
        }
        if (tid == 0) {
            st.nelim = 0;
            st.m = p >= 2 ? 1 : 0;
            st.accepted = 0;
        }
    }
    int round = 0;
    if (!grid_sync(ctl, &s_ok, a.spin)) goto done;

    for (;;) {
        const int cur = round & 1, nxt = cur ^ 1;
        // ---------------- decide (CTA 0)
        if (blockIdx.x == 0) {
            for (int k = tid; k < p; k += kT) {
                st.M[k] = __ldcg(&a.M21[cur * p + k]);
                a.M21[nxt * p + k] = 0;  // next maxima start from zero
            }
            __syncthreads();
            Dec out;
            out.kind = D_STOP;
            for (;;) {
                // uniform control state read by all threads
                int nl = st.nelim, mm = st.m;
                if (nl >= p) break;
                while (mm < p && !st.live[mm]) mm++;
                if (mm >= p) {
                    if (!st.accepted) break;
                    __syncthreads();
                    if (tid == 0) {
                        st.accepted = 0;
                        st.m = 0;
                    }
                    __syncthreads();
                    continue;
                }
                if (tid == 0) {
                    int k = 0, hi = p;
                    for (int c = mm; c < p; c++) {
                        if (!st.live[c]) continue;
                        if (k < kNW)
                            st.cand[k++] = c;
                        else {
                            hi = c;
                            break;
                        }
                    }
                    for (int w = k; w < kNW; w++) st.cand[w] = -1;
                    st.hi = hi;
                }
                __syncthreads();
                {
                    const int c = st.cand[warp];
                    if (c >= 0) {
                        Dec d = test_candidate(c, a.W11, st.M, st.live, p, a.u, a.small);
                        if (lane == 0) st.res[warp] = d;
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    int cs = -1;
                    for (int w = 0; w < kNW; w++)
                        if (st.cand[w] >= 0 && st.res[w].kind != D_REJECT) {
                            cs = w;
                            break;
                        }
                    st.cstar = cs;
                    if (cs < 0) {
                        st.m = st.hi;
                    } else {
                        const Dec d = st.res[cs];
                        const int e = st.nelim;
                        st.accepted = 1;
                        st.m = d.m + 1;
                        if (d.kind == D_ZERO) {
                            st.live[d.m] = 0;
                            st.order[e] = d.m;
                            st.kind[e] = CTP_PIVKIND_ZERO;
                            st.sD[2 * e] = st.sD[2 * e + 1] = 0.0;
                            st.sInv[2 * e] = st.sInv[2 * e + 1] = 0.0;
                            st.nelim = e + 1;
                        } else if (d.kind == D_1X1) {
                            st.live[d.m] = 0;
                            st.order[e] = d.m;
                            st.kind[e] = CTP_PIVKIND_1X1;
                            st.sD[2 * e] = d.d0;
                            st.sD[2 * e + 1] = 0.0;
                            st.sInv[2 * e] = d.i0;
                            st.sInv[2 * e + 1] = 0.0;
                            st.nelim = e + 1;
                        } else {
                            st.live[d.t] = 0;
                            st.live[d.m] = 0;
                            st.order[e] = d.t;
                            st.order[e + 1] = d.m;
                            st.kind[e] = CTP_PIVKIND_2X2_FIRST;
                            st.kind[e + 1] = CTP_PIVKIND_2X2_SECOND;
                            st.sD[2 * e] = d.d0;
                            st.sD[2 * e + 1] = d.d1;
                            st.sD[2 * e + 2] = d.d2;
                            st.sD[2 * e + 3] = 0.0;
                            st.sInv[2 * e] = d.i0;
                            st.sInv[2 * e + 1] = d.i1;
                            st.sInv[2 * e + 2] = d.i2;
                            st.sInv[2 * e + 3] = 0.0;
                            st.nelim = e + 2;
                        }
                    }
                }
                __syncthreads();
                const int cs = st.cstar;
                if (cs >= 0 && st.res[cs].kind != D_ZERO) {
                    out = st.res[cs];
                    break;
                }
            }
            if (out.kind == D_STOP) {
                // publish the pivot order: accepted pivots, then delayed columns in order
                if (tid == 0) {
                    int k = st.nelim;
                    for (int c = 0; c < p; c++)
                        if (st.live[c]) {
                            st.order[k] = c;
                            st.kind[k] = CTP_PIVKIND_DELAYED;
                            st.sD[2 * k] = st.sD[2 * k + 1] = 0.0;
                            st.sInv[2 * k] = st.sInv[2 * k + 1] = 0.0;
                            k++;
                        }
                    *a.nelim = st.nelim;
                }
                __syncthreads();
                for (int k = tid; k < p; k += kT) {
                    a.perm[k] = st.order[k];
                    a.piv[k] = st.kind[k];
                    a.D[2 * k] = st.sD[2 * k];
                    a.D[2 * k + 1] = st.sD[2 * k + 1];
                    a.Dinv[2 * k] = st.sInv[2 * k];
                    a.Dinv[2 * k + 1] = st.sInv[2 * k + 1];
                }
            }
            for (int k = tid; k < p; k += kT) a.live_g[k] = st.live[k];
            if (tid == 0) ctl->dec = out;
        }
        if (!grid_sync(ctl, &s_ok, a.spin)) break;
        if (tid == 0) {
            volatile Dec *vd = &ctl->dec;
            s_dec.kind = vd->kind;
            s_dec.t = vd->t;
            s_dec.m = vd->m;
            s_dec.i0 = vd->i0;
            s_dec.i1 = vd->i1;
            s_dec.i2 = vd->i2;
        }
        __syncthreads();
        const Dec dv = s_dec;
        if (dv.kind == D_STOP) break;

        // ---------------- update: every row of [W11; A21] against the pivot
        const int q0 = dv.kind == D_2X2 ? dv.t : dv.m;
        const int q1 = dv.kind == D_2X2 ? dv.m : -1;
        for (int k = tid; k < p; k += kT) {
            live[k] = (unsigned char)__ldcg(&a.live_g[k]);
            const double b0 = __ldcg(&a.W11[(size_t)q0 * p + k]);
            if (q1 < 0) {
                s0[k] = b0 * dv.i0;
                s1[k] = 0.0;
            } else {
                const double b1 = __ldcg(&a.W11[(size_t)q1 * p + k]);
                s0[k] = dv.i0 * b0 + dv.i1 * b1;
                s1[k] = dv.i1 * b0 + dv.i2 * b1;
            }
            ckey[k] = 0;
        }
        __syncthreads();
        {
            // rows 0..p-1 are W11 rows, rows p..n-1 are A21 rows (A21 row r-p is
            // at A + r); warp gw owns 32-row tiles gw, gw + nw, ...
            const int64_t ntiles = (n + 31) / 32;
            const int64_t gw = (int64_t)blockIdx.x * kNW + warp, nw = (int64_t)gridDim.x * kNW;
            for (int64_t t0 = gw; t0 < ntiles; t0 += nw * kTilesPerWarp) {
                double x0[kTilesPerWarp], x1[kTilesPerWarp];
                bool act[kTilesPerWarp], isw[kTilesPerWarp];
                int64_t rr[kTilesPerWarp];
#pragma unroll
                for (int q = 0; q < kTilesPerWarp; q++) {
                    const int64_t r = (t0 + (int64_t)q * nw) * 32 + lane;
                    rr[q] = r;
                    isw[q] = r < p;
                    act[q] = r < n && (r >= p || (live[r] && r != q0 && r != q1));
                    x0[q] = x1[q] = 0.0;
                    if (act[q]) {
                        const double *src0 = isw[q] ? a.W11 + (size_t)q0 * p + r : a.A + (int64_t)q0 * lda + r;
                        x0[q] = __ldcg(src0);
                        if (q1 >= 0) {
                            const double *src1 = isw[q] ? a.W11 + (size_t)q1 * p + r : a.A + (int64_t)q1 * lda + r;
                            x1[q] = __ldcg(src1);
                        }
                    }
                }
                for (int k = 0; k < p; k++) {
                    if (!live[k] || k == q0 || k == q1) continue;
                    const double sk0 = s0[k], sk1 = s1[k];
                    unsigned long long mx = 0;
#pragma unroll
                    for (int q = 0; q < kTilesPerWarp; q++) {
                        if (!act[q]) continue;
                        double *dst = isw[q] ? a.W11 + (size_t)k * p + rr[q] : a.A + (int64_t)k * lda + rr[q];
                        const double v = __ldcg(dst) - (x0[q] * sk0 + x1[q] * sk1);
                        *dst = v;
                        if (!isw[q]) {
                            const unsigned long long kk = akey(v);
                            mx = kk > mx ? kk : mx;
                        }
                    }
                    mx = warp_max_key(mx);
                    if (lane == 0 && mx) atomicMax(&ckey[k], mx);
                }
                // L21 entries of the pivot column(s) in place (A21 rows only)
#pragma unroll
                for (int q = 0; q < kTilesPerWarp; q++) {
                    if (!act[q] || isw[q]) continue;
                    if (q1 < 0) {
                        a.A[(int64_t)q0 * lda + rr[q]] = x0[q] * dv.i0;
                    } else {
                        a.A[(int64_t)q0 * lda + rr[q]] = x0[q] * dv.i0 + x1[q] * dv.i1;
                        a.A[(int64_t)q1 * lda + rr[q]] = x0[q] * dv.i1 + x1[q] * dv.i2;
                    }
                }
            }
        }
        __syncthreads();
        for (int k = tid; k < p; k += kT)
            if (ckey[k]) atomicMax(&a.M21[nxt * p + k], ckey[k]);
        round++;
        if (!grid_sync(ctl, &s_ok, a.spin)) break;
    }

done:
    if (*(volatile int *)&ctl->abort) {
        if (blockIdx.x == 0 && tid == 0) atomicCAS(a.info, kInfoOk, (int32_t)CTP_ETIMEOUT);
        return;
    }
    // ---- output: A21 columns into pivot order (zero pivots give zero columns),
    // then the A11 block from W11 (frozen pivot columns, delayed Schur block)
    {
        double *tile = dsm + 3 * p + (p + 64) / 8;  // [p][33]
        int *sperm = reinterpret_cast<int *>(tile + (size_t)p * 33);
        int *spiv = sperm + p;
        for (int k = tid; k < p; k += kT) {
            sperm[k] = __ldcg(&a.perm[k]);
            spiv[k] = __ldcg(&a.piv[k]);
        }
        __syncthreads();
        const int64_t ntiles = (m + 31) / 32;
        for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
            const int64_t r = tl * 32 + lane;
            for (int k = warp; k < p; k += kNW) tile[k * 33 + lane] = (r < m) ? __ldcg(a.A + (int64_t)k * lda + p + r) : 0.0;
            __syncthreads();
            if (r < m)
                for (int pos = warp; pos < p; pos += kNW)
                    a.A[(int64_t)pos * lda + p + r] = spiv[pos] == CTP_PIVKIND_ZERO ? 0.0 : tile[sperm[pos] * 33 + lane];
            __syncthreads();
        }
    }
    {
        int *sperm = reinterpret_cast<int *>(dsm + 3 * p + (p + 64) / 8 + (size_t)p * 33);
        int *spiv = sperm + p;
        int *pos_of = spiv + p;
        for (int k = tid; k < p; k += kT) pos_of[sperm[k]] = k;
        __syncthreads();
        for (int c = blockIdx.x; c < p; c += gridDim.x) {
            const int pos = pos_of[c];
            const int kd = spiv[pos];
            const double *col = a.W11 + (size_t)c * p;
            double *out = a.A + (int64_t)pos * lda;
            if (kd == CTP_PIVKIND_DELAYED) {
                for (int i = tid; i < p; i += kT)
                    if (pos_of[i] >= pos) out[pos_of[i]] = __ldcg(col + i);
            } else if (kd == CTP_PIVKIND_ZERO) {
                for (int i = tid; i < p; i += kT)
                    if (pos_of[i] >= pos) out[pos_of[i]] = 0.0;
            } else if (kd == CTP_PIVKIND_1X1) {
                const double inv = __ldcg(&a.Dinv[2 * pos]);
                for (int i = tid; i < p; i += kT)
                    if (pos_of[i] > pos) out[pos_of[i]] = __ldcg(col + i) * inv;
                if (tid == 0) out[pos] = __ldcg(&a.D[2 * pos]);
            } else if (kd == CTP_PIVKIND_2X2_FIRST) {
                const double *cmo = a.W11 + (size_t)sperm[pos + 1] * p;
                const double i11 = __ldcg(&a.Dinv[2 * pos]), i21 = __ldcg(&a.Dinv[2 * pos + 1]);
                for (int i = tid; i < p; i += kT)
                    if (pos_of[i] > pos + 1) out[pos_of[i]] = __ldcg(col + i) * i11 + __ldcg(cmo + i) * i21;
                if (tid == 0) {
                    out[pos] = __ldcg(&a.D[2 * pos]);
                    out[pos + 1] = __ldcg(&a.D[2 * pos + 1]);
                }
            } else {
                const double *cto = a.W11 + (size_t)sperm[pos - 1] * p;
                const double i21 = __ldcg(&a.Dinv[2 * (pos - 1) + 1]), i22 = __ldcg(&a.Dinv[2 * (pos - 1) + 2]);
                for (int i = tid; i < p; i += kT)
                    if (pos_of[i] > pos) out[pos_of[i]] = __ldcg(cto + i) * i21 + __ldcg(col + i) * i22;
                if (tid == 0) out[pos] = __ldcg(&a.D[2 * pos]);
            }
        }
    }
}

}  // namespace

size_t tpp_ws_bytes(int p) {
    return 256 + align256(sizeof(double) * (size_t)p * p) + align256(2 * sizeof(unsigned long long) * (size_t)p) +
           align256(sizeof(int) * (size_t)p);
}

static size_t tpp_smem(int p) {
    // ckey, s0, s1 (3p doubles), live (p bytes, padded), tile [p][33], perm/piv/pos_of
    return sizeof(double) * (3 * (size_t)p + (p + 64) / 8 + (size_t)p * 33) + 3 * sizeof(int) * (size_t)p;
}

cudaError_t launch_tpp(double *A, int64_t n, int p, int64_t lda, double u, double small, void *ws,
                       int32_t *perm, int32_t *piv, double *D, double *Dinv, int32_t *nelim,
                       int32_t *info, int num_sms, int spin, cudaStream_t st) {
    char *w = static_cast<char *>(ws);
    TppArgs a;
    a.spin = spin > 0 ? (long)spin : kBarSpin;
    a.A = A;
    a.lda = lda;
    a.n = n;
    a.p = p;
    a.u = u;
    a.small = small;
    a.ctl = reinterpret_cast<Ctl *>(w);
    a.W11 = reinterpret_cast<double *>(w + 256);
    a.M21 = reinterpret_cast<unsigned long long *>(w + 256 + align256(sizeof(double) * (size_t)p * p));
    a.live_g = reinterpret_cast<int *>(reinterpret_cast<char *>(a.M21) +
                                       align256(2 * sizeof(unsigned long long) * (size_t)p));
    a.perm = perm;
    a.piv = piv;
    a.nelim = nelim;
    a.D = D;
    a.Dinv = Dinv;
    a.info = info;
    cudaError_t err = cudaMemsetAsync(w, 0, 256, st);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(a.M21, 0, 2 * sizeof(unsigned long long) * (size_t)p, st);
    if (err != cudaSuccess) return err;
    const size_t smem = tpp_smem(p);
    err = smem_at_least((const void *)k_tpp, smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tpp, kT, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    if (per_sm > 2) per_sm = 2;
    dim3 grid(num_sms * per_sm), block(kT);
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((void *)k_tpp, grid, block, args, smem, st);
}

}  // namespace ctp
