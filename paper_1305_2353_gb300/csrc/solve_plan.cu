// solve_plan.cu -- the level-planned front-list solve and the residual helpers
// of iterative refinement (declared in solve_plan.cuh).
//
// The solve is the front-by-front substitution of system.cu (eq. (1.2) applied
// front by front: y = L11^{-1} b_f, b_rest -= L_rest y, z = D^{-1} y forward;
// x_f = L11^{-T} (z - L_rest^T x_rest) backward), run one level of independent
// panels per launch.  A level's work is cut into items (panel, chunk of 64
// rows below the pivots) so that the FP64 products of a tall panel spread over
// the SMs:
//   forward   every item solves the panel's small triangular system itself
//             (nothing is exchanged between CTAs), subtracts its rows' share
//             from the variables below with atomics, and the panel's first
//             item stores z in a per-panel buffer (not in X: other items of
//             the panel still read b there);
//   backward  every item writes the partial sums L_rest^T x_rest of its rows;
//             the panel's last item to finish (a fenced counter, no waiting)
//             adds them in chunk order and solves with L11^T.
// The sweeps compute in FP64, or in FP32 (the factors, D and X stay FP64 in
// memory and are rounded as they are loaded; X is updated in FP64): the
// correction solves of a refinement whose residuals are FP64 (Section 7) need
// only to contract the error, and GB300's FP32 pipe is many times its FP64 one.
#include "solve_plan.cuh"

namespace ctp {

namespace {

constexpr int kLT = 256;           // threads per item
constexpr int kRC = 64;            // rows below the pivots per item
constexpr int kLJ = 32;            // columns (forward) / rows (backward) of L11 staged at a time
constexpr int kLD = kMaxP + 1;     // padded length of a staged column / row of L11
constexpr int kWork = kLJ * kLD;   // elements of the staging / reduction area

// A panel of the plan.  pvar[q] = rows[perm[q]] (q < p): the variable at
// position q after pivoting; rows[r] for r >= p.  zoff, poff count doubles
// per right-hand side.
struct LvFront {
    const double *L;
    int64_t ldl;
    int64_t n;
    const int32_t *rows;
    const int32_t *pvar;
    const int32_t *piv;
    const double *D;
    int64_t zoff;  // z of the panel: Z[zoff * nrhs + r * e + q]
    int64_t poff;  // partial sums: part[poff * nrhs + (c * nrhs + r) * e + j] (level-local)
    int32_t e, p, nch, pad;
};

template <typename T, int RG>
struct LvShape {
    static constexpr int kRGP = RG == 1 ? 1 : RG + 1;  // padded stride of reduction rows
    // backward: x of the chunk's rows, L columns of the chunk, slice sums
    static constexpr int kChunk = kRC * RG + kLJ * (kRC + 1) + kLT * kRGP;
    static constexpr int kSmall = kLJ * (kLJ + 1);  // L11 of a panel with e <= kLJ, staged once
    static constexpr int kArea = kWork > kChunk + kSmall ? kWork : kChunk + kSmall;
    static constexpr size_t kSmem = sizeof(T) * ((size_t)RG * kMaxP + kArea);
    static_assert(kSmall + 4 * kRC * kRGP <= kArea, "forward reduction area");
};

// Programmatic dependent launch: a level's kernel loads what no earlier kernel
// writes (descriptors, L, pivot kinds) while the previous level runs, then
// waits for it before touching X, Z or the partial sums.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ int row_var(const LvFront &f, int64_t r) {
    return r < f.p ? f.pvar[r] : f.rows[r];
}

// z = D^{-1} y for pivot q (1x1, either column of a 2x2 block, or a zero pivot -> 0).
template <typename T>
__device__ __forceinline__ T d_solve(const LvFront &f, const int *pk, const T *y, int q) {
    const int k = pk[q];
    if (k == CTP_PIVKIND_1X1) return y[q] / (T)f.D[2 * q];
    if (k == CTP_PIVKIND_2X2_FIRST || k == CTP_PIVKIND_2X2_SECOND) {
        const int a = (k == CTP_PIVKIND_2X2_FIRST) ? q : q - 1;
        const T d11 = (T)f.D[2 * a], d21 = (T)f.D[2 * a + 1], d22 = (T)f.D[2 * a + 2];
        const T det = d11 * d22 - d21 * d21;
        return (k == CTP_PIVKIND_2X2_FIRST) ? (d22 * y[a] - d21 * y[a + 1]) / det
                                            : (d11 * y[a + 1] - d21 * y[a]) / det;
    }
    return T(0);
}

// L11(i, j) as the substitutions use it: strictly below the diagonal, except
// the (j+1, j) slot of a 2x2 block, which holds D.
template <typename T>
__device__ __forceinline__ T l11(const LvFront &f, const int *pk, int i, int j) {
    if (i <= j || (i == j + 1 && pk[j] == CTP_PIVKIND_2X2_FIRST)) return T(0);
    return (T)f.L[(int64_t)j * f.ldl + i];
}

template <typename T, int RG>
__global__ void __launch_bounds__(kLT) k_lv_forward(const LvFront *__restrict__ F, const int2 *__restrict__ items,
                                                    double *X, int64_t ldx, int nrhs, T *__restrict__ Z) {
    constexpr int RGP = LvShape<T, RG>::kRGP;
    constexpr int kPre = kLJ / 4;   // update columns per thread loaded before the wait
    extern __shared__ __align__(16) unsigned char lv_smem[];
    T *sm = reinterpret_cast<T *>(lv_smem);
    T *sy = sm;                // [RG][kMaxP]: b, then y, of the pivot variables
    T *wk = sm + RG * kMaxP;   // L11 columns [kLJ][lds]; slice sums [4][kRC][RGP] after kSmall
    T *red = wk + LvShape<T, RG>::kSmall;
    __shared__ int pvar[kMaxP], pk[kMaxP], rvar[kRC];
    const int2 it = items[blockIdx.x];
    const LvFront f = F[it.x];
    const int e = f.e;
    if (e == 0) return;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int64_t rbase = e + (int64_t)it.y * kRC;
    const int nr = (int)max((int64_t)0, min((int64_t)kRC, f.n - rbase));
    const int lds = e <= kLJ ? kLJ + 1 : kLD;
    for (int q = t; q < e; q += kLT) {
        pvar[q] = f.pvar[q];
        pk[q] = f.piv[q];
    }
    if (t < nr) rvar[t] = row_var(f, rbase + t);
    const int rl = t & (kRC - 1), sl = t / kRC;  // this thread's row of the chunk; its slice of the columns
    const double *lp = f.L + rbase + rl;
    T lpre[kPre];  // L(row, sl + 4k)
#pragma unroll
    for (int k = 0; k < kPre; k++) lpre[k] = (rl < nr && sl + 4 * k < e) ? (T)lp[(int64_t)(sl + 4 * k) * f.ldl] : T(0);
    __syncthreads();
    if (e <= kLJ)  // the whole L11 of a small panel, staged once
        for (int idx = t; idx < e * e; idx += kLT) {
            const int jj = idx / e, i = idx - jj * e;
            wk[jj * lds + i] = l11<T>(f, pk, i, jj);
        }
    pdl_trigger();
    pdl_wait();
    for (int g0 = 0; g0 < nrhs; g0 += RG) {
        const int ng = min(RG, nrhs - g0);
        __syncthreads();
        for (int idx = t; idx < ng * e; idx += kLT) {
            const int r = idx / e, q = idx - r * e;
            sy[r * kMaxP + q] = (T)X[(int64_t)(g0 + r) * ldx + pvar[q]];
        }
        // y = L11^{-1} b: warp w takes right-hand sides w, w + 8, ...; lanes take rows
        for (int j0 = 0; j0 < e; j0 += kLJ) {
            const int nj = min(kLJ, e - j0);
            __syncthreads();
            if (e > kLJ) {
                for (int idx = t; idx < nj * e; idx += kLT) {
                    const int jj = idx / e, i = idx - jj * e;
                    wk[jj * lds + i] = l11<T>(f, pk, i, j0 + jj);
                }
                __syncthreads();
            }
            for (int r = warp; r < ng; r += kLT / 32) {
                T *y = sy + r * kMaxP;
                for (int jj = 0; jj < nj; jj++) {
                    const int j = j0 + jj;
                    const T yj = y[j];
                    for (int i = j + 1 + lane; i < e; i += 32) y[i] -= wk[jj * lds + i] * yj;
                    __syncwarp();
                }
            }
        }
        __syncthreads();
        if (it.y == 0)
            for (int idx = t; idx < ng * e; idx += kLT) {
                const int r = idx / e, q = idx - r * e;
                Z[f.zoff * nrhs + (int64_t)(g0 + r) * e + q] = d_solve<T>(f, pk, sy + r * kMaxP, q);
            }
        if (nr == 0) continue;
        // rows below: b(var(row)) -= L(row, 0:e) y; slice sl takes the columns j = sl mod 4
        T acc[RG];
#pragma unroll
        for (int r = 0; r < RG; r++) acc[r] = T(0);
        if (rl < nr) {
#pragma unroll
            for (int k = 0; k < kPre; k++) {
                const int j = sl + 4 * k;
                if (j < e)
#pragma unroll
                    for (int r = 0; r < RG; r++) acc[r] += lpre[k] * sy[r * kMaxP + j];
            }
            int j = sl + 4 * kPre;
            for (; j + 12 < e; j += 16) {
                const T l0 = (T)lp[(int64_t)j * f.ldl], l1 = (T)lp[(int64_t)(j + 4) * f.ldl];
                const T l2 = (T)lp[(int64_t)(j + 8) * f.ldl], l3 = (T)lp[(int64_t)(j + 12) * f.ldl];
#pragma unroll
                for (int r = 0; r < RG; r++) {
                    const T *y = sy + r * kMaxP;
                    acc[r] += l0 * y[j];
                    acc[r] += l1 * y[j + 4];
                    acc[r] += l2 * y[j + 8];
                    acc[r] += l3 * y[j + 12];
                }
            }
            for (; j < e; j += 4) {
                const T l0 = (T)lp[(int64_t)j * f.ldl];
#pragma unroll
                for (int r = 0; r < RG; r++) acc[r] += l0 * sy[r * kMaxP + j];
            }
        }
#pragma unroll
        for (int r = 0; r < RG; r++) red[(sl * kRC + rl) * RGP + r] = acc[r];
        __syncthreads();
        for (int idx = t; idx < ng * nr; idx += kLT) {
            const int r = idx / nr, q = idx - r * nr;
            T v = red[q * RGP + r];
            v += red[(kRC + q) * RGP + r];
            v += red[(2 * kRC + q) * RGP + r];
            v += red[(3 * kRC + q) * RGP + r];
            atomicAdd(X + (int64_t)(g0 + r) * ldx + rvar[q], -(double)v);  // panels of a level may share rows below
        }
    }
}

// Stage columns j0 .. j0+nj-1 of L over this item's rows: ls[c][row].
template <typename T>
__device__ __forceinline__ void stage_chunk_cols(const LvFront &f, int64_t rbase, int nr, int j0, int nj, T *ls) {
    for (int idx = threadIdx.x; idx < nj * kRC; idx += kLT) {
        const int c = idx / kRC, row = idx - c * kRC;
        ls[c * (kRC + 1) + row] = row < nr ? (T)f.L[(int64_t)(j0 + c) * f.ldl + rbase + row] : T(0);
    }
}

// Sums over this item's rows of L(row, j) x(var(row), g0 + r) for every pivot
// column j: into part (out_part != nullptr) or subtracted from sz[r][j].
// pre0: columns 0 .. kLJ-1 are already staged in ls.
template <typename T, int RG>
__device__ __forceinline__ void chunk_sums(const LvFront &f, const int *rvar, int64_t rbase, int nr, const double *X,
                                           int64_t ldx, int g0, int ng, T *wk, bool pre0, T *out_part,
                                           int nrhs, int chunk, T *sz) {
    constexpr int RGP = LvShape<T, RG>::kRGP;
    constexpr int kS = kLT / kLJ, kRS = kRC / kS;  // row slices, rows per slice
    T *xs = wk;                      // [kRC][RG]
    T *ls = xs + kRC * RG;           // [kLJ][kRC + 1]: L(rbase + row, j0 + jj)
    T *red = ls + kLJ * (kRC + 1);   // [kS][kLJ][RGP]
    const int e = f.e, t = threadIdx.x, jj = t % kLJ, s = t / kLJ;
    __syncthreads();
    for (int idx = t; idx < kRC * RG; idx += kLT) {
        const int row = idx / RG, r = idx - row * RG;
        xs[idx] = (row < nr && r < ng) ? (T)X[(int64_t)(g0 + r) * ldx + rvar[row]] : T(0);
    }
    for (int j0 = 0; j0 < e; j0 += kLJ) {
        const int nj = min(kLJ, e - j0);
        __syncthreads();
        if (!(j0 == 0 && pre0)) {
            stage_chunk_cols(f, rbase, nr, j0, nj, ls);
            __syncthreads();
        }
        T acc[RG];
#pragma unroll
        for (int r = 0; r < RG; r++) acc[r] = T(0);
        if (jj < nj) {
#pragma unroll
            for (int k = 0; k < kRS; k++) {
                const int row = s * kRS + k;
                const T l = ls[jj * (kRC + 1) + row];
#pragma unroll
                for (int r = 0; r < RG; r++) acc[r] += l * xs[row * RG + r];
            }
        }
#pragma unroll
        for (int r = 0; r < RG; r++) red[(s * kLJ + jj) * RGP + r] = acc[r];
        __syncthreads();
        for (int idx = t; idx < ng * nj; idx += kLT) {
            const int r = idx / nj, c = idx - r * nj;
            T v = T(0);
#pragma unroll
            for (int s2 = 0; s2 < kS; s2++) v += red[(s2 * kLJ + c) * RGP + r];
            if (out_part != nullptr)
                out_part[((int64_t)chunk * nrhs + g0 + r) * e + j0 + c] = v;
            else
                sz[r * kMaxP + j0 + c] -= v;
        }
    }
}

template <typename T, int RG>
__global__ void __launch_bounds__(kLT) k_lv_backward(const LvFront *__restrict__ F, const int2 *__restrict__ items,
                                                     double *X, int64_t ldx, int nrhs, const T *__restrict__ Z,
                                                     T *part, int *cnt) {
    extern __shared__ __align__(16) unsigned char lv_smem[];
    T *sm = reinterpret_cast<T *>(lv_smem);
    T *sz = sm;               // [RG][kMaxP]: z - L_rest^T x_rest, then x, of the pivot variables
    T *wk = sm + RG * kMaxP;  // partial sums; then rows of L11 [kLJ][kLD]
    T *l11s = wk + LvShape<T, RG>::kChunk;  // L11 of a panel with e <= kLJ: [e][kLJ + 1] by rows
    __shared__ int pvar[kMaxP], pk[kMaxP], rvar[kRC];
    __shared__ int last;
    const int2 it = items[blockIdx.x];
    const LvFront f = F[it.x];
    const int e = f.e;
    if (e == 0) return;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int64_t rbase = e + (int64_t)it.y * kRC;
    const int nr = (int)max((int64_t)0, min((int64_t)kRC, f.n - rbase));
    for (int q = t; q < e; q += kLT) {
        pvar[q] = f.pvar[q];
        pk[q] = f.piv[q];
    }
    if (t < nr) rvar[t] = row_var(f, rbase + t);
    const bool small = e <= kLJ;
    const bool pre0 = nr > 0;
    if (pre0) stage_chunk_cols<T>(f, rbase, nr, 0, min(kLJ, e), wk + kRC * RG);
    __syncthreads();
    if (small)
        for (int idx = t; idx < e * e; idx += kLT) {
            const int j = idx / e, ii = idx - j * e;
            l11s[ii * (kLJ + 1) + j] = l11<T>(f, pk, ii, j);
        }
    pdl_trigger();
    pdl_wait();
    T *fpart = part + f.poff * nrhs;
    if (f.nch > 1) {
        for (int g0 = 0; g0 < nrhs; g0 += RG)
            chunk_sums<T, RG>(f, rvar, rbase, nr, X, ldx, g0, min(RG, nrhs - g0), wk, pre0 && (small || g0 == 0),
                           fpart, nrhs, it.y, nullptr);
        // the last item of the panel to get here finishes it
        __threadfence();
        __syncthreads();
        if (t == 0) last = atomicAdd(cnt + it.x, 1) == f.nch - 1;
        __syncthreads();
        if (!last) return;
        __threadfence();
        if (t == 0) cnt[it.x] = 0;  // ready for the next solve
    }
    for (int g0 = 0; g0 < nrhs; g0 += RG) {
        const int ng = min(RG, nrhs - g0);
        __syncthreads();
        for (int idx = t; idx < ng * e; idx += kLT) {
            const int r = idx / e, q = idx - r * e;
            T v = Z[f.zoff * nrhs + (int64_t)(g0 + r) * e + q];
            if (f.nch > 1)
                for (int c = 0; c < f.nch; c++) v -= __ldcg(fpart + ((int64_t)c * nrhs + g0 + r) * e + q);
            sz[r * kMaxP + q] = v;
        }
        if (f.nch == 1 && nr > 0)
            chunk_sums<T, RG>(f, rvar, rbase, nr, X, ldx, g0, ng, wk, pre0 && (small || g0 == 0), nullptr, nrhs, 0, sz);
        // L11^T x = z from the last pivot up, kLJ rows of L11 staged at a time;
        // warp w takes right-hand sides w, w + 8, ...; lanes take columns
        for (int i1 = e; i1 > 0; i1 -= kLJ) {
            const int i0 = max(0, i1 - kLJ), ni = i1 - i0;
            const T *rowsL = l11s;
            int ldr = kLJ + 1;
            __syncthreads();
            if (!small) {
                for (int idx = t; idx < ni * i1; idx += kLT) {
                    const int j = idx / ni, ii = idx - j * ni;
                    wk[ii * kLD + j] = l11<T>(f, pk, i0 + ii, j);
                }
                __syncthreads();
                rowsL = wk;
                ldr = kLD;
            }
            for (int r = warp; r < ng; r += kLT / 32) {
                T *z = sz + r * kMaxP;
                for (int ii = ni - 1; ii >= 0; ii--) {
                    const int i = i0 + ii;
                    const T xi = z[i];
                    for (int j = lane; j < i; j += 32) z[j] -= rowsL[ii * ldr + j] * xi;
                    __syncwarp();
                }
            }
        }
        __syncthreads();
        for (int idx = t; idx < ng * e; idx += kLT) {
            const int r = idx / e, q = idx - r * e;
            X[(int64_t)(g0 + r) * ldx + pvar[q]] = (double)sz[r * kMaxP + q];
        }
    }
}

// pvar[off[k] + q] = rows[perm[q]] for the panels' fully-summed positions.
__global__ void k_lv_pvar(const ctp_sfront *__restrict__ sf, const int64_t *__restrict__ off, int32_t *pvar) {
    const ctp_sfront f = sf[blockIdx.x];
    for (int q = threadIdx.x; q < f.p; q += blockDim.x) pvar[off[blockIdx.x] + q] = f.rows[f.perm[q]];
}

template <typename T, int RG>
cudaError_t launch_level(bool forward, const LvFront *F, const int2 *items, int64_t nitems, double *X,
                         int64_t ldx, int nrhs, T *Z, T *part, int *cnt, cudaStream_t st) {
    {
        cudaError_t e = smem_at_least((const void *)k_lv_forward<T, RG>, LvShape<T, RG>::kSmem);
        if (e == cudaSuccess)
            e = smem_at_least((const void *)k_lv_backward<T, RG>, LvShape<T, RG>::kSmem);
        if (e != cudaSuccess) return e;
    }
    if (nitems == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nitems);
    cfg.blockDim = dim3(kLT);
    cfg.dynamicSmemBytes = LvShape<T, RG>::kSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr_pdl[1];
    attr_pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr_pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr_pdl;
    cfg.numAttrs = 1;
    if (forward) return cudaLaunchKernelEx(&cfg, k_lv_forward<T, RG>, F, items, X, ldx, nrhs, Z);
    return cudaLaunchKernelEx(&cfg, k_lv_backward<T, RG>, F, items, X, ldx, nrhs, (const T *)Z, part, cnt);
}

template <typename T>
cudaError_t launch_level_rg(bool forward, const LvFront *F, const int2 *items, int64_t nitems, double *X,
                            int64_t ldx, int nrhs, T *Z, T *part, int *cnt, cudaStream_t st) {
    if (nrhs <= 1) return launch_level<T, 1>(forward, F, items, nitems, X, ldx, nrhs, Z, part, cnt, st);
    if (nrhs <= 2) return launch_level<T, 2>(forward, F, items, nitems, X, ldx, nrhs, Z, part, cnt, st);
    if (nrhs <= 4) return launch_level<T, 4>(forward, F, items, nitems, X, ldx, nrhs, Z, part, cnt, st);
    if (nrhs <= 8) return launch_level<T, 8>(forward, F, items, nitems, X, ldx, nrhs, Z, part, cnt, st);
    if constexpr (sizeof(T) == 4) {  // FP32: 32 right-hand sides per pass fit in shared memory
        if (nrhs > 16) return launch_level<T, 32>(forward, F, items, nitems, X, ldx, nrhs, Z, part, cnt, st);
    }
    return launch_level<T, 16>(forward, F, items, nitems, X, ldx, nrhs, Z, part, cnt, st);
}

}  // namespace

void SolvePlan::clear() {
    if (d_F) cudaFree(d_F);
    if (d_items) cudaFree(d_items);
    if (d_pvar) cudaFree(d_pvar);
    if (d_cnt) cudaFree(d_cnt);
    d_F = nullptr;
    d_items = nullptr;
    d_pvar = nullptr;
    d_cnt = nullptr;
    nf = nlev = 0;
    item_ptr.clear();
    z_per_rhs = 0;
    part_per_rhs = 0;
}

ctp_status SolvePlan::build(const std::vector<ctp_sfront> &fronts, const std::vector<int> &level,
                            const std::vector<int32_t> &nelim, cudaStream_t st) {
    clear();
    nf = (int)fronts.size();
    if (nf == 0) return CTP_OK;
    std::vector<LvFront> lf(nf);
    std::vector<int2> items;
    std::vector<int64_t> poff(nf);
    int64_t pv = 0, zo = 0, level_part = 0;
    item_ptr.push_back(0);
    for (int k = 0; k < nf; k++) {
        const ctp_sfront &s = fronts[k];
        if (k > 0 && level[k] < level[k - 1]) return CTP_EINVAL;
        if (nelim[k] < 0 || nelim[k] > s.p || s.p > kMaxP || s.n < s.p) return CTP_EINVAL;
        if (k > 0 && level[k] != level[k - 1]) {
            item_ptr.push_back((int64_t)items.size());
            level_part = 0;
        }
        LvFront &f = lf[k];
        f.L = s.L;
        f.ldl = s.ldl;
        f.n = s.n;
        f.rows = s.rows;
        f.piv = s.piv;
        f.D = s.D;
        f.e = nelim[k];
        f.p = s.p;
        f.pad = 0;
        poff[k] = pv;
        pv += s.p;
        f.zoff = zo;
        zo += f.e;
        const int64_t below = s.n - f.e;
        const int64_t nch = below > 0 ? (below + kRC - 1) / kRC : 1;
        if (nch > 0x7fffffffLL) return CTP_EINVAL;
        f.nch = (int32_t)nch;
        f.poff = level_part;
        if (nch > 1) level_part += nch * f.e;
        part_per_rhs = level_part > part_per_rhs ? level_part : part_per_rhs;
        if (f.e > 0)
            for (int64_t c = 0; c < nch; c++) items.push_back(make_int2(k, (int)c));
    }
    item_ptr.push_back((int64_t)items.size());
    nlev = (int)item_ptr.size() - 1;
    z_per_rhs = zo;
    ctp_sfront *d_sf = nullptr;
    int64_t *d_off = nullptr;
    bool ok = cudaMalloc(&d_F, sizeof(LvFront) * nf) == cudaSuccess &&
              cudaMalloc(&d_items, sizeof(int2) * (items.empty() ? 1 : items.size())) == cudaSuccess &&
              cudaMalloc(&d_pvar, sizeof(int32_t) * (pv > 0 ? pv : 1)) == cudaSuccess &&
              cudaMalloc(&d_cnt, sizeof(int) * nf) == cudaSuccess &&
              cudaMalloc(&d_sf, sizeof(ctp_sfront) * nf) == cudaSuccess &&
              cudaMalloc(&d_off, sizeof(int64_t) * nf) == cudaSuccess;
    if (!ok) {
        if (d_sf) cudaFree(d_sf);
        if (d_off) cudaFree(d_off);
        return CTP_ENOMEM;
    }
    for (int k = 0; k < nf; k++) lf[k].pvar = d_pvar + poff[k];
    ok = cudaMemcpy(d_F, lf.data(), sizeof(LvFront) * nf, cudaMemcpyHostToDevice) == cudaSuccess &&
         (items.empty() ||
          cudaMemcpy(d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice) == cudaSuccess) &&
         cudaMemcpy(d_sf, fronts.data(), sizeof(ctp_sfront) * nf, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(d_off, poff.data(), sizeof(int64_t) * nf, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemsetAsync(d_cnt, 0, sizeof(int) * nf, st) == cudaSuccess;
    if (ok) {
        k_lv_pvar<<<nf, 128, 0, st>>>(d_sf, d_off, d_pvar);
        ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
    }
    cudaFree(d_sf);
    cudaFree(d_off);
    return ok ? CTP_OK : CTP_ECUDA;
}

size_t SolvePlan::ws_bytes(int nrhs) const {
    return align256(sizeof(double) * (size_t)(z_per_rhs > 0 ? z_per_rhs : 1) * nrhs) +
           align256(sizeof(double) * (size_t)(part_per_rhs > 0 ? part_per_rhs : 1) * nrhs);
}

template <typename T>
static cudaError_t plan_sweeps(ctp_ctx *ctx, const SolvePlan &pl, double *X, int64_t ldx, int nrhs, void *ws,
                               cudaStream_t st) {
    T *Z = (T *)ws;
    T *part = (T *)((char *)ws + align256(sizeof(double) * (size_t)(pl.z_per_rhs > 0 ? pl.z_per_rhs : 1) * nrhs));
    const LvFront *F = (const LvFront *)pl.d_F;
    for (int l = 0; l < pl.nlev; l++) {
        cudaError_t e = timed(ctx, K_SYS_FWD, st, [&] {
            return launch_level_rg<T>(true, F, pl.d_items + pl.item_ptr[l], pl.item_ptr[l + 1] - pl.item_ptr[l], X,
                                      ldx, nrhs, Z, part, pl.d_cnt, st);
        });
        if (e != cudaSuccess) return e;
    }
    for (int l = pl.nlev - 1; l >= 0; l--) {
        cudaError_t e = timed(ctx, K_SYS_BWD, st, [&] {
            return launch_level_rg<T>(false, F, pl.d_items + pl.item_ptr[l], pl.item_ptr[l + 1] - pl.item_ptr[l], X,
                                      ldx, nrhs, Z, part, pl.d_cnt, st);
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t SolvePlan::solve(ctp_ctx *ctx, double *X, int64_t ldx, int nrhs, void *ws, cudaStream_t st,
                             bool fp32) const {
    return fp32 ? plan_sweeps<float>(ctx, *this, X, ldx, nrhs, ws, st)
                : plan_sweeps<double>(ctx, *this, X, ldx, nrhs, ws, st);
}

RefineLayout refine_layout(int64_t N, size_t solve_ws, int nrhs) {
    RefineLayout L;
    size_t off = 0;
    L.solve = off;
    off += align256(solve_ws);
    L.R = off;
    off += align256(sizeof(double) * (size_t)N * nrhs);
    L.rowsum = off;
    off += align256(sizeof(double) * (size_t)N);
    L.mx = off;
    off += align256(sizeof(double) * (3 * (size_t)nrhs + 1));
    L.berr = off;
    off += align256(sizeof(double) * (size_t)nrhs);
    L.total = off;
    return L;
}

static cudaError_t mat_residual(ctp_ctx *ctx, const MatOp &A, int64_t N, int nrhs, const double *X,
                                int64_t ldx, double *R, cudaStream_t st) {
    if (A.sparse())
        return timed(ctx, K_SPMV, st, [&] {
            return launch_spmv_csc_residual(N, A.colptr, A.rowind, A.val, nrhs, X, ldx, R, N, st);
        });
    return timed(ctx, K_SYMV, st, [&] { return launch_symv_residual(N, A.M, A.ldm, nrhs, X, ldx, R, N, st); });
}

cudaError_t mat_abs_rowsum(ctp_ctx *ctx, const MatOp &A, int64_t N, double *rowsum, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(rowsum, 0, sizeof(double) * N, st);
    if (e != cudaSuccess) return e;
    if (A.sparse())
        return timed(ctx, K_SPMV, st, [&] {
            return launch_spmv_csc_abs_rowsum(N, A.colptr, A.rowind, A.val, rowsum, st);
        });
    return timed(ctx, K_SYMV, st, [&] { return launch_abs_rowsum(N, A.M, A.ldm, rowsum, st); });
}

cudaError_t residual_berr(ctp_ctx *ctx, const MatOp &A, int64_t N, int nrhs, const double *B, int64_t ldb,
                          const double *X, int64_t ldx, double *R, const double *rowsum, double *mx,
                          double *berr, cudaStream_t st) {
    cudaError_t e = cudaMemcpy2DAsync(R, sizeof(double) * N, B, sizeof(double) * ldb, sizeof(double) * N, nrhs,
                                      cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    e = mat_residual(ctx, A, N, nrhs, X, ldx, R, st);
    if (e != cudaSuccess) return e;
    return timed(ctx, K_BERR, st, [&] {
        return launch_backward_error(N, nrhs, R, N, X, ldx, B, ldb, rowsum, mx, berr, st);
    });
}

}  // namespace ctp
