// system.cu -- solving a complete system with the supernodes' factors, the FP64
// residual, the backward error of Section 7 and the kernels iterative
// refinement needs.
//
// The factors are a list of fronts in elimination order (a chain or an assembly
// tree, children first).  Front f has n_f rows named by the variable indices
// rows[0..n_f) (rows[0..p) are its fully-summed variables in the order they had
// before pivoting, so front row q < p holds variable rows[perm[q]] afterwards)
// and stores, in ctp_factor_supernode's in-place layout, the unit lower
// factor L (columns 0..e-1), D (1x1 and 2x2 blocks; the (q+1, q) slot of a
// 2x2 block holds D, not L).  With P M P^T = L D L^T the solve is
//   forward   for f in order:   y = L11^{-1} b_f,  b_rest -= L_rest y,  z = D^{-1} y
//   backward  for f reversed:   x_f = L11^{-T} (z - L_rest^T x_rest)
// (Section 1's factorization applied front by front).  Right-hand sides are the
// columns of an N x nrhs column-major array X, solved in place.
#include "ctp_internal.cuh"

namespace ctp {

namespace {

constexpr int kTh = 256;   // threads of every kernel here
constexpr int kRB = 8;     // right-hand sides per pass of the triangular kernels
constexpr int kJB = 32;    // columns of L11 staged per block of the triangular solves

__device__ __forceinline__ int front_var(const ctp_sfront &f, int64_t r) {
    return r < f.p ? f.rows[f.perm[r]] : f.rows[r];
}

// Forward step of one front: gather, unit-lower solve with L11, keep y for the
// update of the rows below, scatter z = D^{-1} y.
__device__ __forceinline__ void dev_fwd_tri(const ctp_sfront &f, double *X, int64_t ldx, int nrhs, double *Y) {
    extern __shared__ double sm[];
    double *sl = sm;                      // [kJB][kMaxP]: L(i, j0 + jj) at sl[jj * kMaxP + i]
    double *sy = sm + kJB * kMaxP;        // [kRB][kMaxP]
    __shared__ int var[kMaxP];
    __shared__ int pv[kMaxP];
    const int e = *f.nelim;
    const int t = threadIdx.x;
    for (int q = t; q < e; q += kTh) {
        var[q] = f.rows[f.perm[q]];
        pv[q] = f.piv[q];
    }
    __syncthreads();
    for (int r0 = 0; r0 < nrhs; r0 += kRB) {
        const int nr = min(kRB, nrhs - r0);
        for (int idx = t; idx < nr * e; idx += kTh) {
            const int r = idx / e, q = idx % e;
            sy[r * kMaxP + q] = X[(int64_t)(r0 + r) * ldx + var[q]];
        }
        __syncthreads();
        for (int j0 = 0; j0 < e; j0 += kJB) {
            const int nj = min(kJB, e - j0);
            for (int idx = t; idx < nj * e; idx += kTh) {
                const int jj = idx / e, i = idx % e;
                sl[jj * kMaxP + i] = (i > j0 + jj) ? f.L[(int64_t)(j0 + jj) * f.ldl + i] : 0.0;
            }
            __syncthreads();
            for (int jj = 0; jj < nj; jj++) {
                const int j = j0 + jj;
                const int i = t;
                if (i > j && i < e && !(i == j + 1 && pv[j] == CTP_PIVKIND_2X2_FIRST)) {
                    const double l = sl[jj * kMaxP + i];
                    for (int r = 0; r < nr; r++) sy[r * kMaxP + i] -= l * sy[r * kMaxP + j];
                }
                __syncthreads();
            }
        }
        for (int idx = t; idx < nr * e; idx += kTh) {
            const int r = idx / e, q = idx % e;
            Y[(int64_t)(r0 + r) * kMaxP + q] = sy[r * kMaxP + q];
        }
        // D solve: 1x1, 2x2 (handled by its first column), zero pivot -> 0
        for (int idx = t; idx < nr * e; idx += kTh) {
            const int r = idx / e, q = idx % e;
            const int k = pv[q];
            double z = 0.0;
            if (k == CTP_PIVKIND_1X1) {
                z = sy[r * kMaxP + q] / f.D[2 * q];
            } else if (k == CTP_PIVKIND_2X2_FIRST || k == CTP_PIVKIND_2X2_SECOND) {
                const int a = (k == CTP_PIVKIND_2X2_FIRST) ? q : q - 1;
                const double d11 = f.D[2 * a], d21 = f.D[2 * a + 1], d22 = f.D[2 * a + 2];
                const double y0 = sy[r * kMaxP + a], y1 = sy[r * kMaxP + a + 1];
                const double det = d11 * d22 - d21 * d21;
                z = (k == CTP_PIVKIND_2X2_FIRST) ? (d22 * y0 - d21 * y1) / det
                                                 : (d11 * y1 - d21 * y0) / det;
            }
            X[(int64_t)(r0 + r) * ldx + var[q]] = z;
        }
        __syncthreads();
    }
}

// Rows below the pivots: b(var(r)) -= L(r, 0:e) y, one row per thread.
__device__ __forceinline__ void dev_fwd_upd(const ctp_sfront &f, double *X, int64_t ldx, int nrhs, const double *Y,
                                            int64_t chunk) {
    __shared__ double sy[kRB][kMaxP];
    const int e = *f.nelim;
    const int64_t r = (int64_t)e + chunk * kTh + threadIdx.x;
    const bool live = r < f.n;
    const int v = live ? front_var(f, r) : 0;
    for (int r0 = 0; r0 < nrhs; r0 += kRB) {
        const int nr = min(kRB, nrhs - r0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nr * e; idx += kTh) {
            const int rr = idx / e, q = idx % e;
            sy[rr][q] = Y[(int64_t)(r0 + rr) * kMaxP + q];
        }
        __syncthreads();
        if (!live) continue;
        double acc[kRB];
#pragma unroll
        for (int rr = 0; rr < kRB; rr++) acc[rr] = 0.0;
        const double *lp = f.L + r;
        for (int j = 0; j < e; j++) {
            const double l = lp[(int64_t)j * f.ldl];
#pragma unroll
            for (int rr = 0; rr < kRB; rr++) acc[rr] += l * sy[rr][j];
        }
        for (int rr = 0; rr < nr; rr++) X[(int64_t)(r0 + rr) * ldx + v] -= acc[rr];
    }
}

// Backward step, part 1: per chunk of kTh rows below the pivots,
// part[c][r][j] = sum over the chunk's rows of L(row, j) x(var(row), r).
__device__ __forceinline__ void dev_bwd_part(const ctp_sfront &f, const double *X, int64_t ldx, int nrhs,
                                             double *part, int64_t c) {
    __shared__ double sx[kRB][kTh];
    const int e = *f.nelim;
    const int64_t below = f.n - e;
    const int64_t nch = (below + kTh - 1) / kTh;
    if (c >= nch) return;
    const int64_t rbase = e + c * kTh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r0 = 0; r0 < nrhs; r0 += kRB) {
        const int nr = min(kRB, nrhs - r0);
        __syncthreads();
        {
            const int64_t row = rbase + threadIdx.x;
            const int v = row < f.n ? front_var(f, row) : 0;
            for (int rr = 0; rr < kRB; rr++)
                sx[rr][threadIdx.x] = (row < f.n && rr < nr) ? X[(int64_t)(r0 + rr) * ldx + v] : 0.0;
        }
        __syncthreads();
        for (int j = warp; j < e; j += kTh / 32) {
            double acc[kRB];
#pragma unroll
            for (int rr = 0; rr < kRB; rr++) acc[rr] = 0.0;
            const double *lp = f.L + (int64_t)j * f.ldl + rbase;
#pragma unroll
            for (int k = 0; k < kTh / 32; k++) {
                const int ro = lane + 32 * k;
                const double l = (rbase + ro < f.n) ? lp[ro] : 0.0;
#pragma unroll
                for (int rr = 0; rr < kRB; rr++) acc[rr] += l * sx[rr][ro];
            }
#pragma unroll
            for (int rr = 0; rr < kRB; rr++)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[rr] += __shfl_xor_sync(0xffffffffu, acc[rr], o);
            if (lane == 0)
                for (int rr = 0; rr < nr; rr++) part[(c * nrhs + r0 + rr) * kMaxP + j] = acc[rr];
        }
    }
}

// Backward step, part 2: z = x(piv vars) - sum of the chunk partials, then
// L11^T x = z, right-looking from the last pivot, 32 rows of L11 staged at a time.
__device__ __forceinline__ void dev_bwd_tri(const ctp_sfront &f, double *X, int64_t ldx, int nrhs,
                                            const double *part) {
    extern __shared__ double sm[];
    double *sl = sm;                  // [kJB][kMaxP]: L(i0 + ii, j) at sl[ii * kMaxP + j]
    double *sz = sm + kJB * kMaxP;    // [kRB][kMaxP]
    __shared__ int var[kMaxP];
    __shared__ int pv[kMaxP];
    const int e = *f.nelim;
    const int64_t nch = (f.n - e + kTh - 1) / kTh;
    const int t = threadIdx.x;
    for (int q = t; q < e; q += kTh) {
        var[q] = f.rows[f.perm[q]];
        pv[q] = f.piv[q];
    }
    __syncthreads();
    for (int r0 = 0; r0 < nrhs; r0 += kRB) {
        const int nr = min(kRB, nrhs - r0);
        for (int idx = t; idx < nr * e; idx += kTh) {
            const int r = idx / e, q = idx % e;
            double s = 0.0;
            for (int64_t c = 0; c < nch; c++) s += part[(c * nrhs + r0 + r) * kMaxP + q];
            sz[r * kMaxP + q] = X[(int64_t)(r0 + r) * ldx + var[q]] - s;
        }
        __syncthreads();
        for (int i1 = e; i1 > 0; i1 -= kJB) {
            const int i0 = max(0, i1 - kJB), ni = i1 - i0;
            for (int idx = t; idx < ni * i1; idx += kTh) {
                const int ii = idx % ni, j = idx / ni;
                sl[ii * kMaxP + j] = f.L[(int64_t)j * f.ldl + i0 + ii];
            }
            __syncthreads();
            for (int ii = ni - 1; ii >= 0; ii--) {
                const int i = i0 + ii;
                const int j = t;
                // x_i is final; remove its contribution from z_j, j < i
                if (j < i && !(i == j + 1 && pv[j] == CTP_PIVKIND_2X2_FIRST)) {
                    const double l = sl[ii * kMaxP + j];
                    for (int r = 0; r < nr; r++) sz[r * kMaxP + j] -= l * sz[r * kMaxP + i];
                }
                __syncthreads();
            }
        }
        for (int idx = t; idx < nr * e; idx += kTh) {
            const int r = idx / e, q = idx % e;
            X[(int64_t)(r0 + r) * ldx + var[q]] = sz[r * kMaxP + q];
        }
        __syncthreads();
    }
}

// One front per launch (the generic front-list solve).
__global__ void __launch_bounds__(kTh) k_sys_fwd_tri(ctp_sfront f, double *X, int64_t ldx, int nrhs,
                                                     double *Y) {
    dev_fwd_tri(f, X, ldx, nrhs, Y);
}
__global__ void __launch_bounds__(kTh) k_sys_fwd_upd(ctp_sfront f, double *X, int64_t ldx, int nrhs,
                                                     const double *Y) {
    dev_fwd_upd(f, X, ldx, nrhs, Y, blockIdx.x);
}
__global__ void __launch_bounds__(kTh) k_sys_bwd_part(ctp_sfront f, const double *X, int64_t ldx,
                                                      int nrhs, double *part) {
    dev_bwd_part(f, X, ldx, nrhs, part, blockIdx.x);
}
__global__ void __launch_bounds__(kTh) k_sys_bwd_tri(ctp_sfront f, double *X, int64_t ldx, int nrhs,
                                                     const double *part) {
    dev_bwd_tri(f, X, ldx, nrhs, part);
}

// R -= M X (kAbs = false) or R += |M| 1 (kAbs = true: the row sums of |M|),
// M symmetric with its lower triangle stored (column-major, ldm), one 64 x 64
// tile of the lower block triangle per CTA; both the tile and its transpose
// contribute, accumulated with FP64 atomics.
constexpr int kRT = 64;
template <bool kAbs>
__global__ void __launch_bounds__(kTh) k_symv(int64_t N, const double *__restrict__ M, int64_t ldm,
                                              int nrhs, const double *__restrict__ X, int64_t ldx,
                                              double *R, int64_t ldr) {
    __shared__ double a[kRT][kRT + 1];
    __shared__ double xi[kRT], xj[kRT];
    const int64_t b = blockIdx.x;
    int64_t ti = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= b) ti++;
    while (ti * (ti + 1) / 2 > b) ti--;
    const int64_t tj = b - ti * (ti + 1) / 2;
    const int64_t i0 = ti * kRT, j0 = tj * kRT;
    const bool diag = ti == tj;
    for (int idx = threadIdx.x; idx < kRT * kRT; idx += kTh) {
        const int ii = idx % kRT, jj = idx / kRT;
        const int64_t gi = i0 + ii, gj = j0 + jj;
        double v = (gi < N && gj < N && (!diag || ii >= jj)) ? M[gj * ldm + gi] : 0.0;
        a[ii][jj] = kAbs ? fabs(v) : v;
    }
    const int nr = kAbs ? 1 : nrhs;
    for (int r = 0; r < nr; r++) {
        __syncthreads();
        if (threadIdx.x < kRT) {
            const int64_t g = j0 + threadIdx.x;
            xj[threadIdx.x] = kAbs ? 1.0 : (g < N ? X[(int64_t)r * ldx + g] : 0.0);
        } else if (threadIdx.x < 2 * kRT) {
            const int64_t g = i0 + threadIdx.x - kRT;
            xi[threadIdx.x - kRT] = kAbs ? 1.0 : (g < N ? X[(int64_t)r * ldx + g] : 0.0);
        }
        __syncthreads();
        if (threadIdx.x < kRT) {
            const int ii = threadIdx.x;
            double s = 0.0;
            for (int jj = 0; jj < kRT; jj++) s += a[ii][jj] * xj[jj];
            if (i0 + ii < N) atomicAdd(R + (int64_t)r * ldr + i0 + ii, kAbs ? s : -s);
        } else if (threadIdx.x < 2 * kRT) {
            const int jj = threadIdx.x - kRT;
            double s = 0.0;
            for (int ii = 0; ii < kRT; ii++)
                if (!diag || ii > jj) s += a[ii][jj] * xi[ii];
            if (j0 + jj < N) atomicAdd(R + (int64_t)r * ldr + j0 + jj, kAbs ? s : -s);
        }
    }
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// mx[3 r + 0..2] = max |R(:, r)|, max |X(:, r)|, max |B(:, r)|; mx[3 nrhs] = max row sum.
__global__ void __launch_bounds__(kTh) k_maxabs(int64_t N, int nrhs, const double *R, int64_t ldr,
                                                const double *X, int64_t ldx, const double *B,
                                                int64_t ldb, const double *rowsum, double *mx) {
    const int r = blockIdx.y;
    double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kTh + threadIdx.x; i < N; i += (int64_t)gridDim.x * kTh) {
        m0 = fmax(m0, fabs(R[(int64_t)r * ldr + i]));
        m1 = fmax(m1, fabs(X[(int64_t)r * ldx + i]));
        m2 = fmax(m2, fabs(B[(int64_t)r * ldb + i]));
        if (r == 0 && rowsum != nullptr) m3 = fmax(m3, rowsum[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        m0 = fmax(m0, __shfl_xor_sync(0xffffffffu, m0, o));
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        m3 = fmax(m3, __shfl_xor_sync(0xffffffffu, m3, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(mx + 3 * r + 0, m0);
        atomic_max_nonneg(mx + 3 * r + 1, m1);
        atomic_max_nonneg(mx + 3 * r + 2, m2);
        if (r == 0 && rowsum != nullptr) atomic_max_nonneg(mx + 3 * nrhs, m3);
    }
}

// berr[r] = ||R||_inf / (||M||_inf ||X||_inf + ||B||_inf)   (Section 7)
__global__ void k_berr(int nrhs, const double *mx, double *berr) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    const double den = mx[3 * nrhs] * mx[3 * r + 1] + mx[3 * r + 2];
    berr[r] = den > 0.0 ? mx[3 * r] / den : 0.0;
}

// X(:, r) += Dx(:, r)
__global__ void k_axpy(int64_t N, int nrhs, double *X, int64_t ldx, const double *Dx, int64_t ldd) {
    const int r = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * kTh + threadIdx.x; i < N; i += (int64_t)gridDim.x * kTh)
        X[(int64_t)r * ldx + i] += Dx[(int64_t)r * ldd + i];
}

// W21 = L21 D11 from the stored L21 and D (used where the pivoting kernel does
// not produce W21 itself, i.e. full-column threshold partial pivoting).
__global__ void __launch_bounds__(kTh) k_w21_from_l(const double *A, int64_t lda, int p, int64_t m,
                                                    const int32_t *piv, const double *D,
                                                    const int32_t *nelim, double *W21, int64_t ldw) {
    const int e = *nelim;
    const int64_t i = (int64_t)blockIdx.x * kTh + threadIdx.x;
    if (i >= m) return;
    const double *L = A + p + i;
    for (int q = 0; q < e; q++) {
        const int k = piv[q];
        double w = 0.0;
        if (k == CTP_PIVKIND_1X1) {
            w = L[(int64_t)q * lda] * D[2 * q];
        } else if (k == CTP_PIVKIND_2X2_FIRST) {
            w = L[(int64_t)q * lda] * D[2 * q] + L[(int64_t)(q + 1) * lda] * D[2 * q + 1];
        } else if (k == CTP_PIVKIND_2X2_SECOND) {
            w = L[(int64_t)(q - 1) * lda] * D[2 * q - 1] + L[(int64_t)q * lda] * D[2 * q];
        }
        W21[(int64_t)q * ldw + i] = w;
    }
}

// Gradient of a loss through x = M^{-1} b with respect to the stored lower
// triangle of the symmetric M (each stored off-diagonal entry stands for both
// m_ij and m_ji): dL/dm_ij = -sum_r (g_ir x_jr + g_jr x_ir) for i > j and
// -sum_r g_ir x_ir on the diagonal, with g = M^{-T} dL/dx.  Dense form: the lower
// triangle of an N x N column-major output (strict upper triangle zeroed).
__global__ void __launch_bounds__(kTh) k_sym_grad_dense(int64_t N, int nrhs, const double *__restrict__ G,
                                                        int64_t ldg, const double *__restrict__ X,
                                                        int64_t ldx, double *__restrict__ out,
                                                        int64_t ldo) {
    for (int64_t j = blockIdx.y; j < N; j += gridDim.y)
    for (int64_t i = (int64_t)blockIdx.x * kTh + threadIdx.x; i < N; i += (int64_t)gridDim.x * kTh) {
        double s = 0.0;
        if (i > j) {
            for (int r = 0; r < nrhs; r++)
                s += G[(int64_t)r * ldg + i] * X[(int64_t)r * ldx + j] +
                     G[(int64_t)r * ldg + j] * X[(int64_t)r * ldx + i];
        } else if (i == j) {
            for (int r = 0; r < nrhs; r++) s += G[(int64_t)r * ldg + i] * X[(int64_t)r * ldx + i];
        }
        out[j * ldo + i] = -s;
    }
}

// The same restricted to a pattern of stored entries (row[k], col[k]), any order;
// an entry with row == col is a diagonal entry, otherwise it stands for both
// (row, col) and (col, row).
__global__ void __launch_bounds__(kTh) k_sym_grad_pattern(int64_t nnz, const int32_t *__restrict__ row,
                                                          const int32_t *__restrict__ col, int nrhs,
                                                          const double *__restrict__ G, int64_t ldg,
                                                          const double *__restrict__ X, int64_t ldx,
                                                          double *__restrict__ out) {
    for (int64_t k = (int64_t)blockIdx.x * kTh + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * kTh) {
        const int64_t i = row[k], j = col[k];
        double s = 0.0;
        // the same expressions as the dense kernel, so both round alike
        if (i != j) {
            for (int r = 0; r < nrhs; r++)
                s += G[(int64_t)r * ldg + i] * X[(int64_t)r * ldx + j] +
                     G[(int64_t)r * ldg + j] * X[(int64_t)r * ldx + i];
        } else {
            for (int r = 0; r < nrhs; r++) s += G[(int64_t)r * ldg + i] * X[(int64_t)r * ldx + i];
        }
        out[k] = -s;
    }
}

// R -= A X for a symmetric A given by its lower triangle in compressed columns
// (kAbs: R += |A| 1, the row sums of |A|).  One warp per column j: the
// column's entries update R(i) (atomics) and their transposes accumulate into
// R(j).
template <bool kAbs>
__global__ void __launch_bounds__(kTh) k_spmv_csc(int64_t N, const int64_t *__restrict__ colptr,
                                                  const int32_t *__restrict__ rowind,
                                                  const double *__restrict__ val, int nrhs,
                                                  const double *__restrict__ X, int64_t ldx, double *R,
                                                  int64_t ldr) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kTh / 32);
    const int nr = kAbs ? 1 : nrhs;
    for (int64_t j = (int64_t)blockIdx.x * (kTh / 32) + (threadIdx.x >> 5); j < N; j += warps) {
        const int64_t q0 = colptr[j], q1 = colptr[j + 1];
        for (int r = 0; r < nr; r++) {
            const double xj = kAbs ? 1.0 : X[(int64_t)r * ldx + j];
            double t = 0.0;
            for (int64_t q = q0 + lane; q < q1; q += 32) {
                const int64_t i = rowind[q];
                const double a = kAbs ? fabs(val[q]) : val[q];
                if (i == j) {
                    t += a * xj;
                } else {
                    atomicAdd(R + (int64_t)r * ldr + i, kAbs ? a : -a * xj);
                    t += a * (kAbs ? 1.0 : X[(int64_t)r * ldx + i]);
                }
            }
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) atomicAdd(R + (int64_t)r * ldr + j, kAbs ? t : -t);
        }
    }
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kTh - 1) / kTh); }

constexpr size_t kTriSmem = sizeof(double) * (size_t)(kJB + kRB) * kMaxP;

}  // namespace

size_t sys_solve_ws_bytes(int64_t nmax, int nrhs) {
    const int64_t nch = (nmax + kTh - 1) / kTh;
    return align256(sizeof(double) * (size_t)kMaxP * nrhs) +
           align256(sizeof(double) * (size_t)nch * nrhs * kMaxP);
}

cudaError_t launch_sys_forward(const ctp_sfront &f, double *X, int64_t ldx, int nrhs, void *ws,
                               cudaStream_t st) {
    {
        cudaError_t e = smem_at_least((const void *)k_sys_fwd_tri, kTriSmem);
        if (e == cudaSuccess) e = smem_at_least((const void *)k_sys_bwd_tri, kTriSmem);
        if (e != cudaSuccess) return e;
    }
    double *Y = (double *)ws;
    k_sys_fwd_tri<<<1, kTh, kTriSmem, st>>>(f, X, ldx, nrhs, Y);
    if (f.n > 0) k_sys_fwd_upd<<<blocks_for(f.n), kTh, 0, st>>>(f, X, ldx, nrhs, Y);
    return cudaGetLastError();
}

cudaError_t launch_sys_backward(const ctp_sfront &f, double *X, int64_t ldx, int nrhs, void *ws,
                                cudaStream_t st) {
    double *part = (double *)((char *)ws + align256(sizeof(double) * (size_t)kMaxP * nrhs));
    const int64_t nch = (f.n + kTh - 1) / kTh;  // upper bound on the chunks below the pivots
    cudaError_t e = smem_at_least((const void *)k_sys_bwd_tri, kTriSmem);
    if (e != cudaSuccess) return e;
    if (nch > 0) k_sys_bwd_part<<<(unsigned)nch, kTh, 0, st>>>(f, X, ldx, nrhs, part);
    k_sys_bwd_tri<<<1, kTh, kTriSmem, st>>>(f, X, ldx, nrhs, part);
    return cudaGetLastError();
}

cudaError_t launch_symv_residual(int64_t N, const double *M, int64_t ldm, int nrhs, const double *X,
                                 int64_t ldx, double *R, int64_t ldr, cudaStream_t st) {
    const int64_t nt = (N + kRT - 1) / kRT;
    const int64_t tiles = nt * (nt + 1) / 2;
    if (tiles == 0) return cudaSuccess;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_symv<false><<<(unsigned)tiles, kTh, 0, st>>>(N, M, ldm, nrhs, X, ldx, R, ldr);
    return cudaGetLastError();
}

cudaError_t launch_abs_rowsum(int64_t N, const double *M, int64_t ldm, double *rowsum,
                              cudaStream_t st) {
    const int64_t nt = (N + kRT - 1) / kRT;
    const int64_t tiles = nt * (nt + 1) / 2;
    if (tiles == 0) return cudaSuccess;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_symv<true><<<(unsigned)tiles, kTh, 0, st>>>(N, M, ldm, 1, nullptr, 0, rowsum, N);
    return cudaGetLastError();
}

cudaError_t launch_backward_error(int64_t N, int nrhs, const double *R, int64_t ldr, const double *X,
                                  int64_t ldx, const double *B, int64_t ldb, const double *rowsum,
                                  double *mx, double *berr, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(double) * (3 * (size_t)nrhs + 1), st);
    if (e != cudaSuccess) return e;
    const unsigned gx = (unsigned)(N < 1 ? 1 : ((N + kTh - 1) / kTh < 304 ? (N + kTh - 1) / kTh : 304));
    k_maxabs<<<dim3(gx, nrhs), kTh, 0, st>>>(N, nrhs, R, ldr, X, ldx, B, ldb, rowsum, mx);
    k_berr<<<(nrhs + 127) / 128, 128, 0, st>>>(nrhs, mx, berr);
    return cudaGetLastError();
}

cudaError_t launch_axpy(int64_t N, int nrhs, double *X, int64_t ldx, const double *Dx, int64_t ldd,
                        cudaStream_t st) {
    if (N == 0 || nrhs == 0) return cudaSuccess;
    const unsigned gx = (unsigned)((N + kTh - 1) / kTh < 1216 ? (N + kTh - 1) / kTh : 1216);
    k_axpy<<<dim3(gx, nrhs), kTh, 0, st>>>(N, nrhs, X, ldx, Dx, ldd);
    return cudaGetLastError();
}

cudaError_t launch_sym_grad_dense(int64_t N, int nrhs, const double *G, int64_t ldg, const double *X,
                                  int64_t ldx, double *out, int64_t ldo, cudaStream_t st) {
    if (N == 0) return cudaSuccess;
    const unsigned gx = blocks_for(N) < 64 ? blocks_for(N) : 64;
    const unsigned gy = N < 65535 ? (unsigned)N : 65535u;
    k_sym_grad_dense<<<dim3(gx, gy), kTh, 0, st>>>(N, nrhs, G, ldg, X, ldx, out, ldo);
    return cudaGetLastError();
}

cudaError_t launch_sym_grad_pattern(int64_t nnz, const int32_t *row, const int32_t *col, int nrhs,
                                    const double *G, int64_t ldg, const double *X, int64_t ldx,
                                    double *out, cudaStream_t st) {
    if (nnz == 0) return cudaSuccess;
    const unsigned g = blocks_for(nnz) < 4096 ? blocks_for(nnz) : 4096;
    k_sym_grad_pattern<<<g, kTh, 0, st>>>(nnz, row, col, nrhs, G, ldg, X, ldx, out);
    return cudaGetLastError();
}

cudaError_t launch_spmv_csc_residual(int64_t N, const int64_t *colptr, const int32_t *rowind,
                                     const double *val, int nrhs, const double *X, int64_t ldx, double *R,
                                     int64_t ldr, cudaStream_t st) {
    const int64_t g = (N + 7) / 8 < 4096 ? (N + 7) / 8 : 4096;
    k_spmv_csc<false><<<(unsigned)g, kTh, 0, st>>>(N, colptr, rowind, val, nrhs, X, ldx, R, ldr);
    return cudaGetLastError();
}

cudaError_t launch_spmv_csc_abs_rowsum(int64_t N, const int64_t *colptr, const int32_t *rowind,
                                       const double *val, double *rowsum, cudaStream_t st) {
    const int64_t g = (N + 7) / 8 < 4096 ? (N + 7) / 8 : 4096;
    k_spmv_csc<true><<<(unsigned)g, kTh, 0, st>>>(N, colptr, rowind, val, 1, nullptr, 0, rowsum, N);
    return cudaGetLastError();
}

cudaError_t launch_w21_from_l(const double *A, int64_t lda, int p, int64_t m, const int32_t *piv,
                              const double *D, const int32_t *nelim, double *W21, int64_t ldw,
                              cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_w21_from_l<<<blocks_for(m), kTh, 0, st>>>(A, lda, p, m, piv, D, nelim, W21, ldw);
    return cudaGetLastError();
}

}  // namespace ctp
