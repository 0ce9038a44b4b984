// solve.cu -- K5: the Solve task L21 = A21 P^T (D11 L11^T)^{-1} (Section 1 task
// list; Figure 4.1 (d),(e)) fused with the update of the delayed columns, in FP64.
//
// Every A21 row is independent: with x = A21(i, perm) the permuted row,
//   Y  = x_e L11^{-T}          (forward substitution, right-looking by column),
//   x_d <- x_d - Y L_d^T        (delayed columns: L_d are the delayed rows of L),
//   L21(i,:) = Y D11^{-1}       (1x1 and 2x2 blocks; zero pivots give 0).
// A CTA owns a tile of kRows consecutive rows; the tile is gathered through the
// permutation with coalesced loads into shared memory (padded [p][kRows+1]),
// eliminated in place, and written back in place (L21 in the first e columns,
// the updated delayed columns after them).  Y = L21 D11 is also written to the
// workspace when the Form step needs it.  Arithmetic is O(p^2) FP64 FMAs per row
// and the GB300 FP64 pipe is the bound; L columns are broadcast from L1.
#include "ctp_internal.cuh"

namespace ctp {

namespace {

constexpr int kRows = 32;     // rows per tile = threads per CTA (one row per thread)
constexpr int kThreadsS = 32;

__global__ void __launch_bounds__(kThreadsS)
    k_solve_fp64(double *__restrict__ A, int64_t n, int p, int64_t lda,
                 const int32_t *__restrict__ perm, const int32_t *__restrict__ piv,
                 const double *__restrict__ Dinv, const int32_t *__restrict__ nelim_p,
                 double *__restrict__ W21, int64_t ldw) {
    extern __shared__ __align__(16) double xs[];  // [p][kRows+1]
    const int64_t m = n - p;
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    if (row0 >= m) return;
    const int r = threadIdx.x;
    const int64_t row = row0 + r;
    const bool valid = row < m;
    const int e = *nelim_p;
    double *A21 = A + p;
    constexpr int LDX = kRows + 1;

    // gather x = A21(rows, perm) (coalesced: consecutive threads, consecutive rows)
    for (int k = 0; k < p; k++) {
        const int c = perm[k];
        xs[k * LDX + r] = valid ? A21[(int64_t)c * lda + row] : 0.0;
    }
    __syncwarp();

    // forward substitution, right-looking over the eliminated positions
    for (int j = 0; j < e;) {
        const int kd = piv[j];
        if (kd == CTP_PIVKIND_2X2_FIRST) {
            const double y0 = xs[j * LDX + r], y1 = xs[(j + 1) * LDX + r];
            const double *l0 = A + (int64_t)j * lda, *l1 = A + (int64_t)(j + 1) * lda;
            for (int k = j + 2; k < p; k++) {
                xs[k * LDX + r] -= y0 * __ldg(l0 + k) + y1 * __ldg(l1 + k);
            }
            j += 2;
        } else {
            if (kd == CTP_PIVKIND_1X1) {
                const double y0 = xs[j * LDX + r];
                const double *l0 = A + (int64_t)j * lda;
                for (int k = j + 1; k < p; k++) xs[k * LDX + r] -= y0 * __ldg(l0 + k);
            }
            j += 1;  // zero pivots have an all-zero L column
        }
    }

    if (valid) {
        // W21 = Y (= L21 D11) for the Form step
        if (W21 != nullptr)
            for (int j = 0; j < e; j++) W21[(int64_t)j * ldw + row] = xs[j * LDX + r];
        // L21 = Y D11^{-1}
        for (int j = 0; j < e;) {
            const int kd = piv[j];
            if (kd == CTP_PIVKIND_2X2_FIRST) {
                const double y0 = xs[j * LDX + r], y1 = xs[(j + 1) * LDX + r];
                const double i11 = Dinv[2 * j], i21 = Dinv[2 * j + 1], i22 = Dinv[2 * j + 2];
                A21[(int64_t)j * lda + row] = y0 * i11 + y1 * i21;
                A21[(int64_t)(j + 1) * lda + row] = y0 * i21 + y1 * i22;
                j += 2;
            } else {
                A21[(int64_t)j * lda + row] =
                    (kd == CTP_PIVKIND_1X1) ? xs[j * LDX + r] * Dinv[2 * j] : 0.0;
                j += 1;
            }
        }
        for (int k = e; k < p; k++) A21[(int64_t)k * lda + row] = xs[k * LDX + r];
    }
}

}  // namespace

cudaError_t launch_solve_fp64(double *A, int64_t n, int p, int64_t lda, const int32_t *perm,
                              const int32_t *piv, const double *Dinv, const int32_t *nelim,
                              double *W21, int64_t ldw, cudaStream_t st) {
    const int64_t m = n - p;
    if (m <= 0) return cudaSuccess;
    size_t smem = sizeof(double) * (size_t)p * (kRows + 1);
    cudaError_t err =
        cudaFuncSetAttribute(k_solve_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int64_t grid = (m + kRows - 1) / kRows;
    k_solve_fp64<<<(unsigned)grid, kThreadsS, smem, st>>>(A, n, p, lda, perm, piv, Dinv, nelim,
                                                          W21, ldw);
    return cudaGetLastError();
}

}  // namespace ctp
