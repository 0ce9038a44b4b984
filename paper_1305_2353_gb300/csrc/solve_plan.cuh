// solve_plan.cuh -- a front-list solve planned by levels (fronts of a level are
// independent: one launch per level and sweep), and FP64 iterative refinement
// (Section 7) around any solve: the helpers shared by the ABI's complete-system
// entry points.
#pragma once

#include <vector>

#include "ctx.cuh"

namespace ctp {

// Fronts in an elimination order grouped by level: the fronts of a level are
// independent (none updates another's pivot rows), so a level is one launch
// per sweep over items (front, chunk of rows below its pivots).
struct SolvePlan {
    int nf = 0, nlev = 0;
    std::vector<int64_t> item_ptr;  // items of level l: [item_ptr[l], item_ptr[l+1])
    void *d_F = nullptr;            // the fronts' descriptors (solve_plan.cu)
    int2 *d_items = nullptr;        // (front, chunk)
    int32_t *d_pvar = nullptr;      // per front: the variables of its pivot positions
    int *d_cnt = nullptr;           // per front: items done in the backward sweep (0 between solves)
    int64_t z_per_rhs = 0;          // doubles per right-hand side: z of every front
    int64_t part_per_rhs = 0;       // doubles per right-hand side: the largest level's partial sums
    SolvePlan() = default;
    SolvePlan(const SolvePlan &) = delete;
    SolvePlan &operator=(const SolvePlan &) = delete;
    ~SolvePlan() { clear(); }
    void clear();
    // fronts with their levels (nondecreasing) and eliminated counts; perm and
    // rows are read on `st` (synchronised before returning)
    ctp_status build(const std::vector<ctp_sfront> &fronts, const std::vector<int> &level,
                     const std::vector<int32_t> &nelim, cudaStream_t st);
    size_t ws_bytes(int nrhs) const;
    // X <- M^{-1} X; fp32: the sweeps' arithmetic in FP32 (X read and written in FP64)
    cudaError_t solve(ctp_ctx *ctx, double *X, int64_t ldx, int nrhs, void *ws, cudaStream_t st,
                      bool fp32 = false) const;
};

// The system matrix of a residual: dense (lower triangle, column-major) or
// sparse (lower triangle in compressed columns), symmetric either way.
struct MatOp {
    const double *M = nullptr;
    int64_t ldm = 0;
    const int64_t *colptr = nullptr;
    const int32_t *rowind = nullptr;
    const double *val = nullptr;
    bool sparse() const { return colptr != nullptr; }
};

struct RefineLayout {
    size_t solve, R, rowsum, mx, berr, total;
};
RefineLayout refine_layout(int64_t N, size_t solve_ws, int nrhs);

// Residual R = B - A X and the Section 7 backward errors into berr (device).
cudaError_t residual_berr(ctp_ctx *ctx, const MatOp &A, int64_t N, int nrhs, const double *B, int64_t ldb,
                          const double *X, int64_t ldx, double *R, const double *rowsum, double *mx,
                          double *berr, cudaStream_t st);
cudaError_t mat_abs_rowsum(ctp_ctx *ctx, const MatOp &A, int64_t N, double *rowsum, cudaStream_t st);

// X = solve(B); while the worst backward error exceeds tol and fewer than
// max_steps corrections were made: X += solve(B - A X).  `solve(Y, ldy, ws)`
// overwrites the N x nrhs array Y with the solution (cudaError_t).
template <typename Solve>
ctp_status refine_core(ctp_ctx *ctx, Solve &&solve, size_t solve_ws, int64_t N, const MatOp &A, int32_t nrhs,
                       const double *B, int64_t ldb, double *X, int64_t ldx, int32_t max_steps, double tol,
                       double *berr_host, int32_t *steps_host, void *workspace, size_t ws_bytes,
                       cudaStream_t st) {
    RefineLayout L = refine_layout(N, solve_ws, nrhs);
    if (ws_bytes < L.total) return CTP_ENOMEM;
    char *w = (char *)workspace;
    void *sws = w + L.solve;
    double *R = (double *)(w + L.R), *rowsum = (double *)(w + L.rowsum);
    double *mx = (double *)(w + L.mx), *berr = (double *)(w + L.berr);
    *steps_host = 0;
    CTP_CUDA(mat_abs_rowsum(ctx, A, N, rowsum, st));
    CTP_CUDA(cudaMemcpy2DAsync(X, sizeof(double) * ldx, B, sizeof(double) * ldb, sizeof(double) * N, nrhs,
                               cudaMemcpyDeviceToDevice, st));
    CTP_CUDA(solve(X, ldx, sws));
    for (int32_t k = 0;; k++) {
        CTP_CUDA(residual_berr(ctx, A, N, nrhs, B, ldb, X, ldx, R, rowsum, mx, berr, st));
        double *bh = berr_host + (size_t)k * nrhs;
        CTP_CUDA(cudaMemcpyAsync(bh, berr, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
        CTP_CUDA(cudaStreamSynchronize(st));
        double worst = 0.0;
        for (int r = 0; r < nrhs; r++) worst = bh[r] > worst || bh[r] != bh[r] ? bh[r] : worst;
        if (!(worst > tol) || k == max_steps) break;
        CTP_CUDA(solve(R, N, sws));
        CTP_CUDA(timed(ctx, K_AXPY, st, [&] { return launch_axpy(N, nrhs, X, ldx, R, N, st); }));
        *steps_host = k + 1;
    }
    return CTP_OK;
}

}  // namespace ctp
