// solve_plan.cu -- the level-planned front-list solve and the residual helpers
// of iterative refinement (declared in solve_plan.cuh).
#include "solve_plan.cuh"

namespace ctp {

void SolvePlan::clear() {
    if (d_F) cudaFree(d_F);
    if (d_items) cudaFree(d_items);
    if (d_poff) cudaFree(d_poff);
    d_F = nullptr;
    d_items = nullptr;
    d_poff = nullptr;
    nf = nlev = 0;
    lev_ptr.clear();
    item_ptr.clear();
    max_fronts = 0;
    max_chunks = 0;
}

ctp_status SolvePlan::build(const std::vector<ctp_sfront> &fronts, const std::vector<int> &level,
                            const std::vector<int32_t> &nelim) {
    clear();
    nf = (int)fronts.size();
    if (nf == 0) return CTP_OK;
    std::vector<int2> items;
    std::vector<int64_t> poff(nf);
    lev_ptr.push_back(0);
    item_ptr.push_back(0);
    int64_t chunks_in_level = 0;
    for (int k = 0; k < nf; k++) {
        if (k > 0 && level[k] < level[k - 1]) return CTP_EINVAL;
        if (k > 0 && level[k] != level[k - 1]) {
            lev_ptr.push_back(k);
            item_ptr.push_back((int64_t)items.size());
            chunks_in_level = 0;
        }
        const int local = k - lev_ptr.back();
        const int64_t below = fronts[k].n - nelim[k];
        const int64_t nch = (below + 255) / 256;
        poff[k] = chunks_in_level;
        for (int64_t c = 0; c < nch; c++) items.push_back(make_int2(local, (int)c));
        chunks_in_level += nch;
        max_chunks = chunks_in_level > max_chunks ? chunks_in_level : max_chunks;
    }
    lev_ptr.push_back(nf);
    item_ptr.push_back((int64_t)items.size());
    nlev = (int)lev_ptr.size() - 1;
    for (int l = 0; l < nlev; l++) {
        const int nfl = lev_ptr[l + 1] - lev_ptr[l];
        max_fronts = nfl > max_fronts ? nfl : max_fronts;
    }
    if (cudaMalloc(&d_F, sizeof(ctp_sfront) * nf) != cudaSuccess ||
        cudaMalloc(&d_items, sizeof(int2) * (items.size() > 0 ? items.size() : 1)) != cudaSuccess ||
        cudaMalloc(&d_poff, sizeof(int64_t) * nf) != cudaSuccess)
        return CTP_ENOMEM;
    if (cudaMemcpy(d_F, fronts.data(), sizeof(ctp_sfront) * nf, cudaMemcpyHostToDevice) != cudaSuccess ||
        (!items.empty() &&
         cudaMemcpy(d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy(d_poff, poff.data(), sizeof(int64_t) * nf, cudaMemcpyHostToDevice) != cudaSuccess)
        return CTP_ECUDA;
    return CTP_OK;
}

size_t SolvePlan::ws_bytes(int nrhs) const {
    return align256(sizeof(double) * (size_t)(max_fronts > 0 ? max_fronts : 1) * kMaxP * nrhs) +
           align256(sizeof(double) * (size_t)(max_chunks > 0 ? max_chunks : 1) * nrhs * kMaxP);
}

cudaError_t SolvePlan::solve(ctp_ctx *ctx, double *X, int64_t ldx, int nrhs, void *ws, cudaStream_t st) const {
    double *Y = (double *)ws;
    double *part = (double *)((char *)ws + align256(sizeof(double) * (size_t)(max_fronts > 0 ? max_fronts : 1) *
                                                    kMaxP * nrhs));
    for (int l = 0; l < nlev; l++) {
        const int f0 = lev_ptr[l], nfl = lev_ptr[l + 1] - f0;
        cudaError_t e = timed(ctx, K_SYS_FWD, st, [&] {
            return launch_sys_level_forward(d_F + f0, nfl, d_items + item_ptr[l], item_ptr[l + 1] - item_ptr[l], X,
                                            ldx, nrhs, Y, st);
        });
        if (e != cudaSuccess) return e;
    }
    for (int l = nlev - 1; l >= 0; l--) {
        const int f0 = lev_ptr[l], nfl = lev_ptr[l + 1] - f0;
        cudaError_t e = timed(ctx, K_SYS_BWD, st, [&] {
            return launch_sys_level_backward(d_F + f0, nfl, d_items + item_ptr[l], item_ptr[l + 1] - item_ptr[l],
                                             d_poff + f0, X, ldx, nrhs, part, st);
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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
