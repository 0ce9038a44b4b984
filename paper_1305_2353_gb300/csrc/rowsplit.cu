// rowsplit.cu -- the row split of one supernode over P processors (Section 6,
// Table 6.1, Appendix A): A21's rows are cut into P blocks, each processor
// compresses its own block, and one exchange builds the compressed matrix of the
// whole supernode.
//  * strict (Section 4.1): c(j,k) is a maximum over the rows with J(i) = j, so
//    the blocks' matrices combine by an elementwise maximum -- exact and
//    independent of the order (an allreduce with the max operation);
//  * relaxed (Section 4.2): column j's choice lies among the j+1 largest
//    |a21(i,j)| of the whole column (at most j rows are flagged before it), and
//    those lie among the union of every block's own j+1 largest.  So each block
//    sends its per-column candidate lists (a gather), one processor runs the
//    greedy on their union, and the owners of the chosen rows send those rows.
// Here the P blocks live on one GPU; the entry points are the per-block steps
// and the exchange steps of that scheme, so that the exchange can be checked
// against the single-pass compression bit for bit.
#include "ctx.cuh"

namespace ctp {

size_t relaxed_candidate_bytes(int nslot, int p);
cudaError_t launch_relaxed_candidates(const double *A21, int64_t m, int p, int64_t lda, int row0, int slot,
                                      int nslot, void *cand, int32_t *info, cudaStream_t st);
cudaError_t launch_relaxed_select(int p, int nslot, const void *cand, int32_t *rows, cudaStream_t st);
cudaError_t launch_gather_rows(const double *A21, int64_t lda, int p, const int32_t *rows, double *C,
                               cudaStream_t st);

namespace {

constexpr int kMaxBlocks = 8;  // candidate lists per column the greedy stages on chip

// C = elementwise max over P blocks of nonnegative matrices, block b at
// Cb + b * stride.  The entries of strict compressed matrices are |a21| values
// or 0, so the maximum is taken on their bit patterns (integer order).
__global__ void k_strict_merge(const double *__restrict__ Cb, int64_t stride, int P, int64_t n,
                               double *__restrict__ C) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long best = 0;
        for (int b = 0; b < P; b++) {
            const unsigned long long k = (unsigned long long)__double_as_longlong(Cb[b * stride + i]);
            best = k > best ? k : best;
        }
        C[i] = __longlong_as_double((long long)best);
    }
}

}  // namespace
}  // namespace ctp

using namespace ctp;

extern "C" {

ctp_status ctp_compress_strict_merge(ctp_ctx *ctx, int32_t P, int32_t p, const double *C_blocks,
                                     int64_t block_stride, double *C, void *stream) {
    if (ctx == nullptr || C_blocks == nullptr || C == nullptr || P < 1 || p < 1) return CTP_EINVAL;
    if (p > kMaxP) return CTP_EUNSUPPORTED;
    if (block_stride < (int64_t)p * p) return CTP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)p * p;
    k_strict_merge<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(C_blocks, block_stride, P, n, C);
    CTP_CUDA(cudaGetLastError());
    return CTP_OK;
}

ctp_status ctp_relaxed_candidates_size(int32_t P, int32_t p, size_t *bytes) {
    if (bytes == nullptr || P < 1 || p < 1) return CTP_EINVAL;
    if (p > kMaxP || P > kMaxBlocks) return CTP_EUNSUPPORTED;
    *bytes = 256 + relaxed_candidate_bytes(P, p);
    return CTP_OK;
}

ctp_status ctp_compress_relaxed_candidates(ctp_ctx *ctx, int64_t m, int32_t p, const double *A21, int64_t lda,
                                           int64_t row0, int32_t P, int32_t block, void *cand,
                                           size_t cand_bytes, void *stream) {
    if (ctx == nullptr || A21 == nullptr || cand == nullptr || P < 1 || p < 1) return CTP_EINVAL;
    if (m < 0 || lda < (m > 0 ? m : 1) || row0 < 0 || block < 0 || block >= P) return CTP_EINVAL;
    if (p > kMaxP || P > kMaxBlocks || row0 + m > 0x7fffffffLL) return CTP_EUNSUPPORTED;
    if (cand_bytes < 256 + relaxed_candidate_bytes(P, p)) return CTP_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    char *c = (char *)cand;
    CTP_CUDA(timed(ctx, K_RELAXED, st, [&] {
        return launch_relaxed_candidates(A21, m, p, lda, (int)row0, block, P, c + 256,
                                         reinterpret_cast<int32_t *>(c), st);
    }));
    return CTP_OK;
}

ctp_status ctp_compress_relaxed_select(ctp_ctx *ctx, int32_t P, int32_t p, const void *cand, size_t cand_bytes,
                                       int32_t *rows, void *stream) {
    if (ctx == nullptr || cand == nullptr || rows == nullptr || P < 1 || p < 1) return CTP_EINVAL;
    if (p > kMaxP || P > kMaxBlocks) return CTP_EUNSUPPORTED;
    if (cand_bytes < 256 + relaxed_candidate_bytes(P, p)) return CTP_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    CTP_CUDA(launch_relaxed_select(p, P, (const char *)cand + 256, rows, st));
    return CTP_OK;
}

ctp_status ctp_gather_rows(ctp_ctx *ctx, int32_t p, const double *A21, int64_t lda, const int32_t *rows, double *C,
                           void *stream) {
    if (ctx == nullptr || A21 == nullptr || rows == nullptr || C == nullptr || p < 1 || lda < 1) return CTP_EINVAL;
    if (p > kMaxP) return CTP_EUNSUPPORTED;
    CTP_CUDA(launch_gather_rows(A21, lda, p, rows, C, (cudaStream_t)stream));
    return CTP_OK;
}

}  // extern "C"
