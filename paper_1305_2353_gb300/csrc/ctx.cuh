// ctx.cuh -- the library context and the per-kernel profiling hook shared by
// the translation units that implement the C ABI.
#pragma once

#include "ctp_internal.cuh"

namespace ctp {
constexpr int kMaxRec = 32768;
constexpr int kSideStreams = 5;  // the batch's pivot-search classes run on these, round robin
enum KernelId {
    K_COMPRESS_STRICT = 0, K_KEYS, K_RELAXED, K_FACTOR, K_SOLVE, K_FORM, K_FORM_TC, K_TPP,
    K_B_PREPARE, K_B_COMPRESS, K_B_FACTOR_G1, K_B_FACTOR_G2, K_B_FACTOR_G4, K_B_FACTOR_G8,
    K_B_FACTOR_G16, K_B_SOLVE, K_B_FORM, K_W21, K_SYS_FWD, K_SYS_BWD, K_SYMV, K_BERR, K_AXPY,
    K_FORM_TC3, K_GRAD, K_MF_ASSEMBLE, K_MF_EXTEND_ADD, K_SPMV, K_FORM_TC6, K_SOLVE_TC, K_B_FACTOR_WARP,
    K_NUM_IDS
};
extern const char *kKernelNames[K_NUM_IDS];
}  // namespace ctp

struct ctp_ctx {
    int device;
    int num_sms;
    int form_walk;      // CTP_TUNE_FORM_WALK
    int batch_smem_kb;  // CTP_TUNE_BATCH_SMEM_KB
    int factor_g;       // CTP_TUNE_FACTOR_G
    int tpp_spin;       // CTP_TUNE_TPP_SPIN (0: the kernel's default)
    bool profiling;
    int nrec;
    int rec_id[ctp::kMaxRec];
    cudaEvent_t ev[2 * ctp::kMaxRec];
    bool events_made;
    // side streams on which a batch's pivot-search classes run side by side
    cudaStream_t side[ctp::kSideStreams];
    cudaEvent_t fork_ev, join_ev[ctp::kSideStreams];
    bool side_made;
};

namespace ctp {
// Launch `launch()` (a cudaError_t expression enqueueing kernels on `st`),
// bracketed by profiling events when enabled.
template <typename F>
static cudaError_t timed(ctp_ctx *ctx, int id, cudaStream_t st, F &&launch) {
    if (!ctx->profiling || ctx->nrec >= kMaxRec) return launch();
    const int r = ctx->nrec++;
    ctx->rec_id[r] = id;
    cudaEventRecord(ctx->ev[2 * r], st);
    cudaError_t e = launch();
    cudaEventRecord(ctx->ev[2 * r + 1], st);
    return e;
}
}  // namespace ctp

#define CTP_CUDA(x)                               \
    do {                                          \
        if ((x) != cudaSuccess) return CTP_ECUDA; \
    } while (0)
