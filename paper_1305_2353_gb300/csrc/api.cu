// api.cu -- the C ABI of libctp (declared in include/ctp.h): argument checks,
// workspace layout and the launch sequence of the per-supernode hot path.
#include <stdlib.h>
#include <string.h>

#include "ctp_internal.cuh"

namespace {
constexpr int kMaxRec = 4096;
enum KernelId {
    K_COMPRESS_STRICT = 0, K_KEYS, K_RELAXED, K_FACTOR, K_SOLVE, K_FORM, K_FORM_TC, K_TPP,
    K_B_PREPARE, K_B_COMPRESS, K_B_FACTOR_G1, K_B_FACTOR_G2, K_B_FACTOR_G4, K_B_FACTOR_G8,
    K_B_FACTOR_G16, K_B_SOLVE, K_B_FORM, K_NUM_IDS
};
const char *kKernelNames[K_NUM_IDS] = {"compress_strict", "keys_to_rowmajor", "compress_relaxed",
                                       "factor_cluster", "solve_fp64", "form_fp64", "form_tc_bf16",
                                       "tpp_full_column", "batch_prepare", "batch_compress_strict",
                                       "batch_factor_g1", "batch_factor_g2", "batch_factor_g4",
                                       "batch_factor_g8", "batch_factor_g16", "batch_solve_fp64",
                                       "batch_form"};
}  // namespace

struct ctp_ctx {
    int device;
    int num_sms;
    bool profiling;
    int nrec;
    int rec_id[kMaxRec];
    cudaEvent_t ev[2 * kMaxRec];
    bool events_made;
};

// Launch `expr` (a cudaError_t expression enqueueing one kernel on `st`),
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

namespace ctp {

WsLayout ws_layout(int64_t n, int p, const ctp_options *opt, int num_sms) {
    WsLayout L;
    const int64_t m = n - p;
    size_t off = 0;
    L.info = off;
    off += 256;
    L.C = off;
    const bool compressed = opt->pivot == CTP_PIV_STRICT || opt->pivot == CTP_PIV_RELAXED;
    off += align256(compressed ? sizeof(double) * (size_t)p * p : 0);
    L.Dinv = off;
    off += align256(sizeof(double) * (2 * (size_t)p + 2));
    const bool tc = opt->prec == CTP_BF16 && opt->smode != CTP_S_NONE;
    L.W21 = off;
    off += align256(opt->smode != CTP_S_NONE && !tc ? sizeof(double) * (size_t)m * p : 0);
    const size_t nb = tc ? 2 * (size_t)m * form_tc_kpad(p) : 0;
    L.Wb = off;
    off += align256(nb);
    L.Lb = off;
    off += align256(nb);
    L.aux = off;
    off += align256(opt->pivot == CTP_PIV_RELAXED ? relaxed_aux_bytes(m, p, num_sms)
                                                  : (opt->pivot == CTP_PIV_TPP ? tpp_ws_bytes(p) : 0));
    L.total = off;
    return L;
}

}  // namespace ctp

using namespace ctp;

#define CTP_CUDA(x)                            \
    do {                                       \
        if ((x) != cudaSuccess) return CTP_ECUDA; \
    } while (0)

extern "C" {

int32_t ctp_max_p(void) { return kMaxP; }

ctp_status ctp_create(ctp_ctx **ctx, int32_t device) {
    if (ctx == nullptr) return CTP_EINVAL;
    *ctx = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return CTP_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return CTP_ECUDA;
    ctp_ctx *c = (ctp_ctx *)malloc(sizeof(ctp_ctx));
    if (c == nullptr) return CTP_ENOMEM;
    c->device = device;
    c->num_sms = sms;
    c->profiling = false;
    c->nrec = 0;
    c->events_made = false;
    *ctx = c;
    return CTP_OK;
}

ctp_status ctp_destroy(ctp_ctx *ctx) {
    if (ctx != nullptr && ctx->events_made)
        for (int i = 0; i < 2 * kMaxRec; i++) cudaEventDestroy(ctx->ev[i]);
    free(ctx);
    return CTP_OK;
}

static ctp_status check_opts(const ctp_options *opt) {
    if (opt == nullptr) return CTP_EINVAL;
    if (!(opt->u > 0.0) || opt->u > 0.5) return CTP_EINVAL;
    if (!(opt->small >= 0.0)) return CTP_EINVAL;
    if (opt->pivot < CTP_PIV_STRICT || opt->pivot > CTP_PIV_RESTRICTED) return CTP_EINVAL;
    if (opt->prec != CTP_FP64 && opt->prec != CTP_BF16) return CTP_EINVAL;
    if (opt->smode < CTP_S_NONE || opt->smode > CTP_S_FP32_TILED) return CTP_EINVAL;
    return CTP_OK;
}

ctp_status ctp_workspace_size(const ctp_ctx *ctx, int64_t n, int32_t p, const ctp_options *opt,
                              size_t *bytes) {
    if (ctx == nullptr || bytes == nullptr || p < 1 || n < p) return CTP_EINVAL;
    ctp_status s = check_opts(opt);
    if (s != CTP_OK) return s;
    *bytes = ws_layout(n, p, opt, ctx->num_sms).total;
    return CTP_OK;
}

ctp_status ctp_compress_strict(ctp_ctx *ctx, int64_t m, int32_t p, const double *A21, int64_t lda,
                               double *C, int32_t *J, void *workspace, size_t ws_bytes,
                               void *stream) {
    if (ctx == nullptr || A21 == nullptr || C == nullptr || workspace == nullptr) return CTP_EINVAL;
    if (m < 0 || p < 1 || lda < (m > 0 ? m : 1)) return CTP_EINVAL;
    if (p > kMaxP) return CTP_EUNSUPPORTED;
    ctp_options o = {0.01, 1e-20, CTP_PIV_STRICT, CTP_FP64, CTP_S_NONE, 0};
    WsLayout L = ws_layout(m + p, p, &o, ctx->num_sms);
    if (ws_bytes < L.total) return CTP_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    int32_t *info = (int32_t *)(ws + L.info);
    unsigned long long *keys = (unsigned long long *)(ws + L.C);
    CTP_CUDA(cudaMemsetAsync(info, 0, sizeof(int32_t), st));
    CTP_CUDA(cudaMemsetAsync(keys, 0, sizeof(double) * (size_t)p * p, st));
    CTP_CUDA(timed(ctx, K_COMPRESS_STRICT, st, [&] {
        return launch_compress_strict(A21, m, p, lda, keys, J, info, ctx->num_sms, st);
    }));
    CTP_CUDA(timed(ctx, K_KEYS, st, [&] { return launch_keys_to_rowmajor(keys, C, p, st); }));
    return CTP_OK;
}

ctp_status ctp_compress_relaxed(ctp_ctx *ctx, int64_t m, int32_t p, const double *A21,
                                int64_t lda, double *C, int32_t *rows, void *workspace,
                                size_t ws_bytes, void *stream) {
    if (ctx == nullptr || A21 == nullptr || C == nullptr || workspace == nullptr) return CTP_EINVAL;
    if (m < 0 || p < 1 || lda < (m > 0 ? m : 1)) return CTP_EINVAL;
    if (p > kMaxP) return CTP_EUNSUPPORTED;
    ctp_options o = {0.01, 1e-20, CTP_PIV_RELAXED, CTP_FP64, CTP_S_NONE, 0};
    WsLayout L = ws_layout(m + p, p, &o, ctx->num_sms);
    if (ws_bytes < L.total) return CTP_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    int32_t *info = (int32_t *)(ws + L.info);
    CTP_CUDA(cudaMemsetAsync(info, 0, sizeof(int32_t), st));
    CTP_CUDA(timed(ctx, K_RELAXED, st, [&] {
        return launch_compress_relaxed(A21, m, p, lda, C, rows, ws + L.aux, info, ctx->num_sms, st);
    }));
    return CTP_OK;
}

ctp_status ctp_factor_supernode(ctp_ctx *ctx, int64_t n, int32_t p, double *A, int64_t lda,
                                const ctp_options *opt, int32_t *perm, int32_t *piv, double *D,
                                int32_t *nelim, void *S, int64_t lds, void *workspace,
                                size_t ws_bytes, void *stream) {
    if (ctx == nullptr || A == nullptr || perm == nullptr || piv == nullptr || D == nullptr ||
        nelim == nullptr || workspace == nullptr)
        return CTP_EINVAL;
    if (p < 1 || n < p || lda < n) return CTP_EINVAL;
    ctp_status s = check_opts(opt);
    if (s != CTP_OK) return s;
    const int64_t m = n - p;
    const bool packed = opt->smode == CTP_S_FP64_PACKED || opt->smode == CTP_S_FP32_PACKED ||
                        opt->smode == CTP_S_FP32_TILED;
    if (opt->smode != CTP_S_NONE && (S == nullptr || (!packed && lds < (m > 0 ? m : 1))))
        return CTP_EINVAL;
    if (p > kMaxP) return CTP_EUNSUPPORTED;
    if (opt->pivot == CTP_PIV_TPP && opt->smode != CTP_S_NONE) return CTP_EUNSUPPORTED;
    const bool tc = opt->prec == CTP_BF16 && opt->smode != CTP_S_NONE;
    if (tc && opt->smode != CTP_S_FP32 && opt->smode != CTP_S_FP32_PACKED &&
        opt->smode != CTP_S_FP32_TILED)
        return CTP_EUNSUPPORTED;  // the tensor-core Form writes FP32
    if (!tc && opt->smode == CTP_S_FP32_TILED) return CTP_EUNSUPPORTED;
    WsLayout L = ws_layout(n, p, opt, ctx->num_sms);
    if (ws_bytes < L.total) return CTP_ENOMEM;

    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    int32_t *info = (int32_t *)(ws + L.info);
    double *Dinv = (double *)(ws + L.Dinv);
    double *W21 = (opt->smode != CTP_S_NONE && !tc) ? (double *)(ws + L.W21) : nullptr;
    void *Wb = tc ? (void *)(ws + L.Wb) : nullptr;
    void *Lbf = tc ? (void *)(ws + L.Lb) : nullptr;
    const int Kp = form_tc_kpad(p);
    CTP_CUDA(cudaMemsetAsync(info, 0, sizeof(int32_t), st));

    if (opt->pivot == CTP_PIV_TPP) {
        // Listing 1 on all n rows: factor and solve in one cooperative kernel
        CTP_CUDA(timed(ctx, K_TPP, st, [&] {
            return launch_tpp(A, n, p, lda, opt->u, opt->small, ws + L.aux, perm, piv, D, Dinv, nelim,
                              info, ctx->num_sms, st);
        }));
        return CTP_OK;
    }
    FactorArgs fa;
    fa.A = A;
    fa.lda = lda;
    fa.p = p;
    fa.u = opt->u;
    fa.small = opt->small;
    fa.perm = perm;
    fa.piv = piv;
    fa.nelim = nelim;
    fa.D = D;
    fa.Dinv = Dinv;
    fa.info = info;
    if (opt->pivot == CTP_PIV_STRICT) {
        unsigned long long *keys = (unsigned long long *)(ws + L.C);
        CTP_CUDA(cudaMemsetAsync(keys, 0, sizeof(double) * (size_t)p * p, st));
        CTP_CUDA(timed(ctx, K_COMPRESS_STRICT, st, [&] {
            return launch_compress_strict(A + p, m, p, lda, keys, nullptr, info, ctx->num_sms, st);
        }));
        fa.R = p;
        fa.abs_update = 1;
        fa.C = (const double *)keys;  // non-negative keys are the doubles themselves
    } else if (opt->pivot == CTP_PIV_RELAXED) {
        double *C = (double *)(ws + L.C);
        CTP_CUDA(timed(ctx, K_RELAXED, st, [&] {
            return launch_compress_relaxed(A + p, m, p, lda, C, nullptr, ws + L.aux, info,
                                           ctx->num_sms, st);
        }));
        fa.R = p;
        fa.abs_update = 0;
        fa.C = C;
    } else {  // restricted: the tests look at A11 only
        fa.R = 0;
        fa.abs_update = 0;
        fa.C = nullptr;
    }
    CTP_CUDA(timed(ctx, K_FACTOR, st, [&] { return launch_factor_cluster(fa, st); }));
    if (m > 0)
        CTP_CUDA(timed(ctx, K_SOLVE, st, [&] {
            return launch_solve_fp64(A, n, p, lda, perm, piv, Dinv, nelim, W21, m, Wb, Lbf, Kp, st);
        }));
    if (opt->smode != CTP_S_NONE && m > 0) {
        if (tc)
            CTP_CUDA(timed(ctx, K_FORM_TC, st, [&] {
                return launch_form_tc(Wb, Lbf, m, Kp, nelim, (float *)S, lds,
                                      opt->smode == CTP_S_FP32_TILED ? 2 : (packed ? 1 : 0), info,
                                      ctx->num_sms, st);
            }));
        else
            CTP_CUDA(timed(ctx, K_FORM, st, [&] {
                return launch_form_fp64(A + p, lda, W21, m, m, nelim, S, lds, opt->smode, st);
            }));
    }
    return CTP_OK;
}

ctp_status ctp_read_info(ctp_ctx *ctx, const void *workspace, int32_t *info_host, void *stream) {
    if (ctx == nullptr || workspace == nullptr || info_host == nullptr) return CTP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    CTP_CUDA(cudaMemcpyAsync(info_host, workspace, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CTP_CUDA(cudaStreamSynchronize(st));
    return CTP_OK;
}

ctp_status ctp_profile_begin(ctp_ctx *ctx) {
    if (ctx == nullptr) return CTP_EINVAL;
    if (!ctx->events_made) {
        for (int i = 0; i < 2 * kMaxRec; i++)
            if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess) return CTP_ECUDA;
        ctx->events_made = true;
    }
    ctx->nrec = 0;
    ctx->profiling = true;
    return CTP_OK;
}

ctp_status ctp_profile_end(ctp_ctx *ctx, int32_t max_kernels, char *names, double *total_ms,
                           int32_t *launches, int32_t *nkernels) {
    if (ctx == nullptr || nkernels == nullptr || max_kernels < 0) return CTP_EINVAL;
    ctx->profiling = false;
    double tot[K_NUM_IDS] = {};
    int cnt[K_NUM_IDS] = {};
    for (int r = 0; r < ctx->nrec; r++) {
        if (cudaEventSynchronize(ctx->ev[2 * r + 1]) != cudaSuccess) return CTP_ECUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev[2 * r], ctx->ev[2 * r + 1]) != cudaSuccess)
            return CTP_ECUDA;
        tot[ctx->rec_id[r]] += ms;
        cnt[ctx->rec_id[r]]++;
    }
    int k = 0;
    for (int id = 0; id < K_NUM_IDS; id++) {
        if (cnt[id] == 0) continue;
        if (k < max_kernels) {
            if (names) {
                strncpy(names + 48 * k, kKernelNames[id], 47);
                names[48 * k + 47] = 0;
            }
            if (total_ms) total_ms[k] = tot[id];
            if (launches) launches[k] = cnt[id];
        }
        k++;
    }
    *nkernels = k;
    ctx->nrec = 0;
    return CTP_OK;
}

ctp_status ctp_factor_batch(ctp_ctx *ctx, const ctp_plan *plan, const ctp_front *fronts,
                            void *workspace, size_t ws_bytes, void *stream) {
    if (ctx == nullptr || plan == nullptr || fronts == nullptr || workspace == nullptr) return CTP_EINVAL;
    if (ws_bytes < batch_total(plan)) return CTP_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)workspace;
    CTP_CUDA(timed(ctx, K_B_PREPARE, st, [&] { return batch_prepare(plan, w, st); }));
    CTP_CUDA(timed(ctx, K_B_COMPRESS, st, [&] { return batch_compress(plan, fronts, w, ctx->num_sms, st); }));
    for (int c = 0; c < batch_num_classes(plan); c++) {
        const int G = batch_class_G(plan, c);
        const int id = K_B_FACTOR_G1 + (G == 1 ? 0 : G == 2 ? 1 : G == 4 ? 2 : G == 8 ? 3 : 4);
        CTP_CUDA(timed(ctx, id, st, [&] { return batch_factor_class(plan, c, fronts, w, st); }));
    }
    CTP_CUDA(timed(ctx, K_B_SOLVE, st, [&] { return batch_solve(plan, fronts, w, st); }));
    CTP_CUDA(timed(ctx, K_B_FORM, st, [&] { return batch_form(plan, fronts, w, ctx->num_sms, st); }));
    return CTP_OK;
}

}  // extern "C"
