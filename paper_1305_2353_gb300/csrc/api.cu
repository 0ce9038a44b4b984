// api.cu -- the C ABI of libctp (declared in include/ctp.h): argument checks,
// workspace layout and the launch sequence of the per-supernode hot path.
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "chain.cuh"
#include "ctx.cuh"
#include "solve_plan.cuh"

namespace ctp {
const char *kKernelNames[K_NUM_IDS] = {"compress_strict", "keys_to_rowmajor", "compress_relaxed",
                                       "factor_cluster", "solve_fp64", "form_fp64", "form_tc_bf16",
                                       "tpp_full_column", "batch_prepare", "batch_compress_strict",
                                       "batch_factor_cta", "batch_factor_g2", "batch_factor_g4",
                                       "batch_factor_g8", "batch_factor_g16", "batch_solve_fp64",
                                       "batch_form", "w21_from_l", "sys_forward", "sys_backward",
                                       "symv_residual", "backward_error", "axpy", "form_tc_bf16x3",
                                       "sym_grad", "mf_assemble", "mf_extend_add", "spmv_residual",
                                       "form_tc_bf16x6", "solve_tc", "batch_factor_warp"};
}  // namespace ctp

namespace ctp {

int ctx_batch_smem_kb(const ctp_ctx *ctx) { return ctx->batch_smem_kb; }

cudaError_t smem_at_least(const void *func, size_t bytes) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);  // query and raise as one step
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

WsLayout ws_layout(int64_t n, int p, const ctp_options *opt, int num_sms) {
    WsLayout L;
    const int64_t m = n - p;
    size_t off = 0;
    L.info = off;
    off += 256;
    L.C = off;
    const bool compressed = opt->pivot == CTP_PIV_STRICT || opt->pivot == CTP_PIV_RELAXED ||
                            opt->pivot == CTP_PIV_SINGLE_ROW;
    off += align256(compressed ? sizeof(double) * (size_t)p * p : 0);
    L.Dinv = off;
    off += align256(sizeof(double) * (2 * (size_t)p + 2));
    const bool tc = opt->prec != CTP_FP64 && opt->smode != CTP_S_NONE;
    L.W21 = off;
    off += align256(opt->smode != CTP_S_NONE && !tc ? sizeof(double) * (size_t)m * p : 0);
    // BF16 operand copies (hi, and for the split form the lo parts after them)
    const size_t nb = tc ? 2 * (size_t)m * form_tc_kpad(p) * prec_pieces(opt->prec) : 0;
    L.Wb = off;
    off += align256(nb);
    L.Lb = off;
    off += align256(nb);
    L.aux = off;
    off += align256(opt->pivot == CTP_PIV_RELAXED ? relaxed_aux_bytes(m, p, num_sms)
                                                  : (opt->pivot == CTP_PIV_TPP ? tpp_ws_bytes(p) : 0));
    // tensor-core Solve: split-BF16 copies of x_e and Z^T
    L.Xs = off;
    off += align256(solve_on_tc(opt) ? solve_tc_ws_bytes(m, p, solve_tc_pieces(opt->prec)) : 0);
    L.flags = off;  // strict: which rows of C receive an A21 row
    off += align256(opt->pivot == CTP_PIV_STRICT ? sizeof(int32_t) * (size_t)p : 0);
    L.total = off;
    return L;
}

}  // namespace ctp

using namespace ctp;


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
    c->form_walk = CTP_WALK_AUTO;
    c->batch_smem_kb = 200;
    c->factor_g = 0;
    c->tpp_spin = 0;
    c->profiling = false;
    c->nrec = 0;
    c->events_made = false;
    c->side_made = false;
    *ctx = c;
    return CTP_OK;
}

ctp_status ctp_destroy(ctp_ctx *ctx) {
    if (ctx != nullptr && ctx->events_made)
        for (int i = 0; i < 2 * kMaxRec; i++) cudaEventDestroy(ctx->ev[i]);
    if (ctx != nullptr && ctx->side_made) {
        for (int i = 0; i < kSideStreams; i++) {
            cudaStreamDestroy(ctx->side[i]);
            cudaEventDestroy(ctx->join_ev[i]);
        }
        cudaEventDestroy(ctx->fork_ev);
    }
    free(ctx);
    return CTP_OK;
}

static ctp_status check_opts(const ctp_options *opt) {
    if (opt == nullptr) return CTP_EINVAL;
    if (!(opt->u > 0.0) || opt->u > 0.5) return CTP_EINVAL;
    if (!(opt->small >= 0.0)) return CTP_EINVAL;
    if (opt->pivot < CTP_PIV_STRICT || opt->pivot > CTP_PIV_SINGLE_ROW) return CTP_EINVAL;
    if (opt->prec < CTP_FP64 || opt->prec > CTP_BF16X6) return CTP_EINVAL;
    if (opt->smode < CTP_S_NONE || opt->smode > CTP_S_FP64_SUB) return CTP_EINVAL;
    if (opt->solve != CTP_SOLVE_FP64 && opt->solve != CTP_SOLVE_TC) return CTP_EINVAL;
    return CTP_OK;
}

ctp_status ctp_tune_set(ctp_ctx *ctx, int32_t key, int32_t value) {
    if (ctx == nullptr) return CTP_EINVAL;
    if (key == CTP_TUNE_FORM_WALK) {
        if (value < CTP_WALK_AUTO || value > CTP_WALK_PANELS) return CTP_EINVAL;
        ctx->form_walk = value;
        return CTP_OK;
    }
    if (key == CTP_TUNE_BATCH_SMEM_KB) {
        if (value < 48 || value > 220) return CTP_EINVAL;
        ctx->batch_smem_kb = value;
        return CTP_OK;
    }
    if (key == CTP_TUNE_FACTOR_G) {
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
            return CTP_EINVAL;
        ctx->factor_g = value;
        return CTP_OK;
    }
    if (key == CTP_TUNE_TPP_SPIN) {
        if (value < 0 || value > (1 << 24)) return CTP_EINVAL;
        ctx->tpp_spin = value;
        return CTP_OK;
    }
    return CTP_EINVAL;
}

ctp_status ctp_tune_get(const ctp_ctx *ctx, int32_t key, int32_t *value) {
    if (ctx == nullptr || value == nullptr) return CTP_EINVAL;
    if (key == CTP_TUNE_FORM_WALK)
        *value = ctx->form_walk;
    else if (key == CTP_TUNE_BATCH_SMEM_KB)
        *value = ctx->batch_smem_kb;
    else if (key == CTP_TUNE_FACTOR_G)
        *value = ctx->factor_g;
    else if (key == CTP_TUNE_TPP_SPIN)
        *value = ctx->tpp_spin;
    else
        return CTP_EINVAL;
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
        return launch_compress_strict(A21, m, p, lda, keys, J, nullptr, info, ctx->num_sms, st);
    }));
    CTP_CUDA(timed(ctx, K_KEYS, st, [&] { return launch_keys_to_rowmajor(keys, C, p, st); }));
    return CTP_OK;
}

ctp_status ctp_compress_relaxed(ctp_ctx *ctx, int64_t m, int32_t p, const double *A21,
                                int64_t lda, double *C, int32_t *rows, void *workspace,
                                size_t ws_bytes, void *stream) {
    if (ctx == nullptr || A21 == nullptr || C == nullptr || workspace == nullptr) return CTP_EINVAL;
    if (m < 0 || p < 1 || lda < (m > 0 ? m : 1)) return CTP_EINVAL;
    if (p > kMaxP || m > 0x7fffffffLL) return CTP_EUNSUPPORTED;  // rows are reported as int32
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
    if (p > kMaxP || n > 0x7fffffffLL) return CTP_EUNSUPPORTED;  // row indices are int32
    const bool tc = opt->prec != CTP_FP64 && opt->smode != CTP_S_NONE;
    if (opt->pivot == CTP_PIV_TPP && tc) return CTP_EUNSUPPORTED;
    if (tc && opt->smode != CTP_S_FP32 && opt->smode != CTP_S_FP32_PACKED &&
        opt->smode != CTP_S_FP32_TILED && opt->smode != CTP_S_FP64_SUB)
        return CTP_EUNSUPPORTED;  // the tensor-core Form writes FP32 (or subtracts into FP64)
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
    const int pieces = tc ? prec_pieces(opt->prec) : 0;
    const int64_t lo_off = pieces > 1 ? m * Kp : 0;
    CTP_CUDA(cudaMemsetAsync(info, 0, sizeof(int32_t), st));

    if (opt->pivot == CTP_PIV_TPP) {
        // Listing 1 on all n rows: factor and solve in one cooperative kernel
        CTP_CUDA(timed(ctx, K_TPP, st, [&] {
            return launch_tpp(A, n, p, lda, opt->u, opt->small, ws + L.aux, perm, piv, D, Dinv, nelim,
                              info, ctx->num_sms, ctx->tpp_spin, st);
        }));
        if (opt->smode != CTP_S_NONE && m > 0) {
            CTP_CUDA(timed(ctx, K_W21, st, [&] {
                return launch_w21_from_l(A, lda, p, m, piv, D, nelim, W21, m, st);
            }));
            CTP_CUDA(timed(ctx, K_FORM, st, [&] {
                return launch_form_fp64(A + p, lda, W21, m, m, nelim, S, lds, opt->smode, st);
            }));
        }
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
    fa.rowbits = nullptr;
    if (opt->pivot == CTP_PIV_STRICT) {
        unsigned long long *keys = (unsigned long long *)(ws + L.C);
        uint32_t *flags = (uint32_t *)(ws + L.flags);
        CTP_CUDA(cudaMemsetAsync(keys, 0, sizeof(double) * (size_t)p * p, st));
        CTP_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (size_t)((p + 31) / 32), st));
        CTP_CUDA(timed(ctx, K_COMPRESS_STRICT, st, [&] {
            return launch_compress_strict(A + p, m, p, lda, keys, nullptr, flags, info, ctx->num_sms, st);
        }));
        fa.rowbits = flags;
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
    } else if (opt->pivot == CTP_PIV_SINGLE_ROW) {
        // one row of column maxima (eq. (4.1) with J = all rows), worst-case update
        unsigned long long *keys = (unsigned long long *)(ws + L.C);
        CTP_CUDA(cudaMemsetAsync(keys, 0, sizeof(double) * (size_t)p, st));
        CTP_CUDA(timed(ctx, K_COMPRESS_STRICT, st, [&] {
            return launch_compress_single_row(A + p, m, p, lda, keys, info, ctx->num_sms, st);
        }));
        fa.R = 1;
        fa.abs_update = 1;
        fa.C = (const double *)keys;
    } else {  // restricted: the tests look at A11 only
        fa.R = 0;
        fa.abs_update = 0;
        fa.C = nullptr;
    }
    CTP_CUDA(timed(ctx, K_FACTOR, st, [&] { return launch_factor_cluster(fa, ctx->factor_g, st); }));
    if (m > 0 && solve_on_tc(opt))
        CTP_CUDA(timed(ctx, K_SOLVE_TC, st, [&] {
            return launch_solve_tc(A, n, p, lda, perm, piv, Dinv, nelim, ws + L.Xs, solve_tc_pieces(opt->prec), Wb,
                                   Lbf, lo_off, pieces, info, ctx->num_sms, st);
        }));
    else if (m > 0)
        CTP_CUDA(timed(ctx, K_SOLVE, st, [&] {
            return launch_solve_fp64(A, n, p, lda, perm, piv, Dinv, nelim, W21, m, Wb, Lbf, Kp, lo_off, pieces,
                                     st);
        }));
    if (opt->smode != CTP_S_NONE && m > 0) {
        if (tc)
            CTP_CUDA(timed(ctx, pieces == 3 ? K_FORM_TC6 : (pieces == 2 ? K_FORM_TC3 : K_FORM_TC), st, [&] {
                return launch_form_tc(Wb, Lbf, lo_off, pieces, m, Kp, nelim, (float *)S, lds,
                                      opt->smode == CTP_S_FP64_SUB ? 3
                                      : opt->smode == CTP_S_FP32_TILED ? 2 : (packed ? 1 : 0), info,
                                      ctx->num_sms, ctx->form_walk, st);
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

// The context's side streams, made on first use outside a stream capture
// (false: run on st alone).  They belong to the context's device: when another
// device is current the batch does not fork (the caller's stream is on the
// current device, and events cannot join streams across devices).  A partial
// failure releases what it made, so a later call may try again.
static bool side_streams(ctp_ctx *ctx, cudaStream_t st) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device) return false;
    if (ctx->side_made) return true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    int ns = 0, ne = 0;
    bool fork = false, ok = true;
    for (; ok && ns < kSideStreams; ns++)
        ok = cudaStreamCreateWithFlags(&ctx->side[ns], cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) ns--;
    for (; ok && ne < kSideStreams; ne++)
        ok = cudaEventCreateWithFlags(&ctx->join_ev[ne], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) ne--;
    if (ok) ok = fork = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        for (int i = 0; i < ns; i++) cudaStreamDestroy(ctx->side[i]);
        for (int i = 0; i < ne; i++) cudaEventDestroy(ctx->join_ev[i]);
        if (fork) cudaEventDestroy(ctx->fork_ev);
        (void)cudaGetLastError();
        return false;
    }
    ctx->side_made = true;
    return true;
}

ctp_status ctp_factor_batch(ctp_ctx *ctx, const ctp_plan *plan, const ctp_front *fronts,
                            void *workspace, size_t ws_bytes, void *stream) {
    if (ctx == nullptr || plan == nullptr || fronts == nullptr || workspace == nullptr) return CTP_EINVAL;
    if (ws_bytes < batch_total(plan)) return CTP_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)workspace;
    CTP_CUDA(timed(ctx, K_B_PREPARE, st, [&] { return batch_prepare(plan, w, st); }));
    CTP_CUDA(timed(ctx, K_B_COMPRESS, st, [&] { return batch_compress(plan, fronts, w, ctx->num_sms, st); }));
    const int ncls = batch_num_classes(plan);
    if (!ctx->profiling && ncls > 1 && side_streams(ctx, st)) {
        // the classes touch disjoint fronts: run them side by side (the plan
        // lists the widest last: launched first, its clusters take SMs before
        // the narrow CTAs fill the rest), each followed on its stream by the
        // FP64 Solve and the Form of its own fronts (which then overlap the
        // classes still searching), joined back into st; capturable as a
        // fork/join
        const bool per_class = batch_solve_per_class(plan);
        CTP_CUDA(cudaEventRecord(ctx->fork_ev, st));
        for (int i = 0; i < ncls; i++) {
            const int c = ncls - 1 - i;
            cudaStream_t s = ctx->side[i % kSideStreams];
            CTP_CUDA(cudaStreamWaitEvent(s, ctx->fork_ev, 0));
            CTP_CUDA(batch_factor_class(plan, c, fronts, w, s));
            if (per_class) {
                CTP_CUDA(batch_solve_class(plan, c, fronts, w, s));
                CTP_CUDA(batch_form_class(plan, c, fronts, w, ctx->num_sms, s));
            }
            CTP_CUDA(cudaEventRecord(ctx->join_ev[i % kSideStreams], s));
        }
        for (int i = 0; i < ncls && i < kSideStreams; i++) CTP_CUDA(cudaStreamWaitEvent(st, ctx->join_ev[i], 0));
        if (!per_class) {
            CTP_CUDA(timed(ctx, K_B_SOLVE, st, [&] { return batch_solve(plan, fronts, w, ctx->num_sms, st); }));
            CTP_CUDA(timed(ctx, K_B_FORM, st, [&] { return batch_form(plan, fronts, w, ctx->num_sms, st); }));
        }
        return CTP_OK;
    } else {
        for (int c = 0; c < ncls; c++) {
            const int G = batch_class_G(plan, c), kind = batch_class_kind(plan, c);
            const int id = kind == kFactorWarp ? K_B_FACTOR_WARP
                         : K_B_FACTOR_G1 + (G == 1 ? 0 : G == 2 ? 1 : G == 4 ? 2 : G == 8 ? 3 : 4);
            CTP_CUDA(timed(ctx, id, st, [&] { return batch_factor_class(plan, c, fronts, w, st); }));
        }
        CTP_CUDA(timed(ctx, K_B_SOLVE, st, [&] { return batch_solve(plan, fronts, w, ctx->num_sms, st); }));
    }
    CTP_CUDA(timed(ctx, K_B_FORM, st, [&] { return batch_form(plan, fronts, w, ctx->num_sms, st); }));
    return CTP_OK;
}

/* ---------------------------------------------------------------------- */
/* Complete systems                                                         */

ctp_status ctp_solve_workspace_size(int64_t nmax, int32_t nrhs, size_t *bytes) {
    if (bytes == nullptr || nmax < 0 || nrhs < 1) return CTP_EINVAL;
    *bytes = sys_solve_ws_bytes(nmax, nrhs);
    return CTP_OK;
}

static ctp_status check_fronts(int32_t nf, const ctp_sfront *fronts, int64_t N, int64_t ws_nmax_cap) {
    if (nf < 0 || (nf > 0 && fronts == nullptr)) return CTP_EINVAL;
    for (int32_t k = 0; k < nf; k++) {
        const ctp_sfront &f = fronts[k];
        if (f.p < 1 || f.p > kMaxP || f.n < f.p || f.n > N || f.n > ws_nmax_cap || f.ldl < f.n ||
            f.L == nullptr || f.perm == nullptr || f.piv == nullptr || f.D == nullptr ||
            f.nelim == nullptr || f.rows == nullptr)
            return CTP_EINVAL;
    }
    return CTP_OK;
}

static cudaError_t solve_fronts(ctp_ctx *ctx, int32_t nf, const ctp_sfront *fronts, int32_t nrhs,
                                double *X, int64_t ldx, void *ws, cudaStream_t st) {
    for (int32_t k = 0; k < nf; k++) {
        cudaError_t e = timed(ctx, K_SYS_FWD, st, [&] {
            return launch_sys_forward(fronts[k], X, ldx, nrhs, ws, st);
        });
        if (e != cudaSuccess) return e;
    }
    for (int32_t k = nf - 1; k >= 0; k--) {
        cudaError_t e = timed(ctx, K_SYS_BWD, st, [&] {
            return launch_sys_backward(fronts[k], X, ldx, nrhs, ws, st);
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

ctp_status ctp_solve(ctp_ctx *ctx, int32_t nf, const ctp_sfront *fronts, int64_t N, int32_t nrhs,
                     double *X, int64_t ldx, void *workspace, size_t ws_bytes, void *stream) {
    if (ctx == nullptr || X == nullptr || workspace == nullptr || N < 1 || nrhs < 1 || ldx < N)
        return CTP_EINVAL;
    int64_t nmax = 0;
    for (int32_t k = 0; k < nf && fronts != nullptr; k++) nmax = fronts[k].n > nmax ? fronts[k].n : nmax;
    ctp_status s = check_fronts(nf, fronts, N, nmax);
    if (s != CTP_OK) return s;
    if (ws_bytes < sys_solve_ws_bytes(nmax, nrhs)) return CTP_ENOMEM;
    CTP_CUDA(solve_fronts(ctx, nf, fronts, nrhs, X, ldx, workspace, (cudaStream_t)stream));
    return CTP_OK;
}

ctp_status ctp_adjoint_solve(ctp_ctx *ctx, int32_t nf, const ctp_sfront *fronts, int64_t N,
                             int32_t nrhs, double *G, int64_t ldg, void *workspace, size_t ws_bytes,
                             void *stream) {
    // M is symmetric and so is its factored form: the adjoint is the same solve
    return ctp_solve(ctx, nf, fronts, N, nrhs, G, ldg, workspace, ws_bytes, stream);
}

ctp_status ctp_sym_grad_dense(ctp_ctx *ctx, int64_t N, int32_t nrhs, const double *Gb, int64_t ldg,
                              const double *X, int64_t ldx, double *out, int64_t ldo, void *stream) {
    if (ctx == nullptr || Gb == nullptr || X == nullptr || out == nullptr || N < 1 || nrhs < 1 ||
        ldg < N || ldx < N || ldo < N)
        return CTP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    CTP_CUDA(timed(ctx, K_GRAD, st, [&] {
        return launch_sym_grad_dense(N, nrhs, Gb, ldg, X, ldx, out, ldo, st);
    }));
    return CTP_OK;
}

ctp_status ctp_sym_grad_pattern(ctp_ctx *ctx, int64_t nnz, const int32_t *row, const int32_t *col,
                                int64_t N, int32_t nrhs, const double *Gb, int64_t ldg,
                                const double *X, int64_t ldx, double *out, void *stream) {
    if (ctx == nullptr || nnz < 0 || (nnz > 0 && (row == nullptr || col == nullptr || out == nullptr)) ||
        Gb == nullptr || X == nullptr || N < 1 || nrhs < 1 || ldg < N || ldx < N)
        return CTP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    CTP_CUDA(timed(ctx, K_GRAD, st, [&] {
        return launch_sym_grad_pattern(nnz, row, col, nrhs, Gb, ldg, X, ldx, out, st);
    }));
    return CTP_OK;
}

ctp_status ctp_refine_workspace_size(int64_t N, int64_t nmax, int32_t nrhs, size_t *bytes) {
    if (bytes == nullptr || N < 1 || nmax < 0 || nrhs < 1) return CTP_EINVAL;
    *bytes = refine_layout(N, sys_solve_ws_bytes(nmax, nrhs), nrhs).total;
    return CTP_OK;
}

static ctp_status backward_error_impl(ctp_ctx *ctx, const MatOp &A, int64_t N, int32_t nrhs,
                                      const double *B, int64_t ldb, const double *X, int64_t ldx,
                                      double *berr, void *workspace, size_t ws_bytes, void *stream) {
    RefineLayout L = refine_layout(N, 0, nrhs);
    if (ws_bytes < L.total) return CTP_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)workspace;
    double *rowsum = (double *)(w + L.rowsum);
    CTP_CUDA(mat_abs_rowsum(ctx, A, N, rowsum, st));
    CTP_CUDA(residual_berr(ctx, A, N, nrhs, B, ldb, X, ldx, (double *)(w + L.R), rowsum,
                           (double *)(w + L.mx), berr, st));
    return CTP_OK;
}

static ctp_status refine_impl(ctp_ctx *ctx, int32_t nf, const ctp_sfront *fronts, int64_t N, const MatOp &A,
                              int32_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx,
                              int32_t max_steps, double tol, double *berr_host, int32_t *steps_host,
                              void *workspace, size_t ws_bytes, void *stream) {
    int64_t nmax = 0;
    for (int32_t k = 0; k < nf && fronts != nullptr; k++) nmax = fronts[k].n > nmax ? fronts[k].n : nmax;
    ctp_status s = check_fronts(nf, fronts, N, nmax);
    if (s != CTP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    auto solve = [&](double *Y, int64_t ldy, void *sws) {
        return solve_fronts(ctx, nf, fronts, nrhs, Y, ldy, sws, st);
    };
    return refine_core(ctx, solve, sys_solve_ws_bytes(nmax, nrhs), N, A, nrhs, B, ldb, X, ldx, max_steps, tol,
                       berr_host, steps_host, workspace, ws_bytes, st);
}

ctp_status ctp_backward_error(ctp_ctx *ctx, int64_t N, const double *M, int64_t ldm, int32_t nrhs,
                              const double *B, int64_t ldb, const double *X, int64_t ldx,
                              double *berr, void *workspace, size_t ws_bytes, void *stream) {
    if (ctx == nullptr || M == nullptr || B == nullptr || X == nullptr || berr == nullptr ||
        workspace == nullptr || N < 1 || nrhs < 1 || ldm < N || ldb < N || ldx < N)
        return CTP_EINVAL;
    MatOp A;
    A.M = M;
    A.ldm = ldm;
    return backward_error_impl(ctx, A, N, nrhs, B, ldb, X, ldx, berr, workspace, ws_bytes, stream);
}

ctp_status ctp_backward_error_csc(ctp_ctx *ctx, int64_t N, const int64_t *colptr, const int32_t *rowind,
                                  const double *val, int32_t nrhs, const double *B, int64_t ldb,
                                  const double *X, int64_t ldx, double *berr, void *workspace,
                                  size_t ws_bytes, void *stream) {
    if (ctx == nullptr || colptr == nullptr || rowind == nullptr || val == nullptr || B == nullptr ||
        X == nullptr || berr == nullptr || workspace == nullptr || N < 1 || nrhs < 1 || ldb < N || ldx < N)
        return CTP_EINVAL;
    MatOp A;
    A.colptr = colptr;
    A.rowind = rowind;
    A.val = val;
    return backward_error_impl(ctx, A, N, nrhs, B, ldb, X, ldx, berr, workspace, ws_bytes, stream);
}

ctp_status ctp_refine(ctp_ctx *ctx, int32_t nf, const ctp_sfront *fronts, int64_t N,
                      const double *M, int64_t ldm, int32_t nrhs, const double *B, int64_t ldb,
                      double *X, int64_t ldx, int32_t max_steps, double tol, double *berr_host,
                      int32_t *steps_host, void *workspace, size_t ws_bytes, void *stream) {
    if (ctx == nullptr || M == nullptr || B == nullptr || X == nullptr || berr_host == nullptr ||
        steps_host == nullptr || workspace == nullptr || N < 1 || nrhs < 1 || ldm < N ||
        ldb < N || ldx < N || max_steps < 0 || max_steps > 100 || !(tol >= 0.0))
        return CTP_EINVAL;
    MatOp A;
    A.M = M;
    A.ldm = ldm;
    return refine_impl(ctx, nf, fronts, N, A, nrhs, B, ldb, X, ldx, max_steps, tol, berr_host, steps_host,
                       workspace, ws_bytes, stream);
}

ctp_status ctp_refine_csc(ctp_ctx *ctx, int32_t nf, const ctp_sfront *fronts, int64_t N,
                          const int64_t *colptr, const int32_t *rowind, const double *val, int32_t nrhs,
                          const double *B, int64_t ldb, double *X, int64_t ldx, int32_t max_steps,
                          double tol, double *berr_host, int32_t *steps_host, void *workspace,
                          size_t ws_bytes, void *stream) {
    if (ctx == nullptr || colptr == nullptr || rowind == nullptr || val == nullptr || B == nullptr ||
        X == nullptr || berr_host == nullptr || steps_host == nullptr || workspace == nullptr || N < 1 ||
        nrhs < 1 || ldb < N || ldx < N || max_steps < 0 || max_steps > 100 || !(tol >= 0.0))
        return CTP_EINVAL;
    MatOp A;
    A.colptr = colptr;
    A.rowind = rowind;
    A.val = val;
    return refine_impl(ctx, nf, fronts, N, A, nrhs, B, ldb, X, ldx, max_steps, tol, berr_host, steps_host,
                       workspace, ws_bytes, stream);
}

}  // extern "C"

struct ctp_chain {
    std::vector<ctp_sfront> fronts;
    std::vector<int32_t> nelim, p, pivot;
    Arena arena;
};

namespace {
void chain_free(ctp_chain *c) {
    if (c == nullptr) return;
    c->arena.release();
    delete c;
}
}  // namespace

namespace ctp {
int ctx_num_sms(const ctp_ctx *ctx) { return ctx->num_sms; }
}  // namespace ctp

extern "C" {

ctp_status ctp_factor_dense(ctp_ctx *ctx, int64_t N, double *M, int64_t ldm, int32_t p_first,
                            const ctp_options *opt_first, int32_t w_rest,
                            const ctp_options *opt_rest, ctp_chain **chain, void *stream) {
    if (ctx == nullptr || M == nullptr || chain == nullptr || N < 1 || ldm < N) return CTP_EINVAL;
    *chain = nullptr;
    if (p_first < 1 || p_first > kMaxP || w_rest < 1 || w_rest > kMaxP) return CTP_EINVAL;
    ctp_status s = check_opts(opt_first);
    if (s == CTP_OK) s = check_opts(opt_rest);
    if (s != CTP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    ChainCfg cfg;
    cfg.w_first = p_first;
    cfg.w_rest = w_rest;
    cfg.o_first = *opt_first;
    cfg.o_rest = *opt_rest;
    cfg.retry_tpp = true;
    cfg.must_finish = true;
    cfg.one_pass = false;
    ctp_chain *c = new ctp_chain();
    c->arena.chunk_bytes = (size_t)64 << 20;
    std::vector<int32_t> ord(N);
    for (int64_t i = 0; i < N; i++) ord[i] = (int32_t)i;
    std::vector<PanelRec> panels;
    int64_t elim = 0;
    ChainWork wk;
    s = chain_factor(ctx, M, N, ldm, N, cfg, ord.data(), c->arena, wk, panels, &elim, st);
    cudaStreamSynchronize(st);
    if (s != CTP_OK) {
        chain_free(c);
        return s;
    }
    for (const PanelRec &r : panels) {
        c->fronts.push_back(r.f);
        c->nelim.push_back(r.e);
        c->p.push_back(r.w);
        c->pivot.push_back(r.pivot);
    }
    *chain = c;
    return CTP_OK;
}

ctp_status ctp_chain_fronts(const ctp_chain *chain, int32_t *nf, const ctp_sfront **fronts) {
    if (chain == nullptr || nf == nullptr || fronts == nullptr) return CTP_EINVAL;
    *nf = (int32_t)chain->fronts.size();
    *fronts = chain->fronts.data();
    return CTP_OK;
}

ctp_status ctp_chain_info(const ctp_chain *chain, int32_t cap, int32_t *nelim, int32_t *p,
                          int32_t *pivot) {
    if (chain == nullptr || cap < 0) return CTP_EINVAL;
    const int32_t n = (int32_t)chain->fronts.size();
    for (int32_t k = 0; k < n && k < cap; k++) {
        if (nelim) nelim[k] = chain->nelim[k];
        if (p) p[k] = chain->p[k];
        if (pivot) pivot[k] = chain->pivot[k];
    }
    return CTP_OK;
}

ctp_status ctp_chain_destroy(ctp_chain *chain) {
    chain_free(chain);
    return CTP_OK;
}

}  // extern "C"
