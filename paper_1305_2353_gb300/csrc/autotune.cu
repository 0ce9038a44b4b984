// autotune.cu -- the library's own autotuner: it picks the launch choices of
// the GB300 kernels (the tuning knobs of a context) for a given workload by
// timing the real calls on the device.  Launch choices never change results,
// so the tuner may run the caller's own inputs: it backs them up once, and
// restores them before every trial and at the end.
#include <string.h>

#include <vector>

#include "ctp_internal.cuh"

using namespace ctp;

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    bool ok = false;
    Timer() { ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess; }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// One n x p column-major block (leading dimension ld) and its backup.
struct Saved {
    double *A;
    int64_t n, ld;
    int p;
    size_t off;
};

// Backup of the caller's inputs; restore() copies them back.
struct Backup {
    std::vector<Saved> blocks;
    double *buf = nullptr;
    cudaStream_t st;
    ~Backup() {
        if (buf) cudaFree(buf);
    }
    ctp_status make(cudaStream_t s) {
        st = s;
        size_t total = 0;
        for (Saved &b : blocks) {
            b.off = total;
            total += (size_t)b.n * b.p;
        }
        if (cudaMalloc(&buf, sizeof(double) * (total > 0 ? total : 1)) != cudaSuccess) return CTP_ENOMEM;
        for (const Saved &b : blocks)
            if (cudaMemcpy2DAsync(buf + b.off, sizeof(double) * b.n, b.A, sizeof(double) * b.ld,
                                  sizeof(double) * b.n, b.p, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return CTP_ECUDA;
        return CTP_OK;
    }
    bool restore() const {
        for (const Saved &b : blocks)
            if (cudaMemcpy2DAsync(b.A, sizeof(double) * b.ld, buf + b.off, sizeof(double) * b.n,
                                  sizeof(double) * b.n, b.p, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return false;
        return true;
    }
};

// The common loop: for each candidate set the knobs, run `trial` twice (warm-up
// and timed) on restored inputs, keep the fastest.  `prepare(c)` runs after the
// knobs are set and before the trials (a plan, say); `finish()` after them.
template <typename Prep, typename Trial, typename Fin>
ctp_status tune_loop(ctp_ctx *ctx, const Backup &bk, cudaStream_t st, int32_t nk, const int32_t *keys,
                     int32_t ncand, const int32_t *values, double *ms_out, int32_t *best, Prep prepare,
                     Trial trial, Fin finish) {
    std::vector<int32_t> old(nk);
    for (int k = 0; k < nk; k++)
        if (ctp_tune_get(ctx, keys[k], &old[k]) != CTP_OK) return CTP_EINVAL;
    Timer tm;
    if (!tm.ok) return CTP_ECUDA;
    ctp_status rc = CTP_OK;
    int bestc = -1;
    double bestms = 1e300;
    for (int c = 0; c < ncand && rc == CTP_OK; c++) {
        for (int k = 0; k < nk && rc == CTP_OK; k++) rc = ctp_tune_set(ctx, keys[k], values[c * nk + k]);
        if (rc != CTP_OK) break;
        rc = prepare(c);
        double ms = 0.0;
        for (int rep = 0; rep < 2 && rc == CTP_OK; rep++) {
            if (!bk.restore()) {
                rc = CTP_ECUDA;
                break;
            }
            cudaEventRecord(tm.a, st);
            rc = trial();
            cudaEventRecord(tm.b, st);
            if (rc == CTP_OK && cudaEventSynchronize(tm.b) == cudaSuccess) {
                float f = 0.f;
                cudaEventElapsedTime(&f, tm.a, tm.b);
                ms = f;
            } else if (rc == CTP_OK) {
                rc = CTP_ECUDA;
            }
        }
        finish();
        if (rc != CTP_OK) break;
        if (ms_out) ms_out[c] = ms;
        if (ms < bestms) {
            bestms = ms;
            bestc = c;
        }
    }
    // put the inputs back whatever happened in the trials
    if (!bk.restore() && rc == CTP_OK) rc = CTP_ECUDA;
    cudaStreamSynchronize(st);
    if (rc == CTP_OK && bestc >= 0) {
        for (int k = 0; k < nk; k++) ctp_tune_set(ctx, keys[k], values[bestc * nk + k]);
        if (best) *best = bestc;
    } else {
        for (int k = 0; k < nk; k++) ctp_tune_set(ctx, keys[k], old[k]);
    }
    return rc;
}

}  // namespace

extern "C" {

ctp_status ctp_autotune_batch(ctp_ctx *ctx, int32_t nb, const int64_t *n_host, const int32_t *p_host,
                              const ctp_options *opt, const ctp_front *fronts_host,
                              const ctp_front *fronts_dev, int32_t nk, const int32_t *keys,
                              int32_t ncand, const int32_t *values, double *ms_out, int32_t *best,
                              void *stream) {
    if (ctx == nullptr || n_host == nullptr || p_host == nullptr || opt == nullptr ||
        fronts_host == nullptr || fronts_dev == nullptr || nb < 1 || nk < 1 || keys == nullptr ||
        ncand < 1 || values == nullptr)
        return CTP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Backup bk;
    for (int f = 0; f < nb; f++) {
        const ctp_front &fr = fronts_host[f];
        if (fr.A == nullptr || fr.n != n_host[f] || fr.p != p_host[f] || fr.lda < fr.n) return CTP_EINVAL;
        bk.blocks.push_back({fr.A, fr.n, fr.lda, fr.p, 0});
    }
    ctp_status rc = bk.make(st);
    if (rc != CTP_OK) return rc;
    ctp_plan *plan = nullptr;
    void *ws = nullptr;
    size_t ws_cap = 0;
    auto prepare = [&](int) -> ctp_status {
        size_t need = 0;
        ctp_status r = ctp_batch_plan_create(ctx, nb, n_host, p_host, opt, &plan, &need);
        if (r != CTP_OK) return r;
        if (need > ws_cap) {
            if (ws) cudaFree(ws);
            ws = nullptr;
            ws_cap = 0;
            if (cudaMalloc(&ws, need) != cudaSuccess) return CTP_ENOMEM;
            ws_cap = need;
        }
        return ctp_batch_upload(ctx, plan, ws, ws_cap, stream);
    };
    auto trial = [&]() { return ctp_factor_batch(ctx, plan, fronts_dev, ws, ws_cap, stream); };
    auto finish = [&]() {
        if (plan) ctp_batch_plan_destroy(plan);
        plan = nullptr;
    };
    rc = tune_loop(ctx, bk, st, nk, keys, ncand, values, ms_out, best, prepare, trial, finish);
    if (ws) cudaFree(ws);
    return rc;
}

ctp_status ctp_autotune_supernode(ctp_ctx *ctx, int64_t n, int32_t p, double *A, int64_t lda,
                                  const ctp_options *opt, int32_t *perm, int32_t *piv, double *D,
                                  int32_t *nelim, void *S, int64_t lds, void *workspace,
                                  size_t ws_bytes, int32_t nk, const int32_t *keys, int32_t ncand,
                                  const int32_t *values, double *ms_out, int32_t *best, void *stream) {
    if (ctx == nullptr || A == nullptr || p < 1 || n < p || lda < n || nk < 1 || keys == nullptr ||
        ncand < 1 || values == nullptr)
        return CTP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Backup bk;
    bk.blocks.push_back({A, n, lda, p, 0});
    ctp_status rc = bk.make(st);
    if (rc != CTP_OK) return rc;
    auto prepare = [&](int) { return CTP_OK; };
    auto trial = [&]() {
        return ctp_factor_supernode(ctx, n, p, A, lda, opt, perm, piv, D, nelim, S, lds, workspace,
                                    ws_bytes, stream);
    };
    auto finish = [&]() {};
    return tune_loop(ctx, bk, st, nk, keys, ncand, values, ms_out, best, prepare, trial, finish);
}

}  // extern "C"
