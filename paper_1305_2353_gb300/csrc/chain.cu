// chain.cu -- elimination of the leading columns of a dense symmetric matrix in
// panels of at most 256 columns (a chain of supernodes), each panel factored by
// ctp_factor_supernode with its Form subtracting into the trailing matrix.
// The columns a panel delays lead the next panel (Section 1: delayed columns
// are passed on).  Used for complete dense systems (ctp_factor_dense) and for
// the fronts of the multifrontal factorization.
#include <string.h>

#include "chain.cuh"

namespace ctp {

void *Arena::alloc(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (chunks.empty() || used + bytes > cap) {
        const size_t sz = bytes > chunk_bytes ? bytes : chunk_bytes;
        void *p = nullptr;
        if (cudaMalloc(&p, sz) != cudaSuccess) return nullptr;
        chunks.push_back(p);
        cap = sz;
        used = 0;
    }
    void *p = (char *)chunks.back() + used;
    used += bytes;
    return p;
}

void Arena::release() {
    for (void *p : chunks) cudaFree(p);
    chunks.clear();
    cap = used = 0;
}

ChainWork::~ChainWork() {
    if (ws) cudaFree(ws);
    if (snap) cudaFree(snap);
    if (hbuf) cudaFreeHost(hbuf);
}

bool ChainWork::reserve(ctp_ctx *ctx, int64_t n, int w, const ctp_options *opts, int nopt) {
    // any panel width up to w can occur (first panel, last panel, and a
    // narrower panel has more rows below it for the same K padding)
    size_t need = 0;
    const int wm = w < n ? w : (int)n;
    for (int k = 0; k < nopt; k++)
        for (int wi = 1; wi <= wm; wi++) {
            const size_t b = ws_layout(n, wi, &opts[k], ctx_num_sms(ctx)).total;
            need = b > need ? b : need;
        }
    if (need > ws_bytes) {
        if (ws) cudaFree(ws);
        ws = nullptr;
        ws_bytes = 0;
        if (cudaMalloc(&ws, need) != cudaSuccess) return false;
        ws_bytes = need;
    }
    const size_t sb = sizeof(double) * (size_t)n * (w < n ? w : n);
    if (sb > snap_bytes) {
        if (snap) cudaFree(snap);
        snap = nullptr;
        snap_bytes = 0;
        if (cudaMalloc(&snap, sb) != cudaSuccess) return false;
        snap_bytes = sb;
    }
    if (hbuf == nullptr && cudaMallocHost((void **)&hbuf, sizeof(int32_t) * (kMaxP + 2)) != cudaSuccess)
        return false;
    return true;
}

ctp_status chain_factor(ctp_ctx *ctx, double *F, int64_t n, int64_t ld, int64_t p_fs, const ChainCfg &cfg,
                        int32_t *ord, Arena &arena, ChainWork &wk, std::vector<PanelRec> &out,
                        int64_t *elim, cudaStream_t st) {
    *elim = 0;
    ctp_options otpp = cfg.o_rest;
    otpp.pivot = CTP_PIV_TPP;
    otpp.prec = CTP_FP64;
    // workspace for the panels as they run: Form subtracting into the trailing matrix
    ctp_options cand[3] = {cfg.o_first, cfg.o_rest, otpp};
    for (ctp_options &c : cand) {
        c.smode = CTP_S_FP64_SUB;
        if (c.pivot == CTP_PIV_TPP) c.prec = CTP_FP64;
    }
    const int wmax = cfg.w_first > cfg.w_rest ? cfg.w_first : cfg.w_rest;
    if (!wk.reserve(ctx, n, wmax, cand, 3)) return CTP_ENOMEM;
    int64_t col = 0, untried = p_fs;  // untried: fully-summed columns not yet in a panel
    bool first = true;
    std::vector<int32_t> tmp(kMaxP);
    while (col < p_fs) {
        const int64_t nk = n - col, p_left = p_fs - col;
        ctp_options ok = first ? cfg.o_first : cfg.o_rest;
        const int64_t wreq = first ? cfg.w_first : cfg.w_rest;
        const int w = (int)(wreq < p_left ? wreq : p_left);
        const int64_t carried = p_left - untried;
        untried -= w > carried ? w - carried : 0;
        first = false;
        ok.smode = nk > w ? CTP_S_FP64_SUB : CTP_S_NONE;
        if (ok.pivot == CTP_PIV_TPP) ok.prec = CTP_FP64;
        // one device block per panel: rows | perm | piv | nelim | D
        const size_t ints = (size_t)nk + 2 * (size_t)w + 2;
        const size_t bytes = align256(sizeof(int32_t) * ints) + sizeof(double) * 2 * (size_t)w;
        char *blk = (char *)arena.alloc(bytes);
        if (blk == nullptr) return CTP_ENOMEM;
        int32_t *rows = (int32_t *)blk, *perm = rows + nk, *piv = perm + w, *nel = piv + w;
        double *D = (double *)(blk + align256(sizeof(int32_t) * ints));
        if (cudaMemcpyAsync(rows, ord + col, sizeof(int32_t) * nk, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return CTP_ECUDA;
        double *A = F + col * ld + col;
        double *S = nk > w ? A + (int64_t)w * ld + w : nullptr;
        const bool may_retry = cfg.retry_tpp || cfg.must_finish;
        if (may_retry && ok.pivot != CTP_PIV_TPP &&
            cudaMemcpy2DAsync(wk.snap, sizeof(double) * nk, A, sizeof(double) * ld, sizeof(double) * nk, w,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return CTP_ECUDA;
        int32_t info = CTP_OK, e = 0;
        for (int attempt = 0; attempt < 2; attempt++) {
            ctp_status rc = ctp_factor_supernode(ctx, nk, w, A, ld, &ok, perm, piv, D, nel, S, ld, wk.ws,
                                                 wk.ws_bytes, st);
            if (rc != CTP_OK) return rc;
            if (cudaMemcpyAsync(wk.hbuf, nel, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(wk.hbuf + 1, perm, sizeof(int32_t) * w, cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaMemcpyAsync(&info, wk.ws, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return CTP_ECUDA;
            if (info != CTP_OK) return (ctp_status)info;
            e = wk.hbuf[0];
            if (e > 0 || ok.pivot == CTP_PIV_TPP || !may_retry) break;
            // nothing eliminated: put the panel back and use full-column pivoting
            if (cudaMemcpy2DAsync(A, sizeof(double) * ld, wk.snap, sizeof(double) * nk, sizeof(double) * nk, w,
                                  cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return CTP_ECUDA;
            const int sm = ok.smode;
            ok = otpp;
            ok.smode = sm;
        }
        if (e == 0) {
            if (cfg.must_finish || cfg.retry_tpp) return CTP_ECAPACITY;
            break;  // a front: the remaining fully-summed columns go to the parent
        }
        if (nk == w && e < w && (cfg.must_finish || cfg.retry_tpp)) return CTP_ECAPACITY;
        for (int q = 0; q < w; q++) tmp[q] = ord[col + wk.hbuf[1 + q]];
        for (int q = 0; q < w; q++) ord[col + q] = tmp[q];
        PanelRec r;
        r.f.n = nk;
        r.f.p = w;
        r.f.reserved = 0;
        r.f.L = A;
        r.f.ldl = ld;
        r.f.perm = perm;
        r.f.piv = piv;
        r.f.D = D;
        r.f.nelim = nel;
        r.f.rows = rows;
        r.e = e;
        r.w = w;
        r.pivot = ok.pivot;
        out.push_back(r);
        col += e;
        if (cfg.one_pass && !cfg.must_finish && untried == 0) break;
    }
    if (cfg.must_finish && col < p_fs) return CTP_ECAPACITY;
    *elim = col;
    return CTP_OK;
}

}  // namespace ctp
