// multifrontal.cu -- the multifrontal factorization of a sparse symmetric
// indefinite matrix around the per-supernode kernels (Section 1: the Factor,
// Solve, Form and Scatter tasks over an assembly tree, delayed columns passed
// to the parent front).
//
// Analysis (host): the caller gives the lower triangle's pattern, an
// elimination order and its supernodes -- consecutive blocks of that order
// (the separators and leaf boxes of nested dissection).  Front s holds its
// block's variables and struct(s), the later variables joined to the block in
// the filled graph: the block's own later neighbours and the later rows of its
// children's fronts.  Its parent is the block of the first variable of
// struct(s).  The original entries each front assembles (those whose earlier
// variable is in its block) are listed once, by local position, and uploaded.
//
// Factorization (device, fronts children first): the frontal matrix (dense,
// lower triangle) receives its original entries and the children's
// contribution blocks (extend-add); its fully-summed columns -- the block's
// variables, then the columns the children delayed -- are eliminated by the
// panel-chain driver, whose Forms subtract into the front's trailing block, so
// that block becomes the front's contribution block in place.  A panel that
// eliminates nothing ends the front: its remaining fully-summed columns lead
// the contribution block and are delayed to the parent.  A root must finish.
#include <string.h>

#include <algorithm>
#include <vector>

#include "chain.cuh"
#include "ctx.cuh"

using namespace ctp;

struct ctp_mf {
    int64_t N = 0, nnz = 0;
    std::vector<int32_t> perm, inv;  // new -> original, original -> new
    struct Blk {
        int64_t lo = 0, hi = 0;
        std::vector<int32_t> st;  // struct (new numbering, ascending)
        int parent = -1;
        std::vector<int> children;
        int64_t e0 = 0, ne = 0;  // this block's entries in the uploaded lists
        // numeric results
        double *F = nullptr;
        int64_t n = 0, p = 0, elim = 0;
        std::vector<int32_t> cb;  // contribution-block variables (new numbering); delayed first
        int64_t ndel = 0;
    };
    std::vector<Blk> blk;
    // assembly lists: local codes (own variables 0..p_own-1, struct rows p_own + t)
    // and value indices, all blocks concatenated, on the device
    int32_t *d_ci = nullptr, *d_cj = nullptr;
    int64_t *d_q = nullptr;
    Arena arena;  // frontal matrices and panel blocks
    std::vector<ctp_sfront> fronts;
    std::vector<PanelRec> panels;
    bool factored = false;
    ~ctp_mf() {
        if (d_ci) cudaFree(d_ci);
        if (d_cj) cudaFree(d_cj);
        if (d_q) cudaFree(d_q);
        arena.release();
    }
};

namespace {

constexpr int kTh = 256;

// Original entries of a front: F(local(ci), local(cj)) += val[q], with struct
// codes shifted by the number of delayed columns the front received.
__global__ void __launch_bounds__(kTh) k_mf_assemble(int64_t ne, const int32_t *__restrict__ ci,
                                                     const int32_t *__restrict__ cj,
                                                     const int64_t *__restrict__ q,
                                                     const double *__restrict__ val, int p_own,
                                                     int64_t d, double *F, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * kTh + threadIdx.x; k < ne; k += (int64_t)gridDim.x * kTh) {
        int64_t a = ci[k], b = cj[k];
        if (a >= p_own) a += d;
        if (b >= p_own) b += d;
        if (a < b) {
            const int64_t t = a;
            a = b;
            b = t;
        }
        F[b * n + a] += val[q[k]];
    }
}

// Extend-add of a child's contribution block C = Fc[e:, e:] (lower triangle,
// m x m, leading dimension ldc) into the parent: F(map[i], map[j]) += C(i, j).
__global__ void __launch_bounds__(kTh) k_mf_extend_add(const double *__restrict__ Fc, int64_t ldc, int64_t m,
                                                       const int32_t *__restrict__ map, double *F, int64_t n) {
    const int64_t j = blockIdx.y;
    for (int64_t jj = j; jj < m; jj += gridDim.y) {
        const int64_t bj = map[jj];
        const double *col = Fc + jj * ldc;
        for (int64_t i = jj + (int64_t)blockIdx.x * kTh + threadIdx.x; i < m; i += (int64_t)gridDim.x * kTh) {
            int64_t a = map[i], b = bj;
            if (a < b) {
                const int64_t t = a;
                a = b;
                b = t;
            }
            F[b * n + a] += col[i];
        }
    }
}

}  // namespace

extern "C" {

ctp_status ctp_mf_analyse(ctp_ctx *ctx, int64_t N, const int64_t *colptr, const int32_t *rowind,
                          const int32_t *perm, int32_t nblocks, const int64_t *blocks, ctp_mf **out) {
    if (ctx == nullptr || out == nullptr || colptr == nullptr || rowind == nullptr || perm == nullptr ||
        blocks == nullptr || N < 1 || nblocks < 1 || N > 0x7fffffffLL)
        return CTP_EINVAL;
    *out = nullptr;
    if (blocks[0] != 0 || blocks[nblocks] != N) return CTP_EINVAL;
    for (int s = 0; s < nblocks; s++)
        if (blocks[s + 1] <= blocks[s]) return CTP_EINVAL;
    ctp_mf *mf = new ctp_mf();
    mf->N = N;
    mf->nnz = colptr[N];
    mf->perm.assign(perm, perm + N);
    mf->inv.assign(N, -1);
    for (int64_t k = 0; k < N; k++) {
        if (perm[k] < 0 || perm[k] >= N || mf->inv[perm[k]] >= 0) {
            delete mf;
            return CTP_EINVAL;
        }
        mf->inv[perm[k]] = (int32_t)k;
    }
    const std::vector<int32_t> &inv = mf->inv;
    // adjacency (both triangles) in the new numbering, compressed
    std::vector<int64_t> deg(N + 1, 0);
    for (int64_t j = 0; j < N; j++)
        for (int64_t q = colptr[j]; q < colptr[j + 1]; q++) {
            const int64_t i = rowind[q];
            if (i < 0 || i >= N || i < j) {
                delete mf;
                return CTP_EINVAL;  // lower triangle expected
            }
            if (i != j) {
                deg[inv[i] + 1]++;
                deg[inv[j] + 1]++;
            }
        }
    for (int64_t v = 0; v < N; v++) deg[v + 1] += deg[v];
    std::vector<int32_t> adj(deg[N]);
    {
        std::vector<int64_t> fill(deg.begin(), deg.end() - 1);
        for (int64_t j = 0; j < N; j++)
            for (int64_t q = colptr[j]; q < colptr[j + 1]; q++) {
                const int64_t i = rowind[q];
                if (i != j) {
                    adj[fill[inv[i]]++] = inv[j];
                    adj[fill[inv[j]]++] = inv[i];
                }
            }
    }
    std::vector<int32_t> owner(N);
    mf->blk.resize(nblocks);
    for (int s = 0; s < nblocks; s++) {
        mf->blk[s].lo = blocks[s];
        mf->blk[s].hi = blocks[s + 1];
        for (int64_t v = blocks[s]; v < blocks[s + 1]; v++) owner[v] = s;
    }
    // struct of each block, children first
    std::vector<int64_t> mark(N, -1);
    for (int s = 0; s < nblocks; s++) {
        ctp_mf::Blk &b = mf->blk[s];
        std::vector<int32_t> rows;
        for (int64_t v = b.lo; v < b.hi; v++)
            for (int64_t q = deg[v]; q < deg[v + 1]; q++) {
                const int32_t w = adj[q];
                if (w >= b.hi && mark[w] != s) {
                    mark[w] = s;
                    rows.push_back(w);
                }
            }
        for (int c : b.children)
            for (int32_t w : mf->blk[c].st)
                if (w >= b.hi && mark[w] != s) {
                    mark[w] = s;
                    rows.push_back(w);
                }
        std::sort(rows.begin(), rows.end());
        b.st.swap(rows);
        if (!b.st.empty()) {
            b.parent = owner[b.st[0]];
            mf->blk[b.parent].children.push_back(s);
        }
    }
    // assembly lists: each original entry (i, j) belongs to the front of the
    // block holding the earlier of its two variables in the new order
    std::vector<int32_t> ci, cj;
    std::vector<int64_t> qv;
    std::vector<int32_t> code(N, -1);
    {
        std::vector<int64_t> cnt(nblocks + 1, 0);
        for (int64_t j = 0; j < N; j++)
            for (int64_t q = colptr[j]; q < colptr[j + 1]; q++) {
                const int64_t a = inv[rowind[q]], c = inv[j];
                cnt[owner[a < c ? a : c] + 1]++;
            }
        for (int s = 0; s < nblocks; s++) cnt[s + 1] += cnt[s];
        const int64_t nnz = cnt[nblocks];
        std::vector<int64_t> ent(nnz), ecol(nnz), fill(cnt.begin(), cnt.end() - 1);
        for (int64_t j = 0; j < N; j++)
            for (int64_t q = colptr[j]; q < colptr[j + 1]; q++) {
                const int64_t a = inv[rowind[q]], c = inv[j];
                const int64_t k = fill[owner[a < c ? a : c]]++;
                ent[k] = q;
                ecol[k] = j;
            }
        ci.resize(nnz);
        cj.resize(nnz);
        qv.resize(nnz);
        for (int s = 0; s < nblocks; s++) {
            ctp_mf::Blk &b = mf->blk[s];
            const int64_t pown = b.hi - b.lo;
            for (int64_t v = b.lo; v < b.hi; v++) code[v] = (int32_t)(v - b.lo);
            for (size_t t = 0; t < b.st.size(); t++) code[b.st[t]] = (int32_t)(pown + t);
            b.e0 = cnt[s];
            b.ne = cnt[s + 1] - cnt[s];
            for (int64_t k = cnt[s]; k < cnt[s + 1]; k++) {
                const int32_t a = code[inv[rowind[ent[k]]]], c = code[inv[ecol[k]]];
                if (a < 0 || c < 0) {  // an entry outside its front: inconsistent input
                    delete mf;
                    return CTP_EINVAL;
                }
                ci[k] = a;
                cj[k] = c;
                qv[k] = ent[k];
            }
            for (int64_t v = b.lo; v < b.hi; v++) code[v] = -1;
            for (int32_t w : b.st) code[w] = -1;
        }
    }
    const size_t ne = ci.size() > 0 ? ci.size() : 1;
    if (cudaMalloc(&mf->d_ci, sizeof(int32_t) * ne) != cudaSuccess ||
        cudaMalloc(&mf->d_cj, sizeof(int32_t) * ne) != cudaSuccess ||
        cudaMalloc(&mf->d_q, sizeof(int64_t) * ne) != cudaSuccess) {
        delete mf;
        return CTP_ENOMEM;
    }
    if (!ci.empty() &&
        (cudaMemcpy(mf->d_ci, ci.data(), sizeof(int32_t) * ci.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(mf->d_cj, cj.data(), sizeof(int32_t) * cj.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(mf->d_q, qv.data(), sizeof(int64_t) * qv.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
        delete mf;
        return CTP_ECUDA;
    }
    *out = mf;
    return CTP_OK;
}

ctp_status ctp_mf_factor(ctp_ctx *ctx, ctp_mf *mf, const double *val, const ctp_options *opt, void *stream) {
    if (ctx == nullptr || mf == nullptr || val == nullptr || opt == nullptr) return CTP_EINVAL;
    if (!(opt->u > 0.0) || opt->u > 0.5 || !(opt->small >= 0.0)) return CTP_EINVAL;
    if (opt->pivot < CTP_PIV_STRICT || opt->pivot > CTP_PIV_RESTRICTED) return CTP_EINVAL;
    if (opt->prec < CTP_FP64 || opt->prec > CTP_BF16X6) return CTP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // a fresh factorization: drop the previous one's memory
    mf->arena.release();
    mf->fronts.clear();
    mf->panels.clear();
    mf->factored = false;
    ChainCfg cfg;
    cfg.w_first = cfg.w_rest = kMaxP;
    cfg.o_first = cfg.o_rest = *opt;
    cfg.retry_tpp = false;
    ChainWork wk;
    std::vector<int32_t> loc(mf->N, -1);
    std::vector<int32_t> rows, ord, map;
    for (size_t s = 0; s < mf->blk.size(); s++) {
        ctp_mf::Blk &b = mf->blk[s];
        const int64_t pown = b.hi - b.lo;
        rows.clear();
        for (int64_t v = b.lo; v < b.hi; v++) rows.push_back((int32_t)v);
        for (int c : b.children) {
            const ctp_mf::Blk &cb = mf->blk[c];
            rows.insert(rows.end(), cb.cb.begin(), cb.cb.begin() + cb.ndel);
        }
        const int64_t d = (int64_t)rows.size() - pown;
        rows.insert(rows.end(), b.st.begin(), b.st.end());
        const int64_t n = (int64_t)rows.size(), pfs = pown + d;
        for (int64_t k = 0; k < n; k++) loc[rows[k]] = (int32_t)k;
        double *F = (double *)mf->arena.alloc(sizeof(double) * (size_t)n * n);
        if (F == nullptr) return CTP_ENOMEM;
        CTP_CUDA(cudaMemsetAsync(F, 0, sizeof(double) * (size_t)n * n, st));
        if (b.ne > 0) {
            const unsigned g = (unsigned)std::min<int64_t>((b.ne + kTh - 1) / kTh, 4096);
            CTP_CUDA(timed(ctx, K_MF_ASSEMBLE, st, [&] {
                k_mf_assemble<<<g, kTh, 0, st>>>(b.ne, mf->d_ci + b.e0, mf->d_cj + b.e0, mf->d_q + b.e0, val,
                                                  (int)pown, d, F, n);
                return cudaGetLastError();
            }));
        }
        for (int c : b.children) {
            ctp_mf::Blk &cb = mf->blk[c];
            const int64_t m = (int64_t)cb.cb.size();
            if (m == 0) continue;
            map.resize(m);
            for (int64_t k = 0; k < m; k++) {
                map[k] = loc[cb.cb[k]];
                if (map[k] < 0 || map[k] >= n) return CTP_EINVAL;  // a row the parent lacks
            }
            int32_t *dmap = (int32_t *)mf->arena.alloc(sizeof(int32_t) * m);
            if (dmap == nullptr) return CTP_ENOMEM;
            CTP_CUDA(cudaMemcpyAsync(dmap, map.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
            const double *C = cb.F + cb.elim * cb.n + cb.elim;
            const unsigned gy = (unsigned)std::min<int64_t>(m, 1024);
            const unsigned gx = (unsigned)std::min<int64_t>((m + kTh - 1) / kTh, 8);
            // (a copy from pageable memory has left `map` when cudaMemcpyAsync returns)
            CTP_CUDA(timed(ctx, K_MF_EXTEND_ADD, st, [&] {
                k_mf_extend_add<<<dim3(gx, gy), kTh, 0, st>>>(C, cb.n, m, dmap, F, n);
                return cudaGetLastError();
            }));
        }
        // eliminate the fully-summed columns (rows named by original variables)
        ord.resize(n);
        for (int64_t k = 0; k < n; k++) ord[k] = mf->perm[rows[k]];
        cfg.must_finish = b.parent < 0;
        int64_t elim = 0;
        const size_t before = mf->panels.size();
        ctp_status rc = chain_factor(ctx, F, n, n, pfs, cfg, ord.data(), mf->arena, wk, mf->panels, &elim, st);
        if (rc != CTP_OK) return rc;
        (void)before;
        b.F = F;
        b.n = n;
        b.p = pfs;
        b.elim = elim;
        b.ndel = pfs - elim;
        b.cb.resize(n - elim);
        for (int64_t k = elim; k < n; k++) b.cb[k - elim] = mf->inv[ord[k]];
        for (int64_t k = 0; k < n; k++) loc[rows[k]] = -1;
    }
    for (const PanelRec &r : mf->panels) mf->fronts.push_back(r.f);
    mf->factored = true;
    CTP_CUDA(cudaStreamSynchronize(st));
    return CTP_OK;
}

ctp_status ctp_mf_fronts(const ctp_mf *mf, int32_t *nf, const ctp_sfront **fronts) {
    if (mf == nullptr || nf == nullptr || fronts == nullptr || !mf->factored) return CTP_EINVAL;
    *nf = (int32_t)mf->fronts.size();
    *fronts = mf->fronts.data();
    return CTP_OK;
}

ctp_status ctp_mf_info(const ctp_mf *mf, int32_t cap, int32_t *nblocks, int32_t *parent, int64_t *n,
                       int64_t *p, int64_t *nelim, int64_t *ndelayed) {
    if (mf == nullptr || cap < 0) return CTP_EINVAL;
    if (nblocks) *nblocks = (int32_t)mf->blk.size();
    for (int32_t s = 0; s < (int32_t)mf->blk.size() && s < cap; s++) {
        const ctp_mf::Blk &b = mf->blk[s];
        if (parent) parent[s] = b.parent;
        if (n) n[s] = mf->factored ? b.n : (int64_t)(b.hi - b.lo + b.st.size());
        if (p) p[s] = mf->factored ? b.p : b.hi - b.lo;
        if (nelim) nelim[s] = b.elim;
        if (ndelayed) ndelayed[s] = b.ndel;
    }
    return CTP_OK;
}

ctp_status ctp_mf_panel_info(const ctp_mf *mf, int32_t cap, int64_t *n, int32_t *p, int32_t *nelim) {
    if (mf == nullptr || cap < 0 || !mf->factored) return CTP_EINVAL;
    for (int32_t k = 0; k < (int32_t)mf->panels.size() && k < cap; k++) {
        if (n) n[k] = mf->panels[k].f.n;
        if (p) p[k] = mf->panels[k].w;
        if (nelim) nelim[k] = mf->panels[k].e;
    }
    return CTP_OK;
}

ctp_status ctp_mf_destroy(ctp_mf *mf) {
    delete mf;
    return CTP_OK;
}

}  // extern "C"
