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
#include "solve_plan.cuh"

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
        int64_t pa = 0, pb = 0;  // this block's panels in the panel list
        int last_level = -1;     // solve level of its last panel
    };
    std::vector<Blk> blk;
    // assembly lists: local codes (own variables 0..p_own-1, struct rows p_own + t)
    // and value indices, all blocks concatenated, on the device
    int32_t *d_ci = nullptr, *d_cj = nullptr;
    int64_t *d_q = nullptr;
    Arena arena;  // frontal matrices and panel blocks
    std::vector<ctp_sfront> fronts;
    std::vector<PanelRec> panels;
    std::vector<int32_t> panel_block;  // block of each panel
    SolvePlan plan;  // the panels grouped into levels of independent panels
    bool factored = false;
    bool mixed = false;  // the last factorization's Form ran on the tensor cores
    ~ctp_mf() {
        if (d_ci) cudaFree(d_ci);
        if (d_cj) cudaFree(d_cj);
        if (d_q) cudaFree(d_q);
        arena.release();
    }
};

namespace {

constexpr int kTh = 256;

// Level versions: one launch for all fronts of a tree level (blockIdx.y picks
// the front, resp. blockIdx.z the child).
struct AsmRowDev {
    int64_t e0, ne;
    double *F;
    int64_t n, d;
    int p_own, pad;
};
struct ExtRowDev {
    const double *C;
    int64_t ldc, m, map_off;
    double *F;
    int64_t n;
};

__global__ void __launch_bounds__(kTh) k_mf_assemble_lv(const AsmRowDev *__restrict__ tab,
                                                        const int32_t *__restrict__ ci,
                                                        const int32_t *__restrict__ cj,
                                                        const int64_t *__restrict__ q,
                                                        const double *__restrict__ val) {
    const AsmRowDev t = tab[blockIdx.y];
    for (int64_t k = (int64_t)blockIdx.x * kTh + threadIdx.x; k < t.ne; k += (int64_t)gridDim.x * kTh) {
        int64_t a = ci[t.e0 + k], b = cj[t.e0 + k];
        if (a >= t.p_own) a += t.d;
        if (b >= t.p_own) b += t.d;
        if (a < b) {
            const int64_t u = a;
            a = b;
            b = u;
        }
        t.F[b * t.n + a] += val[q[t.e0 + k]];
    }
}

__global__ void __launch_bounds__(kTh) k_mf_extend_add_lv(const ExtRowDev *__restrict__ tab,
                                                          const int32_t *__restrict__ maps) {
    const ExtRowDev t = tab[blockIdx.z];
    const int32_t *map = maps + t.map_off;
    for (int64_t jj = blockIdx.y; jj < t.m; jj += gridDim.y) {
        const int64_t bj = map[jj];
        const double *col = t.C + jj * t.ldc;
        for (int64_t i = jj + (int64_t)blockIdx.x * kTh + threadIdx.x; i < t.m; i += (int64_t)gridDim.x * kTh) {
            int64_t a = map[i], b = bj;
            if (a < b) {
                const int64_t u = a;
                a = b;
                b = u;
            }
            t.F[b * t.n + a] += col[i];
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
    mf->panel_block.clear();
    mf->plan.clear();
    mf->factored = false;
    ChainCfg cfg;
    cfg.w_first = cfg.w_rest = kMaxP;
    cfg.o_first = cfg.o_rest = *opt;
    cfg.retry_tpp = false;
    cfg.one_pass = false;
    ChainWork wk;
    // fronts of one tree level are independent: assemble them together, and
    // factor the narrow ones (at most kMaxP fully-summed columns, not a root)
    // in one batch; the batch handles strict and restricted pivoting
    const bool batchable = opt->pivot == CTP_PIV_STRICT || opt->pivot == CTP_PIV_RESTRICTED;
    ctp_options bopt = *opt;
    bopt.smode = CTP_S_FP64_SUB;
    if (bopt.pivot == CTP_PIV_TPP) bopt.prec = CTP_FP64;
    const int nblk = (int)mf->blk.size();
    std::vector<int> lvl(nblk, 0);
    int nlev = 0;
    for (int s2 = 0; s2 < nblk; s2++) {
        for (int c : mf->blk[s2].children) lvl[s2] = std::max(lvl[s2], lvl[c] + 1);
        nlev = std::max(nlev, lvl[s2] + 1);
    }
    std::vector<std::vector<int>> bylev(nlev);
    for (int s2 = 0; s2 < nblk; s2++) bylev[lvl[s2]].push_back(s2);
    std::vector<int32_t> loc(mf->N, -1);
    void *bws = nullptr;
    size_t bws_cap = 0;
    struct AsmRow {
        int64_t e0, ne;
        double *F;
        int64_t n, d;
        int p_own, pad;
    };
    struct ExtRow {
        const double *C;
        int64_t ldc, m, map_off;
        double *F;
        int64_t n;
    };
    ctp_status rc = CTP_OK;
    for (int L = 0; L < nlev && rc == CTP_OK; L++) {
        const std::vector<int> &lv = bylev[L];
        const int nl = (int)lv.size();
        // rows of each front: own variables, delayed columns of its children, struct
        std::vector<std::vector<int32_t>> rows(nl);
        std::vector<int64_t> dcount(nl), offF(nl);
        int64_t total = 0;
        for (int i = 0; i < nl; i++) {
            ctp_mf::Blk &b = mf->blk[lv[i]];
            std::vector<int32_t> &r = rows[i];
            for (int64_t v = b.lo; v < b.hi; v++) r.push_back((int32_t)v);
            for (int c : b.children) {
                const ctp_mf::Blk &cb = mf->blk[c];
                r.insert(r.end(), cb.cb.begin(), cb.cb.begin() + cb.ndel);
            }
            dcount[i] = (int64_t)r.size() - (b.hi - b.lo);
            r.insert(r.end(), b.st.begin(), b.st.end());
            b.n = (int64_t)r.size();
            b.p = (b.hi - b.lo) + dcount[i];
            offF[i] = total;
            total += (b.n * b.n + 31) / 32 * 32;  // 256-byte aligned fronts
        }
        double *Fl = (double *)mf->arena.alloc(sizeof(double) * (size_t)(total > 0 ? total : 1));
        if (Fl == nullptr) {
            rc = CTP_ENOMEM;
            break;
        }
        for (int i = 0; i < nl; i++) mf->blk[lv[i]].F = Fl + offF[i];
        if (cudaMemsetAsync(Fl, 0, sizeof(double) * (size_t)total, st) != cudaSuccess) {
            rc = CTP_ECUDA;
            break;
        }
        // assembly of the original entries, all fronts of the level
        std::vector<AsmRow> at;
        int64_t maxne = 0;
        for (int i = 0; i < nl; i++) {
            const ctp_mf::Blk &b = mf->blk[lv[i]];
            if (b.ne == 0) continue;
            at.push_back({b.e0, b.ne, b.F, b.n, dcount[i], (int)(b.hi - b.lo), 0});
            maxne = std::max(maxne, b.ne);
        }
        // extend-add maps of all children of the level's fronts, grouped by the
        // child's rank among its siblings: siblings add into the same parent
        // entries, so each rank is a launch of its own (no two blocks of a
        // launch add into one front; the sums stay in a fixed order)
        std::vector<ExtRow> et;
        std::vector<int32_t> maps;
        std::vector<int> rank_of;
        int64_t maxm = 0;
        for (int i = 0; i < nl && rc == CTP_OK; i++) {
            const ctp_mf::Blk &b = mf->blk[lv[i]];
            for (int64_t k = 0; k < b.n; k++) loc[rows[i][k]] = (int32_t)k;
            int rank = 0;
            for (int c : b.children) {
                const ctp_mf::Blk &cb = mf->blk[c];
                const int64_t m = (int64_t)cb.cb.size();
                if (m == 0) continue;
                const int64_t off = (int64_t)maps.size();
                for (int64_t k = 0; k < m; k++) {
                    const int32_t t = loc[cb.cb[k]];
                    if (t < 0 || t >= b.n) rc = CTP_EINVAL;  // a row the parent lacks
                    maps.push_back(t);
                }
                et.push_back({cb.F + cb.elim * cb.n + cb.elim, cb.n, m, off, b.F, b.n});
                rank_of.push_back(rank++);
                maxm = std::max(maxm, m);
            }
            for (int64_t k = 0; k < b.n; k++) loc[rows[i][k]] = -1;
        }
        if (rc != CTP_OK) break;
        // order the extend-add rows by sibling rank
        std::vector<int64_t> rank_ptr(1, 0);
        {
            std::vector<int> idx(et.size());
            for (size_t k = 0; k < idx.size(); k++) idx[k] = (int)k;
            std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return rank_of[a] < rank_of[c]; });
            std::vector<ExtRow> sorted;
            sorted.reserve(et.size());
            for (size_t k = 0; k < idx.size(); k++) {
                if (k > 0 && rank_of[idx[k]] != rank_of[idx[k - 1]]) rank_ptr.push_back((int64_t)k);
                sorted.push_back(et[idx[k]]);
            }
            rank_ptr.push_back((int64_t)et.size());
            et.swap(sorted);
        }
        const size_t tbytes = align256(sizeof(AsmRow) * at.size()) + align256(sizeof(ExtRow) * et.size()) +
                              align256(sizeof(int32_t) * maps.size());
        char *tb = (char *)mf->arena.alloc(tbytes > 0 ? tbytes : 256);
        if (tb == nullptr) {
            rc = CTP_ENOMEM;
            break;
        }
        AsmRow *d_at = (AsmRow *)tb;
        ExtRow *d_et = (ExtRow *)(tb + align256(sizeof(AsmRow) * at.size()));
        int32_t *d_maps = (int32_t *)((char *)d_et + align256(sizeof(ExtRow) * et.size()));
        if ((!at.empty() && cudaMemcpyAsync(d_at, at.data(), sizeof(AsmRow) * at.size(), cudaMemcpyHostToDevice,
                                            st) != cudaSuccess) ||
            (!et.empty() && cudaMemcpyAsync(d_et, et.data(), sizeof(ExtRow) * et.size(), cudaMemcpyHostToDevice,
                                            st) != cudaSuccess) ||
            (!maps.empty() && cudaMemcpyAsync(d_maps, maps.data(), sizeof(int32_t) * maps.size(),
                                              cudaMemcpyHostToDevice, st) != cudaSuccess)) {
            rc = CTP_ECUDA;
            break;
        }
        if (!at.empty()) {
            const unsigned gx = (unsigned)std::min<int64_t>((maxne + kTh - 1) / kTh, 64);
            if (timed(ctx, K_MF_ASSEMBLE, st, [&] {
                    k_mf_assemble_lv<<<dim3(gx, (unsigned)at.size()), kTh, 0, st>>>(
                        reinterpret_cast<const AsmRowDev *>(d_at), mf->d_ci, mf->d_cj, mf->d_q, val);
                    return cudaGetLastError();
                }) != cudaSuccess) {
                rc = CTP_ECUDA;
                break;
            }
        }
        for (size_t g = 0; g + 1 < rank_ptr.size() && !et.empty(); g++) {
            const int64_t r0 = rank_ptr[g], r1 = rank_ptr[g + 1];
            if (r1 <= r0) continue;
            const unsigned gx = (unsigned)std::min<int64_t>((maxm + kTh - 1) / kTh, 4);
            const unsigned gy = (unsigned)std::min<int64_t>(maxm, 256);
            if (timed(ctx, K_MF_EXTEND_ADD, st, [&] {
                    k_mf_extend_add_lv<<<dim3(gx, gy, (unsigned)(r1 - r0)), kTh, 0, st>>>(
                        reinterpret_cast<const ExtRowDev *>(d_et) + r0, d_maps);
                    return cudaGetLastError();
                }) != cudaSuccess) {
                rc = CTP_ECUDA;
                break;
            }
        }
        if (rc != CTP_OK) break;
        // the level's fronts other than roots, in batches: each pass factors the
        // next panel (the leading at most kMaxP remaining fully-summed columns)
        // of every front still making progress, until none has columns left or
        // eliminates anything more
        std::vector<int> bi;  // indices into lv
        for (int i = 0; i < nl; i++) {
            const ctp_mf::Blk &b = mf->blk[lv[i]];
            if (batchable && b.parent >= 0 && b.n > b.p) bi.push_back(i);
        }
        std::vector<std::vector<int32_t>> ordb(bi.size());  // current row order (new numbering)
        for (size_t k = 0; k < bi.size(); k++) {
            ctp_mf::Blk &b = mf->blk[lv[bi[k]]];
            ordb[k] = rows[bi[k]];
            b.elim = 0;
            b.pa = b.pb = -1;
        }
        std::vector<int> active(bi.size());
        for (size_t k = 0; k < bi.size(); k++) active[k] = (int)k;
        std::vector<std::vector<PanelRec>> recs(bi.size());
        while (!active.empty() && rc == CTP_OK) {
            const int nb = (int)active.size();
            std::vector<int64_t> nh(nb);
            std::vector<int32_t> ph(nb);
            int64_t sp = 0, sn = 0;
            for (int k = 0; k < nb; k++) {
                const ctp_mf::Blk &b = mf->blk[lv[bi[active[k]]]];
                nh[k] = b.n - b.elim;
                ph[k] = (int32_t)std::min<int64_t>(kMaxP, b.p - b.elim);
                sp += ph[k];
                sn += nh[k];
            }
            // per-front outputs, contiguous for one read-back: nelim | perm | piv | rows, then D
            const size_t ib = align256(sizeof(int32_t) * (size_t)(nb + 2 * sp + sn));
            char *ob = (char *)mf->arena.alloc(ib + align256(sizeof(double) * 2 * (size_t)sp) +
                                               sizeof(ctp_front) * nb);
            if (ob == nullptr) {
                rc = CTP_ENOMEM;
                break;
            }
            int32_t *d_nel = (int32_t *)ob, *d_perm = d_nel + nb, *d_piv = d_perm + sp, *d_rows = d_piv + sp;
            double *d_D = (double *)(ob + ib);
            ctp_front *d_fr = (ctp_front *)(ob + ib + align256(sizeof(double) * 2 * (size_t)sp));
            std::vector<ctp_front> fh(nb);
            std::vector<int32_t> rows_h;
            rows_h.reserve(sn);
            int64_t po = 0;
            for (int k = 0; k < nb; k++) {
                ctp_mf::Blk &b = mf->blk[lv[bi[active[k]]]];
                const int64_t e0 = b.elim;
                ctp_front &f = fh[k];
                f.n = nh[k];
                f.p = ph[k];
                f.reserved = 0;
                f.A = b.F + e0 * b.n + e0;
                f.lda = b.n;
                f.perm = d_perm + po;
                f.piv = d_piv + po;
                f.D = d_D + 2 * po;
                f.nelim = d_nel + k;
                f.S = f.A + (int64_t)ph[k] * b.n + ph[k];
                f.lds = b.n;
                for (int64_t q = e0; q < b.n; q++) rows_h.push_back(mf->perm[ordb[active[k]][q]]);
                po += ph[k];
            }
            if (cudaMemcpyAsync(d_rows, rows_h.data(), sizeof(int32_t) * rows_h.size(), cudaMemcpyHostToDevice,
                                st) != cudaSuccess ||
                cudaMemcpyAsync(d_fr, fh.data(), sizeof(ctp_front) * nb, cudaMemcpyHostToDevice, st) != cudaSuccess) {
                rc = CTP_ECUDA;
                break;
            }
            ctp_plan *plan = nullptr;
            size_t need = 0;
            rc = ctp_batch_plan_create(ctx, nb, nh.data(), ph.data(), &bopt, &plan, &need);
            if (rc != CTP_OK) break;
            if (need > bws_cap) {
                if (bws) cudaFree(bws);
                bws = nullptr;
                bws_cap = 0;
                if (cudaMalloc(&bws, need) != cudaSuccess) {
                    ctp_batch_plan_destroy(plan);
                    rc = CTP_ENOMEM;
                    break;
                }
                bws_cap = need;
            }
            rc = ctp_batch_upload(ctx, plan, bws, bws_cap, st);
            if (rc == CTP_OK) rc = ctp_factor_batch(ctx, plan, d_fr, bws, bws_cap, st);
            std::vector<int32_t> flags(nb), outh(nb + sp);
            if (rc == CTP_OK) rc = ctp_batch_read_info(ctx, plan, bws, flags.data(), st);
            ctp_batch_plan_destroy(plan);
            if (rc != CTP_OK) break;
            for (int k = 0; k < nb; k++)
                if (flags[k] != CTP_OK) rc = (ctp_status)flags[k];
            if (rc != CTP_OK) break;
            if (cudaMemcpyAsync(outh.data(), d_nel, sizeof(int32_t) * (nb + sp), cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = CTP_ECUDA;
                break;
            }
            std::vector<int> next;
            std::vector<int32_t> tmp;
            po = 0;
            int64_t ro = 0;
            for (int k = 0; k < nb; k++) {
                const int a = active[k];
                ctp_mf::Blk &b = mf->blk[lv[bi[a]]];
                const int32_t e = outh[k];
                const int64_t e0 = b.elim, pk = ph[k];
                // pivot order of this pass's fully-summed rows
                std::vector<int32_t> &o = ordb[a];
                tmp.assign(o.begin() + e0, o.begin() + e0 + pk);
                for (int64_t q = 0; q < pk; q++) o[e0 + q] = tmp[outh[nb + po + q]];
                if (e > 0) {
                    PanelRec r;
                    r.f = {nh[k], (int32_t)pk, 0, fh[k].A, b.n, d_perm + po, d_piv + po, d_D + 2 * po, d_nel + k,
                           d_rows + ro};
                    r.e = e;
                    r.w = (int32_t)pk;
                    r.pivot = opt->pivot;
                    recs[a].push_back(r);
                    b.elim += e;
                    if (b.elim < b.p) next.push_back(a);
                }
                po += pk;
                ro += nh[k];
            }
            active.swap(next);
        }
        if (rc != CTP_OK) break;
        for (size_t k = 0; k < bi.size(); k++) {
            ctp_mf::Blk &b = mf->blk[lv[bi[k]]];
            b.pa = (int64_t)mf->panels.size();
            for (const PanelRec &r : recs[k]) {
                mf->panels.push_back(r);
                mf->panel_block.push_back(lv[bi[k]]);
            }
            b.pb = (int64_t)mf->panels.size();
            b.ndel = b.p - b.elim;
            b.cb.assign(ordb[k].begin() + b.elim, ordb[k].end());
        }
        // the other fronts (roots, or all fronts when the pivoting cannot be
        // batched) by the panel-chain driver
        for (int i = 0; i < nl && rc == CTP_OK; i++) {
            ctp_mf::Blk &b = mf->blk[lv[i]];
            if (std::find(bi.begin(), bi.end(), i) != bi.end()) continue;
            std::vector<int32_t> ord(b.n);
            for (int64_t k = 0; k < b.n; k++) ord[k] = mf->perm[rows[i][k]];
            cfg.must_finish = b.parent < 0;
            int64_t elim = 0;
            b.pa = (int64_t)mf->panels.size();
            rc = chain_factor(ctx, b.F, b.n, b.n, b.p, cfg, ord.data(), mf->arena, wk, mf->panels, &elim, st);
            if (rc != CTP_OK) break;
            b.pb = (int64_t)mf->panels.size();
            mf->panel_block.resize(mf->panels.size(), lv[i]);
            b.elim = elim;
            b.ndel = b.p - elim;
            b.cb.resize(b.n - elim);
            for (int64_t k = elim; k < b.n; k++) b.cb[k - elim] = mf->inv[ord[k]];
        }
    }
    if (bws) cudaFree(bws);
    if (rc != CTP_OK) {
        cudaStreamSynchronize(st);
        return rc;
    }
    for (const PanelRec &r : mf->panels) mf->fronts.push_back(r.f);
    // solve levels: a block's first panel follows its children's last panels,
    // each further panel follows the one before
    std::vector<int> level(mf->panels.size());
    for (ctp_mf::Blk &b : mf->blk) {
        int lv = -1;
        for (int c : b.children) lv = std::max(lv, mf->blk[c].last_level);
        for (int64_t k = b.pa; k < b.pb; k++) level[k] = ++lv;
        b.last_level = lv;
    }
    std::vector<int> order(mf->panels.size());
    for (size_t k = 0; k < order.size(); k++) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return level[a] < level[c]; });
    std::vector<ctp_sfront> pf;
    std::vector<int> pl;
    std::vector<int32_t> pe;
    for (int k : order) {
        pf.push_back(mf->panels[k].f);
        pl.push_back(level[k]);
        pe.push_back(mf->panels[k].e);
    }
    rc = mf->plan.build(pf, pl, pe, st);
    if (rc != CTP_OK) return rc;
    mf->factored = true;
    mf->mixed = opt->prec != CTP_FP64;
    CTP_CUDA(cudaStreamSynchronize(st));
    return CTP_OK;
}

ctp_status ctp_mf_solve_workspace_size(const ctp_mf *mf, int32_t nrhs, size_t *bytes) {
    if (mf == nullptr || bytes == nullptr || nrhs < 1 || !mf->factored) return CTP_EINVAL;
    *bytes = mf->plan.ws_bytes(nrhs);
    return CTP_OK;
}

ctp_status ctp_mf_solve(ctp_ctx *ctx, const ctp_mf *mf, int32_t nrhs, double *X, int64_t ldx, void *workspace,
                        size_t ws_bytes, void *stream) {
    if (ctx == nullptr || mf == nullptr || X == nullptr || workspace == nullptr || nrhs < 1 || !mf->factored ||
        ldx < mf->N)
        return CTP_EINVAL;
    if (ws_bytes < mf->plan.ws_bytes(nrhs)) return CTP_ENOMEM;
    CTP_CUDA(mf->plan.solve(ctx, X, ldx, nrhs, workspace, (cudaStream_t)stream));
    return CTP_OK;
}

ctp_status ctp_mf_adjoint_solve(ctp_ctx *ctx, const ctp_mf *mf, int32_t nrhs, double *G, int64_t ldg,
                                void *workspace, size_t ws_bytes, void *stream) {
    // M symmetric, D's 2x2 blocks symmetric: M^{-T} = M^{-1}, the same planned solve
    return ctp_mf_solve(ctx, mf, nrhs, G, ldg, workspace, ws_bytes, stream);
}

ctp_status ctp_mf_refine_workspace_size(const ctp_mf *mf, int32_t nrhs, size_t *bytes) {
    if (mf == nullptr || bytes == nullptr || nrhs < 1 || !mf->factored) return CTP_EINVAL;
    *bytes = refine_layout(mf->N, mf->plan.ws_bytes(nrhs), nrhs).total;
    return CTP_OK;
}

ctp_status ctp_mf_refine(ctp_ctx *ctx, const ctp_mf *mf, const int64_t *colptr, const int32_t *rowind,
                         const double *val, int32_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx,
                         int32_t max_steps, double tol, double *berr_host, int32_t *steps_host, void *workspace,
                         size_t ws_bytes, void *stream) {
    if (ctx == nullptr || mf == nullptr || !mf->factored || colptr == nullptr || rowind == nullptr ||
        val == nullptr || B == nullptr || X == nullptr || berr_host == nullptr || steps_host == nullptr ||
        workspace == nullptr || nrhs < 1 || ldb < mf->N || ldx < mf->N || max_steps < 0 || max_steps > 100 ||
        !(tol >= 0.0))
        return CTP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    MatOp A;
    A.colptr = colptr;
    A.rowind = rowind;
    A.val = val;
    // factors of a tensor-core Form: FP32 sweeps (the refinement corrects both errors)
    auto solve = [&](double *Y, int64_t ldy, void *sws) {
        return mf->plan.solve(ctx, Y, ldy, nrhs, sws, st, mf->mixed);
    };
    return refine_core(ctx, solve, mf->plan.ws_bytes(nrhs), mf->N, A, nrhs, B, ldb, X, ldx, max_steps, tol,
                       berr_host, steps_host, workspace, ws_bytes, st);
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

ctp_status ctp_mf_panel_info(const ctp_mf *mf, int32_t cap, int64_t *n, int32_t *p, int32_t *nelim,
                             int32_t *block) {
    if (mf == nullptr || cap < 0 || !mf->factored) return CTP_EINVAL;
    for (int32_t k = 0; k < (int32_t)mf->panels.size() && k < cap; k++) {
        if (n) n[k] = mf->panels[k].f.n;
        if (p) p[k] = mf->panels[k].w;
        if (nelim) nelim[k] = mf->panels[k].e;
        if (block) block[k] = mf->panel_block[k];
    }
    return CTP_OK;
}

ctp_status ctp_mf_destroy(ctp_mf *mf) {
    delete mf;
    return CTP_OK;
}

}  // extern "C"
