// batch.cu -- factorization of many independent supernodes (fronts) in a few
// launches: the batched path of the per-supernode hot path.
//
// The host builds a plan once from the fronts' shapes: a workspace section per
// front, the work-item tables of every batched kernel (item -> front maps and
// per-front first items), the fronts grouped by the cluster width of the pivot
// search, and the rows of each front in the stacked BF16 operand buffers of the
// tensor-core Form (each front padded to 256 rows, K stride 256).  The tables
// are copied into the workspace once (ctp_batch_upload); ctp_factor_batch then
// only launches kernels -- prepare, compress, one pivot-search launch per
// cluster width, Solve, Form -- so it can be captured into a CUDA graph.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ctp_internal.cuh"

namespace ctp {

int64_t form_fp64_tiles(int64_t m);
int64_t form_tc_tiles(int64_t m, int pieces);

namespace {

constexpr int kTR = 32;     // rows per compression item
constexpr int kThreads = 256;
constexpr unsigned long long kAbsMask = 0x7FFFFFFFFFFFFFFFull;

__device__ __forceinline__ unsigned long long abs_key(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x)) & kAbsMask;
}

// clear every front's info word and (strict) compressed-matrix keys, and the
// batch-wide info word
__global__ void k_batch_prepare(const BFront *__restrict__ tab, char *ws, BatchOpts o, int32_t *ginfo) {
    const int f = blockIdx.x;
    if (f == 0 && threadIdx.x == 0) *ginfo = 0;
    const BFront bt = tab[f];
    ctp_options oo;
    oo.pivot = o.pivot;
    oo.smode = o.smode;
    oo.prec = o.prec;
    const BSection sec = bsection(bt.n, bt.p, &oo);
    char *base = ws + bt.ws;
    if (threadIdx.x == 0) *reinterpret_cast<int32_t *>(base + sec.info) = 0;
    if (o.pivot == CTP_PIV_STRICT) {
        unsigned long long *keys = reinterpret_cast<unsigned long long *>(base + sec.C);
        for (int i = threadIdx.x; i < bt.p * bt.p; i += blockDim.x) keys[i] = 0;
        int32_t *nz = reinterpret_cast<int32_t *>(base + sec.nz);  // covers the ceil(p/32) words of bits
        for (int i = threadIdx.x; i < bt.p; i += blockDim.x) nz[i] = 0;
    }
}

// Lowest index among the lanes' (key, index) pairs with the largest key
// (keys compared as unsigned 64-bit integers by their 32-bit halves).
__device__ __forceinline__ int warp_argmax_key(unsigned long long key, int idx, unsigned &hi_out) {
    const unsigned h = (unsigned)(key >> 32), l = (unsigned)key;
    const unsigned H = __reduce_max_sync(0xffffffffu, h);
    const unsigned L = __reduce_max_sync(0xffffffffu, h == H ? l : 0u);
    hi_out = H;
    return __reduce_min_sync(0xffffffffu, (h == H && l == L) ? idx : 0x7fffffff);
}

// Strict compression (Section 4.1, eq. (4.1)), one 32-row tile of one front per
// CTA and no shared-memory tile: warp w takes rows 4w..4w+3 of the tile, two at
// a time.  Lane l loads columns l, l+32, ... of both rows with 8-byte loads
// through L1 (a 32-byte sector holds four consecutive rows of a column, so the
// tile's sectors come from memory once), the rows' maxima come from warp
// reductions on the 32-bit halves of the integer keys (lowest column on ties),
// then test-then-atomicMax into the front's C.  The rows of C that receive a
// row are gathered as bits in shared memory and published once per CTA.
// The items come bucketed by p (KPL = ceil(p / 32) columns per lane at most):
// this launch takes items ibase + blockIdx.x.
template <int KPL>
__global__ void __launch_bounds__(kThreads, KPL <= 2 ? 6 : (KPL == 4 ? 4 : 3))
    k_compress_strict_batch(const ctp_front *__restrict__ fronts, const BFront *__restrict__ tab,
                            char *ws, const int *__restrict__ item_front, int64_t ibase, BatchOpts o) {
    __shared__ unsigned rbits[kMaxP / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < kMaxP / 32) rbits[threadIdx.x] = 0u;
    const int64_t item = ibase + blockIdx.x;
    const int f = item_front[item];
    const BFront bt = tab[f];
    const ctp_front fr = fronts[f];
    ctp_options oo;
    oo.pivot = o.pivot;
    oo.smode = o.smode;
    oo.prec = o.prec;
    const BSection sec = bsection(bt.n, bt.p, &oo);
    char *base = ws + bt.ws;
    unsigned long long *Ckeys = reinterpret_cast<unsigned long long *>(base + sec.C);
    const int p = bt.p;
    const int64_t m = bt.m;
    const int64_t row0 = (item - bt.c0) * (int64_t)kTR;
    const double *A21 = fr.A + p;
    const int64_t lda = fr.lda;
    const int nrows = (int)((m - row0) < kTR ? (m - row0) : kTR);
    __syncthreads();
    bool nonfinite = false;
#pragma unroll 1
    for (int pass = 0; pass < 2; pass++) {
        const int ra = 4 * warp + 2 * pass;
        if (ra >= nrows) break;  // warp-uniform
        const bool vb = ra + 1 < nrows;
        const double *pa = A21 + row0 + ra;
        unsigned long long xa[KPL], xb[KPL];
#pragma unroll
        for (int u = 0; u < KPL; u++) {
            const int kc = lane + 32 * u;
            xa[u] = kc < p ? abs_key(pa[(int64_t)kc * lda]) : 0ull;
            xb[u] = (vb && kc < p) ? abs_key(pa[(int64_t)kc * lda + 1]) : 0ull;
        }
        // per lane: the largest key of its columns (ascending, so the lowest
        // column wins ties); lanes without a column offer none
        unsigned long long ba = xa[0], bb = xb[0];
        int ia = lane < p ? lane : 0x7fffffff, ib = ia;
#pragma unroll
        for (int u = 1; u < KPL; u++) {
            const int kc = lane + 32 * u;
            if (kc < p) {
                if (xa[u] > ba) {
                    ba = xa[u];
                    ia = kc;
                }
                if (xb[u] > bb) {
                    bb = xb[u];
                    ib = kc;
                }
            }
        }
        unsigned ha, hb;
        const int Ia = warp_argmax_key(ba, ia, ha), Ib = warp_argmax_key(bb, ib, hb);
        // an Inf or NaN anywhere in a row is its maximum key
        nonfinite |= ha >= 0x7FF00000u || (vb && hb >= 0x7FF00000u);
        if (lane == 0) {
            atomicOr(&rbits[Ia >> 5], 1u << (Ia & 31));
            if (vb) atomicOr(&rbits[Ib >> 5], 1u << (Ib & 31));
        }
        // every C key is loaded before any compare (the L2 round trips overlap);
        // the atomic fires only on a new maximum
        unsigned long long *ca = Ckeys + (int64_t)Ia * p, *cb = Ckeys + (int64_t)(vb ? Ib : Ia) * p;
        unsigned long long cura[KPL], curb[KPL];
#pragma unroll
        for (int u = 0; u < KPL; u++) {
            const int kc = lane + 32 * u;
            cura[u] = kc < p ? __ldcg(ca + kc) : ~0ull;
            curb[u] = (vb && kc < p) ? __ldcg(cb + kc) : ~0ull;
        }
#pragma unroll
        for (int u = 0; u < KPL; u++) {
            const int kc = lane + 32 * u;
            if (xa[u] > cura[u]) atomicMax(ca + kc, xa[u]);
            if (xb[u] > curb[u]) atomicMax(cb + kc, xb[u]);
        }
    }
    __syncthreads();
    // row bi of C has a member: the pivot search keeps only such rows
    if (threadIdx.x < (p + 31) / 32 && rbits[threadIdx.x] != 0u)
        atomicOr(reinterpret_cast<uint32_t *>(base + sec.nz) + threadIdx.x, rbits[threadIdx.x]);
    if (nonfinite) atomicCAS(reinterpret_cast<int32_t *>(base + sec.info), kInfoOk, (int32_t)CTP_ENONFINITE);
}

// gather the per-front info words into one array (a batch-wide condition, such
// as a timeout in the batched Form, is reported for every front still OK)
__global__ void k_batch_flags(const BFront *__restrict__ tab, const char *ws, BatchOpts o, int nb,
                              const int32_t *ginfo, int32_t *flags) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nb) return;
    const BFront bt = tab[f];
    ctp_options oo;
    oo.pivot = o.pivot;
    oo.smode = o.smode;
    oo.prec = o.prec;
    const BSection sec = bsection(bt.n, bt.p, &oo);
    const int32_t v = *reinterpret_cast<const int32_t *>(ws + bt.ws + sec.info);
    flags[f] = v != kInfoOk ? v : *ginfo;
}

}  // namespace

cudaError_t launch_compress_strict_batch(const ctp_front *fronts, const BFront *tab, char *ws,
                                         const int *item_front, const int64_t (&bucket)[5], BatchOpts o,
                                         cudaStream_t st) {
    // bucket[b] .. bucket[b+1]: the items of fronts with p <= 32 << b
    for (int b = 0; b < 4; b++) {
        const int64_t n = bucket[b + 1] - bucket[b];
        if (n == 0) continue;
        const unsigned g = (unsigned)n;
        if (b == 0)
            k_compress_strict_batch<1><<<g, kThreads, 0, st>>>(fronts, tab, ws, item_front, bucket[b], o);
        else if (b == 1)
            k_compress_strict_batch<2><<<g, kThreads, 0, st>>>(fronts, tab, ws, item_front, bucket[b], o);
        else if (b == 2)
            k_compress_strict_batch<4><<<g, kThreads, 0, st>>>(fronts, tab, ws, item_front, bucket[b], o);
        else
            k_compress_strict_batch<8><<<g, kThreads, 0, st>>>(fronts, tab, ws, item_front, bucket[b], o);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace ctp

// ---------------------------------------------------------------------------
// plan

using namespace ctp;

struct ctp_plan {
    int nb;
    ctp_options opt;
    BatchOpts bo;
    int pmax;
    bool tc;
    // workspace layout
    size_t off_ginfo, off_tab, off_citem, off_sitem, off_fitem, off_lists, off_flags, off_sections, off_wb,
        off_lb, off_qitem, off_ritem, off_xt, off_zt, off_csitem, off_cstile, off_cfitem, off_cftile;
    size_t total;
    int64_t c_items, s_items, f_items, total_rows, q_items, r_items, nxt, nzt;
    int64_t cbucket[5] = {0, 0, 0, 0, 0};  // compression items of fronts with p <= 32, 64, 128, 256
    struct Class {
        int kind, G, count;  // kFactor*, cluster width
        size_t smem;         // dynamic shared memory per CTA
        int pcap, ldcap;     // warp kernel: largest p and p + R of the class
        size_t list_off;     // element offset in the class-list array
        int pmax;            // largest p of the class
        int64_t s_off, s_count;  // the class's Solve items (front, tile) in the class Solve lists
        int64_t f_off, f_count;  // the class's Form items (front, tile) in the class Form lists
    };
    std::vector<Class> classes;
    std::vector<unsigned char> blob;  // tables, in workspace order (up to off_sections)
};

// Pivot-search class of a front.  Its working matrix [A11; C] has p + R rows,
// where R counts the rows of C that can be nonzero: at most min(p, m) for
// strict compression (each A21 row lands in one row of C), none for restricted
// pivoting.  Small fronts go to the warp kernel; fronts whose working matrix
// fits one CTA under the shared-memory budget go to the CTA kernel, bucketed
// by the shared memory they need (one launch per bucket, so that a launch's
// CTAs are of similar size); the rest to the narrowest cluster whose CTAs fit
// the budget.
struct ClassKey {
    int kind, G, bucket;
};
static ClassKey batch_class_of(int p, int64_t m, int pivot, size_t budget) {
    const int R = pivot == CTP_PIV_STRICT ? (int)(m < p ? m : p) : 0;
    if (p <= 32 && p + R <= 64) return {kFactorWarp, 1, p + R <= 32 ? 0 : 1};
    const size_t need = factor_smem_bytes(p, R, 1);
    if (need <= budget) return {kFactorCta, 1, need <= 60 * 1024 ? 0 : (need <= 98 * 1024 ? 1 : 2)};
    int G = 2;
    while (G < 16 && factor_smem_bytes(p, R, G) > budget) G <<= 1;
    return {kFactorCluster, G, 0};
}

extern "C" {

ctp_status ctp_batch_plan_create(ctp_ctx *ctx, int32_t nb, const int64_t *n_host,
                                 const int32_t *p_host, const ctp_options *opt, ctp_plan **plan,
                                 size_t *ws_bytes) {
    if (ctx == nullptr || plan == nullptr || opt == nullptr || nb < 1 || n_host == nullptr ||
        p_host == nullptr)
        return CTP_EINVAL;
    *plan = nullptr;
    if (!(opt->u > 0.0) || opt->u > 0.5 || !(opt->small >= 0.0)) return CTP_EINVAL;
    if (opt->pivot != CTP_PIV_STRICT && opt->pivot != CTP_PIV_RESTRICTED) return CTP_EUNSUPPORTED;
    if (opt->prec < CTP_FP64 || opt->prec > CTP_BF16X6) return CTP_EINVAL;
    const bool tc = opt->prec != CTP_FP64 && opt->smode != CTP_S_NONE;
    const int pieces = tc ? prec_pieces(opt->prec) : 0;
    const bool stc = solve_on_tc(opt);
    if (tc && opt->smode != CTP_S_FP32_TILED && opt->smode != CTP_S_FP64_SUB) return CTP_EUNSUPPORTED;
    if (!tc && opt->smode != CTP_S_NONE && opt->smode != CTP_S_FP64_PACKED &&
        opt->smode != CTP_S_FP32_PACKED && opt->smode != CTP_S_FP64_SUB)
        return CTP_EUNSUPPORTED;
    for (int f = 0; f < nb; f++) {
        if (p_host[f] < 1 || n_host[f] < p_host[f]) return CTP_EINVAL;
        if (p_host[f] > kMaxP) return CTP_EUNSUPPORTED;
        if (n_host[f] - p_host[f] > 0x7fffffffLL) return CTP_EUNSUPPORTED;
    }
    ctp_plan *P = new ctp_plan();
    P->nb = nb;
    P->opt = *opt;
    P->bo.u = opt->u;
    P->bo.small = opt->small;
    P->bo.pivot = opt->pivot;
    P->bo.smode = opt->smode;
    P->bo.prec = opt->prec;
    P->tc = tc;
    P->pmax = 1;
    std::vector<BFront> tab(nb);
    std::vector<int> citem, sitem, fitem, qitem, ritem;
    size_t sec_off = 0;
    int64_t row0 = 0, xt = 0, zt = 0;
    for (int f = 0; f < nb; f++) {
        BFront &b = tab[f];
        b.n = n_host[f];
        b.p = p_host[f];
        b.m = b.n - b.p;
        b.nM = (int)((b.m + 127) / 128);
        b.ws = (int64_t)sec_off;
        sec_off += bsection(b.n, b.p, opt).total;
        b.row0 = row0;
        if (tc) row0 += (b.m + 255) / 256 * 256;
        const int64_t nt = (b.m + kTR - 1) / kTR;
        b.s0 = (int64_t)sitem.size();
        for (int64_t t = 0; t < nt; t++) sitem.push_back(f);
        b.f0 = (int64_t)fitem.size();
        if (opt->smode != CTP_S_NONE) {
            const int64_t ft = tc ? form_tc_tiles(b.m, pieces) : form_fp64_tiles(b.m);
            for (int64_t t = 0; t < ft; t++) fitem.push_back(f);
        }
        b.kbx = (b.p + 63) / 64;
        b.nwz = stc ? solve_tc_windows(b.p) : 0;
        b.xt0 = xt;
        b.zt0 = zt;
        b.q0 = (int64_t)qitem.size();
        b.r0 = (int64_t)ritem.size();
        if (stc && b.m > 0) {
            const int64_t nrb = (b.m + 127) / 128;
            xt += nrb * b.kbx;
            zt += (int64_t)b.nwz * b.kbx;
            for (int64_t t = 0; t < nrb * b.nwz; t++) qitem.push_back(f);
            for (int64_t t = 0; t < (int64_t)b.kbx * 8; t++) ritem.push_back(f);  // 8 rows per item
        }
        P->pmax = std::max(P->pmax, b.p);
    }
    // compression items (32-row tiles), bucketed by p so that each launch's
    // kernel holds no more columns per lane than its fronts need
    if (opt->pivot == CTP_PIV_STRICT) {
        for (int bk = 0; bk < 4; bk++) {
            P->cbucket[bk] = (int64_t)citem.size();
            for (int f = 0; f < nb; f++) {
                const int p = tab[f].p;
                const int fb = p <= 32 ? 0 : (p <= 64 ? 1 : (p <= 128 ? 2 : 3));
                if (fb != bk) continue;
                tab[f].c0 = (int64_t)citem.size();
                for (int64_t t = 0; t < (tab[f].m + kTR - 1) / kTR; t++) citem.push_back(f);
            }
        }
    }
    P->cbucket[4] = (int64_t)citem.size();
    // fronts by pivot-search class: warp (2 buckets), CTA (3 buckets), cluster
    // (G = 2, 4, 8, 16), in this order; the launch sequence starts from the end
    size_t budget = (size_t)ctx_batch_smem_kb(ctx) * 1024;
    if (budget > factor_batch_max_dynamic_smem()) budget = factor_batch_max_dynamic_smem();
    constexpr int kNumKeys = 2 + 3 + 4;
    std::vector<std::vector<int>> byKey(kNumKeys);
    std::vector<int> pmaxK(kNumKeys, 1), ldmaxK(kNumKeys, 1);
    std::vector<size_t> smemK(kNumKeys, 0);
    for (int f = 0; f < nb; f++) {
        const int p = tab[f].p;
        const int64_t m = tab[f].m;
        const ClassKey k = batch_class_of(p, m, opt->pivot, budget);
        const int R = opt->pivot == CTP_PIV_STRICT ? (int)(m < p ? m : p) : 0;
        const int gi = k.G == 2 ? 0 : k.G == 4 ? 1 : k.G == 8 ? 2 : 3;
        const int key = k.kind == kFactorWarp ? k.bucket : (k.kind == kFactorCta ? 2 + k.bucket : 5 + gi);
        byKey[key].push_back(f);
        pmaxK[key] = std::max(pmaxK[key], p);
        ldmaxK[key] = std::max(ldmaxK[key], p + R);
        if (k.kind != kFactorWarp) smemK[key] = std::max(smemK[key], factor_smem_bytes(p, R, k.G));
    }
    // within a class, the fronts with the most pivot-search work first (about
    // p^2 (p + R) terms), so that no large front starts in the launch's last
    // wave; the results do not depend on the order
    for (int key = 0; key < kNumKeys; key++) {
        auto work = [&](int f) {
            const int64_t p = tab[f].p, m = tab[f].m;
            const int64_t R = opt->pivot == CTP_PIV_STRICT ? (m < p ? m : p) : 0;
            return p * p * (p + R);
        };
        std::stable_sort(byKey[key].begin(), byKey[key].end(), [&](int x, int y) { return work(x) > work(y); });
    }
    std::vector<int> lists, csitem, cstile, cfitem, cftile;
    for (int key = 0; key < kNumKeys; key++) {
        if (byKey[key].empty()) continue;
        ctp_plan::Class c;
        c.pmax = pmaxK[key];
        c.s_off = (int64_t)csitem.size();
        for (int f : byKey[key])
            for (int64_t t = 0; t < (tab[f].m + kTR - 1) / kTR; t++) {
                csitem.push_back(f);
                cstile.push_back((int)t);
            }
        c.s_count = (int64_t)csitem.size() - c.s_off;
        c.f_off = (int64_t)cfitem.size();
        if (opt->smode != CTP_S_NONE)
            for (int f : byKey[key]) {
                const int64_t ft = tc ? form_tc_tiles(tab[f].m, pieces) : form_fp64_tiles(tab[f].m);
                for (int64_t t = 0; t < ft; t++) {
                    cfitem.push_back(f);
                    cftile.push_back((int)t);
                }
            }
        c.f_count = (int64_t)cfitem.size() - c.f_off;
        c.kind = key < 2 ? kFactorWarp : (key < 5 ? kFactorCta : kFactorCluster);
        c.G = key < 5 ? 1 : (2 << (key - 5));
        c.pcap = pmaxK[key];
        c.ldcap = ldmaxK[key];
        c.smem = c.kind == kFactorWarp ? factor_warp_smem_bytes(c.pcap, c.ldcap) : smemK[key];
        c.count = (int)byKey[key].size();
        c.list_off = lists.size();
        lists.insert(lists.end(), byKey[key].begin(), byKey[key].end());
        P->classes.push_back(c);
    }
    P->c_items = (int64_t)citem.size();
    P->s_items = (int64_t)sitem.size();
    P->f_items = (int64_t)fitem.size();
    P->q_items = (int64_t)qitem.size();
    P->r_items = (int64_t)ritem.size();
    P->nxt = xt;
    P->nzt = zt;
    P->total_rows = row0;
    // workspace layout
    size_t off = 0;
    P->off_ginfo = off;  // batch-wide info word (tensor-core Form timeouts)
    off += 256;
    P->off_tab = off;
    off += align256(sizeof(BFront) * (size_t)nb);
    P->off_citem = off;
    off += align256(sizeof(int) * citem.size());
    P->off_sitem = off;
    off += align256(sizeof(int) * sitem.size());
    P->off_fitem = off;
    off += align256(sizeof(int) * fitem.size());
    P->off_lists = off;
    off += align256(sizeof(int) * lists.size());
    P->off_qitem = off;
    off += align256(sizeof(int) * qitem.size());
    P->off_ritem = off;
    off += align256(sizeof(int) * ritem.size());
    P->off_csitem = off;
    off += align256(sizeof(int) * csitem.size());
    P->off_cstile = off;
    off += align256(sizeof(int) * cstile.size());
    P->off_cfitem = off;
    off += align256(sizeof(int) * cfitem.size());
    P->off_cftile = off;
    off += align256(sizeof(int) * cftile.size());
    P->off_flags = off;
    off += align256(sizeof(int32_t) * (size_t)nb);
    const size_t tables_end = off;
    P->off_sections = off;
    off += align256(sec_off);
    // BF16 operand copies: hi rows, then (split) the lo rows
    const size_t copies = pieces > 0 ? pieces : 1;
    P->off_wb = off;
    off += align256(tc ? 2 * copies * (size_t)row0 * kBatchKp : 0);
    P->off_lb = off;
    off += align256(tc ? 2 * copies * (size_t)row0 * kBatchKp : 0);
    P->bo.lo_off = pieces > 1 ? row0 * kBatchKp : 0;
    P->bo.pieces = pieces;
    // tensor-core Solve: x_e and Z^T tiles, three pieces each
    P->bo.stc = stc ? 1 : 0;
    P->bo.xoff = (int64_t)xt * (int64_t)solve_tc_tile_elems();
    P->bo.zoff = (int64_t)zt * (int64_t)solve_tc_tile_elems();
    P->off_xt = off;
    off += align256(stc ? 2 * 3 * (size_t)P->bo.xoff : 0);
    P->off_zt = off;
    off += align256(stc ? 2 * 3 * (size_t)P->bo.zoff : 0);
    P->total = off;
    // section offsets are relative to the sections base: shift them to the workspace base
    for (int f = 0; f < nb; f++) tab[f].ws += (int64_t)P->off_sections;
    P->blob.assign(tables_end, 0);
    memcpy(P->blob.data() + P->off_tab, tab.data(), sizeof(BFront) * (size_t)nb);
    if (!citem.empty()) memcpy(P->blob.data() + P->off_citem, citem.data(), sizeof(int) * citem.size());
    if (!sitem.empty()) memcpy(P->blob.data() + P->off_sitem, sitem.data(), sizeof(int) * sitem.size());
    if (!fitem.empty()) memcpy(P->blob.data() + P->off_fitem, fitem.data(), sizeof(int) * fitem.size());
    if (!lists.empty()) memcpy(P->blob.data() + P->off_lists, lists.data(), sizeof(int) * lists.size());
    if (!qitem.empty()) memcpy(P->blob.data() + P->off_qitem, qitem.data(), sizeof(int) * qitem.size());
    if (!ritem.empty()) memcpy(P->blob.data() + P->off_ritem, ritem.data(), sizeof(int) * ritem.size());
    if (!csitem.empty()) {
        memcpy(P->blob.data() + P->off_csitem, csitem.data(), sizeof(int) * csitem.size());
        memcpy(P->blob.data() + P->off_cstile, cstile.data(), sizeof(int) * cstile.size());
    }
    if (!cfitem.empty()) {
        memcpy(P->blob.data() + P->off_cfitem, cfitem.data(), sizeof(int) * cfitem.size());
        memcpy(P->blob.data() + P->off_cftile, cftile.data(), sizeof(int) * cftile.size());
    }
    *plan = P;
    if (ws_bytes) *ws_bytes = P->total;
    return CTP_OK;
}

ctp_status ctp_batch_plan_destroy(ctp_plan *plan) {
    delete plan;
    return CTP_OK;
}

ctp_status ctp_batch_upload(ctp_ctx *ctx, const ctp_plan *plan, void *workspace, size_t ws_bytes,
                            void *stream) {
    if (ctx == nullptr || plan == nullptr || workspace == nullptr) return CTP_EINVAL;
    if (ws_bytes < plan->total) return CTP_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)workspace;
    if (cudaMemcpyAsync(w, plan->blob.data(), plan->blob.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return CTP_ECUDA;
    if (plan->tc) {
        // padding rows of the stacked operands must read as zero
        if (cudaMemsetAsync(w + plan->off_wb, 0, plan->off_lb - plan->off_wb, st) != cudaSuccess ||
            cudaMemsetAsync(w + plan->off_lb, 0, plan->off_xt - plan->off_lb, st) != cudaSuccess)
            return CTP_ECUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return CTP_ECUDA;  // the blob is pageable
    return CTP_OK;
}

ctp_status ctp_batch_read_info(ctp_ctx *ctx, const ctp_plan *plan, const void *workspace,
                               int32_t *flags_host, void *stream) {
    if (ctx == nullptr || plan == nullptr || workspace == nullptr || flags_host == nullptr)
        return CTP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)const_cast<void *>(workspace);
    k_batch_flags<<<(plan->nb + 255) / 256, 256, 0, st>>>(
        reinterpret_cast<const BFront *>(w + plan->off_tab), w, plan->bo, plan->nb,
        reinterpret_cast<const int32_t *>(w + plan->off_ginfo), reinterpret_cast<int32_t *>(w + plan->off_flags));
    if (cudaGetLastError() != cudaSuccess) return CTP_ECUDA;
    if (cudaMemcpyAsync(flags_host, w + plan->off_flags, sizeof(int32_t) * (size_t)plan->nb,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return CTP_ECUDA;
    return CTP_OK;
}

}  // extern "C"

// The launch sequence (called from api.cu, which owns the profiling hooks).
namespace ctp {

struct BatchLaunch {
    const ctp_plan *P;
    const ctp_front *fronts;
    char *w;
};

int batch_num_classes(const ctp_plan *P) { return (int)P->classes.size(); }
int batch_class_kind(const ctp_plan *P, int c) { return P->classes[c].kind; }
int batch_class_G(const ctp_plan *P, int c) { return P->classes[c].G; }
size_t batch_total(const ctp_plan *P) { return P->total; }

cudaError_t batch_prepare(const ctp_plan *P, char *w, cudaStream_t st) {
    k_batch_prepare<<<P->nb, 256, 0, st>>>(reinterpret_cast<const BFront *>(w + P->off_tab), w, P->bo,
                                            reinterpret_cast<int32_t *>(w + P->off_ginfo));
    return cudaGetLastError();
}
cudaError_t batch_compress(const ctp_plan *P, const ctp_front *fr, char *w, int num_sms, cudaStream_t st) {
    if (P->opt.pivot != CTP_PIV_STRICT) return cudaSuccess;
    (void)num_sms;
    return launch_compress_strict_batch(fr, reinterpret_cast<const BFront *>(w + P->off_tab), w,
                                        reinterpret_cast<const int *>(w + P->off_citem), P->cbucket, P->bo, st);
}
cudaError_t batch_factor_class(const ctp_plan *P, int ci, const ctp_front *fr, char *w, cudaStream_t st) {
    const ctp_plan::Class &c = P->classes[ci];
    return launch_factor_batch(fr, reinterpret_cast<const BFront *>(w + P->off_tab), w,
                               reinterpret_cast<const int *>(w + P->off_lists) + c.list_off, c.count, c.kind,
                               c.G, c.smem, c.pcap, c.ldcap, P->bo, st);
}
cudaError_t batch_solve(const ctp_plan *P, const ctp_front *fr, char *w, int num_sms, cudaStream_t st) {
    if (P->bo.stc)
        return launch_solve_tc_batch(fr, reinterpret_cast<const BFront *>(w + P->off_tab), w,
                                     reinterpret_cast<const int *>(w + P->off_sitem), P->s_items,
                                     reinterpret_cast<const int *>(w + P->off_qitem), P->q_items,
                                     reinterpret_cast<const int *>(w + P->off_ritem), P->r_items, P->bo,
                                     w + P->off_xt, w + P->off_zt, P->nxt, P->nzt, w + P->off_wb, w + P->off_lb,
                                     reinterpret_cast<int32_t *>(w + P->off_ginfo), num_sms, st);
    return launch_solve_batch(fr, reinterpret_cast<const BFront *>(w + P->off_tab), w,
                              reinterpret_cast<const int *>(w + P->off_sitem), P->s_items, P->bo,
                              P->tc ? w + P->off_wb : nullptr, P->tc ? w + P->off_lb : nullptr, P->pmax,
                              st);
}
// The FP64 Solve of one pivot-search class's fronts (false when the batch
// solves on the tensor cores: that Solve runs once over all fronts)
bool batch_solve_per_class(const ctp_plan *P) { return !P->bo.stc; }
cudaError_t batch_solve_class(const ctp_plan *P, int ci, const ctp_front *fr, char *w, cudaStream_t st) {
    const ctp_plan::Class &c = P->classes[ci];
    return launch_solve_batch(fr, reinterpret_cast<const BFront *>(w + P->off_tab), w,
                              reinterpret_cast<const int *>(w + P->off_csitem) + c.s_off, c.s_count, P->bo,
                              P->tc ? w + P->off_wb : nullptr, P->tc ? w + P->off_lb : nullptr, c.pmax, st,
                              reinterpret_cast<const int *>(w + P->off_cstile) + c.s_off);
}
// The Form of one pivot-search class's fronts (after that class's Solve)
cudaError_t batch_form_class(const ctp_plan *P, int ci, const ctp_front *fr, char *w, int num_sms,
                             cudaStream_t st) {
    if (P->opt.smode == CTP_S_NONE) return cudaSuccess;
    const ctp_plan::Class &c = P->classes[ci];
    const BFront *tab = reinterpret_cast<const BFront *>(w + P->off_tab);
    const int *fitem = reinterpret_cast<const int *>(w + P->off_cfitem) + c.f_off;
    const int *ftile = reinterpret_cast<const int *>(w + P->off_cftile) + c.f_off;
    if (P->tc)
        return launch_form_tc_batch(fr, tab, fitem, c.f_count, P->total_rows, w + P->off_wb, w + P->off_lb,
                                    P->bo.pieces, P->opt.smode == CTP_S_FP64_SUB ? 3 : 2,
                                    reinterpret_cast<int32_t *>(w + P->off_ginfo), num_sms, st, ftile);
    return launch_form_fp64_batch(fr, tab, w, fitem, c.f_count, P->bo, st, ftile);
}
cudaError_t batch_form(const ctp_plan *P, const ctp_front *fr, char *w, int num_sms, cudaStream_t st) {
    if (P->opt.smode == CTP_S_NONE) return cudaSuccess;
    const BFront *tab = reinterpret_cast<const BFront *>(w + P->off_tab);
    const int *fitem = reinterpret_cast<const int *>(w + P->off_fitem);
    if (P->tc)
        return launch_form_tc_batch(fr, tab, fitem, P->f_items, P->total_rows, w + P->off_wb, w + P->off_lb,
                                    P->bo.pieces, P->opt.smode == CTP_S_FP64_SUB ? 3 : 2,
                                    reinterpret_cast<int32_t *>(w + P->off_ginfo), num_sms, st);
    return launch_form_fp64_batch(fr, tab, w, fitem, P->f_items, P->bo, st);
}

}  // namespace ctp
