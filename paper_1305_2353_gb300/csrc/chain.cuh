// chain.cuh -- the panel-chain driver shared by dense systems and multifrontal
// fronts, and the device arena their factors live in.
#pragma once

#include <vector>

#include "ctp_internal.cuh"

namespace ctp {

int ctx_num_sms(const ctp_ctx *ctx);

// Device bump allocator: chunks of at least chunk_bytes, freed together.
struct Arena {
    std::vector<void *> chunks;
    size_t cap = 0, used = 0, chunk_bytes = (size_t)256 << 20;
    void *alloc(size_t bytes);
    void release();
};

// Scratch of the driver (grown on demand): the per-panel factor workspace, a
// copy of a panel for a retry, a pinned host buffer for nelim and perm.
struct ChainWork {
    void *ws = nullptr;
    size_t ws_bytes = 0;
    double *snap = nullptr;
    size_t snap_bytes = 0;
    int32_t *hbuf = nullptr;
    ~ChainWork();
    bool reserve(ctp_ctx *ctx, int64_t n, int w, const ctp_options *opts, int nopt);
};

struct ChainCfg {
    int w_first, w_rest;          // panel widths (first panel, the rest)
    ctp_options o_first, o_rest;  // their options (smode is set per panel)
    bool retry_tpp;    // dense system: a panel that eliminates nothing is retried with
                       // TPP and is an error if it still eliminates nothing
    bool must_finish;  // every column must be eliminated (a root front: retry with TPP)
    bool one_pass;     // a front (not a root): stop after the panel that takes the
                       // last untried fully-summed column (the rest go to the parent)
};

struct PanelRec {
    ctp_sfront f;
    int32_t e, w, pivot;
};

// Eliminate up to p_fs leading columns of the dense symmetric n x n matrix F
// (lower triangle, column-major, ld) in panels.  ord[0..n) names the rows
// (variable ids for the solve) and is permuted in step with the panels.  A
// panel that eliminates nothing stops the chain (its columns stay in F,
// leading the trailing matrix) unless cfg asks for a retry or completion.
// *elim receives the number of columns eliminated.
ctp_status chain_factor(ctp_ctx *ctx, double *F, int64_t n, int64_t ld, int64_t p_fs, const ChainCfg &cfg,
                        int32_t *ord, Arena &arena, ChainWork &wk, std::vector<PanelRec> &out,
                        int64_t *elim, cudaStream_t st);

}  // namespace ctp
