/*
 * ctp.h -- C ABI of libctp: compressed threshold pivoting for supernodal LDL^T
 * on NVIDIA GB300 (sm_103a).
 *
 * Method: J. D. Hogg and J. A. Scott, "Compressed threshold pivoting for sparse
 * symmetric indefinite systems", arXiv 1305.2353.  Section numbers below refer
 * to that paper.
 *
 * A supernode (Section 1, eq. (1.1)) is a dense n x p trapezoid A = [A11; A21]:
 * A11 is p x p symmetric (only its lower triangle is read), A21 is (n-p) x p.
 * All matrices are column-major double precision with leading dimension
 * lda >= n.  m = n - p is the number of A21 rows, e = nelim the number of
 * eliminated columns, d = p - e the number of delayed columns.
 *
 * Conventions shared by every entry point:
 *  - Pointers named d_* (and A, C, S, D, perm, piv, nelim, workspace) are
 *    DEVICE pointers owned by the caller; pointers named *_host are host
 *    pointers.  The library never frees caller memory.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Every entry
 *    point only enqueues work on it and returns without synchronising, except
 *    where stated ("synchronises").
 *  - Argument errors detected on the host return CTP_EINVAL (or
 *    CTP_EUNSUPPORTED) before anything is launched.  Conditions found on the
 *    device (non-finite input, a bounded wait that ran out) are recorded in the
 *    info word at the start of the workspace and read back by ctp_read_info().
 *    No kernel traps.
 *  - The workspace is caller-allocated device memory of at least the size
 *    returned by ctp_workspace_size(), 256-byte aligned.
 */
#ifndef CTP_H
#define CTP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CTP_OK = 0,
    CTP_EINVAL = 1,       /* bad argument (null pointer, n < p, lda < n, u not in (0, 0.5], ...) */
    CTP_ENOMEM = 2,       /* workspace too small */
    CTP_ECUDA = 3,        /* a CUDA runtime call failed */
    CTP_ENONFINITE = 4,   /* device: an input entry was Inf or NaN */
    CTP_ETIMEOUT = 5,     /* device: a bounded wait gave up */
    CTP_ECAPACITY = 6,    /* device: a size limit was exceeded */
    CTP_EUNSUPPORTED = 7  /* valid request this build does not handle (e.g. p above the limit) */
} ctp_status;

/* Pivoting strategy. */
typedef enum {
    CTP_PIV_STRICT = 0,     /* strict compressed pivoting, Section 4.1 (eq. (4.1), eq. (4.3)) */
    CTP_PIV_RELAXED = 1,    /* relaxed compressed pivoting, Section 4.2 */
    CTP_PIV_TPP = 2,        /* threshold partial pivoting on all n rows, Listing 1 (Section 2);
                               the comparator of the compressed strategies (FP64 only;
                               any smode but CTP_S_FP32_TILED) */
    CTP_PIV_RESTRICTED = 3, /* restricted pivoting: tests look at A11 only, Section 3.2 */
    CTP_PIV_SINGLE_ROW = 4  /* single-row compression, the variant Section 4.1 closes with:
                               eq. (4.1) with one set J = all A21 rows, so C is the one
                               row of column maxima of |A21|, with the worst-case update
                               eq. (4.3); single supernodes only (not in batches) */
} ctp_pivot;

/* Arithmetic of the Form step.  Compression, pivot selection, the 2x2 pivot
 * inversions and D11 are always FP64; the Solve is FP64 unless the options ask
 * for the tensor-core Solve (ctp_solve_kind below). */
typedef enum {
    CTP_FP64 = 0,  /* FP64 throughout */
    CTP_BF16 = 1,  /* Form on the tensor cores: BF16 operands, FP32 accumulation and
                      FP32 S (requires smode CTP_S_FP32, CTP_S_FP32_PACKED,
                      CTP_S_FP32_TILED or CTP_S_FP64_SUB); products carry the
                      BF16 rounding of L21 and W21 (relative 2^-8) */
    CTP_BF16X3 = 2, /* as CTP_BF16, with each operand split into hi = bf16(x) and
                       lo = bf16(x - hi) and the three products hi*hi + hi*lo + lo*hi
                       accumulated in FP32 (Henry, Tang & Heinecke, 2019): products
                       to about 2^-17 relative at the same bytes of S */
    CTP_BF16X6 = 3  /* three pieces hi, mid = bf16(x - hi), lo = bf16(x - hi - mid)
                       and the six products of total order <= 2 (hi*hi, hi*mid,
                       mid*hi, hi*lo, lo*hi, mid*mid): products close to FP32
                       accuracy, what FP64 refinement needs on worse-conditioned
                       systems (e.g. the shifted 3D Laplacian) */
} ctp_prec;

/* Storage of the Schur complement S (its lower triangle only):
 *  CTP_S_FP64 / CTP_S_FP32: m x m column-major, leading dimension lds >= m; the
 *    strict upper triangle is not written;
 *  CTP_S_FP64_PACKED / CTP_S_FP32_PACKED: lower-packed by columns (LAPACK 'L'
 *    packed): S(i,j), i >= j, at index j*m - j*(j-1)/2 + (i-j); m*(m+1)/2
 *    entries; lds is ignored.
 *  CTP_S_FP32_TILED: the lower block triangle in 128 x 128 blocks, each block
 *    stored contiguously and column-major inside: with nb = ceil(m/128),
 *    block (bi, bj), bi >= bj, starts at element
 *    16384 * (bj*nb - bj*(bj-1)/2 + (bi - bj)), and S(i,j) sits at
 *    (j mod 128)*128 + (i mod 128) inside it; nb*(nb+1)/2 blocks in all.
 *    Diagonal blocks hold both triangles (S is symmetric); rows past m in the
 *    last block row are zero.  Only with CTP_BF16 (the tensor-core Form writes
 *    whole blocks front to back, which HBM absorbs at full speed, unlike the
 *    column pieces of the full or packed layouts).  lds is ignored. */
typedef enum {
    CTP_S_NONE = 0,
    CTP_S_FP64 = 1,
    CTP_S_FP32 = 2,
    CTP_S_FP64_PACKED = 3,
    CTP_S_FP32_PACKED = 4,
    CTP_S_FP32_TILED = 5,
    CTP_S_FP64_SUB = 6
} ctp_smode;

/* Per-position pivot kinds written to piv[] (CTP_S_* above). */
#define CTP_PIVKIND_1X1 1
#define CTP_PIVKIND_2X2_FIRST 2
#define CTP_PIVKIND_2X2_SECOND 0
#define CTP_PIVKIND_ZERO (-1)
#define CTP_PIVKIND_DELAYED 3

/* Arithmetic of the Solve step (L21 = A21 P^T (D11 L11^T)^{-1} and the update
 * of the delayed columns, Section 1 task list).
 *  CTP_SOLVE_FP64: FP64 right-looking substitution per row (default).
 *  CTP_SOLVE_TC: one tensor-core product per supernode, x_e [U D11^{-1} | U |
 *    -U L_d^T] with U = L11^{-T} formed in FP64 on chip, split-BF16 operands
 *    (three pieces: products close to FP32) and FP32 accumulation; the outputs (L21 in
 *    FP64, the Form's BF16 operands, x_d plus its correction in FP64) carry the
 *    split's rounding, which FP64 iterative refinement on the complete system
 *    removes.  It applies with a tensor-core Form (prec != CTP_FP64, smode !=
 *    CTP_S_NONE) and compressed or restricted pivoting; otherwise the Solve is
 *    FP64.  Pivots do not change. */
typedef enum { CTP_SOLVE_FP64 = 0, CTP_SOLVE_TC = 1 } ctp_solve_kind;

typedef struct {
    double u;       /* threshold, 0 < u <= 0.5 (Section 2; default 0.01) */
    double small;   /* entries below `small` count as zero (default 1e-20) */
    int32_t pivot;  /* ctp_pivot */
    int32_t prec;   /* ctp_prec */
    int32_t smode;  /* ctp_smode */
    int32_t solve;  /* ctp_solve_kind (0: FP64) */
} ctp_options;

typedef struct ctp_ctx ctp_ctx;

/* Largest p this build factors (the pivot search keeps [A11; C] on chip). */
int32_t ctp_max_p(void);

/* Create a context bound to CUDA device `device` (it queries the device and
 * caches launch limits; it allocates no device memory).  Returns CTP_ECUDA if
 * the device is unusable. */
ctp_status ctp_create(ctp_ctx **ctx, int32_t device);
ctp_status ctp_destroy(ctp_ctx *ctx);

/* Bytes of device workspace needed by ctp_factor_supernode / ctp_compress_* for
 * an n x p supernode with these options. */
ctp_status ctp_workspace_size(const ctp_ctx *ctx, int64_t n, int32_t p, const ctp_options *opt,
                              size_t *bytes);

/* Strict compression of A21 (Section 4.1, eq. (4.1)): for every A21 row i,
 * J(i) = argmax_k |a21(i,k)| with ties to the lowest k, and
 * c(j,k) = max_{i : J(i) = j} |a21(i,k)|, or 0 when no row has J(i) = j.
 * A21: m x p device matrix (lda >= m).  C: p x p device output, ROW-major
 * (C[j*p + k] = c(j,k)); every entry is exactly |a21(i,k)| of some row or 0.
 * J: device int32[m] output, or NULL.  Exact: no rounding takes place. */
ctp_status ctp_compress_strict(ctp_ctx *ctx, int64_t m, int32_t p, const double *A21, int64_t lda,
                               double *C, int32_t *J, void *workspace, size_t ws_bytes,
                               void *stream);

/* Strict compression that allocates nothing (the paper has no counterpart:
 * this is a service of the library, not a step of the method).  For callers
 * that cannot allocate device memory at the call site -- e.g. a plugin inside
 * an application that owns every device allocation through its own pool, or a
 * latency-critical path that must not pay for cudaMalloc -- the kernel's
 * scratch (an info word and the p x p keys of C, 512 KiB at the largest p) is a
 * fixed array inside this library that every GPU holds from the moment the
 * library is loaded on it until the process exits.  Same inputs and outputs as
 * ctp_compress_strict, on the CURRENT device, with no context and no
 * workspace.  p above ctp_max_p() returns CTP_ECAPACITY.  The first call on a
 * device looks up the array's device address (a one-time set-up; make that
 * first call before any stream capture; the address stays cached for the life
 * of the process, so a program that resets the device -- cudaDeviceReset, or
 * releasing and re-creating the primary context -- must not call this entry
 * point afterwards).  All calls share the one array and
 * every call clears it first: calls that overlap on the GPU (two streams, or
 * two threads) race and must be serialised by the caller.  If info_host is not
 * NULL the call synchronises `stream` and stores the device info word there
 * (CTP_OK or CTP_ENONFINITE). */
ctp_status ctp_compress_strict_noalloc(int64_t m, int32_t p, const double *A21, int64_t lda,
                                       double *C, int32_t *J, int32_t *info_host, void *stream);

/* Relaxed compression of A21 (Section 4.2): for j = 1..p in turn, the A21 row
 * holding the largest |a21(i,j)| among rows not chosen yet (lowest row on ties)
 * becomes row j of C, with its signs.  A21: m x p device matrix (lda >= m).
 * C: p x p device output, ROW-major.  rows: device int32[p] output (the chosen
 * A21 row per C row, -1 when every row was already taken and C's row is zero),
 * or NULL.  Exact: entries of C are copies of entries of A21. */
ctp_status ctp_compress_relaxed(ctp_ctx *ctx, int64_t m, int32_t p, const double *A21,
                                int64_t lda, double *C, int32_t *rows, void *workspace,
                                size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Row split of one supernode (Section 6, Table 6.1; Appendix A): the rows of
 * A21 are cut into P blocks (one per processor), each block is compressed on
 * its own, and one exchange builds the compressed matrix C of the whole
 * supernode.  These are the per-block steps and the exchange steps of that
 * scheme; with every block on one GPU they reproduce ctp_compress_strict and
 * ctp_compress_relaxed bit for bit.  A block is rows [row0, row0 + m) of A21,
 * passed as the pointer to its first row (A21 + row0) with A21's lda.
 *
 * Strict (Section 4.1, eq. (4.1)): every block runs ctp_compress_strict on its
 * rows; C is the elementwise maximum of the blocks' matrices, exact and
 * independent of order (an allreduce with max across processors).
 * C_blocks: P row-major p x p matrices, block b at C_blocks + b * block_stride
 * (block_stride >= p*p elements); C: p x p output.  Device pointers. */
ctp_status ctp_compress_strict_merge(ctp_ctx *ctx, int32_t P, int32_t p, const double *C_blocks,
                                     int64_t block_stride, double *C, void *stream);

/* Relaxed (Section 4.2): column j's row lies among the j+1 largest |a21(i,j)|
 * of the column (ties to the lower row), and so among the union of every
 * block's j+1 largest.  Each block writes its per-column candidate lists into
 * slot `block` of a shared candidate buffer (a gather across processors);
 * ctp_compress_relaxed_select runs the paper's greedy over the union and gives
 * the chosen A21 row of every row of C (-1 when every row was already taken);
 * ctp_gather_rows copies those rows, with their signs, into C (the owners of
 * the rows send them).  P <= 8.  cand: device buffer of
 * ctp_relaxed_candidates_size(P, p) bytes, opaque except that its first int32
 * is an info word: it must be zero before the first block's call (clear the
 * buffer once), a block that meets Inf or NaN sets it to CTP_ENONFINITE, and
 * ctp_read_info(ctx, cand, ...) reads it.  Rows are reported as row0 + local
 * row, so row0 + m must stay below 2^31. */
ctp_status ctp_relaxed_candidates_size(int32_t P, int32_t p, size_t *bytes);
ctp_status ctp_compress_relaxed_candidates(ctp_ctx *ctx, int64_t m, int32_t p, const double *A21, int64_t lda,
                                           int64_t row0, int32_t P, int32_t block, void *cand,
                                           size_t cand_bytes, void *stream);
ctp_status ctp_compress_relaxed_select(ctp_ctx *ctx, int32_t P, int32_t p, const void *cand, size_t cand_bytes,
                                       int32_t *rows, void *stream);
/* C(j, :) = A21(rows[j], :) for j < p (a zero row where rows[j] < 0), C
 * row-major p x p; A21 with leading dimension lda.  Device pointers. */
ctp_status ctp_gather_rows(ctp_ctx *ctx, int32_t p, const double *A21, int64_t lda, const int32_t *rows, double *C,
                           void *stream);

/* The whole per-supernode hot path (Section 1 task list; Figure 4.1):
 * compression of A21 (strict or relaxed), pivot selection by Listing 1 on
 * [A11; C] in FP64 (with the worst-case update eq. (4.3) of C for strict), the
 * Solve L21 = A21 P^T (D11 L11^T)^{-1}, the update of the delayed columns and
 * the Form S = L21 D11 L21^T.
 *
 * In:  A (n x p, lda) holds [A11 lower; A21].
 * Out: A, in place and in pivot order:
 *        rows 0..p-1, lower triangle: unit lower L11 (diagonal implied) in the
 *          first e columns, D on the diagonal and in the (q+1, q) slot of each
 *          2x2 block, L rows of the delayed columns, and the updated delayed
 *          block (Schur complement of the eliminated pivots) in the last d
 *          columns; the strict upper triangle is unspecified;
 *        rows p..n-1: L21 in columns 0..e-1, updated delayed columns after.
 *      perm[p] (int32): perm[k] = original column at position k (0-based);
 *        positions e..p-1 are the delayed columns in their original order.
 *      piv[p] (int32): CTP_PIVKIND_* per position.
 *      D[2p] (double): D[2k] = D(k,k); D[2k+1] = D(k+1,k) for the first column
 *        of a 2x2 block, else 0.  Zero pivots have D = 0 and an all-zero L column.
 *      nelim[1] (int32): e.
 *      S, written iff opt->smode != CTP_S_NONE: lower triangle of L21 D11 L21^T
 *        in FP64 or FP32, full (lds) or packed storage (see ctp_smode).
 * All of perm, piv, D, nelim, S are device pointers.  Nothing is synchronised:
 * e is only known on the device, and the Solve and Form kernels read it there. */
ctp_status ctp_factor_supernode(ctp_ctx *ctx, int64_t n, int32_t p, double *A, int64_t lda,
                                const ctp_options *opt, int32_t *perm, int32_t *piv, double *D,
                                int32_t *nelim, void *S, int64_t lds, void *workspace,
                                size_t ws_bytes, void *stream);

/* Read the device info word of a workspace used by the calls above
 * (synchronises `stream`).  *info_host receives CTP_OK or the first device-side
 * condition (CTP_ENONFINITE, CTP_ETIMEOUT, CTP_ECAPACITY).  The word is cleared
 * at the start of every factor or compress call. */
ctp_status ctp_read_info(ctp_ctx *ctx, const void *workspace, int32_t *info_host, void *stream);


/* ------------------------------------------------------------------------ */
/* Batched factorization of many independent supernodes (the fronts of an
 * assembly tree), each exactly as ctp_factor_supernode would factor it.
 *
 * Device-visible descriptor of one front (an array of them lives in device
 * memory); all pointers are device pointers with the meaning they have in
 * ctp_factor_supernode.  S is written in the layout given by opt->smode. */
typedef struct {
    int64_t n;
    int32_t p;
    int32_t reserved;
    double *A;
    int64_t lda;
    int32_t *perm;
    int32_t *piv;
    double *D;
    int32_t *nelim;
    void *S;
    int64_t lds;
} ctp_front;

typedef struct ctp_plan ctp_plan;

/* Plan a batch from the fronts' shapes (host arrays n_host[nb], p_host[nb];
 * 1 <= p <= ctp_max_p(), n >= p).  The plan holds the launch geometry and the
 * tables the kernels need; *ws_bytes receives the device workspace the batch
 * needs.  Pivoting: CTP_PIV_STRICT or CTP_PIV_RESTRICTED; prec/smode: FP64
 * with CTP_S_NONE / CTP_S_FP64_PACKED / CTP_S_FP32_PACKED / CTP_S_FP64_SUB, or
 * CTP_BF16 / CTP_BF16X3 / CTP_BF16X6 with CTP_S_FP32_TILED or CTP_S_FP64_SUB
 * (Form on the tensor cores).  With CTP_S_FP64_SUB each front's S is the full
 * column-major FP64 matrix at ctp_front.S (leading dimension lds) from which
 * L21 D11 L21^T is subtracted (lower triangle). */
ctp_status ctp_batch_plan_create(ctp_ctx *ctx, int32_t nb, const int64_t *n_host,
                                 const int32_t *p_host, const ctp_options *opt, ctp_plan **plan,
                                 size_t *ws_bytes);
ctp_status ctp_batch_plan_destroy(ctp_plan *plan);

/* Copy the plan's tables into the workspace (one host-to-device copy on
 * `stream`); required once per workspace before ctp_factor_batch. */
ctp_status ctp_batch_upload(ctp_ctx *ctx, const ctp_plan *plan, void *workspace, size_t ws_bytes,
                            void *stream);

/* Factor every front of the batch: only kernel launches on `stream` (no host
 * synchronisation, no copy, no allocation), so the call can be captured into
 * a CUDA graph and replayed.  fronts: device array of nb descriptors. */
ctp_status ctp_factor_batch(ctp_ctx *ctx, const ctp_plan *plan, const ctp_front *fronts,
                            void *workspace, size_t ws_bytes, void *stream);

/* Per-front device info words of the last ctp_factor_batch on this workspace
 * (synchronises `stream`): flags_host[nb] receives CTP_OK or a device-side
 * condition per front. */
ctp_status ctp_batch_read_info(ctp_ctx *ctx, const ctp_plan *plan, const void *workspace,
                               int32_t *flags_host, void *stream);

/* ------------------------------------------------------------------------ */
/* Complete systems: solve, backward error and iterative refinement (Section 7).
 *
 * A factored system is a list of fronts in elimination order (children before
 * parents).  Front f covers n rows of the system, named by the variable indices
 * rows[0..n): rows[0..p) are its p fully-summed variables in the order they had
 * when the front was factored, rows[p..n) the variables of the rows below.
 * L (leading dimension ldl), perm, piv, D and nelim are ctp_factor_supernode's
 * in-place outputs for that front.  All pointers are device pointers.  The
 * fronts together give P M P^T = L D L^T for the system matrix M of order N
 * (eq. (1.2) applied front by front; a front's delayed variables are
 * eliminated by a later front). */
typedef struct {
    int64_t n;
    int32_t p;
    int32_t reserved;
    const double *L;
    int64_t ldl;
    const int32_t *perm;
    const int32_t *piv;
    const double *D;
    const int32_t *nelim;
    const int32_t *rows;
} ctp_sfront;

/* Workspace of ctp_solve for fronts of at most nmax rows and nrhs right-hand sides. */
ctp_status ctp_solve_workspace_size(int64_t nmax, int32_t nrhs, size_t *bytes);

/* X <- M^{-1} X in place (N x nrhs, column-major, ldx >= N) with the factors in
 * fronts[0..nf) (a HOST array of descriptors): forward substitution with the
 * unit lower factors, the block-diagonal solve with D (1x1 and 2x2 blocks; a
 * zero pivot gives a zero component) and back substitution, front by front.
 * Kernel launches only; nothing is synchronised. */
ctp_status ctp_solve(ctp_ctx *ctx, int32_t nf, const ctp_sfront *fronts, int64_t N, int32_t nrhs,
                     double *X, int64_t ldx, void *workspace, size_t ws_bytes, void *stream);

/* Workspace of ctp_backward_error and ctp_refine (systems of order N, fronts
 * of at most nmax rows, nrhs right-hand sides). */
ctp_status ctp_refine_workspace_size(int64_t N, int64_t nmax, int32_t nrhs, size_t *bytes);

/* Scaled backward error of Section 7 per right-hand side, in FP64 on the device:
 *   berr[r] = ||M x_r - b_r||_inf / (||M||_inf ||x_r||_inf + ||b_r||_inf).
 * M: symmetric, lower triangle stored column-major (ldm >= N; the strict upper
 * triangle is not read).  berr: device array of nrhs doubles. */
ctp_status ctp_backward_error(ctp_ctx *ctx, int64_t N, const double *M, int64_t ldm, int32_t nrhs,
                              const double *B, int64_t ldb, const double *X, int64_t ldx,
                              double *berr, void *workspace, size_t ws_bytes, void *stream);

/* Solve M X = B by the factors in fronts[0..nf) with iterative refinement
 * (Section 7: FP64 residuals, at most max_steps corrections, max_steps <= 100):
 *   X = solve(B);  while max_r berr_r > tol and fewer than max_steps
 *   corrections were made:  X += solve(B - M X).
 * M (lower triangle, as in ctp_backward_error) is the matrix before
 * factorization; the factors may be those of a perturbed M (a low-precision
 * Form), refinement then converges to the solution of M.  berr_host (host,
 * capacity (max_steps+1)*nrhs) receives the backward error of every iterate,
 * *steps_host the corrections made.  Synchronises `stream` once per iterate. */
ctp_status ctp_refine(ctp_ctx *ctx, int32_t nf, const ctp_sfront *fronts, int64_t N,
                      const double *M, int64_t ldm, int32_t nrhs, const double *B, int64_t ldb,
                      double *X, int64_t ldx, int32_t max_steps, double tol, double *berr_host,
                      int32_t *steps_host, void *workspace, size_t ws_bytes, void *stream);

/* Adjoint solve: G <- M^{-T} G with the same factors and pivot sequence.  For
 * the symmetric M of these factorizations (P M P^T = L D L^T with D symmetric:
 * its 2x2 blocks are symmetric) M^{-T} = M^{-1}, so this is the solve of
 * ctp_solve applied to G (N x nrhs, column-major, ldg >= N); it is the call the
 * backward pass of a differentiated solve makes.  Arguments as ctp_solve. */
ctp_status ctp_adjoint_solve(ctp_ctx *ctx, int32_t nf, const ctp_sfront *fronts, int64_t N,
                             int32_t nrhs, double *G, int64_t ldg, void *workspace, size_t ws_bytes,
                             void *stream);

/* Gradient of a loss through X = M^{-1} B with respect to the stored entries of
 * the symmetric M, given Gb = M^{-T} dloss/dX (from ctp_adjoint_solve) and X:
 * a stored off-diagonal entry m_ij (it stands for both m_ij and m_ji) gets
 *   -sum_r (Gb(i,r) X(j,r) + Gb(j,r) X(i,r)),
 * a diagonal entry -sum_r Gb(i,r) X(i,r)  (d(M^{-1}B) = -M^{-1} dM M^{-1}B).
 * ctp_sym_grad_dense: out is N x N column-major (ldo >= N); its lower triangle
 *   receives the gradient of the stored lower triangle, its strict upper
 *   triangle zeros (those entries are never read by the factorization).
 * ctp_sym_grad_pattern: out[k] for the stored entries (row[k], col[k]), k < nnz
 *   (int32 device arrays; row == col marks a diagonal entry).
 * All arrays are device memory; launches only. */
ctp_status ctp_sym_grad_dense(ctp_ctx *ctx, int64_t N, int32_t nrhs, const double *Gb, int64_t ldg,
                              const double *X, int64_t ldx, double *out, int64_t ldo, void *stream);
ctp_status ctp_sym_grad_pattern(ctp_ctx *ctx, int64_t nnz, const int32_t *row, const int32_t *col,
                                int64_t N, int32_t nrhs, const double *Gb, int64_t ldg,
                                const double *X, int64_t ldx, double *out, void *stream);

/* The same for a sparse M given by its lower triangle in compressed columns
 * (device arrays: colptr int64[N+1], rowind int32[nnz] with rows >= the column,
 * val float64[nnz]); the residual applies both triangles. */
ctp_status ctp_backward_error_csc(ctp_ctx *ctx, int64_t N, const int64_t *colptr, const int32_t *rowind,
                                  const double *val, int32_t nrhs, const double *B, int64_t ldb,
                                  const double *X, int64_t ldx, double *berr, void *workspace,
                                  size_t ws_bytes, void *stream);
ctp_status ctp_refine_csc(ctp_ctx *ctx, int32_t nf, const ctp_sfront *fronts, int64_t N,
                          const int64_t *colptr, const int32_t *rowind, const double *val, int32_t nrhs,
                          const double *B, int64_t ldb, double *X, int64_t ldx, int32_t max_steps,
                          double tol, double *berr_host, int32_t *steps_host, void *workspace,
                          size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Multifrontal factorization of a sparse symmetric indefinite matrix (Section
 * 1: Factor, Solve, Form and Scatter tasks over an assembly tree; delayed
 * columns passed to the parent front).
 *
 * ctp_mf_analyse (host only): the lower triangle's pattern in compressed
 *   columns (HOST arrays colptr int64[N+1], rowind int32[nnz], rows >= column),
 *   an elimination order perm[q] = variable eliminated q-th, and its supernodes
 *   as nblocks consecutive blocks of that order (blocks[0] = 0 < ... <
 *   blocks[nblocks] = N; e.g. the separators and leaf boxes of nested
 *   dissection).  Front s holds block s and struct(s), the later variables
 *   joined to the block in the filled graph; its parent is the block of
 *   struct(s)'s first variable.  *mf receives the analysis (owns host tables
 *   and small device tables).
 * ctp_mf_factor: the numeric factorization with values val (DEVICE float64[nnz],
 *   in the pattern's order).  Fronts are processed children first: assembly of
 *   original entries, extend-add of the children's contribution blocks, then
 *   the fully-summed columns (the block's, then the children's delayed ones)
 *   eliminated in panels of at most ctp_max_p() columns by ctp_factor_supernode
 *   with opt (its smode is ignored: each panel's Form subtracts into the front,
 *   whose trailing block becomes the contribution block).  A front is a chain
 *   of panels: each panel takes the leading at most ctp_max_p() remaining
 *   fully-summed columns (those the previous panel delayed first) with a fresh
 *   compression, and the front keeps starting panels while they eliminate
 *   something; after a panel that eliminates nothing the columns left are
 *   delayed to the parent.  A root front must eliminate all its columns: a
 *   panel there that eliminates nothing is retried with CTP_PIV_TPP; otherwise
 *   CTP_ECAPACITY.  The fronts of a tree level are assembled together, and
 *   with strict or restricted pivoting the non-root fronts of a level are
 *   factored in batched passes (one panel per front still making progress per
 *   pass).
 *   Device memory for the fronts is allocated by the call and held by *mf.
 *   Synchronises `stream` once per panel.
 * ctp_mf_fronts: the factored panels, in elimination order, as fronts for
 *   ctp_solve / ctp_refine_csc (host array valid until the next factor or
 *   destroy; rows name the ORIGINAL variables).
 * ctp_mf_info: per block (up to cap): parent, front rows n, fully-summed
 *   columns p (including delayed ones received), eliminated, delayed to parent. */
typedef struct ctp_mf ctp_mf;
ctp_status ctp_mf_analyse(ctp_ctx *ctx, int64_t N, const int64_t *colptr, const int32_t *rowind,
                          const int32_t *perm, int32_t nblocks, const int64_t *blocks, ctp_mf **mf);
ctp_status ctp_mf_factor(ctp_ctx *ctx, ctp_mf *mf, const double *val, const ctp_options *opt, void *stream);
ctp_status ctp_mf_fronts(const ctp_mf *mf, int32_t *nf, const ctp_sfront **fronts);
ctp_status ctp_mf_info(const ctp_mf *mf, int32_t cap, int32_t *nblocks, int32_t *parent, int64_t *n,
                       int64_t *p, int64_t *nelim, int64_t *ndelayed);
/* Solve with the factors, planned by levels of independent panels (one launch
 * per level and sweep, over items of 64 rows below a panel's pivots, instead
 * of one per panel), in FP64: X <- M^{-1} X in place (N x nrhs, device,
 * ldx >= N).  The forward sweep adds into rows shared by the panels of a level
 * with atomics, so two solves agree to rounding, not bit for bit.  Launches
 * only. */
ctp_status ctp_mf_solve_workspace_size(const ctp_mf *mf, int32_t nrhs, size_t *bytes);
ctp_status ctp_mf_solve(ctp_ctx *ctx, const ctp_mf *mf, int32_t nrhs, double *X, int64_t ldx, void *workspace,
                        size_t ws_bytes, void *stream);
/* Adjoint solve with the multifrontal factors: G <- M^{-T} G (N x nrhs,
 * device, column-major, ldg >= N) by the planned solve, with the same factors
 * and pivot sequence.  M is symmetric and so is its factored form (the 2x2
 * blocks of D are symmetric), so M^{-T} = M^{-1}: this is the solve that the
 * backward pass of a differentiated sparse solve x = M^{-1} b makes for
 * grad_b = M^{-T} grad_x (Section 1's Solve task run on the adjoint system);
 * its refined form is ctp_mf_refine with G as the right-hand sides.  The
 * gradient of the stored entries then comes from ctp_sym_grad_pattern with
 * the pattern's (row, column) pairs.  Workspace from
 * ctp_mf_solve_workspace_size.  Launches only. */
ctp_status ctp_mf_adjoint_solve(ctp_ctx *ctx, const ctp_mf *mf, int32_t nrhs, double *G, int64_t ldg,
                                void *workspace, size_t ws_bytes, void *stream);
/* ctp_refine_csc with the planned solve (arguments as there; colptr, rowind,
 * val: the matrix in device memory).  When the last ctp_mf_factor ran with a
 * tensor-core Form (opt->prec other than CTP_FP64), the solves inside the
 * refinement compute in FP32 arithmetic on the FP64 factors: X, the residuals
 * and the backward errors stay FP64 (Section 7), and the refinement contracts
 * the solves' rounding together with the factorization's.  After an FP64
 * factorization the solves are FP64. */
ctp_status ctp_mf_refine_workspace_size(const ctp_mf *mf, int32_t nrhs, size_t *bytes);
ctp_status ctp_mf_refine(ctp_ctx *ctx, const ctp_mf *mf, const int64_t *colptr, const int32_t *rowind,
                         const double *val, int32_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx,
                         int32_t max_steps, double tol, double *berr_host, int32_t *steps_host, void *workspace,
                         size_t ws_bytes, void *stream);
/* Per factored panel (up to cap, in the order of ctp_mf_fronts, an elimination
 * order): rows n, columns p, eliminated, and the block (front) it belongs to.
 * The fronts of a tree level are factored together (their narrow fronts in one
 * batch), so panels come level by level. */
ctp_status ctp_mf_panel_info(const ctp_mf *mf, int32_t cap, int64_t *n, int32_t *p, int32_t *nelim,
                             int32_t *block);
ctp_status ctp_mf_destroy(ctp_mf *mf);

typedef struct ctp_chain ctp_chain;

/* Factor a dense symmetric matrix M (order N, lower triangle, column-major,
 * ldm >= N) in place as a chain of fronts.  The first front takes the leading
 * p_first columns and all N rows -- the supernode [A11; A21] of Section 1 --
 * with opt_first; every later one takes the leading min(w_rest, rows left)
 * columns of the current Schur complement, which begin with the columns the
 * previous front delayed, with opt_rest.  Each front is factored by
 * ctp_factor_supernode; its Form subtracts L21 D11 L21^T from the trailing
 * lower triangle in place (CTP_S_FP64_SUB; opt->prec picks the FP64 or the
 * tensor-core Form; opt->smode is ignored).  A compressed or restricted front
 * that eliminates nothing is factored again with CTP_PIV_TPP (FP64).
 * Returns CTP_ECAPACITY if a front with rows below still eliminates nothing or
 * columns stay delayed with no rows below, or the first device-side condition
 * (CTP_ENONFINITE, CTP_ETIMEOUT).  Synchronises `stream` once per front (its
 * nelim and perm shape the next front).  *chain receives the factors (device
 * memory owned by the chain; M holds L and D); release with ctp_chain_destroy. */
ctp_status ctp_factor_dense(ctp_ctx *ctx, int64_t N, double *M, int64_t ldm, int32_t p_first,
                            const ctp_options *opt_first, int32_t w_rest,
                            const ctp_options *opt_rest, ctp_chain **chain, void *stream);
/* The chain's fronts (a host array valid until ctp_chain_destroy). */
ctp_status ctp_chain_fronts(const ctp_chain *chain, int32_t *nf, const ctp_sfront **fronts);
/* Per front (up to cap): nelim, columns taken and the pivoting actually used. */
ctp_status ctp_chain_info(const ctp_chain *chain, int32_t cap, int32_t *nelim, int32_t *p,
                          int32_t *pivot);
ctp_status ctp_chain_destroy(ctp_chain *chain);

/* ------------------------------------------------------------------------ */
/* Tuning knobs of a context (no counterpart in the paper: launch choices of
 * the GB300 kernels).  They change how work is scheduled, never the result.
 *
 * CTP_TUNE_FORM_WALK: the order in which the persistent tensor-core Form
 *   kernel's CTAs take the tiles of S (a ctp_walk value):
 *   CTP_WALK_AUTO (default): panels for the split form when S has at least
 *     two column blocks per SM, contiguous runs otherwise;
 *   CTP_WALK_ROUND_ROBIN: tile t to CTA t mod G down the column-block-major
 *     list (all CTAs in one column block at a time);
 *   CTP_WALK_CHUNKS: CTA c takes the c-th of G equal contiguous runs of that
 *     list (consecutive tiles share the resident L21 block);
 *   CTP_WALK_PANELS: column blocks G at a time, one per CTA, walked down in
 *     step (the W21 blocks are shared through L2).
 * CTP_TUNE_BATCH_SMEM_KB: shared memory (KB, 48..220; default 200) a CTA of
 *   the batched pivot search may hold (capped at what the kernel can take
 *   beside its static shared memory, about 190 KB); each front gets the
 *   narrowest cluster (1..16 CTAs) whose CTAs fit it.  A larger budget means fewer CTAs per
 *   front (cheaper cluster barriers, fewer parallel tests, fewer co-resident
 *   clusters).  Read when a batch plan is created.
 * CTP_TUNE_FACTOR_G: cluster width of the single-supernode pivot search
 *   (0 = by p, the default; else 1, 2, 4, 8 or 16, widened when the columns do
 *   not fit on chip).
 * CTP_TUNE_TPP_SPIN: how many polls (of about 100 ns) a software grid barrier
 *   of the full-column TPP kernel (CTP_PIV_TPP) waits for the other CTAs
 *   before it gives up: the kernel then stops, every CTA returns and the info
 *   word reads CTP_ETIMEOUT (0 = the default, 2^24 polls, about 1.5 s; else
 *   1..2^24).  Small values exist to exercise that timeout path in tests: the
 *   wait of the CTAs for CTA 0's pivot decision then runs out, and the
 *   factorization's outputs are unspecified. */
typedef enum {
    CTP_TUNE_FORM_WALK = 0,
    CTP_TUNE_BATCH_SMEM_KB = 1,
    CTP_TUNE_FACTOR_G = 2,
    CTP_TUNE_TPP_SPIN = 3
} ctp_tune_key;
typedef enum {
    CTP_WALK_AUTO = 0,
    CTP_WALK_ROUND_ROBIN = 1,
    CTP_WALK_CHUNKS = 2,
    CTP_WALK_PANELS = 3
} ctp_walk;
ctp_status ctp_tune_set(ctp_ctx *ctx, int32_t key, int32_t value);
ctp_status ctp_tune_get(const ctp_ctx *ctx, int32_t key, int32_t *value);

/* The autotuner: time the real calls on the caller's own inputs for each
 * candidate setting of the tuning knobs and keep the fastest in the context.
 * A candidate sets the nk knobs keys[0..nk) to values[c*nk .. c*nk+nk).
 * The inputs are backed up once (a device copy the tuner allocates and frees)
 * and restored before every trial and at the end, so on return they hold
 * their original values; the outputs hold the last trial's results.  Each
 * trial is one warm-up call and one timed call (CUDA events on `stream`).
 *
 * ctp_autotune_batch: trials of ctp_factor_batch, each with a plan created
 *   under the candidate's knobs.  fronts_host / fronts_dev: the same
 *   descriptors in host and device memory.
 * ctp_autotune_supernode: trials of one ctp_factor_supernode call (arguments
 *   as there).
 * ms_out[c] (host, optional) receives each candidate's time, *best (optional)
 * the index chosen.  On failure the knobs keep their previous values. */
ctp_status ctp_autotune_batch(ctp_ctx *ctx, int32_t nb, const int64_t *n_host, const int32_t *p_host,
                              const ctp_options *opt, const ctp_front *fronts_host,
                              const ctp_front *fronts_dev, int32_t nk, const int32_t *keys,
                              int32_t ncand, const int32_t *values, double *ms_out, int32_t *best,
                              void *stream);
ctp_status ctp_autotune_supernode(ctp_ctx *ctx, int64_t n, int32_t p, double *A, int64_t lda,
                                  const ctp_options *opt, int32_t *perm, int32_t *piv, double *D,
                                  int32_t *nelim, void *S, int64_t lds, void *workspace,
                                  size_t ws_bytes, int32_t nk, const int32_t *keys, int32_t ncand,
                                  const int32_t *values, double *ms_out, int32_t *best, void *stream);

/* Optional per-kernel timing.  Between ctp_profile_begin() and ctp_profile_end()
 * every kernel this library launches is bracketed by two CUDA events recorded
 * on its launch stream (at most 32768 launches are recorded).  ctp_profile_end()
 * synchronises those events and reports, per kernel name, the number of
 * launches and their summed device time in milliseconds.  names receives up to
 * max_kernels NUL-terminated names of at most 47 characters, 48 bytes apart;
 * *nkernels receives the number of distinct kernels. */
ctp_status ctp_profile_begin(ctp_ctx *ctx);
ctp_status ctp_profile_end(ctp_ctx *ctx, int32_t max_kernels, char *names, double *total_ms,
                           int32_t *launches, int32_t *nkernels);

#ifdef __cplusplus
}
#endif
#endif /* CTP_H */
