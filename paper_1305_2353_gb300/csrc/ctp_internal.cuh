// ctp_internal.cuh -- internal declarations shared by the libctp translation units.
// Product code only: nothing here is used by, or uses, the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ctp.h"

namespace ctp {

// Largest supernode width handled on chip by the pivot search (kernel K3).
constexpr int kMaxP = 256;

// Device info word codes (first int32 of the workspace).
constexpr int kInfoOk = 0;

// Workspace layout (all offsets 256-byte aligned):
//   [0, 256)            info word + scratch counters
//   C                   p*p doubles, row-major compressed matrix (strict: as uint64 keys)
//   Dinv                2p doubles: inverse pivot blocks, same slots as D
//   W21                 m*p doubles (FP64 Y = L21 D11) when the FP64 Form step runs
//   Wb, Lb              m*Kp BF16 copies of Y and L21 for the tensor-core Form
//   aux                 method-specific scratch (relaxed candidate lists)
struct WsLayout {
    size_t info, C, Dinv, W21, Wb, Lb, aux, Xs, flags, total;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Make sure `func` may launch with `bytes` of dynamic shared memory on the
// current device: raises cudaFuncAttributeMaxDynamicSharedMemorySize when it is
// below `bytes` and never lowers it.  The attribute belongs to the function,
// not to one launch: a CUDA graph node captured with more shared memory than a
// later, lower setting allows fails when the graph is replayed, so no launcher
// may lower it.  (A device reset restores the default; the current value is
// queried each time, so the next launch raises it again.)
cudaError_t smem_at_least(const void *func, size_t bytes);

WsLayout ws_layout(int64_t n, int p, const ctp_options *opt, int num_sms);
int ctx_batch_smem_kb(const ctp_ctx *ctx);  // CTP_TUNE_BATCH_SMEM_KB of a context
// BF16 pieces per operand of the tensor-core Form for a precision (0: FP64 Form)
inline int prec_pieces(int prec) {
    return prec == CTP_BF16 ? 1 : (prec == CTP_BF16X3 ? 2 : (prec == CTP_BF16X6 ? 3 : 0));
}
size_t factor_batch_max_dynamic_smem();     // dynamic shared memory the batched pivot search can take
size_t factor_smem_bytes(int p, int R, int G);  // dynamic shared memory of a pivot-search CTA
size_t factor_warp_smem_bytes(int pcap, int ldcap);  // of a CTA of the warp-per-front kernel
// kinds of batched pivot-search launch: a warp per front (p <= 32, at most 64
// rows of [A11; C]), a CTA per front, a cluster of G CTAs per front
constexpr int kFactorWarp = 0, kFactorCta = 1, kFactorCluster = 2;

// ---------------------------------------------------------------------------
// kernel launchers (each returns cudaError_t of the launch)
// rowbits (optional, ceil(p/32) words cleared by the caller): bit j set for
// every row j of C that receives an A21 row (the rows the pivot search must keep)
cudaError_t launch_compress_strict(const double *A21, int64_t m, int p, int64_t lda,
                                   unsigned long long *Ckeys, int32_t *J, uint32_t *rowbits, int32_t *info,
                                   int num_sms, cudaStream_t st);
// single-row compression: ckey[k] (p keys, zeroed by the caller) = max_i |a21(i,k)|
cudaError_t launch_compress_single_row(const double *A21, int64_t m, int p, int64_t lda,
                                       unsigned long long *ckey, int32_t *info, int num_sms, cudaStream_t st);
int relaxed_block_lg(int64_t m, int p);
size_t relaxed_aux_bytes(int64_t m, int p, int num_sms);
cudaError_t launch_compress_relaxed(const double *A21, int64_t m, int p, int64_t lda, double *C,
                                    int32_t *rows, void *aux, int32_t *info, int num_sms,
                                    cudaStream_t st);
cudaError_t launch_keys_to_rowmajor(const unsigned long long *Ckeys, double *C, int p,
                                    cudaStream_t st);

struct FactorArgs {
    double *A;          // n x p supernode (in/out)
    int64_t lda;
    int p;
    int R;              // outer rows held on chip: p (compressed) or 0 (restricted)
    int abs_update;     // 1: strict worst-case update of the outer rows
    const double *C;    // R x p row-major outer rows (doubles), or nullptr
    const uint32_t *rowbits;  // R bits: set for rows of C that may be nonzero (nullptr: scan C)
    double u, small;
    int32_t *perm, *piv, *nelim;
    double *D, *Dinv;
    int32_t *info;
};
cudaError_t launch_factor_cluster(const FactorArgs &a, int G /* 0: by p */, cudaStream_t st);

// ---------------------------------------------------------------------------
// batched path: per-front table (built on the host by the plan, uploaded into
// the workspace) and the per-front workspace sections
struct BFront {
    int64_t n, m;
    int32_t p, nM;       // nM: 128-row blocks of S (tensor-core Form)
    int64_t ws;          // byte offset of this front's workspace section
    int64_t row0;        // first row of this front in the stacked BF16 operand buffers
    int64_t c0, s0, f0;  // first compression / solve / form work item of this front
    // tensor-core Solve: first 128 x 64 tile of x_e and of Z^T, first GEMM item,
    // K blocks and output windows at most (from p)
    int64_t xt0, zt0, q0, r0;  // r0: first prep item (8 identity rows each)
    int32_t kbx, nwz;
};
// offsets inside a front's section: info word, compressed matrix (strict),
// Dinv, and W21 = L21 D11 when an FP64 Form follows
struct BSection {
    size_t info, C, Dinv, W21, nz, total;
};
__host__ __device__ inline size_t align256hd(size_t x) { return (x + 255) & ~size_t(255); }
__host__ __device__ inline BSection bsection(int64_t n, int p, const ctp_options *opt) {
    BSection s;
    size_t off = 0;
    s.info = off;
    off += 256;
    s.C = off;
    off += align256hd(opt->pivot == CTP_PIV_STRICT ? sizeof(double) * (size_t)p * p : 0);
    s.Dinv = off;
    off += align256hd(sizeof(double) * (2 * (size_t)p + 2));
    s.W21 = off;
    off += align256hd((opt->smode != CTP_S_NONE && opt->prec == CTP_FP64) ? sizeof(double) * (size_t)(n - p) * p : 0);
    s.nz = off;  // strict: which rows of C receive an A21 row (one bit per row)
    off += align256hd(opt->pivot == CTP_PIV_STRICT ? sizeof(int32_t) * (size_t)p : 0);
    s.total = off;
    return s;
}

struct BatchOpts {
    double u, small;
    int pivot;  // ctp_pivot
    int smode, prec;
    int64_t lo_off;  // elements between the BF16 pieces of the operand copies
    int pieces;      // BF16 pieces per operand (1: plain; 2, 3: split)
    int stc;         // the Solve runs on the tensor cores
    int64_t xoff, zoff;  // elements between the pieces of the x_e / Z^T tile arrays
};
// pivot search of the fronts list[0..count) of one class: kind (kFactor*), the
// cluster width G, the dynamic shared memory per CTA, and for the warp kernel
// the largest p and p + R of the class (its per-warp slice)
cudaError_t launch_factor_batch(const ctp_front *fronts, const BFront *tab, char *ws, const int *list,
                                int count, int kind, int G, size_t smem, int pcap, int ldcap, BatchOpts o,
                                cudaStream_t st);
// bucket[b] .. bucket[b+1]: the items (32-row tiles) of the fronts with p <= 32 << b
cudaError_t launch_compress_strict_batch(const ctp_front *fronts, const BFront *tab, char *ws,
                                         const int *item_front, const int64_t (&bucket)[5], BatchOpts o,
                                         cudaStream_t st);
// item_tile (optional): each item's 32-row tile of its front; without it the
// items of a front are consecutive, from tab[front].s0 on
cudaError_t launch_solve_batch(const ctp_front *fronts, const BFront *tab, char *ws,
                               const int *item_front, int64_t items, BatchOpts o, void *Wb, void *Lb,
                               int pmax, cudaStream_t st, const int *item_tile = nullptr);
// item_tile (optional, both batched Forms): each item's tile of its front;
// without it the items of a front are consecutive, from tab[front].f0 on
cudaError_t launch_form_fp64_batch(const ctp_front *fronts, const BFront *tab, char *ws,
                                   const int *item_front, int64_t items, BatchOpts o,
                                   cudaStream_t st, const int *item_tile = nullptr);
cudaError_t launch_form_tc_batch(const ctp_front *fronts, const BFront *tab, const int *item_front,
                                 int64_t items, int64_t total_rows, const void *Wb, const void *Lb,
                                 int pieces, int layout /* 2 tiled, 3 subtract */, int32_t *info, int num_sms,
                                 cudaStream_t st, const int *item_tile = nullptr);
constexpr int kBatchKp = 256;  // K stride of the stacked BF16 operand buffers

// the batched launch sequence (batch.cu); the plan type is declared in ctp.h
int batch_num_classes(const ctp_plan *P);
int batch_class_kind(const ctp_plan *P, int c);  // kFactor*
int batch_class_G(const ctp_plan *P, int c);
size_t batch_total(const ctp_plan *P);
cudaError_t batch_prepare(const ctp_plan *P, char *w, cudaStream_t st);
cudaError_t batch_compress(const ctp_plan *P, const ctp_front *fr, char *w, int num_sms, cudaStream_t st);
cudaError_t batch_factor_class(const ctp_plan *P, int ci, const ctp_front *fr, char *w, cudaStream_t st);
cudaError_t batch_solve(const ctp_plan *P, const ctp_front *fr, char *w, int num_sms, cudaStream_t st);
bool batch_solve_per_class(const ctp_plan *P);
cudaError_t batch_solve_class(const ctp_plan *P, int ci, const ctp_front *fr, char *w, cudaStream_t st);
cudaError_t batch_form_class(const ctp_plan *P, int ci, const ctp_front *fr, char *w, int num_sms, cudaStream_t st);
cudaError_t batch_form(const ctp_plan *P, const ctp_front *fr, char *w, int num_sms, cudaStream_t st);

// Tensor-core Solve (solve_tc.cu): BF16 pieces of its operands, its scratch
// bytes, and the launch sequence (prep of Z^T, gather of x_e, the GEMM with its
// epilogue).  Its outputs are stored factors, so it always takes three pieces
// (products close to FP32, whatever the Form's pieces): with two, a chain of
// fronts whose every Solve and Form was split in two stopped refining at 2e-13.
inline int solve_tc_pieces(int) { return 3; }
// the tensor-core Solve runs when asked for and the Form runs on the tensor cores
inline bool solve_on_tc(const ctp_options *o) {
    return o->solve == CTP_SOLVE_TC && o->prec != CTP_FP64 && o->smode != CTP_S_NONE && o->pivot != CTP_PIV_TPP;
}
size_t solve_tc_ws_bytes(int64_t m, int p, int spieces);
cudaError_t launch_solve_tc(double *A, int64_t n, int p, int64_t lda, const int32_t *perm, const int32_t *piv,
                            const double *Dinv, const int32_t *nelim, void *ws, int spieces, void *Wb, void *Lb,
                            int64_t foff, int fpieces, int32_t *info, int num_sms, cudaStream_t st);

// Batched tensor-core Solve: x_e and Z^T of every front in 128 x 64 BF16 tiles
// (three pieces each), GEMM items (front, 128-row block, output window).
size_t solve_tc_tile_elems();  // elements of one tile
int solve_tc_windows(int p);   // output windows of a front of width p, at most
cudaError_t launch_solve_tc_batch(const ctp_front *fronts, const BFront *tab, char *ws, const int *sitem,
                                  int64_t s_items, const int *qitem, int64_t q_items, const int *ritem,
                                  int64_t r_items, BatchOpts o,
                                  void *Xt, void *Zt, int64_t nxt, int64_t nzt, void *Wb, void *Lb,
                                  int32_t *ginfo, int num_sms, cudaStream_t st);

cudaError_t launch_solve_fp64(double *A, int64_t n, int p, int64_t lda, const int32_t *perm,
                              const int32_t *piv, const double *Dinv, const int32_t *nelim,
                              double *W21, int64_t ldw, void *Wb, void *Lb, int Kp, int64_t lo_off,
                              int pieces, cudaStream_t st);

// Threshold partial pivoting on all n rows (the comparator of the compressed path).
size_t tpp_ws_bytes(int p);
// spin: polls a grid barrier waits before it reports CTP_ETIMEOUT (0: the default)
cudaError_t launch_tpp(double *A, int64_t n, int p, int64_t lda, double u, double small, void *ws,
                       int32_t *perm, int32_t *piv, double *D, double *Dinv, int32_t *nelim,
                       int32_t *info, int num_sms, int spin, cudaStream_t st);

// K-padding of the BF16 operand copies used by the tensor-core Form.
int form_tc_kpad(int p);
// pieces: BF16 pieces per operand (1 plain, 2 or 3 split), piece_off elements apart.
cudaError_t launch_form_tc(const void *Wb, const void *Lb, int64_t piece_off, int pieces, int64_t m, int Kp,
                           const int32_t *nelim, float *S, int64_t lds,
                           int layout /* 0 full, 1 packed, 2 tiled, 3 subtract from FP64 */,
                           int32_t *info, int num_sms, int walk /* ctp_walk */, cudaStream_t st);

cudaError_t launch_form_fp64(const double *L21, int64_t ldl, const double *W21, int64_t ldw,
                             int64_t m, const int32_t *nelim, void *S, int64_t lds, int smode,
                             cudaStream_t st);

// Complete systems: front-list solve, residual, backward error (system.cu).
size_t sys_solve_ws_bytes(int64_t nmax, int nrhs);
cudaError_t launch_sys_forward(const ctp_sfront &f, double *X, int64_t ldx, int nrhs, void *ws,
                               cudaStream_t st);
cudaError_t launch_sys_backward(const ctp_sfront &f, double *X, int64_t ldx, int nrhs, void *ws,
                                cudaStream_t st);
cudaError_t launch_symv_residual(int64_t N, const double *M, int64_t ldm, int nrhs, const double *X,
                                 int64_t ldx, double *R, int64_t ldr, cudaStream_t st);
cudaError_t launch_abs_rowsum(int64_t N, const double *M, int64_t ldm, double *rowsum,
                              cudaStream_t st);
cudaError_t launch_backward_error(int64_t N, int nrhs, const double *R, int64_t ldr, const double *X,
                                  int64_t ldx, const double *B, int64_t ldb, const double *rowsum,
                                  double *mx, double *berr, cudaStream_t st);
cudaError_t launch_axpy(int64_t N, int nrhs, double *X, int64_t ldx, const double *Dx, int64_t ldd,
                        cudaStream_t st);
cudaError_t launch_sym_grad_dense(int64_t N, int nrhs, const double *G, int64_t ldg, const double *X,
                                  int64_t ldx, double *out, int64_t ldo, cudaStream_t st);
cudaError_t launch_sym_grad_pattern(int64_t nnz, const int32_t *row, const int32_t *col, int nrhs,
                                    const double *G, int64_t ldg, const double *X, int64_t ldx,
                                    double *out, cudaStream_t st);
cudaError_t launch_spmv_csc_residual(int64_t N, const int64_t *colptr, const int32_t *rowind,
                                     const double *val, int nrhs, const double *X, int64_t ldx, double *R,
                                     int64_t ldr, cudaStream_t st);
cudaError_t launch_spmv_csc_abs_rowsum(int64_t N, const int64_t *colptr, const int32_t *rowind,
                                       const double *val, double *rowsum, cudaStream_t st);
cudaError_t launch_w21_from_l(const double *A, int64_t lda, int p, int64_t m, const int32_t *piv,
                              const double *D, const int32_t *nelim, double *W21, int64_t ldw,
                              cudaStream_t st);

}  // namespace ctp
