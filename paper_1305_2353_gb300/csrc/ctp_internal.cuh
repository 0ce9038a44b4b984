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
    size_t info, C, Dinv, W21, Wb, Lb, aux, total;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

WsLayout ws_layout(int64_t n, int p, const ctp_options *opt, int num_sms);

// ---------------------------------------------------------------------------
// kernel launchers (each returns cudaError_t of the launch)
cudaError_t launch_compress_strict(const double *A21, int64_t m, int p, int64_t lda,
                                   unsigned long long *Ckeys, int32_t *J, int32_t *info,
                                   int num_sms, cudaStream_t st);
int relaxed_segments(int64_t m, int p, int num_sms);
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
    double u, small;
    int32_t *perm, *piv, *nelim;
    double *D, *Dinv;
    int32_t *info;
};
cudaError_t launch_factor_cluster(const FactorArgs &a, cudaStream_t st);

cudaError_t launch_solve_fp64(double *A, int64_t n, int p, int64_t lda, const int32_t *perm,
                              const int32_t *piv, const double *Dinv, const int32_t *nelim,
                              double *W21, int64_t ldw, void *Wb, void *Lb, int Kp,
                              cudaStream_t st);

// Threshold partial pivoting on all n rows (the comparator of the compressed path).
size_t tpp_ws_bytes(int p);
cudaError_t launch_tpp(double *A, int64_t n, int p, int64_t lda, double u, double small, void *ws,
                       int32_t *perm, int32_t *piv, double *D, double *Dinv, int32_t *nelim,
                       int32_t *info, int num_sms, cudaStream_t st);

// K-padding of the BF16 operand copies used by the tensor-core Form.
int form_tc_kpad(int p);
cudaError_t launch_form_tc(const void *Wb, const void *Lb, int64_t m, int Kp, const int32_t *nelim,
                           float *S, int64_t lds, int layout /* 0 full, 1 packed, 2 tiled */,
                           int32_t *info, int num_sms, cudaStream_t st);

cudaError_t launch_form_fp64(const double *L21, int64_t ldl, const double *W21, int64_t ldw,
                             int64_t m, const int32_t *nelim, void *S, int64_t lds, int smode,
                             cudaStream_t st);

}  // namespace ctp
