"""Thin Python binding of libctp (the C ABI declared in include/ctp.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of libctp.so.  PyTorch provides device memory and streams.  There is
no fallback: if the library is missing, ``load()`` raises.

Matrices cross the boundary column-major.  A column-major n x p device matrix
with leading dimension lda is held here as a torch tensor of shape (p, lda)
(row j of the tensor is column j of the matrix); ``colmajor()`` and
``to_numpy()`` convert.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libctp.so")

CTP_OK, CTP_EINVAL, CTP_ENOMEM, CTP_ECUDA, CTP_ENONFINITE, CTP_ETIMEOUT, CTP_ECAPACITY, \
    CTP_EUNSUPPORTED = range(8)
STATUS = {0: "CTP_OK", 1: "CTP_EINVAL", 2: "CTP_ENOMEM", 3: "CTP_ECUDA", 4: "CTP_ENONFINITE",
          5: "CTP_ETIMEOUT", 6: "CTP_ECAPACITY", 7: "CTP_EUNSUPPORTED"}
PIVOT = {"strict": 0, "relaxed": 1, "tpp": 2, "restricted": 3, "single_row": 4}
PREC = {"fp64": 0, "bf16": 1, "bf16x3": 2, "bf16x6": 3}
SOLVE = {"fp64": 0, "tc": 1}
SMODE = {"none": 0, "fp64": 1, "fp32": 2, "fp64_packed": 3, "fp32_packed": 4, "fp32_tiled": 5,
         "fp64_sub": 6}
PIV_1X1, PIV_2X2_FIRST, PIV_2X2_SECOND, PIV_ZERO, PIV_DELAYED = 1, 2, 0, -1, 3

EXPORTS = ["ctp_max_p", "ctp_create", "ctp_destroy", "ctp_workspace_size", "ctp_compress_strict",
           "ctp_compress_strict_noalloc", "ctp_compress_relaxed", "ctp_factor_supernode",
           "ctp_read_info", "ctp_profile_begin", "ctp_profile_end", "ctp_batch_plan_create",
           "ctp_batch_plan_destroy", "ctp_batch_upload", "ctp_factor_batch", "ctp_batch_read_info",
           "ctp_solve_workspace_size", "ctp_solve", "ctp_refine_workspace_size",
           "ctp_backward_error", "ctp_refine", "ctp_factor_dense", "ctp_chain_fronts",
           "ctp_chain_info", "ctp_chain_destroy", "ctp_tune_set", "ctp_tune_get",
           "ctp_autotune_batch", "ctp_autotune_supernode", "ctp_adjoint_solve",
           "ctp_sym_grad_dense", "ctp_sym_grad_pattern", "ctp_backward_error_csc", "ctp_refine_csc",
           "ctp_mf_analyse", "ctp_mf_factor", "ctp_mf_fronts", "ctp_mf_info", "ctp_mf_destroy",
           "ctp_mf_panel_info", "ctp_mf_solve_workspace_size", "ctp_mf_solve",
           "ctp_mf_refine_workspace_size", "ctp_mf_refine", "ctp_mf_adjoint_solve",
           "ctp_compress_strict_merge", "ctp_relaxed_candidates_size", "ctp_compress_relaxed_candidates",
           "ctp_compress_relaxed_select", "ctp_gather_rows"]
TUNE_FORM_WALK, TUNE_BATCH_SMEM_KB, TUNE_FACTOR_G, TUNE_TPP_SPIN = 0, 1, 2, 3
WALK = {"auto": 0, "round_robin": 1, "chunks": 2, "panels": 3}


class Options(ctypes.Structure):
    _fields_ = [("u", ctypes.c_double), ("small", ctypes.c_double), ("pivot", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("smode", ctypes.c_int32), ("solve", ctypes.c_int32)]


def options(u=0.01, small=1e-20, pivot="strict", prec="fp64", smode="none", solve="fp64"):
    return Options(u, small, PIVOT[pivot], PREC[prec], SMODE[smode], SOLVE[solve])


class Front(ctypes.Structure):
    """Mirror of ctp_front (device-visible descriptor of one front)."""
    _fields_ = [("n", ctypes.c_int64), ("p", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("perm", ctypes.c_void_p),
                ("piv", ctypes.c_void_p), ("D", ctypes.c_void_p), ("nelim", ctypes.c_void_p),
                ("S", ctypes.c_void_p), ("lds", ctypes.c_int64)]


class SFront(ctypes.Structure):
    """Mirror of ctp_sfront (one front of a factored system)."""
    _fields_ = [("n", ctypes.c_int64), ("p", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("L", ctypes.c_void_p), ("ldl", ctypes.c_int64), ("perm", ctypes.c_void_p),
                ("piv", ctypes.c_void_p), ("D", ctypes.c_void_p), ("nelim", ctypes.c_void_p),
                ("rows", ctypes.c_void_p)]


class CtpError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} returned {STATUS.get(code, code)}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libctp.so (built by ``paper_1305_2353_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libctp.so not found at {path}: run __graft_entry__.build() first")
    L = ctypes.CDLL(path)
    i32, i64, sz, P = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
    L.ctp_max_p.restype = i32
    L.ctp_max_p.argtypes = []
    L.ctp_create.argtypes = [ctypes.POINTER(P), i32]
    L.ctp_destroy.argtypes = [P]
    L.ctp_workspace_size.argtypes = [P, i64, i32, ctypes.POINTER(Options), ctypes.POINTER(sz)]
    L.ctp_compress_strict.argtypes = [P, i64, i32, P, i64, P, P, P, sz, P]
    L.ctp_compress_relaxed.argtypes = [P, i64, i32, P, i64, P, P, P, sz, P]
    L.ctp_compress_strict_noalloc.argtypes = [i64, i32, P, i64, P, P, ctypes.POINTER(i32), P]
    L.ctp_factor_supernode.argtypes = [P, i64, i32, P, i64, ctypes.POINTER(Options), P, P, P, P, P,
                                       i64, P, sz, P]
    L.ctp_read_info.argtypes = [P, P, ctypes.POINTER(i32), P]
    L.ctp_batch_plan_create.argtypes = [P, i32, P, P, ctypes.POINTER(Options), ctypes.POINTER(P),
                                        ctypes.POINTER(sz)]
    L.ctp_batch_plan_destroy.argtypes = [P]
    L.ctp_batch_upload.argtypes = [P, P, P, sz, P]
    L.ctp_factor_batch.argtypes = [P, P, P, P, sz, P]
    L.ctp_batch_read_info.argtypes = [P, P, P, P, P]
    L.ctp_solve_workspace_size.argtypes = [i64, i32, ctypes.POINTER(sz)]
    L.ctp_solve.argtypes = [P, i32, P, i64, i32, P, i64, P, sz, P]
    L.ctp_refine_workspace_size.argtypes = [i64, i64, i32, ctypes.POINTER(sz)]
    L.ctp_backward_error.argtypes = [P, i64, P, i64, i32, P, i64, P, i64, P, P, sz, P]
    L.ctp_refine.argtypes = [P, i32, P, i64, P, i64, i32, P, i64, P, i64, i32, ctypes.c_double,
                             P, ctypes.POINTER(i32), P, sz, P]
    L.ctp_factor_dense.argtypes = [P, i64, P, i64, i32, ctypes.POINTER(Options), i32,
                                   ctypes.POINTER(Options), ctypes.POINTER(P), P]
    L.ctp_chain_fronts.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(P)]
    L.ctp_chain_info.argtypes = [P, i32, P, P, P]
    L.ctp_chain_destroy.argtypes = [P]
    L.ctp_adjoint_solve.argtypes = [P, i32, P, i64, i32, P, i64, P, sz, P]
    L.ctp_sym_grad_dense.argtypes = [P, i64, i32, P, i64, P, i64, P, i64, P]
    L.ctp_sym_grad_pattern.argtypes = [P, i64, P, P, i64, i32, P, i64, P, i64, P, P]
    L.ctp_backward_error_csc.argtypes = [P, i64, P, P, P, i32, P, i64, P, i64, P, P, sz, P]
    L.ctp_refine_csc.argtypes = [P, i32, P, i64, P, P, P, i32, P, i64, P, i64, i32, ctypes.c_double,
                                 P, ctypes.POINTER(i32), P, sz, P]
    L.ctp_mf_analyse.argtypes = [P, i64, P, P, P, i32, P, ctypes.POINTER(P)]
    L.ctp_mf_factor.argtypes = [P, P, P, ctypes.POINTER(Options), P]
    L.ctp_mf_fronts.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(P)]
    L.ctp_mf_info.argtypes = [P, i32, ctypes.POINTER(i32), P, P, P, P, P]
    L.ctp_mf_destroy.argtypes = [P]
    L.ctp_mf_panel_info.argtypes = [P, i32, P, P, P, P]
    L.ctp_mf_solve_workspace_size.argtypes = [P, i32, ctypes.POINTER(sz)]
    L.ctp_mf_solve.argtypes = [P, P, i32, P, i64, P, sz, P]
    L.ctp_mf_refine_workspace_size.argtypes = [P, i32, ctypes.POINTER(sz)]
    L.ctp_mf_adjoint_solve.argtypes = [P, P, i32, P, i64, P, sz, P]
    L.ctp_mf_refine.argtypes = [P, P, P, P, P, i32, P, i64, P, i64, i32, ctypes.c_double, P,
                                ctypes.POINTER(i32), P, sz, P]
    L.ctp_tune_set.argtypes = [P, i32, i32]
    L.ctp_tune_get.argtypes = [P, i32, ctypes.POINTER(i32)]
    L.ctp_autotune_batch.argtypes = [P, i32, P, P, ctypes.POINTER(Options), P, P, i32, P, i32, P, P,
                                     ctypes.POINTER(i32), P]
    L.ctp_autotune_supernode.argtypes = [P, i64, i32, P, i64, ctypes.POINTER(Options), P, P, P, P,
                                         P, i64, P, sz, i32, P, i32, P, P, ctypes.POINTER(i32), P]
    L.ctp_compress_strict_merge.argtypes = [P, i32, i32, P, i64, P, P]
    L.ctp_relaxed_candidates_size.argtypes = [i32, i32, ctypes.POINTER(sz)]
    L.ctp_compress_relaxed_candidates.argtypes = [P, i64, i32, P, i64, i64, i32, i32, P, sz, P]
    L.ctp_compress_relaxed_select.argtypes = [P, i32, i32, P, sz, P, P]
    L.ctp_gather_rows.argtypes = [P, i32, P, i64, P, P, P]
    L.ctp_profile_begin.argtypes = [P]
    L.ctp_profile_end.argtypes = [P, i32, P, P, P, ctypes.POINTER(i32)]
    for f in EXPORTS[1:]:
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _check(fn, code):
    if code != CTP_OK:
        raise CtpError(fn, code)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """A libctp context bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        _check("ctp_create", self.lib.ctp_create(ctypes.byref(h), device))
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            self.lib.ctp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_size(self, n, p, opt):
        b = ctypes.c_size_t()
        _check("ctp_workspace_size",
               self.lib.ctp_workspace_size(self.handle, n, p, ctypes.byref(opt), ctypes.byref(b)))
        return int(b.value)

    def workspace(self, n, p, opt):
        import torch
        nbytes = self.workspace_size(n, p, opt)
        return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=f"cuda:{self.device}")

    def compress_strict(self, A21, m, p, lda, C, J=None, ws=None, stream=None):
        """A21: device tensor holding the m x p column-major A21 (leading dim lda);
        C: device float64 tensor of p*p (row-major output); J: int32[m] or None."""
        if ws is None:
            ws = self.workspace(m + p, p, options())
        _check("ctp_compress_strict",
               self.lib.ctp_compress_strict(self.handle, m, p, _ptr(A21), lda, _ptr(C), _ptr(J),
                                            _ptr(ws), ws.numel(), _stream(stream)))
        return ws

    def compress_relaxed(self, A21, m, p, lda, C, rows=None, ws=None, stream=None):
        """A21: m x p column-major device matrix; C: float64[p*p] (row-major
        output); rows: int32[p] or None."""
        if ws is None:
            ws = self.workspace(m + p, p, options(pivot="relaxed"))
        _check("ctp_compress_relaxed",
               self.lib.ctp_compress_relaxed(self.handle, m, p, _ptr(A21), lda, _ptr(C), _ptr(rows),
                                             _ptr(ws), ws.numel(), _stream(stream)))
        return ws

    def factor_supernode(self, A, n, p, lda, opt, perm, piv, D, nelim, S=None, lds=0, ws=None,
                         stream=None):
        if ws is None:
            ws = self.workspace(n, p, opt)
        _check("ctp_factor_supernode",
               self.lib.ctp_factor_supernode(self.handle, n, p, _ptr(A), lda, ctypes.byref(opt),
                                             _ptr(perm), _ptr(piv), _ptr(D), _ptr(nelim), _ptr(S),
                                             lds, _ptr(ws), ws.numel(), _stream(stream)))
        return ws

    def compress_strict_merge(self, P, p, C_blocks, block_stride, C, stream=None):
        """C = elementwise max of P stacked strict compressed matrices (the
        exchange of the row split, Section 6)."""
        _check("ctp_compress_strict_merge", self.lib.ctp_compress_strict_merge(
            self.handle, P, p, _ptr(C_blocks), block_stride, _ptr(C), _stream(stream)))

    def relaxed_candidates_buffer(self, P, p):
        import torch
        b = ctypes.c_size_t()
        _check("ctp_relaxed_candidates_size", self.lib.ctp_relaxed_candidates_size(P, p, ctypes.byref(b)))
        return torch.zeros(int(b.value), dtype=torch.uint8, device=f"cuda:{self.device}")

    def compress_relaxed_candidates(self, A21_block, m, p, lda, row0, P, block, cand, stream=None):
        """Candidate lists of one row block (rows row0.. of A21) into slot `block`."""
        _check("ctp_compress_relaxed_candidates", self.lib.ctp_compress_relaxed_candidates(
            self.handle, m, p, _ptr(A21_block), lda, row0, P, block, _ptr(cand), cand.numel(), _stream(stream)))

    def compress_relaxed_select(self, P, p, cand, rows, stream=None):
        _check("ctp_compress_relaxed_select", self.lib.ctp_compress_relaxed_select(
            self.handle, P, p, _ptr(cand), cand.numel(), _ptr(rows), _stream(stream)))

    def gather_rows(self, p, A21, lda, rows, C, stream=None):
        _check("ctp_gather_rows", self.lib.ctp_gather_rows(
            self.handle, p, _ptr(A21), lda, _ptr(rows), _ptr(C), _stream(stream)))

    def tune_set(self, key, value):
        _check("ctp_tune_set", self.lib.ctp_tune_set(self.handle, key, value))

    def tune_get(self, key):
        v = ctypes.c_int32()
        _check("ctp_tune_get", self.lib.ctp_tune_get(self.handle, key, ctypes.byref(v)))
        return int(v.value)

    def profile_begin(self):
        _check("ctp_profile_begin", self.lib.ctp_profile_begin(self.handle))

    def profile_end(self):
        """{kernel name: (launches, total device ms)} since profile_begin()."""
        k = 32
        names = ctypes.create_string_buffer(48 * k)
        tot = (ctypes.c_double * k)()
        cnt = (ctypes.c_int32 * k)()
        nk = ctypes.c_int32()
        _check("ctp_profile_end", self.lib.ctp_profile_end(self.handle, k, names, tot, cnt,
                                                            ctypes.byref(nk)))
        out = {}
        for i in range(min(nk.value, k)):
            nm = names.raw[48 * i:48 * i + 48].split(b"\0", 1)[0].decode()
            out[nm] = (int(cnt[i]), float(tot[i]))
        return out

    def read_info(self, ws, stream=None):
        v = ctypes.c_int32()
        _check("ctp_read_info", self.lib.ctp_read_info(self.handle, _ptr(ws), ctypes.byref(v),
                                                        _stream(stream)))
        return int(v.value)


def compress_strict_noalloc(A21, m, p, lda, C, J=None, stream=None):
    """Strict compression with the library's own fixed scratch (no workspace, no
    device allocation) on the current device; returns the device info word.
    For callers that cannot allocate device memory at the call site; calls that
    overlap on the GPU race on the shared scratch."""
    L = load()
    info = ctypes.c_int32(-1)
    _check("ctp_compress_strict_noalloc",
           L.ctp_compress_strict_noalloc(m, p, _ptr(A21), lda, _ptr(C), _ptr(J), ctypes.byref(info),
                                         _stream(stream)))
    return int(info.value)


# ---------------------------------------------------------------------------
# layout helpers (no arithmetic)

class _CudaArray:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2}


def device_view(ptr, n, dtype="int32"):
    """A torch tensor viewing n elements of library-owned device memory (no copy)."""
    import torch
    ts = {"int32": "<i4", "float64": "<f8"}[dtype]
    return torch.as_tensor(_CudaArray(ptr, n, ts), device="cuda")


def colmajor(a: np.ndarray, device="cuda"):
    """numpy (rows x cols) -> device tensor (cols, rows) holding it column-major."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).to(device)


def to_numpy(t) -> np.ndarray:
    """Inverse of ``colmajor``."""
    return t.detach().cpu().numpy().T.copy()


def unpack_lower(packed: np.ndarray, m: int) -> np.ndarray:
    """Lower-packed-by-columns vector -> m x m matrix (upper triangle zero)."""
    S = np.zeros((m, m), dtype=packed.dtype)
    off = 0
    for j in range(m):
        S[j:, j] = packed[off:off + m - j]
        off += m - j
    return S


def unpack_tiled(blocks: np.ndarray, m: int) -> np.ndarray:
    """128 x 128 block layout (lower block triangle, blocks column-major inside)
    -> m x m matrix holding the lower triangle (strict upper part zeroed)."""
    nb = (m + 127) // 128
    S = np.zeros((nb * 128, nb * 128), dtype=blocks.dtype)
    k = 0
    for bj in range(nb):
        for bi in range(bj, nb):
            S[bi * 128:(bi + 1) * 128, bj * 128:(bj + 1) * 128] = \
                blocks[k * 16384:(k + 1) * 16384].reshape(128, 128).T
            k += 1
    return np.tril(S[:m, :m])


class Supernode:
    """Device buffers for one factorization of an n x p supernode."""

    def __init__(self, ctx: Context, A_host: np.ndarray, p: int, opt, s_dtype=None):
        import torch
        self.ctx = ctx
        self.n, self.p = A_host.shape[0], p
        dev = f"cuda:{ctx.device}"
        self.A = colmajor(A_host, dev)
        self.perm = torch.empty(p, dtype=torch.int32, device=dev)
        self.piv = torch.empty(p, dtype=torch.int32, device=dev)
        self.D = torch.empty(2 * p, dtype=torch.float64, device=dev)
        self.nelim = torch.empty(1, dtype=torch.int32, device=dev)
        m = self.n - p
        self.S = None
        if opt.smode != 0:
            dt = torch.float64 if opt.smode in (1, 3, 6) else torch.float32
            if opt.smode in (3, 4):
                self.S = torch.zeros(max(m * (m + 1) // 2, 1), dtype=dt, device=dev)  # packed
            elif opt.smode == 5:
                nb = (m + 127) // 128
                self.S = torch.zeros(max(nb * (nb + 1) // 2 * 16384, 1), dtype=dt, device=dev)
            else:
                self.S = torch.zeros((m, m), dtype=dt, device=dev)  # column-major m x m
        self.opt = opt
        self.ws = ctx.workspace(self.n, p, opt)

    def run(self, stream=None):
        self.ctx.factor_supernode(self.A, self.n, self.p, self.n, self.opt, self.perm, self.piv,
                                  self.D, self.nelim, self.S, max(self.n - self.p, 1), self.ws,
                                  stream)

    def result(self):
        out = dict(A=to_numpy(self.A), perm=self.perm.cpu().numpy(), piv=self.piv.cpu().numpy(),
                   D=self.D.cpu().numpy(), nelim=int(self.nelim.cpu()[0]))
        if self.S is not None:
            if self.opt.smode in (3, 4):
                out["S"] = unpack_lower(self.S.cpu().numpy(), self.n - self.p)
            elif self.opt.smode == 5:
                out["S"] = unpack_tiled(self.S.cpu().numpy(), self.n - self.p)
            else:
                out["S"] = to_numpy(self.S)
        out["info"] = self.ctx.read_info(self.ws)
        return out


class Chain:
    """Factors of a dense symmetric system (``ctp_factor_dense``): a chain of
    fronts, the first being the supernode [A11; A21]."""

    def __init__(self, ctx: Context, handle):
        self.ctx, self.handle = ctx, handle
        L = ctx.lib
        nf = ctypes.c_int32()
        arr = ctypes.c_void_p()
        _check("ctp_chain_fronts", L.ctp_chain_fronts(handle, ctypes.byref(nf), ctypes.byref(arr)))
        self.nf = int(nf.value)
        self.fronts = ctypes.cast(arr, ctypes.POINTER(SFront))
        e = np.zeros(self.nf, np.int32)
        p = np.zeros(self.nf, np.int32)
        piv = np.zeros(self.nf, np.int32)
        _check("ctp_chain_info", L.ctp_chain_info(handle, self.nf, e.ctypes.data, p.ctypes.data,
                                                  piv.ctypes.data))
        self.nelim, self.p, self.pivot = e, p, piv

    def destroy(self):
        if self.handle:
            self.ctx.lib.ctp_chain_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def factor_dense(ctx: Context, M, N, ldm, p_first, opt_first, w_rest, opt_rest, stream=None):
    """Factor the dense symmetric matrix M (device tensor holding it column-major,
    lower triangle read) in place as a chain of fronts; returns a ``Chain``."""
    h = ctypes.c_void_p()
    _check("ctp_factor_dense",
           ctx.lib.ctp_factor_dense(ctx.handle, N, _ptr(M), ldm, p_first, ctypes.byref(opt_first),
                                    w_rest, ctypes.byref(opt_rest), ctypes.byref(h),
                                    _stream(stream)))
    return Chain(ctx, h)


def autotune_supernode(ctx: Context, A, n, p, lda, opt, perm, piv, D, nelim, S, lds, ws, keys,
                       candidates, stream=None):
    """The library's autotuner over candidate settings of the knobs `keys` for
    one supernode factorization (inputs restored afterwards).  Returns
    (per-candidate ms, chosen index)."""
    k = np.array(keys, np.int32)
    v = np.array(candidates, np.int32).reshape(len(candidates), len(keys))
    ms = np.zeros(len(v))
    best = ctypes.c_int32(-1)
    _check("ctp_autotune_supernode", ctx.lib.ctp_autotune_supernode(
        ctx.handle, n, p, _ptr(A), lda, ctypes.byref(opt), _ptr(perm), _ptr(piv), _ptr(D),
        _ptr(nelim), _ptr(S), lds, _ptr(ws), ws.numel(), len(k), k.ctypes.data_as(ctypes.c_void_p),
        len(v), v.ctypes.data_as(ctypes.c_void_p), ms.ctypes.data_as(ctypes.c_void_p),
        ctypes.byref(best), _stream(stream)))
    return ms, int(best.value)


def solve_workspace(ctx: Context, nmax, nrhs):
    import torch
    b = ctypes.c_size_t()
    _check("ctp_solve_workspace_size", ctx.lib.ctp_solve_workspace_size(nmax, nrhs, ctypes.byref(b)))
    return torch.empty(max(b.value, 1), dtype=torch.uint8, device=f"cuda:{ctx.device}")


def refine_workspace(ctx: Context, N, nmax, nrhs):
    import torch
    b = ctypes.c_size_t()
    _check("ctp_refine_workspace_size",
           ctx.lib.ctp_refine_workspace_size(N, nmax, nrhs, ctypes.byref(b)))
    return torch.empty(max(b.value, 1), dtype=torch.uint8, device=f"cuda:{ctx.device}")


def solve(ctx: Context, fronts, nf, N, nrhs, X, ldx, ws, stream=None):
    """X <- M^{-1} X (device tensor, column-major N x nrhs) with the fronts' factors."""
    _check("ctp_solve", ctx.lib.ctp_solve(ctx.handle, nf, ctypes.cast(fronts, ctypes.c_void_p), N,
                                          nrhs, _ptr(X), ldx, _ptr(ws), ws.numel(), _stream(stream)))


def adjoint_solve(ctx: Context, fronts, nf, N, nrhs, G, ldg, ws, stream=None):
    """G <- M^{-T} G with the same factors (M symmetric: the same solve)."""
    _check("ctp_adjoint_solve", ctx.lib.ctp_adjoint_solve(
        ctx.handle, nf, ctypes.cast(fronts, ctypes.c_void_p), N, nrhs, _ptr(G), ldg, _ptr(ws),
        ws.numel(), _stream(stream)))


def sym_grad_dense(ctx: Context, N, nrhs, Gb, ldg, X, ldx, out, ldo, stream=None):
    """Lower triangle of out (column-major) <- gradient with respect to the
    stored lower triangle of M, from Gb = M^{-T} dloss/dX and X."""
    _check("ctp_sym_grad_dense", ctx.lib.ctp_sym_grad_dense(
        ctx.handle, N, nrhs, _ptr(Gb), ldg, _ptr(X), ldx, _ptr(out), ldo, _stream(stream)))


def sym_grad_pattern(ctx: Context, row, col, N, nrhs, Gb, ldg, X, ldx, out, stream=None):
    """out[k] <- gradient with respect to the stored entry (row[k], col[k])."""
    _check("ctp_sym_grad_pattern", ctx.lib.ctp_sym_grad_pattern(
        ctx.handle, row.numel(), _ptr(row), _ptr(col), N, nrhs, _ptr(Gb), ldg, _ptr(X), ldx,
        _ptr(out), _stream(stream)))


_default_ctx = None


def default_context():
    global _default_ctx
    if _default_ctx is None:
        import torch
        _default_ctx = Context(torch.cuda.current_device())
    return _default_ctx


_SymSolve = None


def _sym_solve_fn():
    """torch.autograd.Function: X = M^{-1} B through the chain factorization
    (forward: factor + FP64 refinement; backward: the adjoint solve with the same
    factors, refined, and the gradient of the stored lower triangle of M)."""
    global _SymSolve
    if _SymSolve is not None:
        return _SymSolve
    import torch

    class SymSolve(torch.autograd.Function):
        @staticmethod
        def forward(fctx, A, B, ctx, p_first, opt_first, w_rest, opt_rest, steps, tol):
            N = A.shape[0]
            Mlow = A.detach().t().contiguous()   # column-major storage of the lower triangle
            Md = Mlow.clone()                    # factored in place
            ch = factor_dense(ctx, Md, N, N, min(p_first, N), opt_first, w_rest, opt_rest)
            Bt = B.detach().reshape(N, -1).t().contiguous()
            nrhs = Bt.shape[0]
            X = torch.zeros_like(Bt)
            ws = refine_workspace(ctx, N, N, nrhs)
            hist, k = refine(ctx, ch.fronts, ch.nf, N, Mlow, N, nrhs, Bt, N, X, N, ws, steps, tol)
            fctx.chain, fctx.Md, fctx.Mlow, fctx.ws = ch, Md, Mlow, ws
            fctx.steps, fctx.tol, fctx.ctx, fctx.bshape = steps, tol, ctx, B.shape
            fctx.history = hist
            fctx.save_for_backward(X)
            out = X.t().contiguous()
            return out.reshape(B.shape)

        @staticmethod
        def backward(fctx, gX):
            (X,) = fctx.saved_tensors
            ctx, ch, N = fctx.ctx, fctx.chain, X.shape[1]
            nrhs = X.shape[0]
            G = gX.reshape(N, -1).t().contiguous()
            Gb = torch.zeros_like(G)
            refine(ctx, ch.fronts, ch.nf, N, fctx.Mlow, N, nrhs, G, N, Gb, N, fctx.ws, fctx.steps,
                   fctx.tol)
            gA = None
            if fctx.needs_input_grad[0]:
                out = torch.empty((N, N), dtype=torch.float64, device=X.device)
                sym_grad_dense(ctx, N, nrhs, Gb, N, X, N, out, N)
                gA = out.t()
            gB = Gb.t().reshape(fctx.bshape) if fctx.needs_input_grad[1] else None
            return gA, gB, None, None, None, None, None, None, None

    _SymSolve = SymSolve
    return SymSolve


def sym_solve(A, B, ctx=None, pivot="strict", prec="fp64", p_first=256, w_rest=256,
              pivot_rest="tpp", steps=10, tol=1e-14):
    """Differentiable X = M^{-1} B for a symmetric indefinite M given by the lower
    triangle of the (N, N) float64 CUDA tensor A (the strict upper triangle is
    not read, and its gradient is zero); B is (N,) or (N, nrhs).  The first
    front (p_first columns) uses `pivot`/`prec`, the rest `pivot_rest` in FP64."""
    ctx = ctx or default_context()
    o1 = options(pivot=pivot, prec=prec)
    o2 = options(pivot=pivot_rest)
    return _sym_solve_fn().apply(A, B, ctx, p_first, o1, w_rest, o2, steps, tol)


def backward_error(ctx: Context, N, M, ldm, nrhs, B, ldb, X, ldx, berr, ws, stream=None):
    """Section 7 backward error per right-hand side into the device tensor berr."""
    _check("ctp_backward_error",
           ctx.lib.ctp_backward_error(ctx.handle, N, _ptr(M), ldm, nrhs, _ptr(B), ldb, _ptr(X), ldx,
                                      _ptr(berr), _ptr(ws), ws.numel(), _stream(stream)))


def refine(ctx: Context, fronts, nf, N, M, ldm, nrhs, B, ldb, X, ldx, ws, max_steps=10, tol=1e-14,
           stream=None):
    """Solve with iterative refinement; returns (history of backward errors as
    a (steps+1) x nrhs array, corrections made)."""
    hist = np.zeros((max_steps + 1) * nrhs)
    steps = ctypes.c_int32()
    _check("ctp_refine",
           ctx.lib.ctp_refine(ctx.handle, nf, ctypes.cast(fronts, ctypes.c_void_p), N, _ptr(M), ldm,
                              nrhs, _ptr(B), ldb, _ptr(X), ldx, max_steps, tol, hist.ctypes.data,
                              ctypes.byref(steps), _ptr(ws), ws.numel(), _stream(stream)))
    k = int(steps.value)
    return hist[:(k + 1) * nrhs].reshape(k + 1, nrhs), k


class Multifrontal:
    """A sparse symmetric matrix (lower triangle in compressed columns, host
    numpy arrays), analysed for an elimination order and its supernode blocks,
    factored multifrontally on the device (``ctp_mf_*``)."""

    def __init__(self, ctx: Context, colptr, rowind, val, perm, blocks):
        import torch
        self.ctx = ctx
        dev = f"cuda:{ctx.device}"
        self.N = len(colptr) - 1
        self.colptr = np.ascontiguousarray(colptr, np.int64)
        self.rowind = np.ascontiguousarray(rowind, np.int32)
        self.perm = np.ascontiguousarray(perm, np.int32)
        self.blocks = np.ascontiguousarray(blocks, np.int64)
        self.d_colptr = torch.from_numpy(self.colptr).to(dev)
        self.d_rowind = torch.from_numpy(self.rowind).to(dev)
        self.d_val = torch.from_numpy(np.ascontiguousarray(val, np.float64)).to(dev)
        h = ctypes.c_void_p()
        _check("ctp_mf_analyse", ctx.lib.ctp_mf_analyse(
            ctx.handle, self.N, self.colptr.ctypes.data_as(ctypes.c_void_p),
            self.rowind.ctypes.data_as(ctypes.c_void_p), self.perm.ctypes.data_as(ctypes.c_void_p),
            len(self.blocks) - 1, self.blocks.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
        self.handle = h
        self.nf = 0
        self.fronts = None

    def factor(self, opt, stream=None):
        _check("ctp_mf_factor", self.ctx.lib.ctp_mf_factor(
            self.ctx.handle, self.handle, _ptr(self.d_val), ctypes.byref(opt), _stream(stream)))
        nf = ctypes.c_int32()
        arr = ctypes.c_void_p()
        _check("ctp_mf_fronts", self.ctx.lib.ctp_mf_fronts(self.handle, ctypes.byref(nf),
                                                           ctypes.byref(arr)))
        self.nf = int(nf.value)
        self.fronts = ctypes.cast(arr, ctypes.POINTER(SFront))

    def info(self):
        nb = len(self.blocks) - 1
        par = np.zeros(nb, np.int32)
        n, p, e, d = (np.zeros(nb, np.int64) for _ in range(4))
        k = ctypes.c_int32()
        _check("ctp_mf_info", self.ctx.lib.ctp_mf_info(
            self.handle, nb, ctypes.byref(k), par.ctypes.data_as(ctypes.c_void_p),
            n.ctypes.data_as(ctypes.c_void_p), p.ctypes.data_as(ctypes.c_void_p),
            e.ctypes.data_as(ctypes.c_void_p), d.ctypes.data_as(ctypes.c_void_p)))
        return dict(parent=par, n=n, p=p, nelim=e, delayed=d)

    def panel_info(self):
        """Per panel: rows, columns, eliminated, block."""
        n = np.zeros(self.nf, np.int64)
        p = np.zeros(self.nf, np.int32)
        e = np.zeros(self.nf, np.int32)
        b = np.zeros(self.nf, np.int32)
        _check("ctp_mf_panel_info", self.ctx.lib.ctp_mf_panel_info(
            self.handle, self.nf, n.ctypes.data_as(ctypes.c_void_p), p.ctypes.data_as(ctypes.c_void_p),
            e.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p)))
        return n, p, e, b

    def panel_perms(self):
        return [device_view(self.fronts[k].perm, int(self.fronts[k].p), "int32").cpu().numpy()
                for k in range(self.nf)]

    def refine(self, B, X, ws, max_steps=10, tol=1e-14, stream=None, planned=True):
        """Solve with FP64 refinement against the sparse matrix (device B, X
        column-major N x nrhs tensors), by the level-planned solve (or, with
        planned=False, the generic front-list solve).  Returns (history,
        corrections)."""
        nrhs = B.shape[0]
        hist = np.zeros((max_steps + 1) * nrhs)
        steps = ctypes.c_int32()
        if planned:
            _check("ctp_mf_refine", self.ctx.lib.ctp_mf_refine(
                self.ctx.handle, self.handle, _ptr(self.d_colptr), _ptr(self.d_rowind), _ptr(self.d_val),
                nrhs, _ptr(B), self.N, _ptr(X), self.N, max_steps, tol, hist.ctypes.data,
                ctypes.byref(steps), _ptr(ws), ws.numel(), _stream(stream)))
        else:
            _check("ctp_refine_csc", self.ctx.lib.ctp_refine_csc(
                self.ctx.handle, self.nf, ctypes.cast(self.fronts, ctypes.c_void_p), self.N,
                _ptr(self.d_colptr), _ptr(self.d_rowind), _ptr(self.d_val), nrhs, _ptr(B), self.N,
                _ptr(X), self.N, max_steps, tol, hist.ctypes.data, ctypes.byref(steps), _ptr(ws),
                ws.numel(), _stream(stream)))
        k = int(steps.value)
        return hist[:(k + 1) * nrhs].reshape(k + 1, nrhs), k

    def refine_workspace(self, nrhs):
        import torch
        b1 = ctypes.c_size_t()
        _check("ctp_mf_refine_workspace_size",
               self.ctx.lib.ctp_mf_refine_workspace_size(self.handle, nrhs, ctypes.byref(b1)))
        b2 = ctypes.c_size_t()
        info = self.info()
        _check("ctp_refine_workspace_size",
               self.ctx.lib.ctp_refine_workspace_size(self.N, int(info["n"].max()), nrhs, ctypes.byref(b2)))
        return torch.empty(max(b1.value, b2.value, 1), dtype=torch.uint8, device=f"cuda:{self.ctx.device}")

    def solve(self, X, ws, stream=None):
        """X <- M^{-1} X by the level-planned solve (device, column-major)."""
        _check("ctp_mf_solve", self.ctx.lib.ctp_mf_solve(
            self.ctx.handle, self.handle, X.shape[0], _ptr(X), self.N, _ptr(ws), ws.numel(),
            _stream(stream)))

    def adjoint_solve(self, G, ws, stream=None):
        """G <- M^{-T} G with the same factors and pivots (device, column-major)."""
        _check("ctp_mf_adjoint_solve", self.ctx.lib.ctp_mf_adjoint_solve(
            self.ctx.handle, self.handle, G.shape[0], _ptr(G), self.N, _ptr(ws), ws.numel(),
            _stream(stream)))

    def set_values(self, val):
        """Replace the matrix values (same pattern) before the next factor."""
        self.d_val.copy_(val.reshape(-1))

    def pattern_device(self):
        """(row, col) int32 device arrays of the stored lower-triangle entries,
        in the pattern's order."""
        if getattr(self, "_d_row", None) is None:
            import torch
            dev = f"cuda:{self.ctx.device}"
            col = np.repeat(np.arange(self.N, dtype=np.int32), np.diff(self.colptr))
            self._d_row = torch.from_numpy(self.rowind).to(dev)
            self._d_col = torch.from_numpy(col).to(dev)
        return self._d_row, self._d_col

    def grad_values(self, Gb, X, out, stream=None):
        """Gradient with respect to the stored entries (pattern order) given
        Gb = M^{-T} dloss/dX and X (device, column-major N x nrhs)."""
        row, col = self.pattern_device()
        sym_grad_pattern(self.ctx, row, col, self.N, X.shape[0], Gb, self.N, X, self.N, out, stream)

    def destroy(self):
        if self.handle:
            self.ctx.lib.ctp_mf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class SparseSymSolver:
    """Differentiable solves X = M^{-1} B for a sparse symmetric indefinite M of
    a fixed pattern (lower triangle in compressed columns, host arrays), its
    elimination order and supernode blocks; the values are a float64 CUDA
    tensor in the pattern's order.  Calling the solver factors M
    multifrontally with `pivot`/`prec` and solves with FP64 refinement; the
    backward pass solves the adjoint system with the same factors (refined)
    and gives the gradient of the stored entries only (the sparsity pattern)."""

    def __init__(self, ctx: Context, colptr, rowind, perm, blocks, pivot="strict", prec="fp64",
                 steps=10, tol=1e-14):
        self.ctx = ctx
        self.mf = Multifrontal(ctx, colptr, rowind, np.zeros(len(rowind)), perm, blocks)
        self.opt = options(pivot=pivot, prec=prec)
        self.steps, self.tol = steps, tol
        self.version = 0          # bumped by every factorization
        self.history = None

    def _factor(self, val):
        self.mf.set_values(val.detach())
        self.mf.factor(self.opt)
        self.version += 1
        return self.version

    def __call__(self, val, B):
        return _sparse_sym_solve_fn().apply(val, B, self)


_SparseSymSolve = None


def _sparse_sym_solve_fn():
    global _SparseSymSolve
    if _SparseSymSolve is not None:
        return _SparseSymSolve
    import torch

    class SparseSymSolve(torch.autograd.Function):
        @staticmethod
        def forward(fctx, val, B, solver):
            mf = solver.mf
            N = mf.N
            version = solver._factor(val)
            Bt = B.detach().reshape(N, -1).t().contiguous()
            X = torch.zeros_like(Bt)
            ws = mf.refine_workspace(Bt.shape[0])
            solver.history, _ = mf.refine(Bt, X, ws, solver.steps, solver.tol)
            fctx.solver, fctx.version, fctx.bshape = solver, version, B.shape
            fctx.save_for_backward(val.detach().clone(), X)
            return X.t().contiguous().reshape(B.shape)

        @staticmethod
        def backward(fctx, gX):
            val, X = fctx.saved_tensors
            solver = fctx.solver
            mf = solver.mf
            N = mf.N
            if solver.version != fctx.version:        # factored again since: restore
                fctx.version = solver._factor(val)
            G = gX.reshape(N, -1).t().contiguous()
            Gb = torch.zeros_like(G)
            ws = mf.refine_workspace(G.shape[0])
            mf.refine(G, Gb, ws, solver.steps, solver.tol)     # M^{-T} = M^{-1}
            gval = None
            if fctx.needs_input_grad[0]:
                gval = torch.empty_like(val)
                mf.grad_values(Gb, X, gval)
            gB = Gb.t().reshape(fctx.bshape) if fctx.needs_input_grad[1] else None
            return gval, gB, None

    _SparseSymSolve = SparseSymSolve
    return SparseSymSolve


class Batch:
    """Device buffers and plan for the batched factorization of many fronts.
    All fronts live in a few pooled tensors; the descriptor array is built on
    the host and copied to the device once."""

    def __init__(self, ctx: Context, A_list, p_list, opt):
        import torch
        self.ctx, self.opt = ctx, opt
        dev = f"cuda:{ctx.device}"
        self.nb = len(A_list)
        self.n = np.array([a.shape[0] for a in A_list], np.int64)
        self.p = np.array(p_list, np.int32)
        m = self.n - self.p
        a_off = np.concatenate([[0], np.cumsum(self.n * self.p)])
        p_off = np.concatenate([[0], np.cumsum(self.p)])
        if opt.smode in (3, 4):
            s_len = m * (m + 1) // 2
        elif opt.smode == 5:
            nbk = (m + 127) // 128
            s_len = nbk * (nbk + 1) // 2 * 16384
        else:
            s_len = np.zeros(self.nb, np.int64)
        s_off = np.concatenate([[0], np.cumsum(s_len)])
        host = np.empty(int(a_off[-1]), np.float64)
        for k, a in enumerate(A_list):
            host[a_off[k]:a_off[k + 1]] = np.asarray(a, np.float64).ravel(order="F")
        self.A = torch.from_numpy(host).to(dev)
        self.perm = torch.empty(int(p_off[-1]), dtype=torch.int32, device=dev)
        self.piv = torch.empty(int(p_off[-1]), dtype=torch.int32, device=dev)
        self.D = torch.empty(2 * int(p_off[-1]), dtype=torch.float64, device=dev)
        self.nelim = torch.empty(self.nb, dtype=torch.int32, device=dev)
        sdt = torch.float64 if opt.smode == 3 else torch.float32
        self.S = torch.zeros(max(int(s_off[-1]), 1), dtype=sdt, device=dev) if opt.smode else None
        self.a_off, self.p_off, self.s_off = a_off, p_off, s_off
        fr = (Front * self.nb)()
        base = self.A.data_ptr()
        for k in range(self.nb):
            fr[k].n, fr[k].p = int(self.n[k]), int(self.p[k])
            fr[k].A = base + 8 * int(a_off[k])
            fr[k].lda = int(self.n[k])
            fr[k].perm = self.perm.data_ptr() + 4 * int(p_off[k])
            fr[k].piv = self.piv.data_ptr() + 4 * int(p_off[k])
            fr[k].D = self.D.data_ptr() + 8 * 2 * int(p_off[k])
            fr[k].nelim = self.nelim.data_ptr() + 4 * k
            fr[k].S = (self.S.data_ptr() + self.S.element_size() * int(s_off[k])) if self.S is not None else None
            fr[k].lds = max(int(m[k]), 1)
        raw = np.frombuffer(bytes(fr), dtype=np.uint8)
        self.fronts_host = fr
        self.fronts = torch.from_numpy(raw.copy()).to(dev)
        self.plan = None
        self.replan()
        self.A0 = self.A.clone()

    def replan(self):
        """(Re)create the plan with the context's current tuning knobs."""
        import torch
        if self.plan:
            self.ctx.lib.ctp_batch_plan_destroy(self.plan)
        plan = ctypes.c_void_p()
        wsb = ctypes.c_size_t()
        _check("ctp_batch_plan_create",
               self.ctx.lib.ctp_batch_plan_create(
                   self.ctx.handle, self.nb, self.n.ctypes.data_as(ctypes.c_void_p),
                   self.p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self.opt),
                   ctypes.byref(plan), ctypes.byref(wsb)))
        self.plan = plan
        self.ws = torch.empty(max(int(wsb.value), 256), dtype=torch.uint8,
                              device=f"cuda:{self.ctx.device}")
        _check("ctp_batch_upload", self.ctx.lib.ctp_batch_upload(
            self.ctx.handle, self.plan, _ptr(self.ws), self.ws.numel(), _stream(None)))

    def autotune(self, keys, candidates, stream=None):
        """Run the library's autotuner over candidate settings of the knobs
        `keys` (candidates: one tuple of values per candidate) on this batch's
        own inputs, keep the fastest in the context and re-plan.  Returns
        (per-candidate ms, chosen index)."""
        k = np.array(keys, np.int32)
        v = np.array(candidates, np.int32).reshape(len(candidates), len(keys))
        ms = np.zeros(len(v))
        best = ctypes.c_int32(-1)
        _check("ctp_autotune_batch", self.ctx.lib.ctp_autotune_batch(
            self.ctx.handle, self.nb, self.n.ctypes.data_as(ctypes.c_void_p),
            self.p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self.opt),
            ctypes.cast(self.fronts_host, ctypes.c_void_p), _ptr(self.fronts), len(k),
            k.ctypes.data_as(ctypes.c_void_p), len(v), v.ctypes.data_as(ctypes.c_void_p),
            ms.ctypes.data_as(ctypes.c_void_p), ctypes.byref(best), _stream(stream)))
        self.replan()
        return ms, int(best.value)

    def reset(self):
        self.A.copy_(self.A0)

    def run(self, stream=None):
        _check("ctp_factor_batch", self.ctx.lib.ctp_factor_batch(
            self.ctx.handle, self.plan, _ptr(self.fronts), _ptr(self.ws), self.ws.numel(),
            _stream(stream)))

    def flags(self, stream=None):
        out = np.zeros(self.nb, np.int32)
        _check("ctp_batch_read_info", self.ctx.lib.ctp_batch_read_info(
            self.ctx.handle, self.plan, _ptr(self.ws), out.ctypes.data_as(ctypes.c_void_p),
            _stream(stream)))
        return out

    def result(self, k):
        n, p = int(self.n[k]), int(self.p[k])
        A = self.A[int(self.a_off[k]):int(self.a_off[k + 1])].cpu().numpy().reshape(p, n).T.copy()
        pv = slice(int(self.p_off[k]), int(self.p_off[k + 1]))
        out = dict(A=A, perm=self.perm[pv].cpu().numpy(), piv=self.piv[pv].cpu().numpy(),
                   D=self.D[2 * pv.start:2 * pv.stop].cpu().numpy(),
                   nelim=int(self.nelim[k].cpu()), info=0)
        if self.S is not None:
            seg = self.S[int(self.s_off[k]):int(self.s_off[k + 1])].cpu().numpy()
            m = n - p
            out["S"] = unpack_tiled(seg, m) if self.opt.smode == 5 else unpack_lower(seg, m)
        return out

    def __del__(self):
        try:
            if self.plan:
                self.ctx.lib.ctp_batch_plan_destroy(self.plan)
                self.plan = None
        except Exception:
            pass

