"""Python access to the CPU FP64 oracle (``ctp_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports, links or runs anything from this directory, and this module never
imports the CUDA library.

The oracle follows the paper (Hogg & Scott, arXiv 1305.2353) step by step:
Listing 1 (threshold partial pivoting, Section 2), strict compression
(Section 4.1, eq. (4.1)) with the worst-case update (eq. (4.3)), relaxed
compression (Section 4.2), restricted pivoting (Section 3.2), the Solve and
Form tasks of Section 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ctp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

STRICT, RELAXED, TPP, RESTRICTED, SINGLE_ROW = 0, 1, 2, 3, 4
METHODS = {"strict": STRICT, "relaxed": RELAXED, "tpp": TPP, "restricted": RESTRICTED,
           "single_row": SINGLE_ROW}
PIV_1X1, PIV_2X2_FIRST, PIV_2X2_SECOND, PIV_ZERO, PIV_DELAYED = 1, 2, 0, -1, 3
UPD_NORMAL, UPD_ABS = 0, 1
LOG_KINDS = {0: "zero", 1: "2x2_max", 2: "2x2_det", 3: "2x2_tiny", 4: "2x2_growth", 5: "1x1"}


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "tests_1x1", "tests_2x2", "accepted_1x1", "accepted_2x2", "zero_pivots", "sweeps",
        "ops_colmax", "ops_test", "ops_apply", "ops_update")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


LOG_DTYPE = np.dtype([("kind", np.int32), ("m", np.int32), ("t", np.int32),
                      ("outcome", np.int32), ("lhs", np.float64), ("rhs", np.float64)])


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction) into oracle/_build."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        P = ctypes.c_void_p
        L.orc_compress_strict.argtypes = [i32, i32, P, i64, P, i64, P]
        L.orc_compress_relaxed.argtypes = [i32, i32, P, i64, P, i64, P]
        L.orc_listing1.argtypes = [i32, i32, i32, i32, P, i64, dbl, dbl, i32, P, P, P, P, P, P, i32, P]
        L.orc_factor.argtypes = [i32, i32, P, i64, i32, dbl, dbl, P, P, P, P, P, P, P, i32, P]
        L.orc_form.argtypes = [i32, i32, P, i64, P, P, P, i64]
        L.orc_form_entries.argtypes = [i32, i32, P, i64, P, P, i32, P, P, P]
        L.orc_ldlt_fixed.argtypes = [i32, i32, P, i64, i32, P, P]
        for f in ("orc_ldlt_fixed", "orc_compress_strict", "orc_compress_relaxed", "orc_listing1", "orc_factor",
                  "orc_form", "orc_form_entries"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _fortran(a, dtype=np.float64):
    return np.asfortranarray(np.array(a, dtype=dtype, copy=True))


def compress_strict(A21):
    """Strict compressed matrix C (eq. (4.1)) and the row sets J(i)."""
    A21 = _fortran(A21)
    m, p = A21.shape
    C = np.zeros((p, p), order="F")
    J = np.zeros(m, dtype=np.int32)
    rc = lib().orc_compress_strict(m, p, _p(A21), max(m, 1), _p(C), p, _p(J))
    assert rc == 0
    return C, J


def compress_relaxed(A21):
    """Relaxed compressed matrix C (Section 4.2) and the chosen A21 rows."""
    A21 = _fortran(A21)
    m, p = A21.shape
    C = np.zeros((p, p), order="F")
    rows = np.zeros(p, dtype=np.int32)
    rc = lib().orc_compress_relaxed(m, p, _p(A21), max(m, 1), _p(C), p, _p(rows))
    assert rc == 0
    return C, rows


def listing1(Wfull, p, rt=0, rs=0, tmode=UPD_NORMAL, u=0.01, small=1e-20, stop_nelim=-1,
             log_cap=0):
    """Listing 1 on a working matrix whose first p rows hold A11 in full symmetric
    form, followed by rt tested outer rows and rs shadow rows."""
    W = _fortran(Wfull)
    assert W.shape == (p + rt + rs, p)
    perm = np.zeros(p, np.int32)
    piv = np.zeros(p, np.int32)
    D = np.zeros(2 * p)
    ne = np.zeros(1, np.int32)
    st = Stats()
    log = np.zeros(max(log_cap, 1), LOG_DTYPE)
    loglen = np.zeros(1, np.int32)
    rc = lib().orc_listing1(p, rt, rs, tmode, _p(W), W.shape[0], u, small, stop_nelim, _p(perm),
                            _p(piv), _p(D), _p(ne), ctypes.byref(st), _p(log), log_cap, _p(loglen))
    assert rc == 0, rc
    return dict(W=W, perm=perm, piv=piv, D=D, nelim=int(ne[0]), stats=st.as_dict(),
                log=log[:min(int(loglen[0]), log_cap)], log_len=int(loglen[0]))


def factor(A, p, method="strict", u=0.01, small=1e-20, log_cap=0):
    """Factor an n x p supernode (A11 lower triangle read).  Returns the in-place
    result and the pivot data; see ``orc_factor`` for the layout."""
    A = _fortran(A)
    n = A.shape[0]
    assert A.shape[1] == p
    perm = np.zeros(p, np.int32)
    piv = np.zeros(p, np.int32)
    D = np.zeros(2 * p)
    ne = np.zeros(1, np.int32)
    C = np.zeros((p, p), order="F")
    st = Stats()
    log = np.zeros(max(log_cap, 1), LOG_DTYPE)
    loglen = np.zeros(1, np.int32)
    rc = lib().orc_factor(n, p, _p(A), n, METHODS[method], u, small, _p(perm), _p(piv), _p(D),
                          _p(ne), _p(C), ctypes.byref(st), _p(log), log_cap, _p(loglen))
    assert rc == 0, rc
    return dict(A=A, perm=perm, piv=piv, D=D, nelim=int(ne[0]), C=C, stats=st.as_dict(),
                log=log[:min(int(loglen[0]), log_cap)], log_len=int(loglen[0]))


def ldlt_fixed(A, p, piv_in):
    """Factor with a prescribed pivot sequence in natural order (no tests)."""
    A = _fortran(A)
    n = A.shape[0]
    piv_in = np.ascontiguousarray(piv_in, dtype=np.int32)
    D = np.zeros(2 * p)
    rc = lib().orc_ldlt_fixed(n, p, _p(A), n, len(piv_in), _p(piv_in), _p(D))
    assert rc == 0
    piv = np.full(p, PIV_DELAYED, np.int32)
    piv[:len(piv_in)] = piv_in
    return dict(A=A, perm=np.arange(p, dtype=np.int32), piv=piv, D=D, nelim=len(piv_in))


def form(L21, piv, D):
    """S = L21 D11 L21^T (lower triangle; the strict upper part is zero)."""
    L21 = _fortran(L21)
    m, e = L21.shape
    S = np.zeros((m, m), order="F")
    piv = np.ascontiguousarray(piv, dtype=np.int32)
    D = np.ascontiguousarray(D, dtype=np.float64)
    rc = lib().orc_form(m, e, _p(L21), max(m, 1), _p(piv), _p(D), _p(S), max(m, 1))
    assert rc == 0
    return S


def form_entries(L21, piv, D, ii, jj):
    """Entries S(ii[t], jj[t]) of S = L21 D11 L21^T."""
    L21 = _fortran(L21)
    m, e = L21.shape
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    val = np.zeros(len(ii))
    piv = np.ascontiguousarray(piv, dtype=np.int32)
    D = np.ascontiguousarray(D, dtype=np.float64)
    rc = lib().orc_form_entries(m, e, _p(L21), max(m, 1), _p(piv), _p(D), len(ii), _p(ii), _p(jj),
                                _p(val))
    assert rc == 0
    return val


# ---------------------------------------------------------------------------
# Helpers that read the oracle's outputs back into matrices (no arithmetic of
# the method: only unpacking of the in-place layout).

def unpack(res, p):
    """Split the in-place result into (L, Dmat, R): L is n x e unit lower (in
    pivot order for the A11 rows), Dmat the e x e block diagonal, R the n x d
    delayed columns (A11 rows in pivot order; its top e rows are zero)."""
    A, piv, D, e = res["A"], res["piv"], res["D"], res["nelim"]
    n = A.shape[0]
    L = np.zeros((n, e))
    Dm = np.zeros((e, e))
    for j in range(e):
        L[j, j] = 1.0
        L[j + 1:, j] = A[j + 1:, j]
        if piv[j] == PIV_2X2_FIRST:
            L[j + 1, j] = 0.0
    for j in range(e):
        if piv[j] == PIV_1X1:
            Dm[j, j] = D[2 * j]
        elif piv[j] == PIV_2X2_FIRST:
            Dm[j, j] = D[2 * j]
            Dm[j + 1, j] = Dm[j, j + 1] = D[2 * j + 1]
            Dm[j + 1, j + 1] = D[2 * j + 2]
    R = np.zeros((n, p - e))
    for k in range(e, p):
        R[k:, k - e] = A[k:, k]
    return L, Dm, R


def permuted_supernode(A, p, perm):
    """The supernode with its columns (and A11 rows) in pivot order, A11 made
    symmetric from its lower triangle: rows 0..p-1 = P A11 P^T, rows p.. = A21 P^T."""
    A = np.array(A, dtype=np.float64)
    A11 = np.tril(A[:p, :p]) + np.tril(A[:p, :p], -1).T
    out = np.zeros_like(A)
    out[:p, :] = A11[np.ix_(perm, perm)]
    out[p:, :] = A[p:, :][:, perm]
    return out
