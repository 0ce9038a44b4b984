"""Complete-system oracle: a supernode embedded in a symmetric indefinite system,
factored as a chain of supernodes, solved, refined.

TEST INFRASTRUCTURE ONLY (same rule as ``oracle.py``): the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs are the only callers;
the CUDA library never uses it.

What is computed (Hogg & Scott, Section 1 and Section 7):

* ``factor_chain``: a dense symmetric matrix M of order N is factored as
  P M P^T = L D L^T by a chain of supernodes.  The first one is the paper's
  supernode [A11; A21] (its p columns and all N rows); each later one takes up
  to ``w_rest`` leading columns of the current Schur complement, which starts
  with the columns the previous supernode delayed (Section 1: delayed columns
  are passed to the parent, here the next supernode of the chain).  Each
  supernode is factored by the oracle's per-supernode routine (``oracle.factor``:
  Listing 1 with compressed, restricted or full-column pivot tests); the Schur
  complement update T <- T - L21 D11 L21^T is the Form step, applied in full
  (both triangles) here.  When a compressed/restricted supernode eliminates
  nothing it is factored again with threshold partial pivoting; a supernode
  that still eliminates nothing with rows below, or leaves columns delayed with
  no rows below, is an error.
* ``solve``: forward substitution with the unit lower factors, the block
  diagonal solve (1x1 and 2x2 blocks; a zero pivot gives a zero component), and
  back substitution, front by front, with every front's rows named by their
  variable indices.
* ``backward_error``: the scaled backward error of Section 7,
  ||M x - b||_inf / (||M||_inf ||x||_inf + ||b||_inf).
* ``refine``: iterative refinement with FP64 residuals (Section 7: at most ten
  steps), stopping once the backward error reaches ``tol``.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import oracle as _orc


class ChainError(RuntimeError):
    pass


def factor_chain(M, first_p, method_first="strict", method_rest="tpp", w_rest=256, u=0.01,
                 small=1e-20, Mfactor=None):
    """Factor the symmetric matrix M (full storage; only its values are read,
    both triangles) as a chain of supernodes.  ``Mfactor`` (default M) is the
    matrix whose factors are computed -- a perturbed copy stands in for a
    low-precision factorization in the refinement tests.

    Returns a list of fronts, each a dict with ``vars`` (variable index of each
    front row, pivot order for the fully-summed ones), ``L`` (n_k x e unit
    lower), ``Dm`` (e x e block diagonal), ``piv``, ``e``, ``p`` (columns taken),
    ``method`` (the pivoting actually used)."""
    T = np.array(M if Mfactor is None else Mfactor, dtype=np.float64, copy=True)
    N = T.shape[0]
    ordv = np.arange(N)
    fronts = []
    first = True
    while T.shape[0] > 0:
        n = T.shape[0]
        w = min(first_p if first else w_rest, n)
        method = method_first if first else method_rest
        first = False
        panel = np.asfortranarray(T[:, :w])
        res = _orc.factor(panel, w, method, u=u, small=small)
        if res["nelim"] == 0 and method != "tpp":
            method = "tpp"
            res = _orc.factor(np.asfortranarray(T[:, :w]), w, method, u=u, small=small)
        e = res["nelim"]
        if e == 0 and n > w:
            raise ChainError("a supernode with rows below eliminated no column")
        if e < w and n == w:
            raise ChainError("columns left delayed with no rows below")
        L, Dm, _ = _orc.unpack(res, w)
        perm = np.asarray(res["perm"], dtype=np.int64)
        rows = np.concatenate([perm, np.arange(w, n)])
        fronts.append(dict(vars=ordv[rows].copy(), L=L, Dm=Dm, piv=np.array(res["piv"][:e]),
                           e=e, p=w, method=method, perm=perm.copy()))
        # Schur complement of the e pivots, rows/columns in the new order
        q = rows[e:]
        L2 = L[e:, :]
        T = T[np.ix_(q, q)] - L2 @ Dm @ L2.T
        ordv = ordv[q]
    return fronts


def global_factors(fronts, N):
    """Assemble (order, L, D): P M P^T = L D L^T with P the pivot order."""
    order = np.concatenate([f["vars"][:f["e"]] for f in fronts])
    pos = np.empty(N, dtype=np.int64)
    pos[order] = np.arange(N)
    L = np.zeros((N, N))
    D = np.zeros((N, N))
    c = 0
    for f in fronts:
        e = f["e"]
        r = pos[f["vars"]]
        L[np.ix_(r, np.arange(c, c + e))] = f["L"]
        D[c:c + e, c:c + e] = f["Dm"]
        c += e
    return order, L, D


def _dsolve(Dm, piv, y):
    """y <- D^{-1} y for one front (1x1 and 2x2 blocks; zero pivots give 0)."""
    e = Dm.shape[0]
    out = np.zeros_like(y)
    j = 0
    while j < e:
        if piv[j] == _orc.PIV_2X2_FIRST:
            out[j:j + 2] = np.linalg.solve(Dm[j:j + 2, j:j + 2], y[j:j + 2])
            j += 2
        else:
            out[j] = y[j] / Dm[j, j] if Dm[j, j] != 0.0 else 0.0
            j += 1
    return out


def solve(fronts, b):
    """x = M^{-1} b from the chain's factors (b: N or N x nrhs)."""
    x = np.array(b, dtype=np.float64, copy=True)
    for f in fronts:                      # L y = b
        e, v, L = f["e"], f["vars"], f["L"]
        y = scipy.linalg.solve_triangular(L[:e, :], x[v[:e]], lower=True, unit_diagonal=True)
        x[v[:e]] = y
        x[v[e:]] -= L[e:, :] @ y
    for f in fronts:                      # D z = y
        v, e = f["vars"], f["e"]
        x[v[:e]] = _dsolve(f["Dm"], f["piv"], x[v[:e]])
    for f in reversed(fronts):            # L^T x = z
        e, v, L = f["e"], f["vars"], f["L"]
        z = x[v[:e]] - L[e:, :].T @ x[v[e:]]
        x[v[:e]] = scipy.linalg.solve_triangular(L[:e, :].T, z, lower=False, unit_diagonal=True)
    return x


def backward_error(M, x, b):
    """||M x - b||_inf / (||M||_inf ||x||_inf + ||b||_inf), per right-hand side."""
    M = np.asarray(M, dtype=np.float64)
    x2 = x.reshape(x.shape[0], -1)
    b2 = b.reshape(b.shape[0], -1)
    r = M @ x2 - b2
    nM = np.abs(M).sum(axis=1).max()
    out = np.abs(r).max(axis=0) / (nM * np.abs(x2).max(axis=0) + np.abs(b2).max(axis=0))
    return out if x.ndim > 1 else float(out[0])


def refine(M, fronts, b, steps=10, tol=1e-14):
    """Iterative refinement: x0 = solve(b); x <- x + solve(b - M x) until the
    backward error is at most ``tol`` or ``steps`` corrections were made.
    Returns (x, history of backward errors, corrections made)."""
    x = solve(fronts, b)
    hist = [backward_error(M, x, b)]
    k = 0
    while k < steps and np.max(hist[-1]) > tol:
        r = b - np.asarray(M) @ x
        x = x + solve(fronts, r)
        hist.append(backward_error(M, x, b))
        k += 1
    return x, hist, k


def solve_gradient(fronts, x, gx):
    """Gradient of a loss through x = M^{-1} b (Section 1's factors reused),
    given gx = dloss/dx: returns (gb, gM) with gb = M^{-T} gx (M symmetric, so
    the same solve) and gM the gradient with respect to the stored lower
    triangle of M -- an off-diagonal stored entry m_ij stands for both m_ij and
    m_ji, so it gets -(gb_i x_j + gb_j x_i); a diagonal entry gets -gb_i x_i
    (from d(M^{-1} b) = -M^{-1} dM M^{-1} b).  The strict upper triangle of gM
    is zero."""
    gb = solve(fronts, gx)
    G = np.atleast_2d(gb.T).T
    X = np.atleast_2d(np.asarray(x).T).T
    full = -(G @ X.T)
    gM = np.tril(full + full.T)
    np.fill_diagonal(gM, np.diag(full))
    return gb, gM


def solve_gradient_pattern(fronts, x, gx, row, col):
    """``solve_gradient`` restricted to a pattern of stored lower-triangle
    entries (row[k] >= col[k]): returns (gb, g) with g[k] the gradient with
    respect to the stored entry (row[k], col[k]) -- for an off-diagonal entry
    -sum_r (gb_ir x_jr + gb_jr x_ir), for a diagonal one -sum_r gb_ir x_ir
    (the same derivative of x = M^{-1} b as ``solve_gradient``, evaluated only
    where the sparse matrix stores an entry)."""
    gb = solve(fronts, gx)
    G = np.atleast_2d(gb.T).T
    X = np.atleast_2d(np.asarray(x).T).T
    row = np.asarray(row, np.int64)
    col = np.asarray(col, np.int64)
    g = np.empty(len(row))
    for k in range(len(row)):
        i, j = row[k], col[k]
        if i == j:
            g[k] = -np.dot(G[i], X[i])
        else:
            g[k] = -(np.dot(G[i], X[j]) + np.dot(G[j], X[i]))
    return gb, g
