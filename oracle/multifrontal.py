"""Multifrontal oracle: a sparse symmetric indefinite system factored front by
front over its assembly tree, each front's fully-summed columns eliminated by
the oracle's per-supernode routine (compressed, restricted or full-column
pivoting), delayed columns passed to the parent front.

TEST INFRASTRUCTURE ONLY (same rule as ``oracle.py``): the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs are the only callers.

What is computed (Hogg & Scott, Section 1: the Factor, Solve, Form and Scatter
tasks of a multifrontal code, and the passing of delayed columns to the parent):

* ``analyse``: the fronts of a given elimination order whose consecutive
  blocks (the separators and leaf boxes of nested dissection) are taken as
  supernodes.  Front s holds its block's variables and the rows below them,
  struct(s) = later variables joined to the block in the filled graph: the
  block's own later neighbours and the later rows of its children's fronts.
  Its parent is the block holding the first variable of struct(s).
* ``factor``: for each front, children first: the frontal matrix gets the
  original entries of its own variables' columns (entries whose earlier
  variable is in this block), then the children's contribution blocks
  (extend-add, the Scatter task).  Its fully-summed columns -- the block's
  variables, then the columns the children delayed -- are eliminated in panels
  of at most ``w`` columns: a panel is the leading columns of the current
  Schur complement (the columns the previous panel delayed come first),
  factored by ``oracle.factor``, and the Schur complement is updated (Form).
  A panel that eliminates nothing ends the front: its remaining fully-summed
  columns are delayed to the parent.  The root must eliminate everything: a
  panel there that eliminates nothing is factored again with threshold partial
  pivoting, and if that also fails the factorization stops with an error.
* The resulting fronts (panels) have the same form as ``system.factor_chain``'s,
  so ``system.solve``, ``system.refine`` and ``system.backward_error`` apply.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import oracle as _orc
from .system import ChainError


def sym_csc(colptr, rowind, val, N):
    """The full symmetric matrix from its lower triangle in compressed columns."""
    L = sp.csc_matrix((val, rowind, colptr), shape=(N, N))
    return (L + sp.tril(L, -1).T).tocsr()


def analyse(colptr, rowind, N, perm, blocks):
    """Fronts of the order `perm` with supernodes `blocks` (start positions,
    blocks[-1] = N).  Returns a list of dicts (one per block, children first):
    vars (new indices), struct (new indices, ascending), parent (block index or
    -1), children."""
    inv = np.empty(N, np.int64)
    inv[perm] = np.arange(N)
    # adjacency in new numbering (both triangles)
    adj = [[] for _ in range(N)]
    for j in range(N):
        for q in range(colptr[j], colptr[j + 1]):
            i = rowind[q]
            if i != j:
                a, b = inv[i], inv[j]
                adj[a].append(b)
                adj[b].append(a)
    nb = len(blocks) - 1
    owner = np.empty(N, np.int64)
    for s in range(nb):
        owner[blocks[s]:blocks[s + 1]] = s
    fronts = [dict(vars=np.arange(blocks[s], blocks[s + 1]), children=[], parent=-1)
              for s in range(nb)]
    for s in range(nb):
        lo, hi = blocks[s], blocks[s + 1]
        rows = set()
        for v in range(lo, hi):
            rows.update(w for w in adj[v] if w >= hi)
        for c in fronts[s]["children"]:
            rows.update(w for w in fronts[c]["struct"] if w >= hi)
        st = np.array(sorted(rows), np.int64)
        fronts[s]["struct"] = st
        if len(st):
            par = int(owner[st[0]])
            fronts[s]["parent"] = par
            fronts[par]["children"].append(s)
    return fronts


def factor(colptr, rowind, val, N, perm, blocks, method="strict", w=256, u=0.01, small=1e-20):
    """Numeric multifrontal factorization.  Returns (panels, info): panels in
    elimination order, each a dict as ``system.factor_chain`` returns (vars in
    the ORIGINAL numbering); info per front: nelim, delayed count, n, p."""
    A = sym_csc(colptr, rowind, val, N)
    inv = np.empty(N, np.int64)
    inv[perm] = np.arange(N)
    fr = analyse(colptr, rowind, N, perm, blocks)
    cb = {}        # front -> (vars of its contribution block (new numbering), matrix)
    panels, info = [], []
    for s, f in enumerate(fr):
        own = f["vars"]
        delayed = [v for c in f["children"] for v in cb[c][0][: cb[c][2]]]
        fs = np.concatenate([own, np.array(delayed, np.int64)])
        rows = np.concatenate([fs, f["struct"]])
        n = len(rows)
        loc = {int(v): k for k, v in enumerate(rows)}
        F = np.zeros((n, n))
        # original entries of the own variables' columns: entries whose earlier
        # variable (new numbering) is one of this block's
        for v in own:
            ov = perm[v]
            row = A.getrow(ov)
            for oj, a in zip(row.indices, row.data):
                w_ = inv[oj]
                if w_ >= v and w_ in loc:
                    i, j = loc[int(w_)], loc[int(v)]
                    F[i, j] += a
                    if i != j:
                        F[j, i] += a
        # extend-add of the children's contribution blocks
        for c in f["children"]:
            cv, C, _ = cb[c]
            idx = np.array([loc[int(v)] for v in cv], np.int64)
            F[np.ix_(idx, idx)] += C
            del cb[c]
        # eliminate the fully-summed columns in panels
        T = F
        ordv = rows.copy()
        p_left = len(fs)
        root = f["parent"] < 0
        e_front = 0
        while p_left > 0:
            m_rows = T.shape[0]
            wd = min(w, p_left)
            meth = method
            res = _orc.factor(np.asfortranarray(T[:, :wd]), wd, meth, u=u, small=small)
            if res["nelim"] == 0 and root and meth != "tpp":
                meth = "tpp"
                res = _orc.factor(np.asfortranarray(T[:, :wd]), wd, meth, u=u, small=small)
            e = res["nelim"]
            if e == 0:
                if root:
                    raise ChainError("the root front eliminated nothing")
                break
            L, Dm, _ = _orc.unpack(res, wd)
            pm = np.asarray(res["perm"], np.int64)
            prow = np.concatenate([pm, np.arange(wd, m_rows)])
            panels.append(dict(vars=perm[ordv[prow]], L=L, Dm=Dm, piv=np.array(res["piv"][:e]), e=e,
                               p=wd, method=meth, perm=pm.copy(), front=s))
            q = prow[e:]
            L2 = L[e:, :]
            T = T[np.ix_(q, q)] - L2 @ Dm @ L2.T
            ordv = ordv[q]
            p_left -= e
            e_front += e
        if root and p_left > 0:
            raise ChainError("columns left at the root")
        info.append(dict(n=n, p=len(fs), own=len(own), nelim=e_front, delayed=p_left))
        if not root:
            cb[s] = (ordv, T, p_left)   # the first p_left are the delayed columns
    return panels, info


def residual_csc(colptr, rowind, val, N, x, b):
    """b - A x with A given by its lower triangle (both triangles applied)."""
    A = sym_csc(colptr, rowind, val, N)
    return b - A @ x
