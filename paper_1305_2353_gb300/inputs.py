"""Seeded synthetic supernodes.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic.  Both the CUDA path's tests and the oracle's tests take
their inputs from here, so the two sides see identical matrices.

A supernode is an n x p column-major float64 array (Section 1, eq. (1.1)):
rows 0..p-1 hold A11 (symmetric; both triangles are filled here, only the lower
one is read), rows p..n-1 hold A21.

Workloads (shapes and value distributions of the paper's random experiments,
Section 7.1, and of the build's configurations):
  * ``single_small``: n=2000, p=64, N(0,1) entries, u = 0.01; eight A11
    rows/columns scaled by 1e-8 (diagonal entry by 1e-16) to force delays.
  * ``single_large``: n=200000, p=256, entries uniform in [-1, 1].
  * ``batch``: 8192 supernodes, p log-uniform in [8, 256], n-p log-uniform in
    [0, 16p] (drawn as floor(exp(U(0, ln(16p+1)))) - 1), N(0,1) entries with 2%
    of the A11 diagonal set to zero.
"""
from __future__ import annotations

import numpy as np


def supernode(n, p, seed=0, dist="normal", scale_cols=0, scale=1e-8, zero_diag_frac=0.0,
              diag_boost=0.0):
    """One n x p supernode.  ``dist`` is ``normal`` (N(0,1)) or ``uniform`` (U[-1,1]).
    ``scale_cols`` A11 rows/columns (chosen by the seeded generator) are scaled by
    ``scale``; a fraction ``zero_diag_frac`` of the A11 diagonal is set to zero;
    ``diag_boost`` adds boost*sign(a_jj) to each diagonal entry."""
    rng = np.random.default_rng(seed)
    if dist == "normal":
        A = rng.standard_normal((n, p))
    elif dist == "uniform":
        A = rng.uniform(-1.0, 1.0, (n, p))
    else:
        raise ValueError(dist)
    A = np.asfortranarray(A)
    # symmetric A11 from the lower triangle that was drawn
    A11 = np.tril(A[:p, :p])
    A[:p, :p] = A11 + np.tril(A11, -1).T
    if scale_cols:
        idx = rng.choice(p, size=min(scale_cols, p), replace=False)
        for j in idx:
            A[:p, j] *= scale
            A[j, :p] *= scale
    if zero_diag_frac > 0.0:
        nz = int(round(zero_diag_frac * p))
        if nz > 0:
            idx = rng.choice(p, size=nz, replace=False)
            A[idx, idx] = 0.0
    if diag_boost:
        d = np.arange(p)
        A[d, d] += diag_boost * np.where(A[d, d] >= 0, 1.0, -1.0)
    return A


def single_small(seed=0):
    return supernode(2000, 64, seed=seed, dist="normal", scale_cols=8, scale=1e-8)


def single_large(seed=0, n=200000, p=256):
    return supernode(n, p, seed=seed, dist="uniform")


def batch_shapes(count=8192, seed=0, pmin=8, pmax=256, ratio=16):
    """(n, p) pairs of the uneven batch: p log-uniform in [pmin, pmax], n-p
    log-uniform in [0, ratio*p]."""
    rng = np.random.default_rng(seed)
    p = np.floor(np.exp(rng.uniform(np.log(pmin), np.log(pmax + 1), count))).astype(np.int64)
    p = np.clip(p, pmin, pmax)
    m = np.floor(np.exp(rng.uniform(0.0, np.log(ratio * p + 1.0)))).astype(np.int64) - 1
    m = np.clip(m, 0, ratio * p)
    return np.stack([p + m, p], axis=1)


def batch(count=8192, seed=0, pmin=8, pmax=256, ratio=16, zero_diag_frac=0.02):
    """List of supernodes of the uneven batch (N(0,1), 2% zero diagonals)."""
    shapes = batch_shapes(count, seed, pmin, pmax, ratio)
    return [supernode(int(n), int(p), seed=seed * 1_000_003 + k + 1, dist="normal",
                      zero_diag_frac=zero_diag_frac) for k, (n, p) in enumerate(shapes)]


def symmetric(n, seed=0, dist="normal"):
    """Dense symmetric n x n matrix (both triangles)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n)) if dist == "normal" else rng.uniform(-1, 1, (n, n))
    L = np.tril(X)
    return np.asfortranarray(L + np.tril(L, -1).T)


def rhs(n, k=1, seed=0):
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, k)))


def two_node(A, seed=0):
    """The symmetric matrix M = [[A11, A21^T], [A21, A22]] of order n in which an
    n x p supernode A is the first block column; A22 is symmetric with N(0,1)
    entries drawn from ``seed``.  Full storage, column-major."""
    A = np.asarray(A, dtype=np.float64)
    n, p = A.shape
    rng = np.random.default_rng(seed + 7_919)
    A22 = rng.standard_normal((n - p, n - p))
    A22 = np.tril(A22) + np.tril(A22, -1).T
    M = np.zeros((n, n), order="F")
    A11 = np.tril(A[:p, :p]) + np.tril(A[:p, :p], -1).T
    M[:p, :p] = A11
    M[p:, :p] = A[p:, :]
    M[:p, p:] = A[p:, :].T
    M[p:, p:] = A22
    return M


def dense_symmetric(N, seed=0, dist="normal"):
    """A dense symmetric N x N matrix with N(0,1) (or U[-1,1]) entries."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, N)) if dist == "normal" else rng.uniform(-1.0, 1.0, (N, N))
    return np.asfortranarray(np.tril(X) + np.tril(X, -1).T)


def laplacian_3d(k, sigma=3.0):
    """The 7-point Laplacian on a k x k x k grid (Dirichlet boundary) shifted by
    -sigma I: diagonal 6 - sigma, -1 for each grid neighbour.  sigma = 3 is half
    the mean eigenvalue (trace/N = 6), which makes the matrix indefinite.
    Variable of grid point (x, y, z) is x + k (y + k z).  Returns the lower
    triangle in compressed-column form: (colptr int64[N+1], rowind int32[nnz],
    val float64[nnz]), rows ascending within a column, the diagonal first."""
    N = k ** 3
    idx = np.arange(N).reshape(k, k, k)  # [z, y, x]
    cols = [[] for _ in range(N)]
    rows, cidx, vals = [], [], []
    for (dz, dy, dx) in ((0, 0, 1), (0, 1, 0), (1, 0, 0)):
        a = idx[: k - dz, : k - dy, : k - dx].ravel()
        b = idx[dz:, dy:, dx:].ravel()
        rows.append(b)
        cidx.append(a)
    r = np.concatenate([np.arange(N)] + rows)
    c = np.concatenate([np.arange(N)] + cidx)
    v = np.concatenate([np.full(N, 6.0 - sigma), -np.ones(sum(len(x) for x in rows))])
    order = np.lexsort((r, c))
    r, c, v = r[order], c[order], v[order]
    colptr = np.zeros(N + 1, np.int64)
    np.add.at(colptr, c + 1, 1)
    colptr = np.cumsum(colptr)
    return colptr, r.astype(np.int32), v


def nested_dissection_3d(k, leaf=64):
    """Geometric nested dissection of the k x k x k grid: a box is cut by the
    middle plane across its longest side; the two halves are ordered first (each
    recursively), the plane last.  Boxes of at most `leaf` points are not cut.
    Returns (perm, blocks): perm[q] = variable eliminated q-th; blocks = start
    positions of the blocks in that order (each leaf box and each plane is one
    block, children before parents), with blocks[-1] = N."""
    perm, blocks = [], []

    def rec(x0, x1, y0, y1, z0, z1):
        sx, sy, sz = x1 - x0, y1 - y0, z1 - z0
        if sx <= 0 or sy <= 0 or sz <= 0:
            return
        if sx * sy * sz <= leaf or max(sx, sy, sz) < 3:
            blocks.append(len(perm))
            for z in range(z0, z1):
                for y in range(y0, y1):
                    for x in range(x0, x1):
                        perm.append(x + k * (y + k * z))
            return
        if sx >= sy and sx >= sz:
            m = x0 + sx // 2
            rec(x0, m, y0, y1, z0, z1)
            rec(m + 1, x1, y0, y1, z0, z1)
            blocks.append(len(perm))
            for z in range(z0, z1):
                for y in range(y0, y1):
                    perm.append(m + k * (y + k * z))
        elif sy >= sz:
            m = y0 + sy // 2
            rec(x0, x1, y0, m, z0, z1)
            rec(x0, x1, m + 1, y1, z0, z1)
            blocks.append(len(perm))
            for z in range(z0, z1):
                for x in range(x0, x1):
                    perm.append(x + k * (m + k * z))
        else:
            m = z0 + sz // 2
            rec(x0, x1, y0, y1, z0, m)
            rec(x0, x1, y0, y1, m + 1, z1)
            blocks.append(len(perm))
            for y in range(y0, y1):
                for x in range(x0, x1):
                    perm.append(x + k * (y + k * m))

    rec(0, k, 0, k, 0, k)
    blocks.append(len(perm))
    return np.asarray(perm, np.int32), np.asarray(blocks, np.int64)
