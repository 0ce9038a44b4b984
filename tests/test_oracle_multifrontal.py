"""Pins of the multifrontal oracle against what mathematics fixes: solutions of
LAPACK/SuperLU, the reconstruction P A P^T = L D L^T, Sylvester's inertia, a
brute-force symbolic elimination, and refinement to the Section 7 criterion."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import multifrontal as MF
from oracle import system as S
from paper_1305_2353_gb300 import inputs


def _problem(k, sigma=3.0, leaf=64):
    cp, ri, v = inputs.laplacian_3d(k, sigma)
    perm, blocks = inputs.nested_dissection_3d(k, leaf)
    return cp, ri, v, k ** 3, perm, blocks


def test_symbolic_matches_brute_force_elimination():
    """Each front's rows below its block equal the later neighbours of the
    block's variables in the filled graph of a brute-force elimination."""
    cp, ri, v, N, perm, blocks = _problem(6, leaf=16)
    A = MF.sym_csc(cp, ri, v, N).toarray() != 0
    P = A[np.ix_(perm, perm)].copy()
    for j in range(N):                      # eliminate j: its later neighbours become a clique
        nb = np.nonzero(P[j, j + 1:])[0] + j + 1
        P[np.ix_(nb, nb)] = True
    fr = MF.analyse(cp, ri, N, perm, blocks)
    for s, f in enumerate(fr):
        lo, hi = blocks[s], blocks[s + 1]
        want = np.nonzero(P[lo:hi, hi:].any(axis=0))[0] + hi
        assert np.array_equal(f["struct"], want), s
        if len(want):
            assert blocks[f["parent"]] <= want[0] < blocks[f["parent"] + 1]


# grid sizes whose shifted Laplacian is safely nonsingular (some k give exact
# zero eigenvalues, e.g. k = 8, sigma = 3: three cosines of pi/3 sum to 1.5)
@pytest.mark.parametrize("k,sigma,method", [(7, 3.0, "strict"), (9, 3.0, "tpp"), (10, 3.0, "relaxed"),
                                            (10, 6.0, "strict"), (6, 6.0, "tpp")])
def test_factor_reconstructs_and_inertia(k, sigma, method):
    """P A P^T = L D L^T for the assembled panels, every variable eliminated once,
    and the inertia of D equals the eigenvalue count of A (Sylvester).  sigma = 6
    zeroes the diagonal: only 2x2 pivots exist and fronts delay columns."""
    cp, ri, v, N, perm, blocks = _problem(k, sigma, leaf=32)
    panels, info = MF.factor(cp, ri, v, N, perm, blocks, method, w=48)
    order, L, D = S.global_factors(panels, N)
    assert sorted(order.tolist()) == list(range(N))
    A = MF.sym_csc(cp, ri, v, N).toarray()
    Ap = A[np.ix_(order, order)]
    rec = np.abs(Ap - L @ D @ L.T).max() / (np.abs(L) @ np.abs(D) @ np.abs(L.T)).max()
    assert rec <= 1e-14
    ev = np.linalg.eigvalsh(A)
    assert np.abs(ev).min() > 1e-3
    dv = np.linalg.eigvalsh(D)
    assert (dv < 0).sum() == (ev < 0).sum() and (dv > 0).sum() == (ev > 0).sum()
    if sigma == 6.0 and method == "strict":
        assert sum(i["delayed"] for i in info) > 0


def test_solution_and_refinement():
    """The multifrontal solve against SuperLU, and FP64 refinement to 1e-14."""
    cp, ri, v, N, perm, blocks = _problem(12)
    panels, _ = MF.factor(cp, ri, v, N, perm, blocks, "strict", w=64)
    A = MF.sym_csc(cp, ri, v, N)
    rng = np.random.default_rng(0)
    b = rng.standard_normal(N)
    xr = spla.spsolve(A.tocsc(), b)
    x = S.solve(panels, b)
    assert np.abs(x - xr).max() <= 1e-10 * np.abs(xr).max()
    Ad = A.toarray()
    x2, hist, k = S.refine(Ad, panels, b)
    assert hist[-1] <= 1e-14


def test_panels_split_wide_fronts():
    """A front wider than the panel width becomes a chain of panels whose
    columns follow one another (the root plane of a 12^3 grid is 144 wide)."""
    cp, ri, v, N, perm, blocks = _problem(12)
    panels, info = MF.factor(cp, ri, v, N, perm, blocks, "tpp", w=40)
    root = len(info) - 1
    rp = [p for p in panels if p["front"] == root]
    assert len(rp) >= 4 and all(p["p"] <= 40 for p in rp)
    assert sum(p["e"] for p in rp) == info[root]["nelim"] == info[root]["p"]


def _fd_loss(cp, ri, N, vals, B):
    """loss = ||A^{-1} B||_F^2 by SuperLU (a library solve, not the oracle)."""
    X = spla.splu(MF.sym_csc(cp, ri, vals, N).tocsc()).solve(B)
    return float((X * X).sum())


@pytest.mark.parametrize("k,leaf,nrhs,sample", [(4, 8, 3, None), (16, 64, 32, 10)])
def test_pattern_gradient_against_finite_differences(k, leaf, nrhs, sample):
    """The gradient of loss = ||x||^2, x = A^{-1} B, through the multifrontal
    panels (adjoint solve with the same factors, then the pattern formula):
    every stored entry of a 4^3 grid and a sample of the 16^3 grid with 32
    right-hand sides, and entries of B, against central differences (h = 1e-6)
    of SuperLU solves.  A stored off-diagonal value stands for both of its
    symmetric entries, so perturbing it perturbs both."""
    cp, ri, v, N, perm, blocks = _problem(k, leaf=leaf)
    panels, _ = MF.factor(cp, ri, v, N, perm, blocks, "strict", w=256)
    rng = np.random.default_rng(k)
    B = rng.standard_normal((N, nrhs))
    x, hist, _ = S.refine(MF.sym_csc(cp, ri, v, N).toarray(), panels, B)
    assert np.max(hist[-1]) <= 1e-14
    col = np.repeat(np.arange(N), np.diff(cp))
    gb, g = S.solve_gradient_pattern(panels, x, 2.0 * x, ri, col)
    h = 1e-6
    qs = range(len(v)) if sample is None else rng.choice(len(v), sample, replace=False)
    for q in qs:
        vp, vm = v.copy(), v.copy()
        vp[q] += h
        vm[q] -= h
        fd = (_fd_loss(cp, ri, N, vp, B) - _fd_loss(cp, ri, N, vm, B)) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * np.abs(g).max(), (q, fd, g[q])
    for _ in range(4):
        i, r = rng.integers(N), rng.integers(nrhs)
        Bp, Bm = B.copy(), B.copy()
        Bp[i, r] += h
        Bm[i, r] -= h
        fd = (_fd_loss(cp, ri, N, v, Bp) - _fd_loss(cp, ri, N, v, Bm)) / (2 * h)
        assert abs(fd - gb[i, r]) <= 1e-6 * np.abs(gb).max(), (i, r, fd, gb[i, r])


def _closed_form_eigs(k, sigma):
    """Eigenvalues of the 7-point Dirichlet Laplacian on k^3 minus sigma I:
    sum over the three axes of 2 - 2 cos(pi i / (k + 1)), i = 1..k, minus sigma."""
    lam = 2.0 - 2.0 * np.cos(np.pi * np.arange(1, k + 1) / (k + 1))
    return (lam[:, None, None] + lam[None, :, None] + lam[None, None, :]).ravel() - sigma


@pytest.mark.parametrize("k", [3, 4, 5])
def test_shifted_laplacian_spectrum(k):
    """The input generator's matrix has the closed-form spectrum (checked with a
    dense symmetric eigensolver), including the exact zero eigenvalue that
    sigma = 3 gives when 3 divides k + 1 (here k = 5)."""
    cp, ri, v = inputs.laplacian_3d(k, 3.0)
    M = MF.sym_csc(cp, ri, v, k ** 3).toarray()
    got = np.sort(np.linalg.eigvalsh(M))
    want = np.sort(_closed_form_eigs(k, 3.0))
    assert np.abs(got - want).max() <= 1e-12
    assert (np.abs(want).min() <= 1e-14) == ((k + 1) % 3 == 0)


def test_grids_in_use_are_nonsingular():
    """Every grid of the GPU tests and the benchmark keeps the shift away from
    the spectrum; 8^3 and 32^3, which do not, are singular."""
    for k in (4, 6, 7, 9, 10, 12, 16, 24, 64):
        assert np.abs(_closed_form_eigs(k, 3.0)).min() > 1e-4, k
    assert np.abs(_closed_form_eigs(10, 6.0)).min() > 1e-4
    assert np.abs(_closed_form_eigs(12, 6.0)).min() > 1e-4
    for k in (8, 32):
        assert np.abs(_closed_form_eigs(k, 3.0)).min() < 1e-14, k
