"""Pins of the complete-system oracle (chain factorization, solve, backward
error, iterative refinement) against mathematics it does not share: a library
dense solver, hand-computed values, reconstructions and structural facts."""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle import system as S
from paper_1305_2353_gb300 import inputs


def _recon(M, fronts):
    order, L, D = S.global_factors(fronts, M.shape[0])
    Mp = M[np.ix_(order, order)]
    return np.abs(Mp - L @ D @ L.T).max() / (np.abs(L) @ np.abs(D) @ np.abs(L.T)).max()


def _embedded(n=500, p=48, seed=0, scale_cols=6):
    A = inputs.supernode(n, p, seed=seed, scale_cols=scale_cols)
    return A, inputs.two_node(A, seed)


@pytest.mark.parametrize("mf,mr,w", [("strict", "tpp", 64), ("strict", "strict", 32),
                                     ("relaxed", "relaxed", 64), ("tpp", "tpp", 40),
                                     ("restricted", "tpp", 64)])
def test_chain_reconstructs(mf, mr, w):
    """P M P^T = L D L^T for the assembled chain factors (Section 1 eq. (1.2)
    applied supernode by supernode), and every variable eliminated once."""
    A, M = _embedded()
    fr = S.factor_chain(M, A.shape[1], mf, mr, w_rest=w)
    order, _, _ = S.global_factors(fr, M.shape[0])
    assert sorted(order.tolist()) == list(range(M.shape[0]))
    assert _recon(M, fr) <= 1e-14


def test_first_front_is_the_supernode():
    """The chain's first front is the stand-alone factorization of [A11; A21]."""
    A, M = _embedded()
    p = A.shape[1]
    fr = S.factor_chain(M, p, "strict", "tpp")
    ref = orc.factor(A.copy(order="F"), p, "strict")
    assert fr[0]["e"] == ref["nelim"]
    assert np.array_equal(fr[0]["perm"], ref["perm"])
    assert np.array_equal(fr[0]["piv"], ref["piv"][:ref["nelim"]])


def test_delays_roll_into_the_next_front():
    """Columns a front delays are the leading fully-summed columns of the next."""
    A, M = _embedded(scale_cols=10)
    fr = S.factor_chain(M, A.shape[1], "strict", "strict", w_rest=32)
    for a, b in zip(fr[:-1], fr[1:]):
        d = min(a["p"] - a["e"], b["p"])
        if d:
            assert np.array_equal(b["vars"][np.argsort(b["perm"])][:d],
                                  a["vars"][a["e"]:a["e"] + d])


def test_solve_matches_library_solver():
    """x = M^{-1} b against LAPACK's dense solver (LU with partial pivoting)."""
    A, M = _embedded()
    rng = np.random.default_rng(3)
    B = rng.standard_normal((M.shape[0], 3))
    xr = np.linalg.solve(M, B)
    cond = np.linalg.cond(M)
    for mf, mr in [("strict", "tpp"), ("tpp", "tpp"), ("relaxed", "relaxed")]:
        fr = S.factor_chain(M, A.shape[1], mf, mr)
        x = S.solve(fr, B)
        assert np.abs(x - xr).max() / np.abs(xr).max() <= 1e-13 * cond


def test_backward_error_hand_value():
    """Section 7 formula on a 2 x 2 case worked by hand: M x = (3, -2), b = (3, -1):
    ||r|| = 1, ||M||_inf = 4, ||x|| = 1, ||b|| = 3  =>  1/7."""
    M = np.array([[2.0, 1.0], [1.0, -3.0]])
    assert S.backward_error(M, np.array([1.0, 1.0]), np.array([3.0, -1.0])) == pytest.approx(1 / 7)
    assert S.backward_error(M, np.array([1.0, 1.0]), np.array([3.0, -2.0])) == 0.0


def test_zero_pivot_component_is_zero():
    """A decoupled zero row/column is a zero pivot: its solution component is 0
    and the rest solves the nonsingular block."""
    rng = np.random.default_rng(5)
    B = rng.standard_normal((40, 40))
    B = B + B.T
    M = np.zeros((41, 41))
    M[:40, :40] = B
    b = np.concatenate([rng.standard_normal(40), [0.0]])
    fr = S.factor_chain(M, 41, "tpp", "tpp")
    x = S.solve(fr, b)
    assert x[40] == 0.0
    np.testing.assert_allclose(x[:40], np.linalg.solve(B, b[:40]), rtol=1e-10, atol=1e-12)


def test_two_by_two_pivots_in_solve():
    """Zero diagonal forces 2x2 pivots; the block solve must use them."""
    rng = np.random.default_rng(6)
    n = 30
    M = rng.standard_normal((n, n))
    M = M + M.T
    np.fill_diagonal(M, 0.0)
    fr = S.factor_chain(M, n, "tpp", "tpp")
    assert any((f["piv"] == orc.PIV_2X2_FIRST).any() for f in fr)
    b = rng.standard_normal(n)
    np.testing.assert_allclose(S.solve(fr, b), np.linalg.solve(M, b), rtol=1e-9, atol=1e-11)


def test_refinement_uses_the_true_matrix():
    """Factors of a perturbed matrix M + E (the effect of a low-precision Form)
    refine to the solution of M, not of M + E, with backward error <= 1e-14."""
    A, M = _embedded()
    rng = np.random.default_rng(8)
    E = rng.standard_normal(M.shape) * 1e-6
    E = E + E.T
    fr = S.factor_chain(M, A.shape[1], "strict", "tpp", Mfactor=M + E)
    b = rng.standard_normal(M.shape[0])
    x, hist, k = S.refine(M, fr, b)
    assert hist[0] > 1e-12 and hist[-1] <= 1e-14 and 1 <= k <= 10
    xr = np.linalg.solve(M, b)
    assert np.abs(x - xr).max() / np.abs(xr).max() <= 1e-10
    assert np.abs(x - np.linalg.solve(M + E, b)).max() / np.abs(xr).max() > 1e-8


def test_restricted_fails_where_strict_succeeds():
    """Section 7: restricted pivoting can fail to reach a backward error of
    1e-14 after ten refinement steps, while strict compressed pivoting and
    threshold partial pivoting do not.  The eight tiny columns of the
    n = 2000, p = 64 supernode are such a case."""
    A = inputs.single_small(0)
    M = inputs.two_node(A, 0)
    b = np.random.default_rng(1).standard_normal(M.shape[0])
    for mf, ok in [("strict", True), ("tpp", True), ("restricted", False)]:
        fr = S.factor_chain(M, 64, mf, "tpp")
        _, hist, _ = S.refine(M, fr, b)
        assert (hist[-1] <= 1e-14) == ok, (mf, hist)


def test_gradient_matches_finite_differences():
    """The oracle's gradient of w^T M^{-1} b with respect to b and to the stored
    lower triangle of M (an off-diagonal entry moves m_ij and m_ji together)
    against central differences of a dense library solve, every entry."""
    A = inputs.supernode(40, 8, seed=21, zero_diag_frac=0.25)
    M = inputs.two_node(A, 21)
    N = M.shape[0]
    rng = np.random.default_rng(22)
    b = rng.standard_normal(N)
    w = rng.standard_normal(N)
    fr = S.factor_chain(M, 8, "strict", "tpp", w_rest=16)
    x = S.solve(fr, b)
    gb, gM = S.solve_gradient(fr, x, w)

    def loss(Mm, bb):
        return w @ np.linalg.solve(Mm, bb)

    h = 1e-6
    fd_b = np.array([(loss(M, b + h * e) - loss(M, b - h * e)) / (2 * h) for e in np.eye(N)])
    np.testing.assert_allclose(gb, fd_b, rtol=1e-6, atol=1e-7 * np.abs(fd_b).max())
    fd_M = np.zeros_like(M)
    for i in range(N):
        for j in range(i + 1):
            E = np.zeros_like(M)
            E[i, j] = E[j, i] = h
            fd_M[i, j] = (loss(M + E, b) - loss(M - E, b)) / (2 * h)
    np.testing.assert_allclose(gM, fd_M, rtol=1e-5, atol=1e-7 * np.abs(fd_M).max())
    assert np.all(np.triu(gM, 1) == 0)
