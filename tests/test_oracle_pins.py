"""Pins of the CPU oracle to what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is a value printed
in the paper (worked examples, Figures 4.2 and 4.3, the counterexample of
Section 5), a theorem (Lemma 5.1, Theorem 5.2, Sylvester's law of inertia), an
identity (PAP^T = LDL^T, the Schur complement), a closed-form count
(Appendix A), a special case that reduces to another method, or an
independent restatement on tiny inputs.
"""
import numpy as np
import pytest

from listing_restated import restated_listing
from oracle import oracle as O
from paper_1305_2353_gb300 import inputs

METHODS = ["strict", "relaxed", "tpp", "restricted", "single_row"]


# --------------------------------------------------------------------------
# worked examples

def test_fig42_strict_compression(golden):
    g = golden("fig4_2_strict.txt")
    C, J = O.compress_strict(g["A21"])
    assert np.array_equal(C, g["C"])
    assert np.array_equal(J + 1, g["J"].ravel().astype(int))


def test_fig43_relaxed_compression(golden):
    g = golden("fig4_3_relaxed.txt")
    C, rows = O.compress_relaxed(g["A21"])
    assert np.array_equal(C, g["C"])
    assert np.array_equal(rows + 1, g["rows"].ravel().astype(int))


def test_counterexample_natural_pivots(golden):
    """Section 5: with 1x1 pivots in natural order, L reaches 2(1/u - eps) > 1/u."""
    g = golden("counterexample_relaxed.txt")
    u = g["u"]
    res = O.ldlt_fixed(g["A"], 2, [O.PIV_1X1, O.PIV_1X1])
    L, Dm, R = O.unpack(res, 2)
    assert np.array_equal(L, g["L"])
    assert np.array_equal(np.diag(Dm), [1.0, 1.0])
    assert np.abs(L).max() > 1.0 / u


def test_counterexample_under_listing1(golden):
    """The same matrix under Listing 1: the 2x2 candidate (1,2) trips the
    cancellation guard at equality (|detpiv| = |detpiv0|/2 = 1/2), column 2 is
    accepted as a 1x1 (2 >= u * 1/u), column 1 then fails (1/2 < 1) and is
    delayed.  Strict pivoting keeps every |l| <= 1/u (Theorem 5.2)."""
    g = golden("counterexample_relaxed.txt")
    u = g["u"]
    res = O.factor(g["A"], 2, "relaxed", u=u, log_cap=32)
    assert res["nelim"] == 1
    assert list(res["perm"]) == [1, 0]
    assert list(res["piv"]) == [O.PIV_1X1, O.PIV_DELAYED]
    kinds = [(O.LOG_KINDS[k], int(o)) for k, o in zip(res["log"]["kind"], res["log"]["outcome"])]
    assert ("2x2_det", 0) in kinds
    det = res["log"][res["log"]["kind"] == 2][0]
    assert det["lhs"] == det["rhs"] == 0.5
    for method in ("strict", "tpp"):
        r = O.factor(g["A"], 2, method, u=u)
        L, _, _ = O.unpack(r, 2)
        assert np.abs(L).max() <= 1.0 / u


# --------------------------------------------------------------------------
# exact factor identity and the threshold bound

def _recon_error(A, p, res):
    """max |(PAP^T) - (LDL^T + [0; R])| over the stored trapezoid, / max |A|."""
    n = A.shape[0]
    e = res["nelim"]
    L, Dm, R = O.unpack(res, p)
    Ap = O.permuted_supernode(A, p, res["perm"])
    rec = L @ Dm @ L[:p, :].T
    rec[:, e:] += R
    mask = np.ones((n, p), bool)
    mask[:p, :] = np.tril(np.ones((p, p), bool))
    err = np.abs(Ap - rec)[mask].max()
    return err / np.abs(A).max()


def _tough(n, p, seed):
    A = inputs.supernode(n, p, seed=seed, dist="normal", scale_cols=max(1, p // 6), scale=1e-3,
                         zero_diag_frac=0.2)
    A[p:, :] *= 5.0
    return A


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("seed", range(6))
def test_reconstruction(method, seed):
    n, p = 90, 17
    A = _tough(n, p, seed)
    res = O.factor(A, p, method)
    assert 0 <= res["nelim"] <= p
    assert sorted(res["perm"]) == list(range(p))
    # restricted pivoting ignores A21 when it tests pivots (Section 3.2), so its
    # L21 is unbounded and the rounding error grows with it
    tol = 1e-11 if method == "restricted" else 1e-13
    assert _recon_error(A, p, res) <= tol


@pytest.mark.parametrize("method", ["strict", "tpp", "single_row"])
@pytest.mark.parametrize("seed", range(8))
def test_threshold_bound_all_rows(method, seed):
    """Theorem 5.2 (strict) and the classical TPP bound: |l_ij| <= 1/u for every
    row, A21 included.  Theorem 5.2's proof holds for any partition of the A21
    rows into the sets J_j, so it covers single-row compression too (one set)."""
    n, p, u = 80, 16, 0.1
    A = _tough(n, p, seed)
    res = O.factor(A, p, method, u=u)
    L, _, _ = O.unpack(res, p)
    assert np.abs(L).max() <= (1.0 / u) * (1 + 1e-12)


def test_relaxed_can_break_bound_strict_cannot():
    """Relaxed compression is a heuristic (Section 5): rows left out of C are not
    tested, and on small random supernodes with large A21 rows the relaxed L
    exceeds 1/u; strict pivoting on the same inputs never does (Theorem 5.2)."""
    u = 0.1
    violations = 0
    for seed in range(300):
        rng = np.random.default_rng(seed)
        p = 3
        n = p + int(rng.integers(p + 1, 3 * p + 1))
        A = rng.standard_normal((n, p))
        A11 = np.tril(A[:p, :p])
        A[:p, :p] = A11 + np.tril(A11, -1).T
        A[p:] *= rng.choice([1, 5, 20])
        L, _, _ = O.unpack(O.factor(A, p, "relaxed", u=u), p)
        violations += np.abs(L).max(initial=0.0) > (1 / u) * (1 + 1e-9)
        Ls, _, _ = O.unpack(O.factor(A, p, "strict", u=u), p)
        assert np.abs(Ls).max(initial=0.0) <= (1 / u) * (1 + 1e-12)
    assert violations >= 1


# --------------------------------------------------------------------------
# Lemma 5.1 and the growth bound (5.1) at every stage

def _stages(A, p, u, tmode, outer, shadow):
    """Run Listing 1 stopped after each pivot block; yield (nelim, W, piv)."""
    A11 = np.tril(A[:p, :p]) + np.tril(A[:p, :p], -1).T
    Wfull = np.vstack([A11, outer, shadow])
    seen = set()
    out = []
    for s in range(0, p + 1):
        r = O.listing1(Wfull, p, rt=outer.shape[0], rs=shadow.shape[0], tmode=tmode, u=u,
                       stop_nelim=s)
        if r["nelim"] in seen:
            continue
        seen.add(r["nelim"])
        out.append(r)
    return out


@pytest.mark.parametrize("seed", range(5))
def test_lemma51_and_growth_strict(seed):
    n, p, u = 70, 12, 0.05
    A = _tough(n, p, seed)
    m = n - p
    C, J = O.compress_strict(A[p:, :])
    stages = _stages(A, p, u, O.UPD_ABS, C, A[p:, :])
    prev = None
    for r in stages:
        W, e = r["W"], r["nelim"]
        Cq = W[p:2 * p, :]
        Sh = W[2 * p:, :]
        # Lemma 5.1: |a^(q)(i,k)| <= c^(q)(J(i),k) for every column (eliminated
        # columns hold l and chat)
        bound = Cq[J, :]
        assert np.all(np.abs(Sh) <= bound * (1 + 1e-12) + 1e-300)
        # growth over the uneliminated part of [A11; C]
        mu = max(np.abs(W[e:p, e:p]).max(initial=0.0), np.abs(Cq[:, e:]).max(initial=0.0))
        if prev is not None:
            pe, pmu = prev
            k = e - pe
            kinds = r["piv"][pe:e]
            factor_ = 1.0 if kinds[0] == O.PIV_ZERO else (1 + k / u)
            assert mu <= pmu * factor_ * (1 + 1e-12)
        prev = (e, mu)


@pytest.mark.parametrize("seed", range(5))
def test_growth_tpp(seed):
    n, p, u = 60, 12, 0.05
    A = _tough(n, p, seed)
    stages = _stages(A, p, u, O.UPD_NORMAL, A[p:, :], np.zeros((0, p)))
    prev = None
    for r in stages:
        W, e = r["W"], r["nelim"]
        mu = max(np.abs(W[e:p, e:p]).max(initial=0.0), np.abs(W[p:, e:]).max(initial=0.0))
        if prev is not None:
            pe, pmu = prev
            k = e - pe
            factor_ = 1.0 if r["piv"][pe] == O.PIV_ZERO else (1 + k / u)
            assert mu <= pmu * factor_ * (1 + 1e-12)
        prev = (e, mu)


# --------------------------------------------------------------------------
# reductions to known cases

@pytest.mark.parametrize("seed", range(4))
def test_n_equals_p_all_methods_identical(seed):
    p = 24
    A = _tough(p, p, seed)
    ref = O.factor(A, p, "tpp")
    for method in ("strict", "relaxed", "restricted", "single_row"):
        r = O.factor(A, p, method)
        assert np.array_equal(r["perm"], ref["perm"])
        assert np.array_equal(r["piv"], ref["piv"])
        assert np.array_equal(r["A"], ref["A"])


@pytest.mark.parametrize("seed", range(6))
def test_relaxed_with_few_rows_is_tpp(seed):
    """m <= p: every A21 row lands in C, normal update, same maxima => TPP."""
    p = 20
    n = p + 7 + seed
    A = _tough(n, p, seed)
    r = O.factor(A, p, "relaxed")
    t = O.factor(A, p, "tpp")
    assert np.array_equal(r["perm"], t["perm"])
    assert np.array_equal(r["piv"], t["piv"])
    assert np.allclose(r["A"], t["A"], rtol=1e-11, atol=1e-11 * np.abs(A).max())


@pytest.mark.parametrize("seed", range(4))
def test_restricted_is_tpp_on_a11(seed):
    n, p = 50, 16
    A = _tough(n, p, seed)
    r = O.factor(A, p, "restricted")
    t = O.factor(A[:p, :], p, "tpp")
    assert np.array_equal(r["perm"], t["perm"])
    assert np.array_equal(r["piv"], t["piv"])
    assert np.array_equal(r["A"][:p], t["A"])


@pytest.mark.parametrize("seed", range(5))
def test_inertia_sylvester(seed):
    """n = p, no delays: the inertia of D equals that of A."""
    p = 30
    A = inputs.supernode(p, p, seed=seed)
    r = O.factor(A, p, "tpp")
    if r["nelim"] != p:
        pytest.skip("delays")
    _, Dm, _ = O.unpack(r, p)
    ev_d = np.linalg.eigvalsh(Dm)
    ev_a = np.linalg.eigvalsh(A)
    assert (ev_d > 0).sum() == (ev_a > 0).sum()
    assert (ev_d < 0).sum() == (ev_a < 0).sum()


# --------------------------------------------------------------------------
# Solve and Form identities

@pytest.mark.parametrize("method", ["strict", "relaxed", "restricted"])
@pytest.mark.parametrize("seed", range(4))
def test_solve_equals_fixed_pivot_elimination(method, seed):
    """L21 = A21 P^T (D11 L11^T)^-1 and the delayed update equal the rows of A21
    eliminated right-looking with the same pivots (shadow rows)."""
    n, p = 64, 14
    A = _tough(n, p, seed)
    r = O.factor(A, p, method)
    if method == "strict":
        outer, tmode = O.compress_strict(A[p:])[0], O.UPD_ABS
    elif method == "relaxed":
        outer, tmode = O.compress_relaxed(A[p:])[0], O.UPD_NORMAL
    else:
        outer, tmode = np.zeros((0, p)), O.UPD_NORMAL
    A11 = np.tril(A[:p, :p]) + np.tril(A[:p, :p], -1).T
    s = O.listing1(np.vstack([A11, outer, A[p:]]), p, rt=outer.shape[0], rs=n - p, tmode=tmode)
    assert np.array_equal(s["perm"], r["perm"])
    sh = s["W"][p + outer.shape[0]:, :]
    assert np.allclose(r["A"][p:], sh, rtol=1e-12, atol=1e-12 * np.abs(sh).max())


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("seed", range(3))
def test_form_is_schur_complement(method, seed):
    """S = L21 D11 L21^T = A21_e (P A11 P^T)_ee^{-1} A21_e^T (numpy solve)."""
    n, p = 70, 15
    A = _tough(n, p, seed)
    r = O.factor(A, p, method)
    e = r["nelim"]
    L, Dm, _ = O.unpack(r, p)
    S = O.form(r["A"][p:, :e], r["piv"][:e], r["D"])
    Ap = O.permuted_supernode(A, p, r["perm"])
    Aee = Ap[:e, :e]
    A2e = Ap[p:, :e]
    # zero pivots contribute nothing: drop them from the Schur complement
    keep = [j for j in range(e) if r["piv"][j] != O.PIV_ZERO]
    Sref = A2e[:, keep] @ np.linalg.solve(Aee[np.ix_(keep, keep)], A2e[:, keep].T)
    lo = np.tril(np.ones_like(S, bool))
    assert np.allclose(S[lo], Sref[lo], rtol=1e-9, atol=1e-9 * np.abs(Sref).max())
    assert np.all(np.triu(S, 1) == 0)
    ii, jj = np.nonzero(lo)
    sel = np.arange(0, len(ii), 37)
    v = O.form_entries(r["A"][p:, :e], r["piv"][:e], r["D"], ii[sel], jj[sel])
    assert np.allclose(v, S[ii[sel], jj[sel]], rtol=1e-13, atol=1e-13 * np.abs(S).max())


# --------------------------------------------------------------------------
# special cases

def test_zero_pivot_recorded():
    n, p = 20, 5
    A = inputs.supernode(n, p, seed=3)
    A[:, 2] = 0.0
    A[2, :p] = 0.0
    r = O.factor(A, p, "strict")
    j = list(r["perm"]).index(2)
    assert r["piv"][j] == O.PIV_ZERO
    assert r["D"][2 * j] == 0.0
    assert np.all(r["A"][j + 1:, j] == 0.0)


def test_relaxed_more_columns_than_rows():
    A21 = np.array([[3.0, -1.0, 2.0, 0.5], [1.0, 4.0, -2.0, 1.0]])
    C, rows = O.compress_relaxed(A21)
    assert list(rows) == [0, 1, -1, -1]
    assert np.array_equal(C[2:], np.zeros((2, 4)))
    assert np.array_equal(C[0], A21[0]) and np.array_equal(C[1], A21[1])


def _relaxed_restated(A21):
    """Section 4.2 restated directly: column by column, the largest |a(i, j)|
    among rows not yet taken (the lowest row on ties) is taken; its signed row
    is row j of C; with every row taken, the remaining rows of C are zero."""
    m, p = A21.shape
    taken = np.zeros(m, dtype=bool)
    C = np.zeros((p, p))
    rows = -np.ones(p, dtype=np.int64)
    for j in range(p):
        if taken.all():
            break
        mag = np.where(taken, -1.0, np.abs(A21[:, j]))
        r = int(np.argmax(mag))          # first maximum: the lowest row on ties
        taken[r] = True
        rows[j] = r
        C[j] = A21[r]
    return C, rows


@pytest.mark.parametrize("seed", range(6))
def test_relaxed_compression_brute_force(seed):
    """Tie-heavy inputs (small integers) of several shapes, including fewer rows
    than columns: the oracle's relaxed compression equals the restatement."""
    rng = np.random.default_rng(100 + seed)
    for m, p in ((1, 1), (3, 5), (7, 4), (40, 6), (200, 16), (5, 5)):
        A21 = rng.integers(-3, 4, size=(m, p)).astype(float)
        C, rows = O.compress_relaxed(A21)
        Cw, rw = _relaxed_restated(A21)
        assert np.array_equal(np.asarray(rows, dtype=np.int64), rw), (m, p)
        assert np.array_equal(C, Cw), (m, p)


def test_strict_compression_entries_are_exact_maxima():
    rng = np.random.default_rng(5)
    A21 = rng.standard_normal((300, 9))
    C, J = O.compress_strict(A21)
    for j in range(9):
        rows = np.nonzero(J == j)[0]
        want = np.abs(A21[rows]).max(axis=0) if len(rows) else np.zeros(9)
        assert np.array_equal(C[j], want)
    assert np.array_equal(J, np.argmax(np.abs(A21), axis=1))


@pytest.mark.parametrize("seed", range(4))
def test_strict_compression_ties_brute_force(seed):
    """Tie-heavy inputs (small integers, whole zero rows): J(i) is the lowest
    column of a row's largest |a| (an all-zero row goes to column 0), and C's
    row j holds the column maxima of |a| over the rows with J(i) = j, zero when
    none (eq. (4.1))."""
    rng = np.random.default_rng(200 + seed)
    for m, p in ((1, 1), (6, 3), (50, 7), (300, 12)):
        A21 = rng.integers(-2, 3, size=(m, p)).astype(float)
        A21[::4] = 0.0
        C, J = O.compress_strict(A21)
        Jw = np.array([int(np.argmax(np.abs(r))) for r in A21])
        assert np.array_equal(np.asarray(J), Jw), (m, p)
        for j in range(p):
            sel = np.abs(A21[Jw == j])
            want = sel.max(axis=0) if len(sel) else np.zeros(p)
            assert np.array_equal(C[j], want), (m, p, j)


def test_app_a_operation_count():
    """Appendix A: with every pivot a 2x2 accepted on its first test, the counted
    operations equal TPP_ops(n,p) = 29/6 p - 3/4 p^2 - 1/3 p^3 + 2np + 1/2 np^2."""
    for n, p in ((40, 8), (100, 12), (64, 16)):
        A = np.zeros((n, p))
        for q in range(0, p, 2):
            A[q + 1, q] = A[q, q + 1] = 1.0
        rng = np.random.default_rng(n + p)
        A[p:, :] = rng.uniform(-1e-3, 1e-3, (n - p, p))
        r = O.factor(A, p, "tpp", u=0.01)
        st = r["stats"]
        assert st["accepted_2x2"] == p // 2 and st["tests_2x2"] == p // 2
        counted = st["ops_colmax"] + st["ops_test"] + st["ops_apply"] + st["ops_update"]
        closed = 29 * p / 6 - 3 * p * p / 4 - p ** 3 / 3 + 2 * n * p + n * p * p / 2
        assert counted == round(closed)


# --------------------------------------------------------------------------
# brute force against an independent restatement of Listing 1

def _tiny_cases():
    rng = np.random.default_rng(1234)
    for case in range(300):
        p = int(rng.integers(1, 6))
        r = int(rng.integers(0, 6))
        A11 = rng.standard_normal((p, p))
        A11 = np.tril(A11) + np.tril(A11, -1).T
        # sprinkle zeros and tiny diagonals to force rejections and 2x2 pivots
        mask = rng.random((p, p)) < 0.25
        mask = np.tril(mask) | np.tril(mask, -1).T
        A11[mask] = 0.0
        d = rng.random(p) < 0.3
        A11[d, d] *= 1e-3
        outer = rng.standard_normal((r, p)) * rng.choice([0.1, 1, 30], size=(r, 1))
        yield case, p, A11, outer


@pytest.mark.parametrize("mode", ["tpp", "strict_abs"])
def test_brute_force_restated_listing(mode):
    u = 0.1
    for case, p, A11, outer in _tiny_cases():
        tmode = O.UPD_ABS if mode == "strict_abs" else O.UPD_NORMAL
        if mode == "strict_abs":
            outer = np.abs(outer)
        res = O.listing1(np.vstack([A11, outer]), p, rt=outer.shape[0], tmode=tmode, u=u)
        order, kinds = restated_listing(A11, outer, u, strict_abs=(mode == "strict_abs"))
        e = res["nelim"]
        assert list(res["perm"][:e]) == order, (case, p)
        code = {"1": O.PIV_1X1, "2a": O.PIV_2X2_FIRST, "2b": O.PIV_2X2_SECOND, "z": O.PIV_ZERO}
        for pos in range(e):
            assert res["piv"][pos] == code[kinds[res["perm"][pos]]], (case, pos)
        assert all(kinds[c] == "d" for c in res["perm"][e:])


# --------------------------------------------------------------------------
# hand-derived cases at the edges of the tests

def test_1x1_threshold_equality_accepts():
    """eq. (2.1) reads |a(q,q)| >= u max|a(i,q)|: equality accepts.  With
    u = 2^-7, a11 = 1 and the only other entry 128, u*128 = 1 exactly."""
    A = np.array([[1.0], [128.0]])
    r = O.factor(A, 1, "tpp", u=2.0 ** -7)
    assert r["nelim"] == 1 and r["piv"][0] == O.PIV_1X1
    assert r["A"][1, 0] == 128.0


def test_partner_ties_go_to_lowest_index():
    """A11 = [[0,0,1],[0,0,1],[1,1,0]]: (1,2) fails as 2x2 (all zero) and column
    2 fails as 1x1; candidate 3 ties |a(3,1)| = |a(3,2)| = 1 and must pair with
    column 1.  (1,3) passes (det -1, growth 1), then column 2 is a zero pivot."""
    A = np.array([[0.0, 0, 1], [0, 0, 1], [1, 1, 0]])
    r = O.factor(A, 3, "tpp", u=0.1)
    assert list(r["perm"]) == [0, 2, 1]
    assert list(r["piv"]) == [O.PIV_2X2_FIRST, O.PIV_2X2_SECOND, O.PIV_ZERO]


def test_2x2_column_maxima_exclude_partner():
    """Listing 1: maxt, maxm exclude rows t and m.  A11 = [[0,1],[1,1]], A21 row
    (3.5, 0.1), u = 1/4: maxt = 3.5, maxm = 0.1, |D^-1| (maxt, maxm) =
    (3.6, 3.5) <= 4, so (1,2) is a 2x2 pivot.  Counting row t in maxm would give
    maxm = 1 and 4.5 > 4."""
    A = np.array([[0.0, 1.0], [1.0, 1.0], [3.5, 0.1]])
    r = O.factor(A, 2, "tpp", u=0.25, log_cap=16)
    assert list(r["piv"]) == [O.PIV_2X2_FIRST, O.PIV_2X2_SECOND]
    g = r["log"][r["log"]["kind"] == 4][0]
    assert abs(g["lhs"] - 3.6) < 1e-15 and g["rhs"] == 4.0


# --------------------------------------------------------------------------
# single-row compression (Section 4.1, closing remark): eq. (4.1) with the one
# set J = all A21 rows, i.e. C is the row of column maxima of |A21|

def test_single_row_on_fig42(golden):
    """The worked example of Figure 4.2 compressed with one set: the column
    maxima of its A21, which are also the column maxima of the strict C the
    figure prints."""
    g = golden("fig4_2_strict.txt")
    A21 = g["A21"]
    p = A21.shape[1]
    A = np.vstack([np.eye(p) * 50.0, A21])
    r = O.factor(A, p, "single_row")
    assert np.array_equal(r["C"][0], [4.0, 10.0, 10.0])
    assert np.array_equal(r["C"][0], g["C"].max(axis=0))
    assert not r["C"][1:].any()


@pytest.mark.parametrize("seed", range(4))
def test_single_row_is_column_max_of_strict(seed):
    A = _tough(400, 24, seed)
    s1 = O.factor(A, 24, "single_row")
    st = O.factor(A, 24, "strict")
    assert np.array_equal(s1["C"][0], st["C"].max(axis=0))


@pytest.mark.parametrize("seed", range(4))
def test_single_row_with_one_a21_row_is_strict(seed):
    """With one A21 row, strict compression has a single nonzero row, |a21|,
    which is also the single row: the factorizations coincide bit for bit."""
    p = 18
    A = _tough(p + 1, p, seed)
    s1 = O.factor(A, p, "single_row")
    st = O.factor(A, p, "strict")
    assert np.array_equal(s1["perm"], st["perm"]) and np.array_equal(s1["piv"], st["piv"])
    assert np.array_equal(s1["A"], st["A"]) and np.array_equal(s1["D"], st["D"])


def test_single_row_rejects_more_than_strict():
    """The paper's observation: one row over-estimates the growth, and most
    pivots beyond the first few are rejected (here: over a seeded sample of the
    uneven N(0,1) fronts with many A21 rows, fewer eliminated than strict)."""
    fr = inputs.batch(200, seed=3)
    tot_s1 = tot_st = 0
    for A in fr:
        if A.shape[0] < 4 * A.shape[1]:
            continue
        tot_s1 += O.factor(A, A.shape[1], "single_row")["nelim"]
        tot_st += O.factor(A, A.shape[1], "strict")["nelim"]
    assert tot_s1 < tot_st
