"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: the strict compressed matrix and the row sets J are bit-exact; pivot
sequences, pivot kinds and nelim are identical (every case is chosen so that no
threshold test of the oracle lies within 1e-10, relative, of its bound, and a
case that does fails); L, D, the delayed block and S agree within FP64 rounding
(1e-10 relative to the largest entry); the GPU factor satisfies
||PAP^T - LDL^T|| <= 1e-14 (max-abs norm over the stored trapezoid, delayed
block counted as residual) relative to max |L||D||L^T| -- the growth-normalised
backward error, which equals the plain ||A||-normalised one when the factor
does not grow -- and its plain (||A||-normalised) backward error is at most
twice the oracle's own on the same input plus 8 units of FP64 rounding at the
factor's growth.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1305_2353_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1305_2353_gb300 import build, ctp
    build.build()
    return ctp.Context(0)


def min_margin(log):
    if len(log) == 0:
        return np.inf
    lhs, rhs = np.abs(log["lhs"]), np.abs(log["rhs"])
    den = np.maximum(np.maximum(lhs, rhs), 1e-300)
    return float(np.min(np.abs(lhs - rhs) / den))


def run_gpu(ctx, A, p, pivot="strict", smode="none", u=0.01):
    from paper_1305_2353_gb300 import ctp
    opt = ctp.options(u=u, pivot=pivot, smode=smode)
    sn = ctp.Supernode(ctx, A, p, opt)
    sn.run()
    torch.cuda.synchronize()
    return sn.result()


def factor_errors(A, p, res):
    """(growth-normalised error, raw error, growth) of a factored supernode over
    the stored trapezoid: the error is max |PAP^T - (LDL^T + [0; R])|, divided by
    max(|L||D||L^T| + |R|) (at least max |A|) or by max |A|; the growth is
    max(|L||D||L^T| + |R|) / max |A|."""
    n = A.shape[0]
    e = res["nelim"]
    L, Dm, R = O.unpack(res, p)
    Ap = O.permuted_supernode(A, p, res["perm"])
    rec = (L @ Dm) @ L[:p, :].T
    scale = np.abs(L) @ (np.abs(Dm) @ np.abs(L[:p, :].T))
    rec[:, e:] += R
    scale[:, e:] += np.abs(R)
    mask = np.ones((n, p), bool)
    mask[:p, :] = np.tril(np.ones((p, p), bool))
    err = np.abs(Ap - rec)[mask].max()
    amax = max(np.abs(A).max(), 1e-300)
    smax = scale[mask].max()
    return err / max(smax, amax), err / amax, smax / amax


def check_backward_error(A, p, got, ref):
    """The GPU factor's growth-normalised backward error is <= 1e-14, and its raw
    error is at most twice the oracle's own raw error on the same input plus 8
    units of FP64 rounding at the factor's growth (the two round in different
    orders, the GPU with fused multiply-adds)."""
    g, raw_g, growth = factor_errors(A, p, got)
    _, raw_o, _ = factor_errors(A, p, ref)
    assert g <= 1e-14
    assert raw_g <= 2.0 * raw_o + 8.0 * 2.0 ** -52 * growth, (raw_g, raw_o, growth)


def compare(ref, got, p, A, check_recon=True):
    """Parity of one GPU factorization with the oracle's.  Pivot sequence, kinds
    and nelim must be identical, and L, D within 1e-10.  The cases in the suite
    are chosen so that no logged threshold test of the oracle lies within 1e-10
    (relative) of its bound; a case that does would make pivot parity depend on
    FP64 rounding order, so it fails here instead of being skipped.  With
    check_recon the backward error is checked as check_backward_error states."""
    assert got["info"] == 0
    assert ref["log_len"] <= len(ref["log"]) or len(ref["log"]) == 0, "oracle decision log truncated"
    margin = min_margin(ref["log"])
    assert margin > 1e-10, f"a threshold test lies within {margin:.1e} of its bound: pick another case"
    assert got["nelim"] == ref["nelim"]
    assert np.array_equal(got["perm"], ref["perm"])
    assert np.array_equal(got["piv"], ref["piv"])
    Ag, Ar = got["A"].copy(), ref["A"].copy()
    # the strict upper triangle of the A11 block is unspecified
    iu = np.triu_indices(p, 1)
    Ag[:p][iu] = 0.0
    Ar[:p][iu] = 0.0
    scale = max(np.abs(Ar).max(), 1.0)
    assert np.allclose(Ag, Ar, rtol=1e-10, atol=1e-10 * scale)
    assert np.allclose(got["D"], ref["D"], rtol=1e-10, atol=1e-10 * np.abs(ref["D"]).max())
    if check_recon:
        check_backward_error(A, p, got, ref)


# --------------------------------------------------------------------------- K1

@pytest.mark.parametrize("m,p", [(5, 3), (1, 1), (17, 1), (100, 7), (1000, 64), (4099, 128),
                                 (20011, 256), (33, 200)])
def test_compress_strict_bit_exact(ctx, m, p):
    from paper_1305_2353_gb300 import ctp
    if (m, p) == (5, 3):
        A21 = np.array([[1, 10, 10], [2, 3, 4], [0, 10, -3], [4, -5, 4], [0, -6, 8]], float)
    else:
        A21 = np.random.default_rng(m * 7 + p).standard_normal((m, p))
        A21[::5, 0] = 0.0  # exact ties between columns
        A21[::7, -1] = A21[::7, 0]
    Cref, Jref = O.compress_strict(A21)
    dA = ctp.colmajor(A21)
    C = torch.empty(p * p, dtype=torch.float64, device="cuda")
    J = torch.empty(m, dtype=torch.int32, device="cuda")
    ws = ctx.compress_strict(dA, m, p, m, C, J)
    torch.cuda.synchronize()
    assert ctx.read_info(ws) == 0
    Cg = C.cpu().numpy().reshape(p, p)  # row-major
    assert np.array_equal(Cg, Cref)
    assert np.array_equal(J.cpu().numpy(), Jref)


def test_compress_strict_flags_nonfinite(ctx):
    from paper_1305_2353_gb300 import ctp
    A21 = np.ones((50, 4))
    A21[13, 2] = np.inf
    C = torch.empty(16, dtype=torch.float64, device="cuda")
    ws = ctx.compress_strict(ctp.colmajor(A21), 50, 4, 50, C)
    assert ctx.read_info(ws) == ctp.CTP_ENONFINITE


@pytest.mark.parametrize("m,p", [(5, 3), (1, 1), (3, 8), (0, 4), (100, 7), (1000, 64),
                                 (40000, 256), (70001, 33)])
def test_compress_relaxed_bit_exact(ctx, m, p):
    from paper_1305_2353_gb300 import ctp
    if (m, p) == (5, 3):
        A21 = np.array([[1, 10, 10], [2, 3, 4], [0, 10, -3], [4, -5, 4], [0, -6, 8]], float)
    else:
        rng = np.random.default_rng(m * 3 + p)
        A21 = rng.standard_normal((m, p))
        if m > 10:
            A21[rng.random((m, p)) < 0.3] = 0.0  # ties at zero
            A21[::11, :] = np.round(A21[::11, :])  # ties between rows
    Cref, rref = O.compress_relaxed(A21) if m > 0 else (np.zeros((p, p)), -np.ones(p, np.int32))
    dA = ctp.colmajor(A21) if m > 0 else torch.zeros((p, 1), dtype=torch.float64, device="cuda")
    C = torch.empty(p * p, dtype=torch.float64, device="cuda")
    rows = torch.empty(p, dtype=torch.int32, device="cuda")
    ws = ctx.compress_relaxed(dA, m, p, max(m, 1), C, rows)
    torch.cuda.synchronize()
    assert ctx.read_info(ws) == 0
    assert np.array_equal(rows.cpu().numpy(), rref)
    assert np.array_equal(C.cpu().numpy().reshape(p, p), Cref)


def _relaxed_input(kind, m, p, rng):
    A21 = rng.standard_normal((m, p))
    if kind == "levels":          # a handful of values: ties everywhere
        A21 = rng.integers(-3, 4, size=(m, p)).astype(float)
    elif kind == "constant":      # every entry of a column ties
        A21 = np.ones((m, p))
        A21[::3] *= -1.0
    elif kind.startswith("front_heavy"):
        # the leading rows are 100x larger: the blocks that hold column maxima
        # are full of candidates (more than one CTA's buffer in the second case)
        lead = 2000 if kind == "front_heavy" else 6000
        A21[:lead] *= 100.0
    return A21


@pytest.mark.parametrize("kind,m,p", [("random", 10000, 256), ("random", 300, 64), ("random", 50, 64),
                                      ("random", 4097, 256), ("levels", 5000, 64), ("constant", 9000, 40),
                                      ("front_heavy", 60000, 256), ("front_heavy_overflow", 60000, 256)])
def test_compress_relaxed_candidate_paths(ctx, kind, m, p):
    """Relaxed compression through block maxima of 1 to 64 rows (the block
    size follows m / p), candidate blocks read again, and the streaming
    fallback when ties or crowded blocks overflow the candidate buffer: C and
    the chosen rows bit-exact with the oracle."""
    from paper_1305_2353_gb300 import ctp
    A21 = _relaxed_input(kind, m, p, np.random.default_rng(m + p))
    Cref, rref = O.compress_relaxed(A21)
    C = torch.empty(p * p, dtype=torch.float64, device="cuda")
    rows = torch.empty(p, dtype=torch.int32, device="cuda")
    ws = ctx.compress_relaxed(ctp.colmajor(A21), m, p, m, C, rows)
    torch.cuda.synchronize()
    assert ctx.read_info(ws) == 0
    assert np.array_equal(rows.cpu().numpy(), rref)
    assert np.array_equal(C.cpu().numpy().reshape(p, p), Cref)


def test_compress_relaxed_flags_nonfinite(ctx):
    from paper_1305_2353_gb300 import ctp
    A21 = np.random.default_rng(3).standard_normal((700, 8))
    A21[613, 5] = -np.inf
    C = torch.empty(64, dtype=torch.float64, device="cuda")
    rows = torch.empty(8, dtype=torch.int32, device="cuda")
    ws = ctx.compress_relaxed(ctp.colmajor(A21), 700, 8, 700, C, rows)
    assert ctx.read_info(ws) == ctp.CTP_ENONFINITE


# --------------------------------------------------------------------------- full path

def _tough(n, p, seed):
    A = inputs.supernode(n, p, seed=seed, dist="normal", scale_cols=max(1, p // 6), scale=1e-3,
                         zero_diag_frac=0.2)
    A[p:, :] *= 5.0
    return A


CASES = [(1, 1), (2, 2), (3, 1), (30, 30), (300, 17), (513, 33), (1200, 100), (800, 200),
         (3000, 256), (700, 129)]


@pytest.mark.parametrize("pivot", ["strict", "relaxed", "restricted", "tpp", "single_row"])
@pytest.mark.parametrize("n,p", CASES)
@pytest.mark.parametrize("seed", [0, 1])
def test_factor_matches_oracle(ctx, pivot, n, p, seed):
    A = _tough(n, p, seed)
    ref = O.factor(A, p, pivot, log_cap=200000)
    got = run_gpu(ctx, A, p, pivot)
    compare(ref, got, p, A)


def _boundary_case(kind, s, delta):
    """A tiny supernode whose first threshold test of the given kind sits a
    relative distance of about delta from its bound, on the side s (+1 or -1):
    1x1: |a_mm| = u (1 + s delta) against u max|a21| = u (Listing 1's 1x1 test);
    det: the 2x2 [[1, x], [x, 1]] with x^2 = (1 + s delta) / 2 against the
         cancellation guard |det| <= max(|d0|, |d1|) / 2;
    grow: the 2x2 [[1, .3], [.3, -1]] with both column maxima v = 109/1.3 (1 + s delta)
         against the growth bound |D^-1| (maxt, maxm)^T <= 1/u (eq. (2.2))."""
    if kind == "1x1":
        return np.array([[0.01 * (1.0 + s * delta)], [1.0]]), 1
    if kind == "det":
        x = np.sqrt(0.5 * (1.0 + s * delta))
        return np.array([[1.0, x], [x, 1.0], [0.01, 0.01]]), 2
    v = 109.0 / 1.3 * (1.0 + s * delta)
    return np.array([[1.0, 0.3], [0.3, -1.0], [v, v]]), 2


@pytest.mark.parametrize("kind,logkind", [("1x1", 5), ("det", 2), ("grow", 4)])
@pytest.mark.parametrize("pivot", ["strict", "relaxed", "tpp"])
def test_threshold_tests_near_their_bounds(ctx, kind, logkind, pivot):
    """Decisions on both sides of each threshold test's bound, from far (1e-2)
    to within 1e-8 of it: the kernels decide the clear cases in FP32 with 2^-16
    margins and leave the close ones to the FP64 test; either way the outcome,
    pivots and factors equal the oracle's (and the two sides differ)."""
    for delta in (1e-2, 1e-4, 3e-6, 1e-8):
        outcomes = []
        for s in (1.0, -1.0):
            A, p = _boundary_case(kind, s, delta)
            ref = O.factor(A, p, pivot, log_cap=1000)
            first = [e for e in ref["log"] if e["kind"] == logkind]
            assert first, (kind, pivot, delta, s)
            outcomes.append(int(first[0]["outcome"]))
            compare(ref, run_gpu(ctx, A, p, pivot), p, A)
        assert outcomes[0] != outcomes[1], (kind, pivot, delta, outcomes)


def test_single_small_workload(ctx):
    """n = 2000, p = 64, N(0,1), eight A11 rows/columns scaled by 1e-8."""
    for seed in range(3):
        A = inputs.single_small(seed)
        ref = O.factor(A, 64, "strict", log_cap=200000)
        got = run_gpu(ctx, A, 64, "strict")
        assert ref["nelim"] < 64  # the scaled columns are delayed
        compare(ref, got, 64, A)


@pytest.mark.parametrize("smode,rtol", [("fp64", 1e-11), ("fp32", 2e-6), ("fp64_packed", 1e-11),
                                        ("fp32_packed", 2e-6)])
@pytest.mark.parametrize("n,p", [(600, 40), (2000, 64), (1500, 130)])
def test_form_matches_oracle(ctx, smode, rtol, n, p):
    A = _tough(n, p, 3)
    ref = O.factor(A, p, "strict")
    got = run_gpu(ctx, A, p, "strict", smode=smode)
    e = ref["nelim"]
    S = O.form(ref["A"][p:, :e], ref["piv"][:e], ref["D"])
    lo = np.tril(np.ones_like(S, dtype=bool))
    scale = np.abs(S).max()
    assert np.allclose(got["S"][lo], S[lo], rtol=rtol, atol=rtol * scale)
    # the strict upper triangle is never written
    assert np.all(np.triu(got["S"], 1) == 0)


def test_large_supernode_relaxed_full_size(ctx):
    """n = 200000, p = 256, U[-1,1]: relaxed compression bit-exact and the whole
    relaxed factorization against the oracle (every pivot is accepted here)."""
    from paper_1305_2353_gb300 import ctp
    n, p = 200000, 256
    A = inputs.single_large(0)
    m = n - p
    Cref, rref = O.compress_relaxed(A[p:])
    dA = ctp.colmajor(A)
    C = torch.empty(p * p, dtype=torch.float64, device="cuda")
    rows = torch.empty(p, dtype=torch.int32, device="cuda")
    ctx.compress_relaxed(dA[:, p:], m, p, n, C, rows)
    torch.cuda.synchronize()
    assert np.array_equal(rows.cpu().numpy(), rref)
    assert np.array_equal(C.cpu().numpy().reshape(p, p), Cref)
    del dA
    ref = O.factor(A, p, "relaxed", log_cap=400000)
    got = run_gpu(ctx, A, p, "relaxed")
    assert ref["nelim"] == p
    compare(ref, got, p, A, check_recon=False)
    rows_s = np.r_[0:p + 64, np.random.default_rng(1).choice(np.arange(p, n), 4000, replace=False)]
    sub, sref = dict(got), dict(ref)
    sub["A"], sref["A"] = got["A"][rows_s], ref["A"][rows_s]
    check_backward_error(A[rows_s], p, sub, sref)
    _form_fp64_packed_full_size(ctx, A, ref)


def _form_fp64_packed_full_size(ctx, A, ref):
    """The benchmarked FP64 Form at full size: S = L21 D11 L21^T of the
    n = 200000, p = 256 relaxed supernode, lower-packed FP64 (m(m+1)/2 =
    1.99e10 entries, 160 GB), sampled entries against the oracle's
    form_entries on the oracle's own factor: the diagonal, the first and last
    rows, the last 64 x 64 tile and 10^4 random entries, each within 1e-11 of
    sum_k |L21(i,k)| |(L21 D11)(j,k)|."""
    from paper_1305_2353_gb300 import ctp
    n, p = A.shape
    m, e = n - p, ref["nelim"]
    opt = ctp.options(pivot="relaxed", smode="fp64_packed")
    dA = ctp.colmajor(A)
    perm = torch.empty(p, dtype=torch.int32, device="cuda")
    piv = torch.empty(p, dtype=torch.int32, device="cuda")
    D = torch.empty(2 * p, dtype=torch.float64, device="cuda")
    nel = torch.empty(1, dtype=torch.int32, device="cuda")
    S = torch.empty(m * (m + 1) // 2, dtype=torch.float64, device="cuda")
    ws = ctx.factor_supernode(dA, n, p, n, opt, perm, piv, D, nel, S, m)
    torch.cuda.synchronize()
    assert ctx.read_info(ws) == 0 and int(nel.cpu()[0]) == e
    del dA, ws
    rng = np.random.default_rng(11)
    ii, jj = rng.integers(0, m, 10000), rng.integers(0, m, 10000)
    ii, jj = np.maximum(ii, jj), np.minimum(ii, jj)
    t = np.arange(m - 64, m)
    ti, tj = np.meshgrid(t, t, indexing="ij")
    keep = ti >= tj
    diag = np.r_[0:64, rng.integers(0, m, 200), m - 64:m]
    ii = np.r_[ii, ti[keep], diag, np.arange(0, m, 997), np.full(64, m - 1)]
    jj = np.r_[jj, tj[keep], diag, np.zeros(len(range(0, m, 997)), np.int64), np.arange(64)]
    lin = jj * m - jj * (jj - 1) // 2 + (ii - jj)
    got = S[torch.as_tensor(lin, device="cuda")].cpu().numpy()
    del S
    torch.cuda.empty_cache()
    L21 = ref["A"][p:, :e]
    want = O.form_entries(L21, ref["piv"][:e], ref["D"], ii, jj)
    _, Dm, _ = O.unpack(ref, p)
    Wd = L21 @ Dm
    bound = np.einsum("tk,tk->t", np.abs(L21[ii]), np.abs(Wd[jj]))
    assert np.all(np.abs(got - want) <= 1e-11 * bound)


def test_large_supernode_tpp_full_size(ctx):
    """Full-column threshold partial pivoting (the comparator) at n = 200000,
    p = 256 against the oracle's Listing 1 on all rows."""
    n, p = 200000, 256
    A = inputs.single_large(0)
    ref = O.factor(A, p, "tpp", log_cap=400000)
    got = run_gpu(ctx, A, p, "tpp")
    assert ref["nelim"] == p
    compare(ref, got, p, A, check_recon=False)
    rows_s = np.r_[0:p + 64, np.random.default_rng(2).choice(np.arange(p, n), 4000, replace=False)]
    sub, sref = dict(got), dict(ref)
    sub["A"], sref["A"] = got["A"][rows_s], ref["A"][rows_s]
    check_backward_error(A[rows_s], p, sub, sref)


def test_large_supernode_full_size(ctx):
    """n = 200000, p = 256, entries U[-1,1], u = 0.01: the benchmarked shape.
    C and J bit-exact on all rows; pivots, nelim and the whole factor against
    the oracle."""
    from paper_1305_2353_gb300 import ctp
    n, p = 200000, 256
    A = inputs.single_large(0)
    m = n - p
    Cref, Jref = O.compress_strict(A[p:])
    dA = ctp.colmajor(A)
    C = torch.empty(p * p, dtype=torch.float64, device="cuda")
    J = torch.empty(m, dtype=torch.int32, device="cuda")
    ctx.compress_strict(dA[:, p:], m, p, n, C, J)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().reshape(p, p), Cref)
    assert np.array_equal(J.cpu().numpy(), Jref)
    del dA
    ref = O.factor(A, p, "strict", log_cap=400000)
    got = run_gpu(ctx, A, p, "strict")
    compare(ref, got, p, A, check_recon=False)
    rows = np.r_[0:p + 64, np.random.default_rng(0).choice(np.arange(p, n), 4000, replace=False)]
    sub, sref = dict(got), dict(ref)
    sub["A"], sref["A"] = got["A"][rows], ref["A"][rows]
    check_backward_error(A[rows], p, sub, sref)


# --------------------------------------------------------------------------- errors

def test_argument_errors(ctx):
    from paper_1305_2353_gb300 import ctp
    A = _tough(100, 10, 0)
    opt = ctp.options()
    sn = ctp.Supernode(ctx, A, 10, opt)
    with pytest.raises(ctp.CtpError) as e:
        ctx.factor_supernode(sn.A, 100, 10, 50, opt, sn.perm, sn.piv, sn.D, sn.nelim, ws=sn.ws)
    assert e.value.code == ctp.CTP_EINVAL
    with pytest.raises(ctp.CtpError) as e:
        ctx.factor_supernode(sn.A, 100, 10, 100, opt, sn.perm, sn.piv, sn.D, sn.nelim,
                             ws=sn.ws[:16])
    assert e.value.code == ctp.CTP_ENOMEM
    big = ctp.options()
    with pytest.raises(ctp.CtpError) as e:
        ctx.factor_supernode(sn.A, 400, 300, 400, big, sn.perm, sn.piv, sn.D, sn.nelim, ws=sn.ws)
    assert e.value.code in (ctp.CTP_EUNSUPPORTED, ctp.CTP_ENOMEM)
    bad_u = ctp.options(u=0.7)
    with pytest.raises(ctp.CtpError) as e:
        ctx.factor_supernode(sn.A, 100, 10, 100, bad_u, sn.perm, sn.piv, sn.D, sn.nelim, ws=sn.ws)
    assert e.value.code == ctp.CTP_EINVAL


def test_nonfinite_input_flagged(ctx):
    A = _tough(200, 12, 1)
    A[150, 3] = np.nan
    got = run_gpu(ctx, A, 12, "strict")
    from paper_1305_2353_gb300 import ctp
    assert got["info"] == ctp.CTP_ENONFINITE


# --------------------------------------------------------------------------- tensor-core Form

def _bf16_bound(Wd, L21):
    """|W||L|^T: the scale of the rounding error of a BF16-operand, FP32-accumulate
    product (each operand is rounded once, relative error 2^-9 each)."""
    return np.abs(Wd) @ np.abs(L21).T


@pytest.mark.parametrize("pivot,smode", [("strict", "fp32"), ("relaxed", "fp32"),
                                         ("relaxed", "fp32_packed"), ("relaxed", "fp32_tiled"),
                                         ("strict", "fp32_tiled")])
@pytest.mark.parametrize("n,p", [(600, 40), (2000, 64), (1500, 130), (3000, 256), (700, 200)])
def test_form_tensor_cores_bf16(ctx, pivot, smode, n, p):
    """S from the tcgen05 kernel (BF16 operands, FP32 accumulation) against the
    oracle's FP64 S: |dS| <= 2^-7 |W21||L21|^T elementwise (lower triangle)."""
    from paper_1305_2353_gb300 import ctp
    A = _tough(n, p, 5)
    ref = O.factor(A, p, pivot)
    opt = ctp.options(pivot=pivot, prec="bf16", smode=smode)
    sn = ctp.Supernode(ctx, A, p, opt)
    sn.run()
    torch.cuda.synchronize()
    got = sn.result()
    assert got["info"] == 0
    e = ref["nelim"]
    assert got["nelim"] == e
    L21 = ref["A"][p:, :e]
    _, Dm, _ = O.unpack(ref, p)
    Wd = L21 @ Dm
    S = O.form(L21, ref["piv"][:e], ref["D"])
    lo = np.tril(np.ones_like(S, dtype=bool))
    bound = _bf16_bound(Wd, L21)
    err = np.abs(got["S"] - S)
    assert np.all(err[lo] <= 2.0 ** -7 * bound[lo] + 1e-30)
    assert np.all(np.triu(got["S"], 1) == 0)


@pytest.mark.parametrize("prec,tol,gain", [("bf16x3", 2.0 ** -13, 64), ("bf16x6", 2.0 ** -19, 4096)])
@pytest.mark.parametrize("smode", ["fp32", "fp32_packed", "fp32_tiled"])
@pytest.mark.parametrize("n,p", [(600, 40), (2000, 64), (3000, 256), (700, 200)])
def test_form_tensor_cores_split(ctx, prec, tol, gain, smode, n, p):
    """Split-operand forms (two pieces: hi*hi + hi*lo + lo*hi; three pieces:
    the six products of total order <= 2): |dS| <= tol |W21||L21|^T
    elementwise, and far below the plain BF16 form's largest error on the same
    supernode (a dropped correction product fails this)."""
    from paper_1305_2353_gb300 import ctp
    A = _tough(n, p, 5)
    ref = O.factor(A, p, "relaxed")
    e = ref["nelim"]
    L21 = ref["A"][p:, :e]
    _, Dm, _ = O.unpack(ref, p)
    S = O.form(L21, ref["piv"][:e], ref["D"])
    lo = np.tril(np.ones_like(S, dtype=bool))
    errs = {}
    for pr in ("bf16", prec):
        sn = ctp.Supernode(ctx, A, p, ctp.options(pivot="relaxed", prec=pr, smode=smode))
        sn.run()
        torch.cuda.synchronize()
        got = sn.result()
        assert got["info"] == 0 and got["nelim"] == e
        errs[pr] = np.abs(got["S"] - S)[lo]
        assert np.all(np.triu(got["S"], 1) == 0)
    bound = _bf16_bound(L21 @ Dm, L21)[lo]
    # FP32 storage of S adds 2^-24 |S|
    assert np.all(errs[prec] <= tol * bound + 2.0 ** -23 * np.abs(S[lo]) + 1e-30)
    assert errs[prec].max() * gain <= errs["bf16"].max()


def test_form_tensor_cores_bf16x3_large(ctx):
    """n = 40000, p = 256: the column-panel walk of the split form (more column
    blocks than twice the SMs), sampled entries against the oracle."""
    from paper_1305_2353_gb300 import ctp
    n, p = 40000, 256
    A = inputs.single_large(3, n=n, p=p)
    ref = O.factor(A, p, "relaxed")
    sn = ctp.Supernode(ctx, A, p, ctp.options(pivot="relaxed", prec="bf16x3", smode="fp32_tiled"))
    sn.run()
    torch.cuda.synchronize()
    assert ctx.read_info(sn.ws) == 0
    m, e = n - p, ref["nelim"]
    rng = np.random.default_rng(1)
    ii = rng.integers(0, m, 6000)
    jj = rng.integers(0, m, 6000)
    ii, jj = np.maximum(ii, jj), np.minimum(ii, jj)
    ii = np.r_[ii, np.arange(m - 300, m), np.arange(0, m, 997)]
    jj = np.r_[jj, np.arange(m - 300, m), np.arange(0, m, 997)]
    L21 = ref["A"][p:, :e]
    want = O.form_entries(L21, ref["piv"][:e], ref["D"], ii, jj)
    nb = (m + 127) // 128
    bi, bj = ii // 128, jj // 128
    blk = bj * nb - bj * (bj - 1) // 2 + (bi - bj)
    idx = blk * 16384 + (jj % 128) * 128 + (ii % 128)
    got = sn.S[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    _, Dm, _ = O.unpack(ref, p)
    bound = np.einsum("tk,tk->t", np.abs((L21 @ Dm)[ii]), np.abs(L21[jj]))
    assert np.all(np.abs(got - want) <= 2.0 ** -13 * bound)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "bf16x6"])
def test_form_walks_are_bit_identical(ctx, prec):
    """The tile walks of the tensor-core Form change which CTA computes a tile,
    not how: S is bit-identical under every walk (n = 40000 so that the panel
    walk is taken)."""
    from paper_1305_2353_gb300 import ctp
    n, p = 40000, 192
    A = inputs.single_large(4, n=n, p=p)
    out = {}
    for w in ("round_robin", "chunks", "panels"):
        ctx.tune_set(ctp.TUNE_FORM_WALK, ctp.WALK[w])
        try:
            sn = ctp.Supernode(ctx, A, p, ctp.options(pivot="relaxed", prec=prec, smode="fp32_tiled"))
            sn.run()
            torch.cuda.synchronize()
            assert ctx.read_info(sn.ws) == 0
            out[w] = sn.S.clone()
            del sn
        finally:
            ctx.tune_set(ctp.TUNE_FORM_WALK, 0)
    assert torch.equal(out["round_robin"], out["chunks"])
    assert torch.equal(out["round_robin"], out["panels"])


def test_supernode_autotune(ctx):
    """The autotuner over Form walks and pivot-search cluster widths restores the
    input and leaves the factorization unchanged."""
    from paper_1305_2353_gb300 import ctp
    n, p = 20000, 128
    A = inputs.single_large(5, n=n, p=p)
    opt = ctp.options(pivot="relaxed", prec="bf16x3", smode="fp32_tiled")
    sn = ctp.Supernode(ctx, A, p, opt)
    before = sn.A.clone()
    cands = [(1, 0), (2, 4), (3, 8), (2, 16)]
    ms, best = ctp.autotune_supernode(ctx, sn.A, n, p, n, opt, sn.perm, sn.piv, sn.D, sn.nelim,
                                      sn.S, n - p, sn.ws, [ctp.TUNE_FORM_WALK, ctp.TUNE_FACTOR_G],
                                      cands)
    torch.cuda.synchronize()
    assert 0 <= best < len(cands) and np.all(ms > 0)
    assert torch.equal(sn.A, before)
    assert ctx.tune_get(ctp.TUNE_FORM_WALK) == cands[best][0]
    assert ctx.tune_get(ctp.TUNE_FACTOR_G) == cands[best][1]
    sn.run()
    torch.cuda.synchronize()
    got = sn.result()
    ctx.tune_set(ctp.TUNE_FORM_WALK, 0)
    ctx.tune_set(ctp.TUNE_FACTOR_G, 0)
    ref = O.factor(A, p, "relaxed")
    assert got["nelim"] == ref["nelim"]
    assert np.array_equal(got["perm"], ref["perm"])


@pytest.mark.parametrize("G", [1, 4, 8])
def test_factor_cluster_width_same_pivots(ctx, G):
    """Any cluster width of the pivot search gives the oracle's pivots."""
    from paper_1305_2353_gb300 import ctp
    A = _tough(3000, 200, 8)
    ctx.tune_set(ctp.TUNE_FACTOR_G, G)
    try:
        got = run_gpu(ctx, A, 200, "strict")
    finally:
        ctx.tune_set(ctp.TUNE_FACTOR_G, 0)
    ref = O.factor(A, 200, "strict", log_cap=100000)
    compare(ref, got, 200, A)


def test_form_tensor_cores_large(ctx):
    """n = 20000, p = 256, relaxed (e = 256): 610 tiles per row band region, sampled
    entries of S against the oracle, including the diagonal and the last rows."""
    from paper_1305_2353_gb300 import ctp
    n, p = 20000, 256
    A = inputs.single_large(2, n=n, p=p)
    ref = O.factor(A, p, "relaxed")
    opt = ctp.options(pivot="relaxed", prec="bf16", smode="fp32")
    sn = ctp.Supernode(ctx, A, p, opt)
    sn.run()
    torch.cuda.synchronize()
    assert ctx.read_info(sn.ws) == 0
    m, e = n - p, ref["nelim"]
    rng = np.random.default_rng(0)
    ii = rng.integers(0, m, 6000)
    jj = rng.integers(0, m, 6000)
    ii, jj = np.maximum(ii, jj), np.minimum(ii, jj)
    ii = np.r_[ii, np.arange(m - 300, m), np.arange(0, m, 997)]
    jj = np.r_[jj, np.arange(m - 300, m), np.arange(0, m, 997)]
    L21 = ref["A"][p:, :e]
    want = O.form_entries(L21, ref["piv"][:e], ref["D"], ii, jj)
    Sg = sn.S  # (m, m) tensor holding S column-major: element (i, j) at [j, i]
    got = Sg[torch.as_tensor(jj, device="cuda"), torch.as_tensor(ii, device="cuda")].cpu().numpy()
    _, Dm, _ = O.unpack(ref, p)
    Wd = L21 @ Dm
    bound = np.einsum("tk,tk->t", np.abs(Wd[ii]), np.abs(L21[jj]))
    assert np.all(np.abs(got - want) <= 2.0 ** -7 * bound)
