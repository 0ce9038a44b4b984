"""The tensor-core Solve (CTP_SOLVE_TC): L21 and the delayed columns from one
split-BF16 product x_e [U D11^{-1} | U | -U L_d^T] per supernode (U = L11^{-T}),
against the oracle's FP64 Solve within the split's error bound; pivots and the
A11 block unchanged; the Form's S from the tensor-core operands; and complete
systems factored with it refined to FP64 accuracy."""
import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_1305_2353_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# Error of the Solve's split-BF16 product with FP32 accumulation, relative to
# sum_k |x_k||z_k|: three pieces represent an operand to 2^-25 and drop the
# products of order >= 3 (about 2^-23); FP32 accumulation over K <= 256 terms
# adds at most 256 * 2^-24 = 2^-16 in the worst case.  The Solve takes three
# pieces whatever the Form's precision.
TOL_SOLVE = 2.0 ** -15
TOL_FORM = {"bf16": 2.0 ** -7, "bf16x3": 2.0 ** -13, "bf16x6": 2.0 ** -19}


@pytest.fixture(scope="module")
def ctx():
    from paper_1305_2353_gb300 import build, ctp
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return ctp.Context(0)


def _tough(n, p, seed):
    A = inputs.supernode(n, p, seed=seed, dist="normal", scale_cols=max(1, p // 6), scale=1e-3,
                         zero_diag_frac=0.2)
    A[p:, :] *= 5.0
    return A


def _operands(A, ref, p):
    """x_e, |x_e||Z| for the L21, Y and delayed blocks, and the oracle's L21, W21."""
    e, perm = ref["nelim"], np.asarray(ref["perm"])
    L, Dm, _ = O.unpack(ref, p)
    L11, Ld = L[:e, :e], L[e:p, :e]
    U = scipy.linalg.solve_triangular(L11.T, np.eye(e), lower=False, unit_diagonal=True)
    Dinv = np.zeros_like(Dm)
    j = 0
    while j < e:   # block inverse; a zero pivot keeps a zero block
        if j + 1 < e and Dm[j + 1, j] != 0.0:
            Dinv[j:j + 2, j:j + 2] = np.linalg.inv(Dm[j:j + 2, j:j + 2])
            j += 2
        else:
            Dinv[j, j] = 1.0 / Dm[j, j] if Dm[j, j] != 0.0 else 0.0
            j += 1
    xe = np.abs(A[p:, perm[:e]])
    return dict(bL=xe @ np.abs(U @ Dinv), bY=xe @ np.abs(U), bd=xe @ np.abs(U @ Ld.T),
                L21=ref["A"][p:, :e], W21=ref["A"][p:, :e] @ Dm, e=e)


def _run(ctx, A, p, pivot, prec, solve, smode="fp32"):
    from paper_1305_2353_gb300 import ctp
    sn = ctp.Supernode(ctx, A, p, ctp.options(pivot=pivot, prec=prec, smode=smode, solve=solve))
    sn.run()
    torch.cuda.synchronize()
    return sn.result()


@pytest.mark.parametrize("pivot", ["strict", "relaxed", "restricted"])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "bf16x6"])
@pytest.mark.parametrize("n,p", [(600, 40), (2000, 64), (1500, 130), (3000, 256), (700, 200), (300, 17),
                                 (1000, 97)])
def test_solve_tc_matches_oracle(ctx, pivot, prec, n, p):
    A = _tough(n, p, 11)
    ref = O.factor(A, p, pivot)
    got = _run(ctx, A, p, pivot, prec, "tc")
    fp = _run(ctx, A, p, pivot, prec, "fp64")
    assert got["info"] == 0
    e = ref["nelim"]
    assert got["nelim"] == e
    assert np.array_equal(got["perm"], ref["perm"]) and np.array_equal(got["piv"], ref["piv"])
    # the A11 rows and D come from the pivot search: bit for bit the FP64-Solve run's
    assert np.array_equal(got["A"][:p], fp["A"][:p]) and np.array_equal(got["D"], fp["D"])
    ops = _operands(A, ref, p)
    tol = TOL_SOLVE
    err_L = np.abs(got["A"][p:, :e] - ops["L21"])
    assert np.all(err_L <= tol * ops["bL"] + 1e-300)
    want_d = ref["A"][p:, e:p]
    err_d = np.abs(got["A"][p:, e:p] - want_d)
    assert np.all(err_d <= tol * ops["bd"] + 2.0 ** -52 * np.abs(want_d) + 1e-300)
    # S = W21 L21^T from the Solve's operands: the Form's own rounding plus the
    # Solve's errors carried through both operands
    S = O.form(ops["L21"], ref["piv"][:e], ref["D"])
    lo = np.tril(np.ones_like(S, dtype=bool))
    aL, aW = np.abs(ops["L21"]), np.abs(ops["W21"])
    bound = (TOL_FORM[prec] * (aW @ aL.T) + 2 * tol * (ops["bY"] @ aL.T + aW @ ops["bL"].T)
             + 2.0 ** -23 * np.abs(S))
    assert np.all(np.abs(got["S"] - S)[lo] <= bound[lo] + 1e-300)


@pytest.mark.parametrize("smode", ["fp32_packed", "fp32_tiled"])
def test_solve_tc_s_layouts(ctx, smode):
    """The Form's other S layouts read the same operands: S equals the full
    layout's S bit for bit."""
    A = _tough(1500, 130, 13)
    full = _run(ctx, A, 130, "strict", "bf16x3", "tc", smode="fp32")
    other = _run(ctx, A, 130, "strict", "bf16x3", "tc", smode=smode)
    lo = np.tril(np.ones_like(full["S"], dtype=bool))
    assert np.array_equal(full["S"][lo], other["S"][lo])


def test_solve_tc_large_sampled(ctx):
    """n = 200000, p = 256 (the single-supernode bench workload): sampled rows of
    L21 against the oracle's Solve of those rows (FP64 substitution with the
    oracle's factors)."""
    from paper_1305_2353_gb300 import ctp
    n, p = 200000, 256
    A = inputs.single_large(0, n=n, p=p)
    sn = ctp.Supernode(ctx, A, p, ctp.options(pivot="relaxed", prec="bf16x6", smode="fp32_tiled", solve="tc"))
    sn.run()
    torch.cuda.synchronize()
    assert ctx.read_info(sn.ws) == 0
    # (S is 80 GB: nothing of it comes to the host)
    # the pivots depend on C, which a sample of rows does not reproduce, so the
    # GPU's pivots (checked against the oracle elsewhere) go into an FP64
    # substitution of the sampled rows
    e = int(sn.nelim.cpu()[0])
    perm, piv, D = sn.perm.cpu().numpy(), sn.piv.cpu().numpy(), sn.D.cpu().numpy()
    assert e == p
    rows = np.r_[np.random.default_rng(3).integers(0, n - p, 400), np.arange(n - p - 50, n - p)]
    Acm = sn.A  # column-major n x p: element (i, j) at [j, i]
    top = Acm[:, :p].cpu().numpy().T
    got_rows = Acm[:, torch.as_tensor(p + rows, device="cuda")].cpu().numpy().T
    del sn
    torch.cuda.empty_cache()
    L11 = np.tril(top, -1) + np.eye(p)
    for j in range(p - 1):
        if piv[j] == 2:
            L11[j + 1, j] = 0.0
    X = A[p + rows][:, perm]
    Y = scipy.linalg.solve_triangular(L11, X.T, lower=True, unit_diagonal=True).T
    Dm = np.zeros((p, p))
    j = 0
    while j < p:
        if piv[j] == 2:
            Dm[j:j + 2, j:j + 2] = [[D[2 * j], D[2 * j + 1]], [D[2 * j + 1], D[2 * j + 2]]]
            j += 2
        else:
            Dm[j, j] = D[2 * j]
            j += 1
    L21 = np.linalg.solve(Dm, Y.T).T
    U = scipy.linalg.solve_triangular(L11.T, np.eye(p), lower=False, unit_diagonal=True)
    bound = np.abs(X) @ np.abs(U @ np.linalg.inv(Dm))
    assert np.all(np.abs(got_rows - L21) <= TOL_SOLVE * bound)


def _refine_chain(ctx, M, p_first, mf, prec_first, mr, w_rest, prec_rest="fp64"):
    from paper_1305_2353_gb300 import ctp
    N = M.shape[0]
    Md = ctp.colmajor(M)
    ch = ctp.factor_dense(ctx, Md, N, N, p_first, ctp.options(pivot=mf, prec=prec_first, solve="tc"),
                          w_rest, ctp.options(pivot=mr, prec=prec_rest, solve="tc"))
    b = np.random.default_rng(1).standard_normal((N, 1))
    X = torch.zeros((1, N), dtype=torch.float64, device="cuda")
    ws = ctp.refine_workspace(ctx, N, N, 1)
    hist, k = ctp.refine(ctx, ch.fronts, ch.nf, N, ctp.colmajor(np.tril(M)), N, 1, ctp.colmajor(b), N,
                         X, N, ws)
    ch.destroy()
    return hist, k


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_solve_tc_system_refines(ctx, prec):
    """The n = 2000, p = 64 supernode (eight tiny columns) in its complete system,
    its Solve and Form on the tensor cores: FP64 refinement reaches the Section 7
    criterion (<= 1e-14) in at most ten corrections.  A chain whose every front
    is compressed with its Solve and Form on the tensor cores does the same with
    the three-piece Form; with the two-piece Form each correction contracts the
    error about tenfold (measured 2e-4, 6e-6, 7e-7, ... 3e-14 after ten), so
    there the bar is the 1e-12 of mixed precision with a steady contraction."""
    A = inputs.single_small(0)
    M = inputs.two_node(A, 0)
    h, k = _refine_chain(ctx, M, 64, "strict", prec, "tpp", 256)
    assert h[-1].max() <= 1e-14 and k <= 10, (h.max(axis=1).tolist(), k)
    A2 = inputs.supernode(1500, 96, seed=7)
    M2 = inputs.two_node(A2, 7)
    h2, k2 = _refine_chain(ctx, M2, 96, "strict", prec, "strict", 128, prec_rest=prec)
    hist = h2.max(axis=1)
    if prec == "bf16x6":
        assert hist[-1] <= 1e-14 and k2 <= 10, (hist.tolist(), k2)
    else:
        assert hist[-1] <= 1e-12 and np.all(hist[1:] <= 0.25 * hist[:-1]), (hist.tolist(), k2)


def _batch_fronts(count, seed):
    """Uneven fronts with the tough structure (rejections, 2x2 and zero pivots,
    delayed columns), plus edge cases: a 1x1 front, a front without A21 rows,
    the widest front, and a front whose p is just above 2 K blocks."""
    shapes = inputs.batch_shapes(count, seed=seed, pmax=256)
    fr = [_tough(int(n), int(p), seed * 7919 + k) for k, (n, p) in enumerate(shapes)]
    fr += [inputs.supernode(1, 1, seed=5), inputs.supernode(40, 40, seed=6), _tough(700, 256, 7),
           _tough(500, 129, 8)]
    return fr


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "bf16x6"])
def test_batch_solve_tc_matches_oracle(ctx, prec):
    """The batched tensor-core Solve (one prep per front, tiles of x_e and Z^T,
    one GEMM launch over every front's (row block, window) items), front by
    front: pivots and A11 as the oracle's, L21 and the delayed columns within the
    split's bound, S within the Form's bound plus the Solve's error."""
    from paper_1305_2353_gb300 import ctp
    fr = _batch_fronts(50, 11)
    b = ctp.Batch(ctx, fr, [a.shape[1] for a in fr],
                  ctp.options(pivot="strict", prec=prec, smode="fp32_tiled", solve="tc"))
    b.run()
    torch.cuda.synchronize()
    assert np.all(b.flags() == 0)
    for k, A in enumerate(fr):
        p = A.shape[1]
        ref = O.factor(A, p, "strict", log_cap=200000)
        got = b.result(k)
        e = ref["nelim"]
        assert got["nelim"] == e
        assert np.array_equal(got["perm"], ref["perm"]) and np.array_equal(got["piv"], ref["piv"])
        if A.shape[0] == p or e == 0:
            continue
        ops = _operands(A, ref, p)
        err_L = np.abs(got["A"][p:, :e] - ops["L21"])
        assert np.all(err_L <= TOL_SOLVE * ops["bL"] + 1e-300), k
        want_d = ref["A"][p:, e:p]
        assert np.all(np.abs(got["A"][p:, e:p] - want_d) <= TOL_SOLVE * ops["bd"] + 2.0 ** -52 * np.abs(want_d)
                      + 1e-300), k
        S = O.form(ops["L21"], ref["piv"][:e], ref["D"])
        lo = np.tril(np.ones_like(S, dtype=bool))
        aL, aW = np.abs(ops["L21"]), np.abs(ops["W21"])
        bound = (TOL_FORM[prec] * (aW @ aL.T) + 2 * TOL_SOLVE * (ops["bY"] @ aL.T + aW @ ops["bL"].T)
                 + 2.0 ** -23 * np.abs(S))
        assert np.all(np.abs(got["S"] - S)[lo] <= bound[lo] + 1e-300), k


def test_multifrontal_solve_tc_refines(ctx):
    """The shifted 24^3 Laplacian factored multifrontally with every panel's
    Solve and Form on the tensor cores (batched fronts and root chains):
    refinement against the sparse matrix reaches 1e-14 with the three-piece
    Form, and leaf fronts keep the FP64 run's pivots."""
    from paper_1305_2353_gb300 import ctp
    cp, ri, v = inputs.laplacian_3d(24, 3.0)
    perm, blocks = inputs.nested_dissection_3d(24, 64)
    N = 24 ** 3
    mf64 = ctp.Multifrontal(ctx, cp, ri, v, perm, blocks)
    mf64.factor(ctp.options(pivot="strict"))
    mf = ctp.Multifrontal(ctx, cp, ri, v, perm, blocks)
    mf.factor(ctp.options(pivot="strict", prec="bf16x6", solve="tc"))
    gi, g64 = mf.info(), mf64.info()
    leaves = [s for s in range(len(gi["parent"])) if s not in set(gi["parent"].tolist())]
    assert [gi["nelim"][s] for s in leaves] == [g64["nelim"][s] for s in leaves]
    B = np.random.default_rng(5).standard_normal((N, 3))
    X = torch.zeros((3, N), dtype=torch.float64, device="cuda")
    hist, steps = mf.refine(ctp.colmajor(B), X, mf.refine_workspace(3))
    assert hist[-1].max() <= 1e-14 and steps <= 6, hist.max(axis=1)
    mf.destroy()
    mf64.destroy()
