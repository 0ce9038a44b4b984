"""The multifrontal factorization on the GPU against the multifrontal oracle:
fronts, eliminated and delayed counts, panel pivot orders, the solution and
FP64 refinement on the shifted 3D Laplacian with nested dissection."""
import numpy as np
import pytest

from oracle import multifrontal as MF
from oracle import system as S
from paper_1305_2353_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_1305_2353_gb300 import build, ctp
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return ctp.Context(0)


def _problem(k, sigma=3.0, leaf=64):
    cp, ri, v = inputs.laplacian_3d(k, sigma)
    perm, blocks = inputs.nested_dissection_3d(k, leaf)
    return cp, ri, v, k ** 3, perm, blocks


# grid sizes whose shifted Laplacian is nonsingular (see the oracle's tests);
# 24^3 and 31^3 have separators of 576 and 961 columns, wider than the 256
# columns of one panel, so their fronts are chains of panels
@pytest.mark.parametrize("k,sigma,method", [(10, 3.0, "strict"), (10, 6.0, "strict"), (12, 3.0, "tpp"),
                                            (12, 6.0, "relaxed"), (7, 3.0, "restricted"),
                                            (24, 3.0, "strict"), (24, 3.0, "tpp"), (31, 3.0, "relaxed")])
def test_multifrontal_matches_oracle(ctx, k, sigma, method):
    from paper_1305_2353_gb300 import ctp
    cp, ri, v, N, perm, blocks = _problem(k, sigma)
    panels, info = MF.factor(cp, ri, v, N, perm, blocks, method, w=256)
    if k >= 24:
        assert max(i["p"] for i in info) > 256   # some front is a chain of panels
    mf = ctp.Multifrontal(ctx, cp, ri, v, perm, blocks)
    mf.factor(ctp.options(pivot=method))
    gi = mf.info()
    assert gi["nelim"].tolist() == [i["nelim"] for i in info]
    assert gi["delayed"].tolist() == [i["delayed"] for i in info]
    assert gi["n"].tolist() == [i["n"] for i in info]
    assert mf.nf == len(panels)
    # panels come level by level on the GPU, block by block in the oracle:
    # compare them per block, in order within a block
    _, _, _, blk = mf.panel_info()
    order = sorted(range(mf.nf), key=lambda k_: (blk[k_], k_))
    perms = mf.panel_perms()
    assert [int(blk[k_]) for k_ in order] == [po["front"] for po in panels]
    for k_, po in zip(order, panels):
        assert np.array_equal(perms[k_], po["perm"]), k_
    rng = np.random.default_rng(4)
    B = rng.standard_normal((N, 2))
    X = ctp.colmajor(B)
    ws = ctp.solve_workspace(ctx, int(gi["n"].max()), 2)
    ctp.solve(ctx, mf.fronts, mf.nf, N, 2, X, N, ws)
    xo = S.solve(panels, B)
    xg = ctp.to_numpy(X)
    assert np.abs(xg - xo).max() <= 1e-9 * np.abs(xo).max()
    # the level-planned solve (independent panels of a level in one launch)
    X2 = ctp.colmajor(B)
    wsr = mf.refine_workspace(2)
    mf.solve(X2, wsr)
    assert np.abs(ctp.to_numpy(X2) - xo).max() <= 1e-9 * np.abs(xo).max()
    if method != "restricted":
        for planned in (True, False):
            Xr = torch.zeros_like(X)
            hist, steps = mf.refine(ctp.colmajor(B), Xr, wsr, planned=planned)
            assert hist[-1].max() <= 1e-14
    mf.destroy()


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3", "bf16"])
def test_multifrontal_mixed_refines(ctx, prec):
    """Panels' Forms on the tensor cores (subtracting into the fronts).  Leaf
    fronts see only FP64 original entries, so their pivots are the FP64 run's;
    a parent's data carries its children's low-precision Forms, so its pivots
    may differ.  With the split form refinement reaches 1e-14 against the
    sparse matrix."""
    from paper_1305_2353_gb300 import ctp
    cp, ri, v, N, perm, blocks = _problem(24, 3.0)
    mf64 = ctp.Multifrontal(ctx, cp, ri, v, perm, blocks)
    mf64.factor(ctp.options(pivot="strict"))
    mf = ctp.Multifrontal(ctx, cp, ri, v, perm, blocks)
    mf.factor(ctp.options(pivot="strict", prec=prec))
    gi, g64 = mf.info(), mf64.info()
    leaves = [s for s in range(len(gi["parent"])) if s not in set(gi["parent"].tolist())]
    assert len(leaves) > 10
    assert [gi["nelim"][s] for s in leaves] == [g64["nelim"][s] for s in leaves]
    B = np.random.default_rng(5).standard_normal((N, 3))
    X = torch.zeros((3, N), dtype=torch.float64, device="cuda")
    wsr = mf.refine_workspace(3)
    hist, steps = mf.refine(ctp.colmajor(B), X, wsr)
    if prec == "bf16x6":
        assert hist[-1].max() <= 1e-14 and steps <= 3
    if prec == "bf16x3":
        assert hist[-1].max() <= 1e-14 and steps <= 10
    mf.destroy()
    mf64.destroy()


@pytest.mark.parametrize("nrhs", [1, 17, 40])
def test_planned_solve_many_rhs(ctx, nrhs):
    """The level-planned solve takes the right-hand sides in groups (16 per pass
    in FP64, 32 in the FP32 sweeps of a mixed refinement); partial and several
    groups give the generic front-list solve's result, and the FP32 sweeps
    still refine split-BF16 factors to 1e-14."""
    from paper_1305_2353_gb300 import ctp
    cp, ri, v, N, perm, blocks = _problem(12, 3.0, leaf=32)
    mf = ctp.Multifrontal(ctx, cp, ri, v, perm, blocks)
    mf.factor(ctp.options(pivot="strict"))
    B = np.random.default_rng(nrhs).standard_normal((N, nrhs))
    X1 = ctp.colmajor(B)
    mf.solve(X1, mf.refine_workspace(nrhs))
    X2 = ctp.colmajor(B)
    ws = ctp.solve_workspace(ctx, int(mf.info()["n"].max()), nrhs)
    ctp.solve(ctx, mf.fronts, mf.nf, N, nrhs, X2, N, ws)
    torch.cuda.synchronize()
    x1, x2 = ctp.to_numpy(X1), ctp.to_numpy(X2)
    assert np.abs(x1 - x2).max() <= 1e-10 * np.abs(x2).max()
    mf.factor(ctp.options(pivot="strict", prec="bf16x6"))
    X = torch.zeros((nrhs, N), dtype=torch.float64, device="cuda")
    hist, steps = mf.refine(ctp.colmajor(B), X, mf.refine_workspace(nrhs))
    assert hist[-1].max() <= 1e-14 and steps <= 6
    mf.destroy()
