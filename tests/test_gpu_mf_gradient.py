"""Differentiation through the multifrontal factorization (the shifted 3D
Laplacian on a 16^3 grid with nested dissection, 32 right-hand sides,
loss = ||x||^2): the adjoint solve with the same factors, the gradient of the
stored entries (the sparsity pattern) and of B, against the oracle's gradient
and central finite differences (h = 1e-6) of the GPU solve, in FP64 and with
the split-BF16 tensor-core Form refined to FP64 accuracy."""
import numpy as np
import pytest

from oracle import multifrontal as MF
from oracle import system as S
from paper_1305_2353_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K, NRHS = 16, 32


@pytest.fixture(scope="module")
def ctx():
    from paper_1305_2353_gb300 import build, ctp
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return ctp.Context(0)


def _problem(k, leaf=64):
    cp, ri, v = inputs.laplacian_3d(k, 3.0)
    perm, blocks = inputs.nested_dissection_3d(k, leaf)
    return cp, ri, v, k ** 3, perm, blocks


@pytest.fixture(scope="module")
def oracle_grad():
    cp, ri, v, N, perm, blocks = _problem(K)
    B = np.random.default_rng(50).standard_normal((N, NRHS))
    panels, _ = MF.factor(cp, ri, v, N, perm, blocks, "strict", w=256)
    x, hist, _ = S.refine(MF.sym_csc(cp, ri, v, N).toarray(), panels, B)
    col = np.repeat(np.arange(N), np.diff(cp))
    gb, g = S.solve_gradient_pattern(panels, x, 2.0 * x, ri, col)
    return B, x, gb, g


def test_mf_adjoint_solve_is_the_solve(ctx):
    """M symmetric: the planned adjoint solve is the planned solve.  Its forward
    sweep adds into shared ancestor rows with atomics, so two calls agree to
    rounding (amplified by the condition number, about 2.5e3 here), not bit
    for bit."""
    from paper_1305_2353_gb300 import ctp
    cp, ri, v, N, perm, blocks = _problem(12)
    mf = ctp.Multifrontal(ctx, cp, ri, v, perm, blocks)
    mf.factor(ctp.options(pivot="strict"))
    B = np.random.default_rng(3).standard_normal((N, 4))
    X1, X2 = ctp.colmajor(B), ctp.colmajor(B)
    ws = mf.refine_workspace(4)
    mf.solve(X1, ws)
    mf.adjoint_solve(X2, ws)
    torch.cuda.synchronize()
    assert torch.allclose(X1, X2, rtol=0, atol=1e-10 * float(X1.abs().max()))
    mf.destroy()


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_mf_gradient_matches_oracle(ctx, oracle_grad, prec):
    from paper_1305_2353_gb300 import ctp
    cp, ri, v, N, perm, blocks = _problem(K)
    B, xo, gbo, go = oracle_grad
    solver = ctp.SparseSymSolver(ctx, cp, ri, perm, blocks, pivot="strict", prec=prec)
    val = torch.tensor(v, device="cuda", requires_grad=True)
    Bt = torch.tensor(B, device="cuda", requires_grad=True)
    X = solver(val, Bt)
    assert solver.history[-1].max() <= 1e-14
    (X * X).sum().backward()
    np.testing.assert_allclose(X.detach().cpu().numpy(), xo, rtol=0, atol=1e-10 * np.abs(xo).max())
    np.testing.assert_allclose(Bt.grad.cpu().numpy(), gbo, rtol=0, atol=1e-10 * np.abs(gbo).max())
    np.testing.assert_allclose(val.grad.cpu().numpy(), go, rtol=0, atol=1e-10 * np.abs(go).max())
    solver.mf.destroy()


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_mf_gradient_finite_differences(ctx, prec):
    """Central differences of the GPU solve itself (factor + refinement per
    evaluation) on a sample of stored entries and of B."""
    from paper_1305_2353_gb300 import ctp
    cp, ri, v, N, perm, blocks = _problem(K)
    B = np.random.default_rng(51).standard_normal((N, NRHS))
    solver = ctp.SparseSymSolver(ctx, cp, ri, perm, blocks, pivot="strict", prec=prec)
    val = torch.tensor(v, device="cuda", requires_grad=True)
    Bt = torch.tensor(B, device="cuda", requires_grad=True)
    X = solver(val, Bt)
    (X * X).sum().backward()
    g, gb = val.grad.cpu().numpy(), Bt.grad.cpu().numpy()

    def loss(vv, BB):
        with torch.no_grad():
            Y = solver(torch.tensor(vv, device="cuda"), torch.tensor(BB, device="cuda"))
            return float((Y * Y).sum())

    h = 1e-6
    rng = np.random.default_rng(52)
    for q in rng.choice(len(v), 8, replace=False):
        vp, vm = v.copy(), v.copy()
        vp[q] += h
        vm[q] -= h
        fd = (loss(vp, B) - loss(vm, B)) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * np.abs(g).max(), (q, fd, g[q])
    for _ in range(4):
        i, r = rng.integers(N), rng.integers(NRHS)
        Bp, Bm = B.copy(), B.copy()
        Bp[i, r] += h
        Bm[i, r] -= h
        fd = (loss(v, Bp) - loss(v, Bm)) / (2 * h)
        assert abs(fd - gb[i, r]) <= 1e-6 * np.abs(gb).max(), (i, r, fd, gb[i, r])
    solver.mf.destroy()


def test_mf_backward_after_refactor(ctx):
    """A second solve with other values before the first backward: the first
    backward still uses its own factors (it factors its values again).  The
    grid is 7^3: with k + 1 divisible by 3 (8^3, 32^3) the shift 3 is an exact
    eigenvalue of the 7-point Laplacian (3 (2 - 2 cos(pi/3))), the system is
    singular and its gradients are rounding noise."""
    from paper_1305_2353_gb300 import ctp
    cp, ri, v, N, perm, blocks = _problem(7, leaf=16)
    B = np.random.default_rng(6).standard_normal((N, 2))
    solver = ctp.SparseSymSolver(ctx, cp, ri, perm, blocks)
    v1 = torch.tensor(v, device="cuda", requires_grad=True)
    v2 = torch.tensor(v * 1.1, device="cuda", requires_grad=True)
    Bt = torch.tensor(B, device="cuda")
    X1 = solver(v1, Bt)
    X2 = solver(v2, Bt)
    (X1 * X1).sum().backward()
    g_interleaved = v1.grad.clone()
    v1.grad = None
    X1b = solver(v1, Bt)
    (X1b * X1b).sum().backward()
    assert torch.allclose(g_interleaved, v1.grad, rtol=0, atol=1e-10 * float(v1.grad.abs().max()))
    del X2
    solver.mf.destroy()


def test_mf_gradcheck_small(ctx):
    """torch.autograd.gradcheck through the multifrontal solve on a 4^3 grid
    cut into leaf boxes of 8 points (a tree of fronts): every stored entry and
    every entry of B."""
    from paper_1305_2353_gb300 import ctp
    cp, ri, v, N, perm, blocks = _problem(4, leaf=8)
    assert len(blocks) > 4
    solver = ctp.SparseSymSolver(ctx, cp, ri, perm, blocks)
    val = torch.tensor(v, device="cuda", requires_grad=True)
    Bt = torch.tensor(np.random.default_rng(2).standard_normal((N, 2)), device="cuda",
                      requires_grad=True)
    assert torch.autograd.gradcheck(lambda a, b: solver(a, b), (val, Bt), eps=1e-6, atol=1e-6,
                                     rtol=1e-5)
    solver.mf.destroy()
