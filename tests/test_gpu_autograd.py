"""Differentiation through the solve: the adjoint solve with the same factors,
the gradient of the stored lower triangle of M (dense and on a pattern), the
torch.autograd.Function, against the oracle's gradient and finite differences."""
import numpy as np
import pytest

from oracle import system as osys
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


def _system(n=400, p=40, seed=3):
    A = inputs.supernode(n, p, seed=seed, scale_cols=4, zero_diag_frac=0.1)
    return inputs.two_node(A, seed)


def test_adjoint_solve_is_the_solve(ctx):
    """M symmetric: the adjoint solve gives the solve's result bit for bit."""
    from paper_1305_2353_gb300 import ctp
    M = _system()
    N = M.shape[0]
    Md = ctp.colmajor(M)
    ch = ctp.factor_dense(ctx, Md, N, N, 40, ctp.options(pivot="strict"), 128, ctp.options(pivot="tpp"))
    B = np.random.default_rng(1).standard_normal((N, 3))
    X1, X2 = ctp.colmajor(B), ctp.colmajor(B)
    ws = ctp.solve_workspace(ctx, N, 3)
    ctp.solve(ctx, ch.fronts, ch.nf, N, 3, X1, N, ws)
    ctp.adjoint_solve(ctx, ch.fronts, ch.nf, N, 3, X2, N, ws)
    torch.cuda.synchronize()
    assert torch.equal(X1, X2)
    ch.destroy()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("nrhs", [1, 4])
def test_gradient_matches_oracle(ctx, prec, nrhs):
    """loss = sum(W * X): the autograd gradients of B and of the lower triangle of
    M equal the oracle's (factors reused, both refined to FP64 accuracy), also
    when the supernode's Form ran on the tensor cores."""
    from paper_1305_2353_gb300 import ctp
    M = _system()
    N = M.shape[0]
    rng = np.random.default_rng(7)
    B = rng.standard_normal((N, nrhs))
    W = rng.standard_normal((N, nrhs))
    At = torch.tensor(np.tril(M) + 17.0 * np.triu(np.ones_like(M), 1), device="cuda",
                      requires_grad=True)   # the strict upper triangle is never read
    Bt = torch.tensor(B, device="cuda", requires_grad=True)
    X = ctp.sym_solve(At, Bt, ctx=ctx, pivot="strict", prec=prec, p_first=40, w_rest=128)
    (X * torch.tensor(W, device="cuda")).sum().backward()
    fo = osys.factor_chain(M, 40, "strict", "tpp", w_rest=128)
    xo, _, _ = osys.refine(M, fo, B)
    gbo, gMo = osys.solve_gradient(fo, xo, W)
    np.testing.assert_allclose(X.detach().cpu().numpy(), xo, rtol=1e-9, atol=1e-9 * np.abs(xo).max())
    np.testing.assert_allclose(Bt.grad.cpu().numpy(), gbo, rtol=1e-9, atol=1e-9 * np.abs(gbo).max())
    gM = At.grad.cpu().numpy()
    assert np.all(np.triu(gM, 1) == 0)
    np.testing.assert_allclose(gM, gMo, rtol=1e-8, atol=1e-9 * np.abs(gMo).max())


def test_gradcheck_small(ctx):
    """torch.autograd.gradcheck (central differences on every entry of A and b)
    through the GPU solve; perturbing the unread upper triangle changes nothing,
    which the zero gradient there matches."""
    from paper_1305_2353_gb300 import ctp
    A = inputs.supernode(24, 6, seed=5, zero_diag_frac=0.3)
    M = inputs.two_node(A, 5)
    At = torch.tensor(M, device="cuda", requires_grad=True)
    Bt = torch.tensor(np.random.default_rng(2).standard_normal((24, 2)), device="cuda",
                      requires_grad=True)

    def f(a, b):
        return ctp.sym_solve(a, b, ctx=ctx, pivot="strict", p_first=6, w_rest=8)

    assert torch.autograd.gradcheck(f, (At, Bt), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_pattern_gradient_equals_dense(ctx):
    """The gradient restricted to a pattern of stored entries equals the dense
    gradient at those entries (diagonal and off-diagonal, any order)."""
    from paper_1305_2353_gb300 import ctp
    N, nrhs = 700, 3
    rng = np.random.default_rng(9)
    G = ctp.colmajor(rng.standard_normal((N, nrhs)))
    X = ctp.colmajor(rng.standard_normal((N, nrhs)))
    dense = torch.empty((N, N), dtype=torch.float64, device="cuda")
    ctp.sym_grad_dense(ctx, N, nrhs, G, N, X, N, dense, N)
    ii = rng.integers(0, N, 5000)
    jj = rng.integers(0, N, 5000)
    ii, jj = np.maximum(ii, jj), np.minimum(ii, jj)
    ii = np.r_[ii, np.arange(N)]
    jj = np.r_[jj, np.arange(N)]
    row = torch.tensor(ii, dtype=torch.int32, device="cuda")
    col = torch.tensor(jj, dtype=torch.int32, device="cuda")
    out = torch.empty(len(ii), dtype=torch.float64, device="cuda")
    ctp.sym_grad_pattern(ctx, row, col, N, nrhs, G, N, X, N, out)
    D = dense.cpu().numpy().T   # element (i, j) of the column-major result
    np.testing.assert_array_equal(out.cpu().numpy(), D[ii, jj])
    g, x = ctp.to_numpy(G), ctp.to_numpy(X)
    full = -(g @ x.T)
    want = np.tril(full + full.T)
    np.fill_diagonal(want, np.diag(full))
    np.testing.assert_allclose(D, want, rtol=1e-13, atol=1e-13)
