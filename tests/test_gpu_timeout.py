"""A bounded wait that runs out, on the GPU, without a fault: the software grid
barrier of the full-column TPP kernel is given a limit of a few polls
(CTP_TUNE_TPP_SPIN), so the CTAs waiting for CTA 0's pivot decision give up.
The kernel must return, the info word must read CTP_ETIMEOUT, and the context
must stay usable: with the default limit the same call then gives the oracle's
factorization."""
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


def _run(ctx, A, p):
    from paper_1305_2353_gb300 import ctp
    n = A.shape[0]
    opt = ctp.options(pivot="tpp")
    dA = ctp.colmajor(A)
    perm = torch.empty(p, dtype=torch.int32, device="cuda")
    piv = torch.empty(p, dtype=torch.int32, device="cuda")
    D = torch.empty(2 * p, dtype=torch.float64, device="cuda")
    nel = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = ctx.factor_supernode(dA, n, p, n, opt, perm, piv, D, nel)
    info = ctx.read_info(ws)
    return info, int(nel.cpu()[0]), perm.cpu().numpy()


def test_tpp_barrier_timeout(ctx):
    from paper_1305_2353_gb300 import ctp
    n, p = 20000, 128
    A = inputs.single_large(4, n=n, p=p)
    assert ctx.tune_get(ctp.TUNE_TPP_SPIN) == 0
    with pytest.raises(ctp.CtpError):
        ctx.tune_set(ctp.TUNE_TPP_SPIN, -1)
    with pytest.raises(ctp.CtpError):
        ctx.tune_set(ctp.TUNE_TPP_SPIN, (1 << 24) + 1)
    ctx.tune_set(ctp.TUNE_TPP_SPIN, 4)
    try:
        assert ctx.tune_get(ctp.TUNE_TPP_SPIN) == 4
        for _ in range(2):
            info, _, _ = _run(ctx, A, p)
            assert info == ctp.CTP_ETIMEOUT
    finally:
        ctx.tune_set(ctp.TUNE_TPP_SPIN, 0)
    info, nelim, perm = _run(ctx, A, p)
    assert info == ctp.CTP_OK
    ref = O.factor(A, p, "tpp")
    assert nelim == ref["nelim"] and np.array_equal(perm, ref["perm"])
