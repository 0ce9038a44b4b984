"""The strict-compression entry point that allocates nothing.

It exists for callers that cannot allocate device memory where they call the
library (for example a plugin whose host application owns every device
allocation).  Its scratch is a fixed array inside libctp, shared by all calls,
so the test makes two calls in a row with different inputs: the second result
must not remember the first.  Both are compared, through the C ABI, with the
workspace-based ctp_compress_strict, bit for bit (compression involves no
rounding).  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _case(seed, m, p, scale):
    A21 = np.random.default_rng(seed).standard_normal((m, p)) * scale
    A21[::9, 0] = 0.0
    return A21


def test_noalloc_matches_workspace_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1305_2353_gb300 import build, ctp
    build.build()
    torch.cuda.set_device(0)
    ctx = ctp.Context(0)
    # first call: large values; second: smaller values and a smaller p, so any
    # maxima left in the shared scratch by the first call would show up
    for seed, m, p, scale in ((1, 50001, 256, 100.0), (2, 30011, 200, 1.0), (3, 777, 256, 1e-3)):
        A21 = _case(seed, m, p, scale)
        dA = ctp.colmajor(A21)
        C_ref = torch.empty(p * p, dtype=torch.float64, device="cuda")
        J_ref = torch.empty(m, dtype=torch.int32, device="cuda")
        ws = ctx.compress_strict(dA, m, p, m, C_ref, J_ref)
        C = torch.full((p * p,), -1.0, dtype=torch.float64, device="cuda")
        J = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        info = ctp.compress_strict_noalloc(dA, m, p, m, C, J)
        torch.cuda.synchronize()
        assert info == 0
        assert ctx.read_info(ws) == 0
        assert torch.equal(C, C_ref)
        assert torch.equal(J, J_ref)


def test_noalloc_rejects_p_above_limit():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1305_2353_gb300 import ctp
    x = torch.zeros((300, 4), dtype=torch.float64, device="cuda")
    C = torch.zeros(300 * 300, dtype=torch.float64, device="cuda")
    with pytest.raises(ctp.CtpError) as e:
        ctp.compress_strict_noalloc(x, 4, 300, 4, C)
    assert e.value.code == ctp.CTP_ECAPACITY
