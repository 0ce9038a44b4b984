"""The row split of one supernode (Section 6, Table 6.1): A21's rows cut into
P blocks, each compressed on its own, then one exchange -- an elementwise
maximum of the blocks' strict compressed matrices, or the greedy of Section 4.2
over the union of the blocks' relaxed candidate lists.  Simulated with every
block on one GPU, through the C ABI, the result must equal the single-pass
compression bit for bit (and so the oracle's), including uneven blocks, empty
blocks and blocks of fewer rows than columns."""
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


def _cuts(m, P, seed):
    """P uneven row blocks of m rows (some may be empty)."""
    rng = np.random.default_rng(seed)
    c = np.sort(rng.integers(0, m + 1, P - 1))
    return np.concatenate([[0], c, [m]]).astype(np.int64)


CASES = [(20000, 256, 2, 0), (20000, 256, 8, 1), (5000, 64, 3, 2), (300, 100, 4, 3), (40, 33, 8, 4),
         (200000, 256, 8, 5)]


def _a21(n, p, seed):
    if n == 200000:
        return inputs.single_large(seed)[p:]
    A = inputs.supernode(n, p, seed=seed)[p:]
    A[::7, 0] = A[::7, 1]          # exact ties between columns (strict argmax) and rows (relaxed)
    A[5::11, 3] = -A[4::11, 3][:len(A[5::11, 3])]
    return A


@pytest.mark.parametrize("n,p,P,seed", CASES)
def test_strict_row_split_equals_single_pass(ctx, n, p, P, seed):
    from paper_1305_2353_gb300 import ctp
    A21 = _a21(n, p, seed)
    m = A21.shape[0]
    dA = ctp.colmajor(A21)
    C1 = torch.empty(p * p, dtype=torch.float64, device="cuda")
    ctx.compress_strict(dA, m, p, m, C1)
    cuts = _cuts(m, P, seed)
    Cb = torch.empty((P, p * p), dtype=torch.float64, device="cuda")
    Jb = torch.empty(m, dtype=torch.int32, device="cuda")
    for b in range(P):
        r0, r1 = int(cuts[b]), int(cuts[b + 1])
        # the block's first row, A21's lda (an empty block still passes a valid pointer)
        blk = dA[:, r0:] if r1 > r0 else dA
        ctx.compress_strict(blk, r1 - r0, p, m, Cb[b], Jb[r0:r1] if r1 > r0 else None)
    C = torch.empty(p * p, dtype=torch.float64, device="cuda")
    ctx.compress_strict_merge(P, p, Cb, p * p, C)
    torch.cuda.synchronize()
    assert torch.equal(C, C1)
    if m <= 20000:
        Cref, Jref = O.compress_strict(A21)
        assert np.array_equal(C.cpu().numpy().reshape(p, p), Cref)
        assert np.array_equal(Jb.cpu().numpy(), Jref)


@pytest.mark.parametrize("n,p,P,seed", CASES)
def test_relaxed_row_split_equals_single_pass(ctx, n, p, P, seed):
    from paper_1305_2353_gb300 import ctp
    A21 = _a21(n, p, seed)
    m = A21.shape[0]
    dA = ctp.colmajor(A21)
    C1 = torch.empty(p * p, dtype=torch.float64, device="cuda")
    rows1 = torch.empty(p, dtype=torch.int32, device="cuda")
    ctx.compress_relaxed(dA, m, p, m, C1, rows1)
    cuts = _cuts(m, P, seed + 100)
    cand = ctx.relaxed_candidates_buffer(P, p)
    for b in range(P):
        r0, r1 = int(cuts[b]), int(cuts[b + 1])
        ctx.compress_relaxed_candidates(dA[:, r0:] if r1 > r0 else dA, r1 - r0, p, m, r0, P, b, cand)
    rows = torch.empty(p, dtype=torch.int32, device="cuda")
    ctx.compress_relaxed_select(P, p, cand, rows)
    C = torch.empty(p * p, dtype=torch.float64, device="cuda")
    ctx.gather_rows(p, dA, m, rows, C)
    torch.cuda.synchronize()
    assert ctx.read_info(cand) == 0
    assert torch.equal(rows, rows1)
    assert torch.equal(C, C1)
    if m <= 20000:
        Cref, rref = O.compress_relaxed(A21)
        assert np.array_equal(rows.cpu().numpy(), rref)
        assert np.array_equal(C.cpu().numpy().reshape(p, p), Cref)
