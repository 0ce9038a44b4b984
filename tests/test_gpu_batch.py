"""The batched path (many fronts in a few launches) against the oracle, front
by front, with the same bars as the single-supernode parity tests."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1305_2353_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from test_gpu_supernode import check_backward_error, compare, min_margin, _bf16_bound  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1305_2353_gb300 import build, ctp
    build.build()
    return ctp.Context(0)


def _fronts(count, seed, pmax=256):
    shapes = inputs.batch_shapes(count, seed=seed, pmax=pmax)
    fr = [inputs.supernode(int(n), int(p), seed=seed * 7919 + k, zero_diag_frac=0.02)
          for k, (n, p) in enumerate(shapes)]
    # edge cases: a 1x1 front, a front without A21 rows, the widest front
    fr += [inputs.supernode(1, 1, seed=5), inputs.supernode(40, 40, seed=6),
           inputs.supernode(700, 256, seed=7, zero_diag_frac=0.02)]
    return fr


@pytest.mark.parametrize("pivot", ["strict", "restricted"])
def test_batch_factor_matches_oracle(ctx, pivot):
    from paper_1305_2353_gb300 import ctp
    fr = _fronts(60, seed=3)
    b = ctp.Batch(ctx, fr, [a.shape[1] for a in fr], ctp.options(pivot=pivot))
    b.run()
    torch.cuda.synchronize()
    assert np.all(b.flags() == 0)
    for k, A in enumerate(fr):
        p = A.shape[1]
        ref = O.factor(A, p, pivot, log_cap=200000)
        compare(ref, b.result(k), p, A)


def test_batch_graph_replay(ctx):
    """The batch call only launches kernels: capture it once, replay it."""
    from paper_1305_2353_gb300 import ctp
    fr = _fronts(30, seed=4)
    b = ctp.Batch(ctx, fr, [a.shape[1] for a in fr], ctp.options(pivot="strict", smode="fp64_packed"))
    s = torch.cuda.Stream()
    b.run()  # warm-up outside the capture (kernel attributes are set once)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(stream=s)
    for _ in range(2):
        b.reset()
        g.replay()
    torch.cuda.synchronize()
    for k, A in enumerate(fr):
        p = A.shape[1]
        ref = O.factor(A, p, "strict")
        got = b.result(k)
        compare(ref, got, p, A)
        e = ref["nelim"]
        S = O.form(ref["A"][p:, :e], ref["piv"][:e], ref["D"])
        if S.size:
            assert np.allclose(got["S"], np.tril(S), rtol=1e-11, atol=1e-11 * max(np.abs(S).max(), 1))


@pytest.mark.parametrize("prec,tol", [("bf16", 2.0 ** -7), ("bf16x3", 2.0 ** -13), ("bf16x6", 2.0 ** -19)])
def test_batch_tensor_core_form(ctx, prec, tol):
    from paper_1305_2353_gb300 import ctp
    fr = _fronts(40, seed=5)
    b = ctp.Batch(ctx, fr, [a.shape[1] for a in fr],
                  ctp.options(pivot="strict", prec=prec, smode="fp32_tiled"))
    b.run()
    torch.cuda.synchronize()
    assert np.all(b.flags() == 0)
    for k, A in enumerate(fr):
        p = A.shape[1]
        ref = O.factor(A, p, "strict")
        got = b.result(k)
        compare(ref, got, p, A)
        e = ref["nelim"]
        L21 = ref["A"][p:, :e]
        _, Dm, _ = O.unpack(ref, p)
        S = O.form(L21, ref["piv"][:e], ref["D"])
        if S.size == 0:
            continue
        bound = _bf16_bound(L21 @ Dm, L21)
        lo = np.tril(np.ones_like(S, dtype=bool))
        assert np.all(np.abs(got["S"] - S)[lo] <= tol * bound[lo] + 2.0 ** -23 * np.abs(S[lo]) + 1e-30)


def test_batch_autotune_keeps_inputs_and_results(ctx):
    """The autotuner times candidate launch settings on the batch's own inputs,
    restores them, keeps the fastest setting; the re-planned batch gives the
    oracle's results."""
    from paper_1305_2353_gb300 import ctp
    fr = _fronts(30, seed=9)
    b = ctp.Batch(ctx, fr, [a.shape[1] for a in fr],
                  ctp.options(pivot="strict", prec="bf16x3", smode="fp32_tiled"))
    before = b.A.clone()
    cands = [(64, 2), (100, 1), (220, 2)]
    ms, best = b.autotune([ctp.TUNE_BATCH_SMEM_KB, ctp.TUNE_FORM_WALK], cands)
    torch.cuda.synchronize()
    assert torch.equal(b.A, before)
    assert 0 <= best < 3 and np.all(ms > 0)
    assert ctx.tune_get(ctp.TUNE_BATCH_SMEM_KB) == cands[best][0]
    assert ctx.tune_get(ctp.TUNE_FORM_WALK) == cands[best][1]
    b.run()
    torch.cuda.synchronize()
    assert np.all(b.flags() == 0)
    for k, A in enumerate(fr):
        p = A.shape[1]
        compare(O.factor(A, p, "strict"), b.result(k), p, A)
    ctx.tune_set(ctp.TUNE_BATCH_SMEM_KB, 200)
    ctx.tune_set(ctp.TUNE_FORM_WALK, 0)


@pytest.mark.parametrize("kb", [64, 220])
def test_batch_cluster_budget_same_results(ctx, kb):
    """Another shared-memory budget changes the cluster widths of the pivot
    search, never the pivots."""
    from paper_1305_2353_gb300 import ctp
    fr = _fronts(30, seed=11)
    ctx.tune_set(ctp.TUNE_BATCH_SMEM_KB, kb)
    try:
        b = ctp.Batch(ctx, fr, [a.shape[1] for a in fr], ctp.options(pivot="strict", smode="none"))
    finally:
        ctx.tune_set(ctp.TUNE_BATCH_SMEM_KB, 200)
    b.run()
    torch.cuda.synchronize()
    assert np.all(b.flags() == 0)
    for k, A in enumerate(fr):
        p = A.shape[1]
        compare(O.factor(A, p, "strict"), b.result(k), p, A)



def test_batch_8192_fronts_every_front_matches_oracle(ctx):
    """The full 8192-front batch of the benchmark (p log-uniform in [8, 256],
    n - p log-uniform in [0, 16p], N(0,1), 2% zero diagonals), strict
    compressed pivoting: every front's pivot sequence, kinds and nelim equal the
    oracle's, in FP64 and with the split-BF16 tensor-core Form (pivots do not
    depend on the Form's precision), and every FP64 factor passes the backward
    error bars of check_backward_error.  (No threshold test of the oracle on this
    batch lies within 1e-10 of its bound.  L itself is not compared entry by
    entry here: some fronts grow by 4e3, and then two valid rounding orders
    already differ by more than 1e-10 of max |L|.)"""
    from paper_1305_2353_gb300 import ctp
    fr = inputs.batch(8192, seed=0)
    refs = [O.factor(A, A.shape[1], "strict") for A in fr]
    for prec, smode in (("fp64", "none"), ("bf16x3", "fp32_tiled")):
        b = ctp.Batch(ctx, fr, [a.shape[1] for a in fr], ctp.options(pivot="strict", prec=prec, smode=smode))
        b.run()
        torch.cuda.synchronize()
        assert np.all(b.flags() == 0)
        Ah, perm, piv = b.A.cpu().numpy(), b.perm.cpu().numpy(), b.piv.cpu().numpy()
        D, ne = b.D.cpu().numpy(), b.nelim.cpu().numpy()
        bad = []
        for k, (A, ref) in enumerate(zip(fr, refs)):
            n, p = A.shape
            pv = slice(int(b.p_off[k]), int(b.p_off[k + 1]))
            if (ne[k] != ref["nelim"] or not np.array_equal(perm[pv], ref["perm"])
                    or not np.array_equal(piv[pv], ref["piv"])):
                bad.append(k)
                continue
            if prec != "fp64":
                continue
            got = dict(A=Ah[int(b.a_off[k]):int(b.a_off[k + 1])].reshape(p, n).T.copy(), perm=perm[pv],
                       piv=piv[pv], D=D[2 * pv.start:2 * pv.stop], nelim=int(ne[k]))
            check_backward_error(A, p, got, ref)
        assert bad == [], (prec, bad[:10])
        del b
        torch.cuda.empty_cache()


def test_graph_replay_after_a_smaller_budget(ctx):
    """A captured batch graph still replays after another batch launched the
    same pivot-search kernel with less dynamic shared memory: the launchers only
    ever raise a kernel's shared-memory limit (a limit lowered below what a
    captured node uses would make that node fail on replay)."""
    from paper_1305_2353_gb300 import ctp
    fr = _fronts(30, seed=12)
    ctx.tune_set(ctp.TUNE_BATCH_SMEM_KB, 220)
    try:
        b1 = ctp.Batch(ctx, fr, [a.shape[1] for a in fr], ctp.options(pivot="strict"))
        s = torch.cuda.Stream()
        b1.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b1.run(stream=s)
        ctx.tune_set(ctp.TUNE_BATCH_SMEM_KB, 48)
        fr2 = _fronts(20, seed=13)
        b2 = ctp.Batch(ctx, fr2, [a.shape[1] for a in fr2], ctp.options(pivot="strict"))
        b2.run()
        torch.cuda.synchronize()
        assert np.all(b2.flags() == 0)
        b1.reset()
        g.replay()
        torch.cuda.synchronize()
    finally:
        ctx.tune_set(ctp.TUNE_BATCH_SMEM_KB, 200)
    assert np.all(b1.flags() == 0)
    for k, A in enumerate(fr):
        p = A.shape[1]
        compare(O.factor(A, p, "strict"), b1.result(k), p, A)
    for k, A in enumerate(fr2):
        p = A.shape[1]
        compare(O.factor(A, p, "strict"), b2.result(k), p, A)
