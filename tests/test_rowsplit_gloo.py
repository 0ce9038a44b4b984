"""The row split's exchange (Section 6, Table 6.1; Appendix A) as two gloo
processes on CPU, each holding half of A21's rows:
  strict   each rank compresses its rows (eq. (4.1)); one allreduce with max
           gives the compressed matrix of the whole supernode; rank 0 runs
           Listing 1 on [A11; C] and broadcasts perm, the pivot kinds, D and
           L11; each rank then solves for its own rows of L21;
  relaxed  each rank sends the full rows of its per-column top-(j+1)
           candidates (at most j rows are flagged before column j, so its choice
           lies among them); the greedy of Section 4.2 on their union picks the
           same rows as on all of A21.
Everything is compared with the single-process oracle: C, rows and pivots bit
for bit, L21 and the delayed columns to FP64 rounding."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

N, P_COLS, SEED = 3000, 48, 17


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _supernode():
    from paper_1305_2353_gb300 import inputs
    A = inputs.supernode(N, P_COLS, seed=SEED, dist="normal", scale_cols=6, scale=1e-3, zero_diag_frac=0.1)
    A[P_COLS:] *= 3.0
    return A


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        A = _supernode()
        p = P_COLS
        A11, A21 = A[:p], A[p:]
        m = A21.shape[0]
        cut = [0, m // 2 + 7, m]
        lo, hi = cut[rank], cut[rank + 1]
        mine = A21[lo:hi]
        res = {}
        # ---- strict: local compression, allreduce max
        Cl, _ = O.compress_strict(mine)
        C = torch.from_numpy(np.ascontiguousarray(Cl))
        dist.all_reduce(C, op=dist.ReduceOp.MAX)
        C = C.numpy()
        res["C_equal"] = np.array_equal(C, O.compress_strict(A21)[0])
        # rank 0: Listing 1 on [A11 (symmetric); C] with the worst-case update, then broadcast
        piv_t = torch.zeros(p, dtype=torch.int32)
        perm_t = torch.zeros(p, dtype=torch.int32)
        ne_t = torch.zeros(1, dtype=torch.int32)
        if rank == 0:
            A11s = np.tril(A11) + np.tril(A11, -1).T
            r = O.listing1(np.vstack([A11s, C]), p, rt=p, tmode=O.UPD_ABS)
            perm_t = torch.from_numpy(r["perm"].astype(np.int32))
            piv_t = torch.from_numpy(r["piv"].astype(np.int32))
            ne_t[0] = r["nelim"]
        for t in (perm_t, piv_t, ne_t):
            dist.broadcast(t, 0)
        perm, piv, e = perm_t.numpy(), piv_t.numpy(), int(ne_t[0])
        ref = O.factor(A, p, "strict")
        res["pivots_equal"] = (e == ref["nelim"] and np.array_equal(perm, ref["perm"])
                               and np.array_equal(piv, ref["piv"]))
        # each rank: its rows of L21 and of the delayed columns, from the
        # broadcast pivot sequence (the Solve with fixed pivots)
        A11p = (np.tril(A11) + np.tril(A11, -1).T)[np.ix_(perm, perm)]
        loc = np.vstack([A11p, mine[:, perm]])
        f = O.ldlt_fixed(loc, p, piv[:e])
        got = f["A"][p:]
        want = ref["A"][p + lo:p + hi]
        scale = max(np.abs(want).max(), 1.0)
        res["L21_close"] = bool(np.allclose(got, want, rtol=1e-12, atol=1e-12 * scale))
        # ---- relaxed: the full rows of every per-column top-(j+1) candidate
        cand = set()
        for j in range(p):
            order = np.lexsort((np.arange(lo, hi), -np.abs(mine[:, j])))  # |a| desc, row asc
            cand.update((lo + order[:j + 1]).tolist())
        ids = torch.tensor(sorted(cand), dtype=torch.int64)
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([len(ids)], dtype=torch.int64))
        cap = int(max(s.item() for s in sizes))
        pad = torch.full((cap,), -1, dtype=torch.int64)
        pad[:len(ids)] = ids
        vals = torch.zeros((cap, p), dtype=torch.float64)
        vals[:len(ids)] = torch.from_numpy(A21[ids.numpy()])
        all_ids = [torch.zeros(cap, dtype=torch.int64) for _ in range(world)]
        all_vals = [torch.zeros((cap, p), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(all_ids, pad)
        dist.all_gather(all_vals, vals)
        gid = torch.cat(all_ids).numpy()
        gv = torch.cat(all_vals).numpy()
        keep = gid >= 0
        gid, gv = gid[keep], gv[keep]
        o = np.argsort(gid, kind="stable")   # the union in A21's row order
        gid, gv = gid[o], gv[o]
        Cu, ru = O.compress_relaxed(gv)
        Cf, rf = O.compress_relaxed(A21)
        rows = np.where(ru >= 0, gid[np.maximum(ru, 0)], -1)
        res["relaxed_equal"] = bool(np.array_equal(rows, rf) and np.array_equal(Cu, Cf))
        res["candidates"] = int(len(ids))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_row_split_exchange_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        r = got[rank]
        assert r["C_equal"] and r["pivots_equal"] and r["L21_close"] and r["relaxed_equal"], (rank, r)
        assert r["candidates"] < (N - P_COLS) // 2   # the exchange moves far fewer rows than a rank holds
