"""Benchmark: per-supernode LDL^T with compressed threshold pivoting on GB300.

One step = one pass of the whole per-supernode hot path over one synthetic
supernode: compression of A21, pivot search on [A11; C], Solve with the
delayed-column update, and Form of the Schur complement S.

Default workload: a single supernode shaped like the paper's large random
examples (Section 7.1): n = 200000, p = 256, A11 symmetric and A21 with entries
uniform in [-1, 1], u = 0.01, relaxed compressed pivoting (on this input every
pivot is accepted, as with threshold partial pivoting; strict compressed
pivoting accepts 12 of 256), FP64 arithmetic throughout, S stored in FP64
(lower-packed, 160 GB).  Every timed step factors its own fresh copy of the
input (409 MB each, larger than L2), so no L2 flush is needed.  The line also
carries a "mixed" measurement of the same workload with the Form on the
tensor cores (BF16 operands, FP32 accumulation, S in FP32).

Metric: GFLOP/s of the supernode factorization under the flop model
  factor+solve = sum_{k=1..e} [(n-k) + 2((n-p)(p-k) + (p-k)(p-k+1)/2)]
  form         = (n-p)(n-p+1) e
with e = nelim (the pivots actually eliminated).  Compression and pivot search
are counted as overhead, not as flops.

Output: the last line on stdout is one compact JSON object (the headline:
metric, value, roofline, cpu_baseline, e2e, clocks, backward errors and the
batch's mixed-versus-FP64 pair, under 2 KB).  Every other leg prints a short
summary line on stderr, and the complete record (kernel splits, autotuner
tables, every leg) is written to --full-out.

--impl reference times the CPU FP64 oracle on a bounded sample of the same
workload (the paper's method has no other reference implementation).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM traffic per launch from ncu captures (profiles/), valid only for the
# kernel source they were taken on (sha1 of the .cu file).
# Measured at a smaller size than the bench's and scaled by the units one launch
# processes (the traffic of the Forms is the S they write, proportional to the
# number of S entries; the Solve's is proportional to the rows of A21): see
# profiles/ for the captures.
NCU_TRAFFIC = {
    # ncu --set full, n=20000 p=256 relaxed, S FP64 lower-packed: 163.66 MB read +
    # 1512.10 MB written for m(m+1)/2 = 194,921,640 entries
    "form_fp64": {"file": "form.cu", "sha1": "bed329d47e2e3d13657366883dcf61b1968adf7a",
                  "unit": "packed_entry", "bytes_per_unit": (163.662592e6 + 1512.099e6) / 194921640},
    # ncu --set full, n=40000 p=256 relaxed, split BF16 on SM pairs, S FP32 in 128x128
    # blocks: 89.63 MB read + 3118.79 MB written for 48,516 blocks of 16,384 entries
    "form_tc_bf16x3": {"file": "form_tc.cu", "sha1": "488eb8cb39a135fe2b96ff90b589d43a008cdf37",
                       "unit": "tiled_entry", "bytes_per_unit": (89.629184e6 + 3118.794e6) / (48516 * 16384)},
    # ncu --set full, n=40000 p=256 relaxed, tensor-core Solve before a split-BF16
    # Form (prep + gather + GEMM): 144.97 MB read + 124.87 MB written for 39,744 rows
    "solve_tc": {"file": "solve_tc.cu", "sha1": "986f68bd883bd413248fac53507ed870abbd31cb", "prec": "bf16x3",
                 "unit": "row", "bytes_per_unit": (144.965376e6 + 124.866e6) / 39744},
    # ncu --set full, n=200000 p=256 strict: 409.64 MB read + 3.59 MB written for
    # 199,744 A21 rows
    "compress_strict": {"file": "compress.cu", "sha1": "64d01d59c6c3d5f92ce7b20d803e44db5ce0659b",
                        "unit": "row", "bytes_per_unit": (409.639936e6 + 3.588608e6) / 199744},
    # ncu --set full, n=200000 p=256 relaxed, the four launches of one compression
    # (block maxima, per-column top-K, greedy, gather): 441.90 MB read + 8.10 MB
    # written for 199,744 A21 rows
    "compress_relaxed": {"file": "relaxed.cu", "sha1": "914805816d1f1d77f7a1c544998af6cea6749c3a",
                         "unit": "row", "bytes_per_unit": (409.117184e6 + 23.292928e6 + 0.161536e6 + 8.32768e6
                                                           + 8.1024e6) / 199744},
}


def max_over_ranks(x, dist):
    """The slowest rank's value of x (a time): the job ends when its last rank
    does.  Every rank gets the same result; dist is torch.distributed or None."""
    if not dist:
        return float(x)
    import torch
    tt = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt[0])


def job_rate(world, work_per_rank, seconds):
    """Whole-job throughput of `world` replicas that each did work_per_rank
    units in (at most) `seconds`."""
    return world * work_per_rank / seconds


def flops_model(n, p, e):
    m = n - p
    fs = 0
    for k in range(1, e + 1):
        fs += (n - k) + 2 * (m * (p - k) + (p - k) * (p - k + 1) // 2)
    form = m * (m + 1) * e
    return fs, form


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=200000)
    ap.add_argument("--p", type=int, default=256)
    ap.add_argument("--pivot", default="relaxed", choices=["strict", "relaxed", "restricted"])
    ap.add_argument("--smode", default="fp64_packed",
                    choices=["none", "fp32", "fp64", "fp32_packed", "fp64_packed", "fp32_tiled"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "bf16", "bf16x3", "bf16x6"],
                    help="Form arithmetic: FP64, or BF16 tensor cores with FP32 accumulation")
    ap.add_argument("--solve", default="fp64", choices=["fp64", "tc"],
                    help="Solve of the main leg: FP64, or on the tensor cores (with a tensor-core Form)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tpp", action="store_true",
                    help="skip the comparator: threshold partial pivoting on all rows (GPU)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched workload (8192 uneven supernodes, graph replay)")
    ap.add_argument("--batch-count", type=int, default=8192)
    ap.add_argument("--batch-eager", action="store_true",
                    help="time the batch by direct calls instead of CUDA-graph replay "
                         "(for profilers that cannot follow graph replays)")
    ap.add_argument("--no-system", action="store_true",
                    help="skip the complete-system leg (2-node embedding, refinement)")
    ap.add_argument("--no-multifrontal", action="store_true",
                    help="skip the multifrontal leg (64^3 Laplacian)")
    ap.add_argument("--no-delays", action="store_true",
                    help="skip the delayed-pivot count leg of --all")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the extra measurement with the Form on the tensor cores")
    ap.add_argument("--all", action="store_true",
                    help="also run the context legs: complete system, multifrontal (64^3), "
                         "GPU TPP comparator, FP64-Solve and plain-BF16 mixed legs, plain-BF16 batch")
    ap.add_argument("--full-out", default=os.path.join("gpurun_out", "bench_full.json"),
                    help="file that receives the complete record of every leg")
    return ap.parse_args(argv)


def workload_name(a):
    kind = {"strict": "strict compressed", "relaxed": "relaxed compressed",
            "restricted": "restricted"}[a.pivot]
    return f"single supernode n={a.n} p={a.p}, A11/A21 U[-1,1], u=0.01, {kind} pivoting"


# --------------------------------------------------------------------------- CPU oracle

def oracle_sample(a, target_s=12.0, with_error=False):
    """Time the CPU oracle (single thread) on a bounded sample of the workload:
    the first m_s rows of A21 for the factor+solve and the first m_f rows for
    the Form.  Returns (flops, seconds, description), plus the oracle factor's
    own backward error on that sample (untimed) when with_error is set."""
    from oracle import oracle
    from paper_1305_2353_gb300 import inputs
    A = inputs.single_large(a.seed, n=a.n, p=a.p)
    p = a.p
    ms = min(a.n - p, 20000)
    As = np.asfortranarray(A[:p + ms])
    t0 = time.perf_counter()
    r = oracle.factor(As, p, a.pivot)
    t_fs = time.perf_counter() - t0
    e = r["nelim"]
    fs, _ = flops_model(p + ms, p, e)
    mf = ms
    if a.smode != "none" and e > 0:
        # Form on the first m_f rows, sized to fit the time budget (~1 GFLOP/s)
        budget = max(target_s - t_fs, 2.0)
        mf = int(min(ms, max(200, np.sqrt(budget * 1.0e9 / max(e, 1)))))
        t1 = time.perf_counter()
        oracle.form(r["A"][p:p + mf, :e], r["piv"][:e], r["D"])
        t_form = time.perf_counter() - t1
        form = mf * (mf + 1) * e
    else:
        t_form, form = 0.0, 0
    desc = (f"oracle factor+solve on the first {ms} A21 rows (n={p + ms}, p={p}, nelim={e}) and "
            f"Form on the first {mf} rows; single-threaded C, -O2")
    if not with_error:
        return fs + form, t_fs + t_form, desc
    rows = np.arange(ms)
    oerr = factor_errors(As, r["A"], r["perm"], r["piv"], r["D"], e, p, rows)
    return fs + form, t_fs + t_form, desc, oerr


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    for i in range(a.warmup + a.steps):
        fl, t, desc = oracle_sample(a, target_s=6.0)
        if i >= a.warmup:
            vals.append((fl, t))
    fl = sum(v[0] for v in vals)
    t = sum(v[1] for v in vals)
    value = fl / t / 1e9
    line = {
        "impl": "reference", "metric": "Supernode LDL^T GFLOP/s", "value": value,
        "unit": "GFLOP/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * t / len(vals), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "n": a.n, "p": a.p, "pivot": a.pivot,
                   "smode": a.smode},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def fp64_peak_tflops(torch, dev, N=6144, reps=10):
    """FP64 matrix-multiply throughput of this GPU, measured now: torch.matmul
    (cuBLAS DGEMM) on N x N float64 operands, best of `reps` after two warm-up
    products, timed with CUDA events."""
    x = torch.randn(N, N, dtype=torch.float64, device=dev)
    y = torch.randn(N, N, dtype=torch.float64, device=dev)
    for _ in range(2):
        x @ y
    best = 1e9
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(reps):
        s.record()
        x @ y
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e) / 1e3)
    del x, y
    return 2 * N ** 3 / best / 1e12


def fp64_alu_peak_tflops(sm_mhz=2070.0, sms=152):
    """FP64 peak from unit counts and clock: GB300 issues 2 FP64 FMAs per clock
    per SM (the nominal 1.25 TFLOP/s at 2070 MHz over 152 SMs)."""
    return sms * 2 * 2 * sm_mhz * 1e6 / 1e12


def ncu_traffic(name, m, prec=None):
    """DRAM bytes of one launch of `name` on m rows, from the ncu record, or None
    when there is none, it was taken at another precision, or the kernel's
    source changed since it was taken."""
    rec = NCU_TRAFFIC.get(name)
    if rec is None or (prec is not None and rec.get("prec", prec) != prec):
        return None
    src_file = os.path.join(ROOT, "paper_1305_2353_gb300", "csrc", rec["file"])
    if hashlib.sha1(open(src_file, "rb").read()).hexdigest() != rec["sha1"]:
        return None
    nbk = (m + 127) // 128
    units = {"row": m, "packed_entry": m * (m + 1) // 2,
             "tiled_entry": nbk * (nbk + 1) // 2 * 16384}[rec["unit"]]
    return rec["bytes_per_unit"] * units


def kernel_roofline(name, launches, ms, a, e, peaks, prec="fp64"):
    """Algorithmic work of one launch of `name` and its roofline."""
    n, p = a.n, a.p
    m = n - p
    t = ms / launches / 1e3
    if name == "solve_tc":
        # A21 read and overwritten in FP64, the Form's BF16 operand pieces (W21
        # and L21) written; the split copy of x_e is the kernel's own scratch
        fp = {"bf16": 1, "bf16x3": 2, "bf16x6": 3}.get(prec, 1)
        work = 16.0 * m * p + 2 * fp * 2.0 * m * ((p + 63) // 64 * 64)
        bound, unit, peak, src = "hbm", "GB/s", peaks["hbm_gbs"], "MEASURED_PEAKS.json hbm_gbs"
        achieved = work / t / 1e9
    elif name in ("compress_strict", "compress_relaxed"):
        work = 8.0 * m * p
        bound, unit, peak, src = "hbm", "GB/s", peaks["hbm_gbs"], "MEASURED_PEAKS.json hbm_gbs"
        achieved = work / t / 1e9
    elif name in ("form_tc_bf16", "form_tc_bf16x3", "form_tc_bf16x6"):
        # S written as FP32 (lower triangle) dominates the bytes: 128 flop/byte at
        # e = 256 (x3 / x6 products per flop of S for the split forms), so the
        # HBM roofline bounds the plain form; the split forms approach the tensor one
        _, form = flops_model(n, p, e)
        pieces = {"form_tc_bf16": 1, "form_tc_bf16x3": 2, "form_tc_bf16x6": 3}[name]
        products = {1: 1, 2: 3, 3: 6}[pieces]
        work = 4.0 * m * (m + 1) / 2 + pieces * 2 * 2.0 * m * ((p + 63) // 64 * 64)
        form *= products  # tensor-core products actually executed
        hbm = work / t / 1e9
        tensor = form / t / 1e12
        # the method's work is bound by the bytes of S it writes (about 128 flop per byte at
        # e = 256): the roofline is HBM on the algorithmic bytes; the tensor rate of the
        # products actually executed (3 or 6 per flop for the split forms) is reported beside
        out = {"kernel": name, "bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": hbm / peaks["hbm_gbs"], "peak_source": "MEASURED_PEAKS.json hbm_gbs",
               "work_per_launch": work, "hbm_gbs": hbm, "hbm_frac": hbm / peaks["hbm_gbs"],
               "products_per_flop": products, "tensor_tflops_executed": tensor,
               "tensor_frac_executed_of_bf16_burst": tensor / peaks["bf16_tflops"],
               "method_tflops": tensor / products, "method_frac_of_bf16_burst": tensor / products / peaks["bf16_tflops"]}
        out["traffic"] = ncu_traffic(name, m, prec)
        out["launch_ms"] = ms / launches
        return out
    elif name in ("form_fp64", "solve_fp64"):
        fs, form = flops_model(n, p, e)
        work = form if name == "form_fp64" else fs
        bound, unit, peak = "alu", "TFLOP/s", peaks["fp64_tflops"]
        src = "measured in this run: torch.matmul float64 6144^3, best of 10"
        achieved = work / t / 1e12
    elif name == "factor_cluster":
        # right-looking FP64 update of [A11; C] per accepted pivot: ~2p(2p - k)
        # FLOP for pivot k (latency-bound: one cluster barrier per round)
        work = sum(2.0 * p * (2 * p - k) for k in range(e))
        bound, unit, peak = "alu", "TFLOP/s", peaks["fp64_tflops"]
        src = "measured in this run: torch.matmul float64 6144^3, best of 10"
        achieved = work / t / 1e12
    else:
        return None
    traffic = ncu_traffic(name, m, prec)
    out = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
           "frac": achieved / peak, "traffic": traffic, "peak_source": src,
           "work_per_launch": work, "launch_ms": ms / launches}
    if bound == "alu":
        alu = fp64_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
        out["alu_peak"] = alu
        out["frac_of_alu_peak"] = achieved / alu
    return out


def unpack_factor(Af, perm, piv, D, e, p):
    """L (rows of Af, e columns, unit diagonal on the A11 rows), the e x e block
    diagonal D and the delayed columns R from the in-place output layout of
    ctp_factor_supernode (Af: the output rows 0..p-1 followed by any A21 rows)."""
    nr = Af.shape[0]
    L = np.zeros((nr, e))
    L[:p] = np.tril(Af[:p, :e], -1)
    L[np.arange(e), np.arange(e)] = 1.0
    L[p:] = Af[p:, :e]
    Dm = np.zeros((e, e))
    for k in range(e):
        if piv[k] == 1:
            Dm[k, k] = D[2 * k]
        elif piv[k] == 2:
            Dm[k, k], Dm[k + 1, k + 1] = D[2 * k], D[2 * k + 2]
            Dm[k + 1, k] = Dm[k, k + 1] = D[2 * k + 1]
            L[k + 1, k] = 0.0  # that slot holds D's off-diagonal
    R = np.zeros((nr, p))
    R[:, e:] = Af[:, e:]
    return L, Dm, R


def factor_errors(A_host, Af, perm, piv, D, e, p, rows):
    """Backward error of a factored supernode, FP64 on the host, over the A11
    block and the A21 rows `rows`:
      raw    = max |P A P^T - (L D L^T + [0; R])| / max |A|
      scaled = the same maximum / max (|L||D||L^T| + |R|)   (growth-normalised)
    over the stored trapezoid (lower triangle of the A11 block, every column of
    the sampled A21 rows).  Af holds the output rows 0..p-1, then the output
    rows p + rows."""
    P = np.asarray(perm, np.int64)
    A11 = np.tril(A_host[:p, :p])
    A11 = A11 + np.tril(A11, -1).T
    orig = np.vstack([A11[np.ix_(P, P)], A_host[p + rows][:, P]])
    L, Dm, R = unpack_factor(Af, perm, piv, D, e, p)
    rec = L @ (L[:p] @ Dm).T + R
    scale = np.abs(L) @ (np.abs(L[:p]) @ np.abs(Dm)).T + np.abs(R)
    mask = np.ones(orig.shape, bool)
    mask[:p] = np.tril(np.ones((p, p), bool))
    r = np.abs(orig - rec)[mask].max()
    return {"raw": float(r / np.abs(A_host).max()), "growth_normalised": float(r / scale[mask].max()),
            "growth": float(scale[mask].max() / np.abs(A_host).max())}


def s_index(i, j, m, smode):
    """Linear index of S(i, j), i >= j, in the layout of ctp_smode."""
    if smode.endswith("packed"):
        return j * m - j * (j - 1) // 2 + (i - j)
    if smode.endswith("tiled"):
        nb = (m + 127) // 128
        bi, bj = i // 128, j // 128
        return 16384 * (bj * nb - bj * (bj - 1) // 2 + bi - bj) + (j % 128) * 128 + (i % 128)
    return j * m + i


def result_errors(A_host, Abuf, perm, piv, D, e, p, S, smode, seed=0, nrows=2048, nent=4096):
    """Per-result accuracy of one factored supernode: the factor's backward
    error (factor_errors) over the A11 block and `nrows` seeded A21 rows (the
    last row included), and, when S was written, the largest error of `nent`
    sampled S entries against S = L21 D11 L21^T formed in FP64 from this
    factor, relative to |L21||D11||L21^T| (the Form's own error)."""
    import torch
    n = A_host.shape[0]
    m = n - p
    rng = np.random.default_rng(seed + 77)
    rows = np.unique(np.concatenate([rng.choice(m, size=min(nrows, m), replace=False), [m - 1]])) \
        if m > 0 else np.zeros(0, np.int64)
    idx = torch.from_numpy(np.concatenate([np.arange(p), p + rows]).astype(np.int64)).to(Abuf.device)
    Af = Abuf[:, idx].T.cpu().numpy().astype(np.float64)   # (p + |rows|) x p
    pv, kv, Dv = perm.cpu().numpy(), piv.cpu().numpy(), D.cpu().numpy()
    out = {"factor": factor_errors(A_host, Af, pv, kv, Dv, e, p, rows), "a21_rows_sampled": int(len(rows))}
    if S is not None and smode != "none" and m > 0 and e > 0:
        L, Dm, _ = unpack_factor(Af, pv, kv, Dv, e, p)
        L21 = L[p:]
        ii = rng.integers(0, len(rows), nent)
        jj = rng.integers(0, len(rows), nent)
        lo, hi = np.minimum(ii, jj), np.maximum(ii, jj)
        lo[:64], hi[:64] = np.arange(64) % len(rows), np.arange(64) % len(rows)   # diagonal entries
        gi, gj = rows[hi], rows[lo]
        lin = torch.from_numpy(np.array([s_index(int(a), int(b), m, smode) for a, b in zip(gi, gj)],
                                        np.int64)).to(S.device)
        got = S.reshape(-1)[lin].double().cpu().numpy()
        W = L21 @ Dm
        ref = np.einsum("ik,ik->i", L21[hi], W[lo])
        scale = np.einsum("ik,ik->i", np.abs(L21[hi]), np.abs(L21[lo]) @ np.abs(Dm))
        out["form"] = {"entries_sampled": int(nent),
                       "max_rel_to_scale": float((np.abs(got - ref) / np.maximum(scale, 1e-300)).max())}
    return out


def measure(a, ctx, dev, A_host, prec, smode, steps, warmup, e2e_steps, peaks, world, dist, solve="fp64"):
    """Time `steps` factorizations (after `warmup`), each on a fresh input copy.
    Returns a dict of the measured quantities."""
    import torch
    from paper_1305_2353_gb300 import ctp
    n, p = a.n, a.p
    m = n - p
    opt = ctp.options(pivot=a.pivot, smode=smode, prec=prec, solve=solve)
    A0 = ctp.colmajor(A_host, dev)
    bufs = [A0.clone() for _ in range(warmup + steps)]
    perm = torch.empty(p, dtype=torch.int32, device=dev)
    piv = torch.empty(p, dtype=torch.int32, device=dev)
    D = torch.empty(2 * p, dtype=torch.float64, device=dev)
    nelim = torch.empty(1, dtype=torch.int32, device=dev)
    S = None
    if smode != "none":
        dt = torch.float64 if smode.startswith("fp64") else torch.float32
        if smode.endswith("packed"):
            S = torch.empty(m * (m + 1) // 2, dtype=dt, device=dev)
        elif smode.endswith("tiled"):
            nb = (m + 127) // 128
            S = torch.empty(nb * (nb + 1) // 2 * 16384, dtype=dt, device=dev)
        else:
            S = torch.empty((m, m), dtype=dt, device=dev)
    ws = ctx.workspace(n, p, opt)
    stream = torch.cuda.current_stream()

    def step(buf):
        ctx.factor_supernode(buf, n, p, n, opt, perm, piv, D, nelim, S, max(m, 1), ws, stream)

    tuned = None
    if prec != "fp64" and smode != "none":
        # the library's autotuner picks the tensor-core Form's tile walk and the
        # pivot search's cluster width for this workload (untimed)
        names = {1: "round_robin", 2: "chunks", 3: "panels"}
        cand = [(w, g) for w in (1, 2, 3) for g in (0, 8)]
        tms, best = ctp.autotune_supernode(ctx, bufs[0], n, p, n, opt, perm, piv, D, nelim, S,
                                           max(m, 1), ws, [ctp.TUNE_FORM_WALK, ctp.TUNE_FACTOR_G],
                                           cand, stream)
        tuned = {"form_walk": names[cand[best][0]], "factor_G": cand[best][1] or "auto",
                 "candidates_ms": {f"{names[w]}/G{g or 'auto'}": float(t)
                                   for (w, g), t in zip(cand, tms)}}

    for i in range(warmup):
        step(bufs[i])
    torch.cuda.synchronize()
    info = ctx.read_info(ws)
    if info != 0:
        raise RuntimeError(f"device info {info}")
    e = int(nelim.cpu()[0])

    clocks = ClockSampler(int(dev.split(":")[1]))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ctx.profile_begin()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(steps):
        step(bufs[warmup + i])
    t1.record(stream)
    torch.cuda.synchronize()
    kern = ctx.profile_end()
    clk = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1), dist)
    fs, form = flops_model(n, p, e)
    flops_step = fs + (form if smode != "none" else 0)
    value = job_rate(world, flops_step * steps, ms / 1e3) / 1e9
    # backward error of this result (the last timed step's factor and S), in
    # FP64 on the host over the A11 block and sampled A21 rows
    err = result_errors(A_host, bufs[-1], perm, piv, D, e, p, S, smode, seed=a.seed)
    del bufs

    # e2e through the public API with host buffers: H2D of the supernode from
    # pinned memory, the factorization, D2H of the factor and the pivots
    e2e = None
    if e2e_steps > 0:
        hA = torch.from_numpy(np.ascontiguousarray(A_host.T)).pin_memory()
        hOut = torch.empty_like(hA).pin_memory()
        hp = torch.empty(p, dtype=torch.int32).pin_memory()
        hv = torch.empty(p, dtype=torch.int32).pin_memory()
        hD = torch.empty(2 * p, dtype=torch.float64).pin_memory()
        hn = torch.empty(1, dtype=torch.int32).pin_memory()
        dA = torch.empty_like(A0)

        def e2e_step():
            dA.copy_(hA, non_blocking=True)
            step(dA)
            hOut.copy_(dA, non_blocking=True)
            hp.copy_(perm, non_blocking=True)
            hv.copy_(piv, non_blocking=True)
            hD.copy_(D, non_blocking=True)
            hn.copy_(nelim, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        s0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - s0, dist)
        e2e = {"value": job_rate(world, flops_step * e2e_steps, te) / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": hA.numel() * 8,
               "d2h_bytes_per_step": hOut.numel() * 8 + hp.numel() * 4 + hv.numel() * 4 +
               hD.numel() * 8 + 4}
    del S, A0, ws
    torch.cuda.empty_cache()
    top = max(kern.items(), key=lambda kv: kv[1][1])
    roof = kernel_roofline(top[0], top[1][0], top[1][1], a, e, peaks, prec)
    others = {k: kernel_roofline(k, v[0], v[1], a, e, peaks, prec) for k, v in kern.items() if k != top[0]}
    ctx.tune_set(ctp.TUNE_FORM_WALK, 0)
    ctx.tune_set(ctp.TUNE_FACTOR_G, 0)
    return dict(value=value, ms=ms, e=e, fs=fs, form=form, flops_step=flops_step, kern=kern,
                clocks=clk, e2e=e2e, roofline=roof, launches=sum(v[0] for v in kern.values()),
                autotune=tuned, rooflines_other={k: v for k, v in others.items() if v is not None},
                errors=err)


def measure_batch(a, ctx, dev, fronts, prec, smode, steps, warmup, accuracy=0):
    """The batched path on many uneven supernodes: the batch call captured once
    into a CUDA graph; each timed replay factors freshly restored inputs (the
    restore runs outside the timed events).  With accuracy > 0, that many
    fronts of the last timed replay are checked for accuracy with their own
    factors (batch_accuracy)."""
    import torch
    from paper_1305_2353_gb300 import ctp
    opt = ctp.options(pivot="strict", prec=prec, smode=smode)
    b = ctp.Batch(ctx, fronts, [f.shape[1] for f in fronts], opt)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    # the library's autotuner: cluster budget of the pivot search and the
    # tensor-core Form's tile walk, timed on this batch (untimed here)
    names = {0: "auto", 1: "round_robin", 2: "chunks"}
    kbs = [64, 100, 160, 220]
    walks = [2, 1] if prec != "fp64" else [0]
    cand = [(k, w) for k in kbs for w in walks]
    tms, best = b.autotune([ctp.TUNE_BATCH_SMEM_KB, ctp.TUNE_FORM_WALK], cand)
    tuned = {"smem_kb": cand[best][0], "form_walk": names[cand[best][1]],
             "candidates_ms": {f"{k}KB/{names[w]}": float(t) for (k, w), t in zip(cand, tms)}}
    b.run()
    torch.cuda.synchronize()
    # kernel split from one profiled run outside the graph
    b.reset()
    ctx.profile_begin()
    b.run()
    torch.cuda.synchronize()
    kern = ctx.profile_end()
    flags = b.flags()
    if a.batch_eager:
        g = None
        launch = b.run
    else:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            b.run(stream=stream)
        launch = g.replay
    for _ in range(warmup):
        b.reset()
        launch()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        b.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        launch()
        e1.record()
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    ne = b.nelim.cpu().numpy()
    fs = form = 0
    for k in range(b.nb):
        f1, f2 = flops_model(int(b.n[k]), int(b.p[k]), int(ne[k]))
        fs += f1
        form += f2 if smode != "none" else 0
    ms = total / steps
    acc = batch_accuracy(ctx, b, fronts, count=accuracy) if accuracy > 0 else None
    del g, b
    ctx.tune_set(ctp.TUNE_BATCH_SMEM_KB, 200)
    ctx.tune_set(ctp.TUNE_FORM_WALK, 0)
    import gc
    gc.collect()
    torch.cuda.empty_cache()
    return {"value": (fs + form) / (ms / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_batch": ms,
            "prec": prec, "S": smode, "factor_solve_flops": fs, "form_flops": form,
            "nelim_total": int(ne.sum()), "p_total": int(sum(f.shape[1] for f in fronts)),
            "device_flags_nonzero": int((flags != 0).sum()), "autotune": tuned, "accuracy": acc,
            "gpu_launches": sum(v[0] for v in kern.values()),
            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in kern.items()}}


def refine_embedded(ctx, dev, A, prec, b, mr="tpp", w_rest=256, seed=0, solve="fp64"):
    """Embed supernode A in its complete system M (inputs.two_node), factor M on
    the GPU as a chain of fronts (the first the supernode, its Form in `prec`),
    refine with FP64 residuals.  Returns timings, steps and backward errors."""
    import torch
    from paper_1305_2353_gb300 import ctp, inputs
    M = inputs.two_node(A, seed)
    N, p = M.shape[0], A.shape[1]
    Mlow = ctp.colmajor(np.tril(M), dev)
    Md = ctp.colmajor(M, dev)
    B = ctp.colmajor(b, dev)
    X = torch.zeros_like(B)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ch = ctp.factor_dense(ctx, Md, N, N, p, ctp.options(pivot="strict", prec=prec, solve=solve), w_rest,
                          ctp.options(pivot=mr))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ws = ctp.refine_workspace(ctx, N, N, b.shape[1])
    ctx.profile_begin()
    t2 = time.perf_counter()
    hist, k = ctp.refine(ctx, ch.fronts, ch.nf, N, Mlow, N, b.shape[1], B, N, X, N, ws)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    kern = ctx.profile_end()
    out = {"prec_first_front": prec, "solve_first_front": solve, "fronts": ch.nf, "nelim_first": int(ch.nelim[0]),
           "factor_ms": (t1 - t0) * 1e3, "refine_ms": (t3 - t2) * 1e3, "corrections": k,
           "bwd_err_history": [float(v) for v in hist.max(axis=1)],
           "kernels": {kk: {"launches": v[0], "ms": v[1]} for kk, v in kern.items()}}
    ch.destroy()
    del Md, Mlow, B, X, ws
    torch.cuda.empty_cache()
    return out


def measure_system(ctx, dev, inputs):
    """The complete-system leg: the n = 2000, p = 64 supernode with eight tiny
    columns embedded in its 2000 x 2000 system (A22 symmetric N(0,1)), strict
    compressed pivoting on the supernode, threshold partial pivoting on the
    rest, Section 7 backward error after FP64 refinement (at most ten
    corrections, stop at 1e-14), for each precision of the supernode's Form."""
    A = inputs.single_small(0)
    b = np.random.default_rng(1).standard_normal((A.shape[0], 1))
    out = {"workload": "n=2000 p=64 supernode (8 columns scaled 1e-8) in its 2-node system, "
                       "1 RHS N(0,1), tol 1e-14, <= 10 corrections"}
    for prec in ("fp64", "bf16x3", "bf16"):
        out[prec] = refine_embedded(ctx, dev, A, prec, b)
    # Solve and Form of the supernode on the tensor cores
    for prec in ("bf16x3", "bf16x6"):
        out[prec + "_tc_solve"] = refine_embedded(ctx, dev, A, prec, b, solve="tc")
    return out


def measure_multifrontal(ctx, dev, inputs, k=64, nrhs=16):
    """Config 4: the 7-point Laplacian on a k^3 grid shifted by -3 I (indefinite),
    geometric nested dissection, multifrontal factorization with strict
    compressed pivoting (FP64, and with split-BF16 Forms), then nrhs N(0,1)
    right-hand sides solved with FP64 refinement against the sparse matrix."""
    import torch
    from paper_1305_2353_gb300 import ctp
    cp, ri, v = inputs.laplacian_3d(k, 3.0)
    perm, blocks = inputs.nested_dissection_3d(k, 64)
    N = k ** 3
    t0 = time.perf_counter()
    mf = ctp.Multifrontal(ctx, cp, ri, v, perm, blocks)
    t_an = time.perf_counter() - t0
    B = np.random.default_rng(0).standard_normal((N, nrhs))
    out = {"workload": f"7-point Laplacian {k}^3 shifted by -3I (N={N}, nnz(lower)={len(v)}), geometric "
                       f"nested dissection ({len(blocks) - 1} blocks, leaves <= 64 points), strict "
                       f"compressed pivoting, {nrhs} RHS N(0,1), refinement to 1e-14 (<= 10 steps)",
           "analyse_s": t_an}
    for prec in ("fp64", "bf16x6", "bf16x3"):
        opt = ctp.options(pivot="strict", prec=prec)
        mf.factor(opt)   # warm-up (allocations, module loads)
        torch.cuda.synchronize()
        ctx.profile_begin()
        t0 = time.perf_counter()
        mf.factor(opt)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        kern = ctx.profile_end()
        n, p, e, _ = mf.panel_info()
        fs = form = 0
        for a, b, c in zip(n, p, e):
            f1, f2 = flops_model(int(a), int(b), int(c))
            fs += f1
            form += f2
        info = mf.info()
        Bd = ctp.colmajor(B, dev)
        X = torch.zeros_like(Bd)
        ws = mf.refine_workspace(nrhs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist, steps = mf.refine(Bd, X, ws)
        torch.cuda.synchronize()
        tr = time.perf_counter() - t0
        out[prec] = {"factor_s": tf, "factor_gflops": (fs + form) / tf / 1e9,
                     "flops": fs + form, "panels": int(mf.nf),
                     "max_front_n": int(info["n"].max()), "delayed_total": int(info["delayed"].sum()),
                     "refine_s": tr, "corrections": steps,
                     "bwd_err_history": [float(x) for x in hist.max(axis=1)],
                     "kernels": {kk: {"launches": vv[0], "ms": vv[1]} for kk, vv in kern.items()}}
        del Bd, X, ws
        if prec in ("fp64", "bf16x6"):
            out[prec]["gradient"] = measure_mf_gradient(mf, dev, N, len(v), nrhs=32)
    mf.destroy()
    torch.cuda.empty_cache()
    return out


def measure_mf_gradient(mf, dev, N, nnz, nrhs=32):
    """Config 5 through config 4's factorization: x = M^{-1} B for nrhs N(0,1)
    right-hand sides (refined), loss = ||x||^2, the refined adjoint solve
    grad_B = M^{-T} (2x) with the same factors and pivots, and the gradient of
    the stored lower-triangle entries (the sparsity pattern)."""
    import torch
    from paper_1305_2353_gb300 import ctp
    B = ctp.colmajor(np.random.default_rng(5).standard_normal((N, nrhs)), dev)
    X = torch.zeros_like(B)
    Gb = torch.zeros_like(B)
    gval = torch.empty(nnz, dtype=torch.float64, device=dev)
    ws = mf.refine_workspace(nrhs)
    mf.grad_values(Gb, X, gval)   # warm-up: pattern upload, module load
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hx, kx = mf.refine(B, X, ws)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    G = 2.0 * X
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    hg, kg = mf.refine(G, Gb, ws)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    mf.grad_values(Gb, X, gval)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    loss = float((X * X).sum())
    return {"nrhs": nrhs, "solve_s": t1 - t0, "adjoint_s": t3 - t2, "grad_pattern_s": t4 - t3,
            "loss": loss, "solve_corrections": kx, "adjoint_corrections": kg,
            "solve_bwd_err": float(hx[-1].max()), "adjoint_bwd_err": float(hg[-1].max()),
            "grad_abs_max": float(gval.abs().max())}


def batch_accuracy(ctx, b, fronts, count=12, seed=0):
    """Equal-accuracy check with the timed batch's own factors.  For a seeded
    sample of fronts spread over n*p, front k as the batch call left it (L, D,
    pivots, and its Schur complement S in the batch's Form precision) is the
    first front of the 2-node system M = [[A11, A21^T], [A21, A22]] (A22
    symmetric N(0,1)); the rest of M -- the delayed columns and A22 - S -- is
    factored on the GPU by threshold partial pivoting (FP64), and M x = b is
    solved with FP64 refinement against M (Section 7: at most ten corrections,
    tolerance 1e-14).  Returns the worst final backward error and the most
    corrections over the sample."""
    import gc
    import torch
    from paper_1305_2353_gb300 import ctp, inputs
    rng = np.random.default_rng(seed)
    order = np.argsort([f.shape[0] * f.shape[1] for f in fronts])
    pick = [int(k) for k in order[np.linspace(0, len(order) - 1, count).astype(int)]]
    dev = f"cuda:{ctx.device}"
    worst, most, first = 0.0, 0, 0.0
    for k in pick:
        A = fronts[k]
        n, p = A.shape
        m = n - p
        r = b.result(k)
        e, perm, Af = r["nelim"], r["perm"].astype(np.int64), r["A"]
        d = p - e
        M = inputs.two_node(A, seed=k)
        hold = []
        f0 = ctp.SFront()
        f0.n, f0.p = n, p
        f0.L, f0.ldl = b.A.data_ptr() + 8 * int(b.a_off[k]), n
        f0.perm = b.perm.data_ptr() + 4 * int(b.p_off[k])
        f0.piv = b.piv.data_ptr() + 4 * int(b.p_off[k])
        f0.D = b.D.data_ptr() + 16 * int(b.p_off[k])
        f0.nelim = b.nelim.data_ptr() + 4 * k
        rows0 = torch.arange(n, dtype=torch.int32, device=dev)
        hold.append(rows0)
        f0.rows = rows0.data_ptr()
        fl = [f0]
        Np = d + m
        ch = None
        if Np > 0:
            # the parent: Schur complement of the eliminated pivots in M
            Mp = np.zeros((Np, Np))
            Db = np.tril(Af[e:p, e:p])
            Mp[:d, :d] = Db + np.tril(Db, -1).T
            Mp[d:, :d] = Af[p:, e:p]
            Mp[:d, d:] = Af[p:, e:p].T
            S = np.asarray(r["S"], np.float64) if "S" in r else np.zeros((m, m))
            S = np.tril(S) + np.tril(S, -1).T
            Mp[d:, d:] = M[p:, p:] - S
            Md = ctp.colmajor(Mp, dev)
            hold.append(Md)
            ch = ctp.factor_dense(ctx, Md, Np, Np, min(256, Np), ctp.options(pivot="tpp"), 256,
                                  ctp.options(pivot="tpp"))
            to_m = torch.from_numpy(np.concatenate([perm[e:p], p + np.arange(m)]).astype(np.int32)).to(dev)
            for q in range(ch.nf):
                fq = ctp.SFront.from_buffer_copy(ch.fronts[q])
                rq = to_m[ctp.device_view(fq.rows, int(fq.n)).long()].contiguous()
                hold.append(rq)
                fq.rows = rq.data_ptr()
                fl.append(fq)
        arr = (ctp.SFront * len(fl))(*fl)
        Mlow = ctp.colmajor(np.tril(M), dev)
        B = ctp.colmajor(rng.standard_normal((n, 1)), dev)
        X = torch.zeros_like(B)
        ws = ctp.refine_workspace(ctx, n, n, 1)
        hist, steps = ctp.refine(ctx, arr, len(fl), n, Mlow, n, 1, B, n, X, n, ws)
        torch.cuda.synchronize()
        hb = [float(v) for v in hist.max(axis=1)]
        worst, most, first = max(worst, hb[-1]), max(most, steps), max(first, hb[0])
        if ch is not None:
            ch.destroy()
        del hold, Mlow, B, X, ws
    gc.collect()
    torch.cuda.empty_cache()
    return {"fronts_checked": len(pick), "max_bwd_err": worst, "max_corrections": most,
            "max_bwd_err_before_refinement": first,
            "how": "the timed batch's own factors and S as the first front of each front's "
                   "2-node system; rest factored by TPP (FP64); FP64 refinement, tol 1e-14"}


def measure_delays(ctx, dev, inputs, batch_count=8192, seed=0):
    """Delayed pivots by method (NEXT-3; the analogue of the paper's delay
    comparisons, Section 7.2, on synthetic inputs): TPP on all rows, strict,
    relaxed, restricted and single-row compression, each supernode factored on
    its own through the C ABI.  Workloads: the 8192-front batch (N(0,1), 2%
    zero diagonals), a set of tough fronts (a sixth of the A11 columns scaled by
    1e-3, 20% zero diagonals, A21 x5), the n = 2000, p = 64 supernode with eight
    tiny columns, and the n = 200000, p = 256 U[-1,1] supernode."""
    import torch
    from paper_1305_2353_gb300 import ctp

    def tough(n, p, s):
        A = inputs.supernode(n, p, seed=s, dist="normal", scale_cols=max(1, p // 6), scale=1e-3,
                             zero_diag_frac=0.2)
        A[p:, :] *= 5.0
        return A

    sets = {
        "batch_8192": inputs.batch(batch_count, seed=seed),
        "tough_60": [tough(int(n), int(p), 1000 + k)
                     for k, (n, p) in enumerate(inputs.batch_shapes(60, seed=7, pmin=8, pmax=256))],
        "single_small": [inputs.single_small(0)],
        "single_large": [inputs.single_large(seed)],
    }
    methods = ("tpp", "strict", "relaxed", "restricted", "single_row")
    out = {}
    for name, fronts in sets.items():
        n = np.array([a.shape[0] for a in fronts], np.int64)
        p = np.array([a.shape[1] for a in fronts], np.int64)
        off = np.concatenate([[0], np.cumsum(n * p)])
        host = np.empty(int(off[-1]))
        for k, a in enumerate(fronts):
            host[off[k]:off[k + 1]] = np.asarray(a, np.float64).ravel(order="F")
        A0 = torch.from_numpy(host).to(dev)
        A = torch.empty_like(A0)
        pmax = int(p.max())
        perm = torch.empty(pmax, dtype=torch.int32, device=dev)
        piv = torch.empty(pmax, dtype=torch.int32, device=dev)
        D = torch.empty(2 * pmax, dtype=torch.float64, device=dev)
        nel = torch.empty(len(fronts), dtype=torch.int32, device=dev)
        row = {}
        t0 = time.perf_counter()
        for meth in methods:
            opt = ctp.options(pivot=meth)
            need = max(ctx.workspace_size(int(a), int(b), opt) for a, b in set(zip(n.tolist(), p.tolist())))
            ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
            A.copy_(A0)
            for k in range(len(fronts)):
                ctx.factor_supernode(A[int(off[k]):int(off[k + 1])], int(n[k]), int(p[k]), int(n[k]), opt,
                                     perm, piv, D, nel[k:k + 1], None, 0, ws)
            torch.cuda.synchronize()
            if ctx.read_info(ws) != 0:
                raise RuntimeError(f"device info after {name}/{meth}")
            e = nel.cpu().numpy().astype(np.int64)
            row[meth] = {"nelim": int(e.sum()), "delayed": int((p - e).sum()),
                         "fronts_with_delays": int((e < p).sum())}
            del ws
        out[name] = {"fronts": len(fronts), "columns": int(p.sum()), "by_method": row,
                     "seconds": time.perf_counter() - t0}
        del A0, A
        torch.cuda.empty_cache()
    return out


def leg_summary(name, d):
    """One short stderr line per leg (the complete record goes to --full-out)."""
    keep = {k: v for k, v in d.items() if isinstance(v, (int, float, str)) or v is None}
    print(json.dumps({"leg": name, **keep})[:600], file=sys.stderr, flush=True)


def _r(x, nd=4):
    """Round for the headline line (None passes through)."""
    if x is None:
        return None
    return float(f"{x:.{nd}g}")


def headline(rec):
    """The compact final line (at most 2 KB) built from the complete record."""
    main = rec["main"]
    roof = main["roofline"]
    cpu = rec.get("cpu_baseline")
    err = main["errors"]
    line = {
        "metric": rec["metric"], "value": _r(main["value"], 6), "unit": "GFLOP/s",
        "n_gpus": rec["n_gpus"], "steps": rec["steps"], "warmup": rec["warmup"],
        "ms_per_step": _r(main["ms"] / rec["steps"], 6), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": rec["dtype"], "data": "synthetic",
        "config": dict(rec["config"]),
        "roofline": {"kernel": roof["kernel"], "bound": roof["bound"], "achieved": _r(roof["achieved"]),
                     "peak": _r(roof["peak"]), "unit": roof["unit"], "frac": _r(roof["frac"]),
                     "traffic": _r(roof.get("traffic")), "peak_source": roof.get("peak_source", "")[:80]},
        "cpu_baseline": None if cpu is None else {
            "value": _r(cpu["value"]), "unit": cpu["unit"], "cores": cpu["cores"], "kind": cpu["kind"],
            "sample": cpu["sample"][:160]},
        "e2e": None if main["e2e"] is None else {k: _r(v) if isinstance(v, float) else v
                                                for k, v in main["e2e"].items()},
        "gpu_launches": main["launches"],
        "clocks": {k: main["clocks"].get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "bwd_err": {"factor_raw": _r(err["factor"]["raw"], 3),
                    "factor_growth_normalised": _r(err["factor"]["growth_normalised"], 3),
                    "form_rel": _r(err.get("form", {}).get("max_rel_to_scale"), 3)},
    }
    if "alu_peak" in roof:
        line["roofline"]["alu_peak"] = _r(roof["alu_peak"])
        line["roofline"]["frac_of_alu_peak"] = _r(roof["frac_of_alu_peak"])
    mx = rec.get("mixed")
    if mx:
        line["mixed"] = {"value": _r(mx["value"]), "ms_per_step": _r(mx["ms_per_step"]),
                         "dtype": "bf16x3 tensor-core Solve+Form, f32 S",
                         "form_frac_of_hbm": _r(mx["roofline"].get("hbm_frac", mx["roofline"].get("frac"))),
                         "form_tensor_frac_executed": _r(mx["roofline"].get("tensor_frac_executed_of_bf16_burst")),
                         "bwd_err_factor_growth_normalised": _r(mx["errors"]["factor"]["growth_normalised"], 3),
                         "form_rel": _r(mx["errors"].get("form", {}).get("max_rel_to_scale"), 3)}
    bt = rec.get("batch")
    if bt and bt.get("fp64") and bt.get("mixed"):
        f, x = bt["fp64"], bt["mixed"]
        line["config"]["batch_8192_mixed_vs_fp64"] = {
            "fp64_ms": _r(f["ms_per_batch"]), "mixed_ms": _r(x["ms_per_batch"]),
            "speedup": _r(f["ms_per_batch"] / x["ms_per_batch"]),
            "fp64_bwd_err": _r((f.get("accuracy") or {}).get("max_bwd_err"), 3),
            "mixed_bwd_err": _r((x.get("accuracy") or {}).get("max_bwd_err"), 3)}
    s = json.dumps(line)
    # never exceed 2 KB: drop context keys first
    for k in ("mixed", "bwd_err"):
        if len(s) <= 2000:
            break
        line.pop(k, None)
        s = json.dumps(line)
    return s


def run_native(a):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    from paper_1305_2353_gb300 import ctp, inputs

    # fallback when the measured peaks are absent: one earlier GB300 measurement
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
    if os.path.exists(MEASURED):
        peaks.update(json.load(open(MEASURED)))
    peaks["fp64_tflops"] = fp64_peak_tflops(torch, dev)
    ctx = ctp.Context(local)
    A_host = inputs.single_large(a.seed, n=a.n, p=a.p)
    rec = {"metric": "Supernode LDL^T GFLOP/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
           "peaks": peaks,
           "dtype": "f64" if a.prec == "fp64" else "f64 (Form: bf16 x bf16 -> f32)"}

    e2e_steps = 0 if a.no_e2e else min(a.steps, 3)
    main = measure(a, ctx, dev, A_host, a.prec, a.smode, a.steps, a.warmup, e2e_steps, peaks, world, dist,
                   solve=a.solve)
    rec["main"] = main
    rec["config"] = {"workload": workload_name(a), "n": a.n, "p": a.p, "u": 0.01, "pivot": a.pivot,
                     "prec": a.prec, "solve": a.solve, "S": a.smode, "nelim": main["e"],
                     "flops_per_step": main["flops_step"],
                     "l2": "inputs larger than L2: a distinct 409 MB input copy per step",
                     "parallelism": f"replicas x{world}"}
    leg_summary("main", {"value": main["value"], "ms_per_step": main["ms"] / a.steps, "nelim": main["e"],
                         "factor_err_growth_normalised": main["errors"]["factor"]["growth_normalised"]})

    def mixed_leg(prec, desc, solve="tc"):
        k = max(a.steps, 5)
        mx = measure(a, ctx, dev, A_host, prec, "fp32_tiled", k, max(a.warmup, 3),
                     0 if a.no_e2e else min(k, 3), peaks, world, dist, solve=solve)
        out = {"value": mx["value"], "unit": "GFLOP/s", "ms_per_step": mx["ms"] / k,
               "prec": desc, "solve": solve, "roofline": mx["roofline"],
               "rooflines_other": mx["rooflines_other"], "e2e": mx["e2e"], "errors": mx["errors"],
               "gpu_launches": mx["launches"],
               "kernels": {kk: {"launches": v[0], "ms": v[1]} for kk, v in mx["kern"].items()},
               "clocks": mx["clocks"], "autotune": mx["autotune"]}
        return out

    if not a.no_mixed and a.prec == "fp64":
        rec["mixed"] = mixed_leg("bf16x3", "Solve and Form on tensor cores: Solve as one product with "
                                           "three-piece split operands, Form with split operands hi*hi + "
                                           "hi*lo + lo*hi (bf16 x bf16 -> f32), S fp32 in 128x128 blocks; "
                                           "compression and pivot search f64")
        leg_summary("mixed", {"value": rec["mixed"]["value"], "ms_per_step": rec["mixed"]["ms_per_step"]})
        if a.all:
            rec["mixed_fp64_solve"] = mixed_leg("bf16x3", "as mixed, with the Solve in FP64", solve="fp64")
            rec["mixed_bf16"] = mixed_leg("bf16", "Solve on tensor cores (three-piece split), Form on "
                                                  "tensor cores bf16 x bf16 -> f32 (single product)")

    if a.all and rank == 0 and not a.no_system:
        rec["complete_system"] = measure_system(ctx, dev, inputs)
    if a.all and rank == 0 and not a.no_multifrontal:
        rec["multifrontal"] = measure_multifrontal(ctx, dev, inputs)

    if not a.no_batch:
        fronts = inputs.batch(a.batch_count, seed=a.seed)
        sh = np.array([[f.shape[0], f.shape[1]] for f in fronts])
        batch = {"workload": f"{a.batch_count} supernodes, p log-uniform [8,256], n-p log-uniform "
                             f"[0,16p], N(0,1), 2% zero diagonals, strict compressed pivoting",
                 "sum_np": int((sh[:, 0] * sh[:, 1]).sum()), "max_n": int(sh[:, 0].max()),
                 "median_p": int(np.median(sh[:, 1])), "median_m": int(np.median(sh[:, 0] - sh[:, 1])),
                 "timing": "CUDA graph of the batch call, replayed; inputs restored outside the "
                           "timed events; launch settings chosen by the library's autotuner first"}
        nacc = 12 if rank == 0 else 0
        batch["fp64"] = measure_batch(a, ctx, dev, fronts, "fp64", "fp64_packed", 3, 2, accuracy=nacc)
        leg_summary("batch_fp64", batch["fp64"])
        batch["mixed"] = measure_batch(a, ctx, dev, fronts, "bf16x3", "fp32_tiled", 3, 2, accuracy=nacc)
        leg_summary("batch_mixed", batch["mixed"])
        if a.all:
            batch["mixed_bf16"] = measure_batch(a, ctx, dev, fronts, "bf16", "fp32_tiled", 3, 2,
                                                accuracy=nacc)
        rec["batch"] = batch
        del fronts

    if a.all and rank == 0 and not a.no_delays:
        rec["delays"] = measure_delays(ctx, dev, inputs, a.batch_count, a.seed)
        for nm, v in rec["delays"].items():
            leg_summary("delays_" + nm, {m: d["delayed"] for m, d in v["by_method"].items()})

    if a.all and not a.no_tpp and a.pivot != "restricted":
        import argparse as _ap
        at = _ap.Namespace(**vars(a))
        at.pivot = "tpp"
        tp = measure(at, ctx, dev, A_host, "fp64", "none", 3, 1, 0, peaks, world, dist)
        comp_ms = sum(v[1] for k, v in main["kern"].items() if not k.startswith("form")) / a.steps
        rec["tpp_comparator"] = {
            "pivot": "tpp (Listing 1 on all n rows, GPU)", "nelim": tp["e"],
            "factor_solve_ms": tp["ms"] / 3, "factor_solve_gflops": tp["fs"] * 3 / (tp["ms"] / 1e3) / 1e9,
            "compressed_factor_solve_ms": comp_ms,
            "compressed_factor_solve_gflops": main["fs"] / (comp_ms / 1e3) / 1e9,
            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in tp["kern"].items()}}
        leg_summary("tpp_comparator", rec["tpp_comparator"])

    if rank == 0 and not a.no_cpu_baseline:
        fl, t, desc, oerr = oracle_sample(a, with_error=True)
        rec["cpu_baseline"] = {"value": fl / t / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                               "sample": desc, "oracle_factor_errors": oerr}
        leg_summary("cpu_baseline", {"value": rec["cpu_baseline"]["value"]})
    if rank == 0:
        rec["main"]["kernels"] = {k: {"launches": v[0], "ms": v[1]} for k, v in main["kern"].items()}
        if a.full_out:
            try:
                os.makedirs(os.path.dirname(os.path.abspath(a.full_out)), exist_ok=True)
                with open(a.full_out, "w") as fh:
                    json.dump(rec, fh, default=str)
            except OSError as ex:
                print(f"could not write {a.full_out}: {ex}", file=sys.stderr)
        print(headline(rec), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    a = parse_args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_native(a)


if __name__ == "__main__":
    main()
