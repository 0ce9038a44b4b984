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
    # ncu --set full, n=20000 p=256 relaxed, S FP64 lower-packed: 163.76 MB read +
    # 1513.69 MB written for m(m+1)/2 = 194,921,640 entries
    "form_fp64": {"file": "form.cu", "sha1": "798d569f67e7e8f417e75b162e2622426e55e05e",
                  "unit": "packed_entry", "bytes_per_unit": (163.760384e6 + 1513.690e6) / 194921640},
    # ncu --set full, n=40000 p=256 relaxed, split BF16, S FP32 in 128x128 blocks:
    # 188.44 MB read + 3118.11 MB written for 48,516 blocks of 16,384 entries
    "form_tc_bf16x3": {"file": "form_tc.cu", "sha1": "f42cb5618b32f27438bd8a88393945b4d1c3750f",
                       "unit": "tiled_entry", "bytes_per_unit": (188.438784e6 + 3118.110e6) / (48516 * 16384)},
    # ncu --set full, n=40000 p=256 relaxed, tensor-core Solve before a split-BF16
    # Form (prep + gather + GEMM): 145.23 MB read + 124.64 MB written for 39,744 rows
    "solve_tc": {"file": "solve_tc.cu", "sha1": "b625943159839444dd75e137c8f4021fbb3e3789", "prec": "bf16x3",
                 "unit": "row", "bytes_per_unit": (145.232896e6 + 124.638e6) / 39744},
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


def parse_args():
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
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the extra measurement with the Form on the tensor cores")
    return ap.parse_args()


def workload_name(a):
    kind = {"strict": "strict compressed", "relaxed": "relaxed compressed",
            "restricted": "restricted"}[a.pivot]
    return f"single supernode n={a.n} p={a.p}, A11/A21 U[-1,1], u=0.01, {kind} pivoting"


# --------------------------------------------------------------------------- CPU oracle

def oracle_sample(a, target_s=12.0):
    """Time the CPU oracle (single thread) on a bounded sample of the workload:
    the first m_s rows of A21 for the factor+solve and the first m_f rows for
    the Form.  Returns (flops, seconds, description)."""
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
    return fs + form, t_fs + t_form, desc


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


def fp64_peak_tflops(torch, dev):
    """cuBLAS DGEMM throughput on this GPU, measured now (best of 5, 4096^3)."""
    N = 4096
    x = torch.randn(N, N, dtype=torch.float64, device=dev)
    y = torch.randn(N, N, dtype=torch.float64, device=dev)
    for _ in range(2):
        x @ y
    best = 1e9
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(5):
        s.record()
        x @ y
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e) / 1e3)
    del x, y
    return 2 * N ** 3 / best / 1e12


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
        if pieces == 1:  # one product per flop: the S stores bound it
            out = {"kernel": name, "bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                   "frac": hbm / peaks["hbm_gbs"], "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                   "work_per_launch": work, "tensor_tflops": tensor}
        else:  # three or six products per flop: the tensor pipe bounds it (launches of ~25 ms: burst peak)
            out = {"kernel": name, "bound": "tensor", "achieved": tensor, "peak": peaks["bf16_tflops"],
                   "unit": "TFLOP/s", "frac": tensor / peaks["bf16_tflops"],
                   "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)", "work_per_launch": form,
                   "products_per_flop": products, "hbm_gbs": hbm, "hbm_frac": hbm / peaks["hbm_gbs"],
                   "hbm_bytes_per_launch": work}
        out["tensor_frac_of_bf16_sustained"] = tensor / peaks.get("bf16_tflops_sustained", 1715.6)
        out["traffic"] = ncu_traffic(name, m, prec)
        out["launch_ms"] = ms / launches
        return out
    elif name in ("form_fp64", "solve_fp64"):
        fs, form = flops_model(n, p, e)
        work = form if name == "form_fp64" else fs
        bound, unit, peak = "alu", "TFLOP/s", 1.25
        src = ("nominal GB300 FP64 1.25 TFLOP/s (profiling recipe table; no FP64 entry in "
               "MEASURED_PEAKS.json); cuBLAS DGEMM 4096^3 in this run: %.3f" % peaks["fp64_tflops"])
        achieved = work / t / 1e12
    elif name == "factor_cluster":
        # right-looking FP64 update of [A11; C] per accepted pivot: ~2p(2p - k)
        # FLOP for pivot k (latency-bound: one cluster barrier per round)
        work = sum(2.0 * p * (2 * p - k) for k in range(e))
        bound, unit, peak = "alu", "TFLOP/s", 1.25
        src = "nominal GB300 FP64 1.25 TFLOP/s (profiling recipe table)"
        achieved = work / t / 1e12
    else:
        return None
    traffic = ncu_traffic(name, m, prec)
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic, "peak_source": src,
            "work_per_launch": work, "launch_ms": ms / launches}


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
                autotune=tuned, rooflines_other={k: v for k, v in others.items() if v is not None})


def measure_batch(a, ctx, dev, fronts, prec, smode, steps, warmup):
    """The batched path on many uneven supernodes: the batch call captured once
    into a CUDA graph; each timed replay factors freshly restored inputs (the
    restore runs outside the timed events)."""
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
    del g, b
    ctx.tune_set(ctp.TUNE_BATCH_SMEM_KB, 200)
    ctx.tune_set(ctp.TUNE_FORM_WALK, 0)
    import gc
    gc.collect()
    torch.cuda.empty_cache()
    return {"value": (fs + form) / (ms / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_batch": ms,
            "prec": prec, "S": smode, "factor_solve_flops": fs, "form_flops": form,
            "nelim_total": int(ne.sum()), "p_total": int(sum(f.shape[1] for f in fronts)),
            "device_flags_nonzero": int((flags != 0).sum()), "autotune": tuned,
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


def batch_accuracy(ctx, fronts, count=12, seed=0):
    """Equal-accuracy check of the batch's precisions: a seeded sample of the
    batch's fronts (spread over sizes), each embedded in its complete system and
    refined; the worst final backward error and the most corrections per precision."""
    rng = np.random.default_rng(seed)
    order = np.argsort([f.shape[0] * f.shape[1] for f in fronts])
    pick = order[np.linspace(0, len(order) - 1, count).astype(int)]
    res = {"sample": f"{count} fronts spread over n*p (n from {fronts[pick[0]].shape[0]} to "
                     f"{fronts[pick[-1]].shape[0]}), 2-node systems, 1 RHS, tol 1e-14"}
    import gc
    import torch
    # the chain driver allocates its fronts itself: hand back what torch caches
    gc.collect()
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info()
    print(f"batch accuracy: {free / 2**30:.1f} GiB free of {total / 2**30:.1f}", file=sys.stderr)
    for prec in ("fp64", "bf16x3", "bf16"):
        worst, steps = 0.0, 0
        for k in pick:
            A = fronts[k]
            b = rng.standard_normal((A.shape[0], 1))
            r = refine_embedded(ctx, "cuda", A, prec, b, seed=int(k))
            worst = max(worst, r["bwd_err_history"][-1])
            steps = max(steps, r["corrections"])
        res[prec] = {"max_bwd_err": worst, "max_corrections": steps}
    return res


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

    main = measure(a, ctx, dev, A_host, a.prec, a.smode, a.steps, a.warmup,
                   0 if a.no_e2e else a.steps, peaks, world, dist, solve=a.solve)
    mixed = mixed_bf16 = mixed_fp64_solve = None
    if not a.no_mixed and a.prec == "fp64":
        def mixed_leg(prec, desc, solve="tc"):
            k = max(a.steps, 5)
            mx = measure(a, ctx, dev, A_host, prec, "fp32_tiled", k, max(a.warmup, 3),
                         0 if a.no_e2e else k, peaks, world, dist, solve=solve)
            return {"value": mx["value"], "unit": "GFLOP/s", "ms_per_step": mx["ms"] / k,
                    "prec": desc, "solve": solve, "roofline": mx["roofline"],
                    "rooflines_other": mx["rooflines_other"], "e2e": mx["e2e"],
                    "gpu_launches": mx["launches"],
                    "kernels": {kk: {"launches": v[0], "ms": v[1]} for kk, v in mx["kern"].items()},
                    "clocks": mx["clocks"], "autotune": mx["autotune"]}
        mixed = mixed_leg("bf16x3", "Solve and Form on tensor cores: Solve as one product with "
                                    "three-piece split operands, Form with split operands hi*hi + "
                                    "hi*lo + lo*hi (bf16 x bf16 -> f32), S fp32 in 128x128 blocks; "
                                    "compression and pivot search f64 (refines to the FP64 backward "
                                    "error, see complete_system)")
        mixed_fp64_solve = mixed_leg("bf16x3", "as mixed, with the Solve in FP64", solve="fp64")
        mixed_bf16 = mixed_leg("bf16", "Solve on tensor cores (three-piece split), Form on tensor "
                                       "cores bf16 x bf16 -> f32 (single product), S fp32 in 128x128 "
                                       "blocks (refinement does not reach 1e-12, see complete_system)")

    system = None
    if not a.no_system and rank == 0:
        system = measure_system(ctx, dev, inputs)
    multifrontal = None
    if not a.no_multifrontal and rank == 0:
        multifrontal = measure_multifrontal(ctx, dev, inputs)

    batch = None
    if not a.no_batch:
        fronts = inputs.batch(a.batch_count, seed=a.seed)
        sh = np.array([[f.shape[0], f.shape[1]] for f in fronts])
        batch = {"workload": f"{a.batch_count} supernodes, p log-uniform [8,256], n-p log-uniform "
                             f"[0,16p], N(0,1), 2% zero diagonals, strict compressed pivoting",
                 "sum_np": int((sh[:, 0] * sh[:, 1]).sum()), "max_n": int(sh[:, 0].max()),
                 "median_p": int(np.median(sh[:, 1])), "median_m": int(np.median(sh[:, 0] - sh[:, 1])),
                 "timing": "CUDA graph of the batch call, replayed; inputs restored outside the "
                           "timed events; launch settings chosen by the library's autotuner first"}
        batch["fp64"] = measure_batch(a, ctx, dev, fronts, "fp64", "fp64_packed", 3, 2)
        batch["mixed"] = measure_batch(a, ctx, dev, fronts, "bf16x3", "fp32_tiled", 3, 2)
        batch["mixed_bf16"] = measure_batch(a, ctx, dev, fronts, "bf16", "fp32_tiled", 3, 2)
        batch["accuracy"] = batch_accuracy(ctx, fronts)
        del fronts

    tpp = None
    if not a.no_tpp and a.pivot != "restricted":
        import argparse as _ap
        at = _ap.Namespace(**vars(a))
        at.pivot = "tpp"
        tp = measure(at, ctx, dev, A_host, "fp64", "none", 3, 1, 0, peaks, world, dist)
        comp_ms = sum(v[1] for k, v in main["kern"].items() if not k.startswith("form")) / a.steps
        tpp = {"pivot": "tpp (Listing 1 on all n rows, GPU)", "nelim": tp["e"],
               "factor_solve_ms": tp["ms"] / 3,
               "factor_solve_gflops": tp["fs"] * 3 / (tp["ms"] / 1e3) / 1e9,
               "compressed_factor_solve_ms": comp_ms,
               "compressed_factor_solve_gflops": main["fs"] / (comp_ms / 1e3) / 1e9,
               "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in tp["kern"].items()}}

    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        fl, t, desc = oracle_sample(a)
        cpu = {"value": fl / t / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
               "sample": desc}
    if rank == 0:
        e = main["e"]
        line = {
            "metric": "Supernode LDL^T GFLOP/s", "value": main["value"], "unit": "GFLOP/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": main["ms"] / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if a.prec == "fp64" else "f64 (Form: bf16 x bf16 -> f32)",
            "data": "synthetic",
            "config": {"workload": workload_name(a), "n": a.n, "p": a.p, "u": 0.01,
                       "pivot": a.pivot, "prec": a.prec, "solve": a.solve, "S": a.smode, "nelim": e,
                       "flops_per_step": main["flops_step"], "factor_solve_flops": main["fs"],
                       "form_flops": main["form"] if a.smode != "none" else 0,
                       "l2": "inputs larger than L2: a distinct 409 MB input copy per step",
                       "parallelism": f"replicas x{world}"},
            "roofline": main["roofline"],
            "cpu_baseline": cpu,
            "e2e": main["e2e"],
            "gpu_launches": main["launches"],
            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in main["kern"].items()},
            "clocks": main["clocks"],
            "fp64_dgemm_tflops": peaks["fp64_tflops"],
            "mixed": mixed,
            "mixed_fp64_solve": mixed_fp64_solve,
            "mixed_bf16": mixed_bf16,
            "complete_system": system,
            "multifrontal": multifrontal,
            "tpp_comparator": tpp,
            "batch": batch,
        }
        print(json.dumps(line), flush=True)
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
