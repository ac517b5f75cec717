#!/usr/bin/env python3
"""Benchmark: S^3TTVc hyperedge-members/s on the power-law rank-25 workload.

Workload (the configuration the headline metric is quoted on): n = 1,000,000
nodes, m = 5,000,000 hyperedges, sizes Zipf(2.5) on {2..25} (rank 25),
Chung-Lu membership with power-law degree exponent 2.1, seeded synthetic
data.  One step is one S^3TTVc call y = B x^(N-1) in FP32 series arithmetic
with the deterministic segmented reduce, x already resident in HBM (x is a
centrality-like positive vector rescaled to max 1).  value = total
hyperedge-members (sum of edge sizes) processed by all ranks / max-over-ranks
time.

Also reported on the same line: the device-time split and the roofline of
the per-edge series kernels (ALU bound), the HBM fraction the metric asks
for, FP64 S^3TTVc, NQZ centrality time-to-tolerance (FP32-mixed vs plain
FP64), the end-to-end number through the host-buffer entry point, clocks
sampled during the timed region, and the FP64 CPU oracle timed on a bounded
sample on this host (``cpu_baseline``).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "powerlaw-hypergraph", "n": 1_000_000, "m": 5_000_000, "rank": 25,
            "edge_sizes": "zipf(2.5) on 2..25", "membership": "chung-lu, degree exponent 2.1", "seed": 2}
METRIC = "S3TTVc hyperedge-members/sec"
WARM_GRAPHS = 48
UNIT = "members/s"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def algorithmic_counts(edges_per_size, N, closed_sizes=(), bern_sizes=(), bern_form="product"):
    """FLOPs of one FP32 S^3TTVc call by the edge-layout algorithm.

    Per edge of size s >= 2 with window W = N - s + 1 (series):
      Toeplitz products: (s-2) prefix + (s-3) suffix windows of W(W+1)/2 FMAs each
                         (s >= 3), plus W FMAs for the last suffix coefficient;
      dots: (W-1) for [t^(N-1)] F_e and W for each of the s-2 interior nodes;
      power tables: 2(s-1) tables of W coefficients, 2 multiplies per coefficient.
    Sizes in bern_sizes count as bernoulli_flops gives them (bern_form: "product" for FP32,
    "powersum" for FP64).
    Per edge of a size in closed_sizes (inclusion-exclusion): for each of the 2^s - 1
    subsets one add (its sum), floor(log2 n) + popcount(n) - 1 multiplies (sum^n,
    n = N-1) and one add (the sum of |terms|), then s 2^(s-1) signed adds.  The
    compensation of the FP32 subset sums is not counted.
    One FMA = 2 flops.  Size-1 edges: ~2 log2(N) multiplies.
    """
    fma = 0
    mul = 0
    n = N - 1
    for s, cnt in enumerate(edges_per_size):
        if cnt == 0 or s == 0:
            continue
        if s == 1:
            mul += cnt * 2 * int(np.ceil(np.log2(max(N, 2))))
            continue
        if s in closed_sizes:
            mul += cnt * ((2 ** s - 1) * (2 + n.bit_length() - 1 + bin(n).count("1") - 1) + s * 2 ** (s - 1))
            continue
        if s in bern_sizes:
            mul += bernoulli_flops(edges_per_size, N, [s], bern_form)
            continue
        W = N - s + 1
        f = (W - 1) + max(s - 2, 0) * W
        if s >= 3:
            f += (s - 2) * W * (W + 1) // 2 + (s - 3) * W * (W + 1) // 2 + W
        fma += cnt * f
        mul += cnt * 2 * (s - 1) * 2 * W
    return 2 * fma + mul, fma


def bernoulli_flops(edges_per_size, N, sizes, form="product"):
    """FLOPs of the Bernoulli-form launch (csrc/s3_bern.cuh) for the edge sizes it takes.

    Per edge of size s, window W = N - s + 1, the product form (FP32): the first member's
    series g (2(W-1) multiplies), then per further member the ratios x/(k+1) (W-1
    multiplies), the truncated product (W(W-1)/2 multiply-adds) and the running product
    (1 multiply); the coefficients H_k = G[W-1-k] beta_k (W multiplies); per member the
    sum in x^4-Horner form (2 + 2 ceil((W-2)/4) + 2 ceil((W-4)/4) + 4 flops with x^2, x^4
    and the two leading terms), the gate (3) and P / x_i times the sum (2).
    The power-sum form (FP64): per member the scaling and running product (2), the powers
    x^2..x^(W-1) (W-2 multiplies) and their sums (W-1 adds); beta_k p_k (W-1 multiplies);
    the recurrences for G and its majorant A (for m = 1..W-1: 2m multiply-adds and 2
    multiplies); H_k and A[W-1-k]|beta_k| (2W multiplies); per member the sum as above, the
    majorant in x^2-Horner form (1 + 2 ceil(W/2) + 2 flops), the gate (2) and the value (2).
    One multiply-add = 2 flops."""
    total = 0
    for s in sizes:
        cnt = edges_per_size[s]
        W = N - s + 1
        horner = 4 + 2 * -(-max(W - 2, 0) // 4) + 2 * -(-max(W - 4, 0) // 4) + 2
        if form == "product":
            per = 2 * (W - 1) + (s - 1) * ((W - 1) + W * (W - 1) + 1) + W
            per += s * (horner + 3 + 2)
        else:
            per = s * (2 + (W - 2) + (W - 1)) + (W - 1) + 2 * W * (W - 1) + 2 * (W - 1) + 2 * W
            per += s * (horner + (1 + 2 * -(-W // 2) + 2) + 2 + 2)
        total += cnt * per
    return total


def hbm_bytes(nnz, n, esz=4, deterministic=True, comp=False):
    """Algorithmic HBM bytes of one call: the int32 member ids
    (4 per member), x gathered once and y written (esz per node each), the FP32
    compensation vector in atomic mode (4 per node), and, in deterministic mode, the
    per-(edge, node) buffer written by the edge kernels and read back by the reduce
    (2 esz per member)."""
    b = 4 * nnz + 2 * esz * n
    if comp:
        b += 4 * n
    if deterministic:
        b += 2 * esz * nnz
    return b


def layout_bytes(nnz, n):
    """Bytes the layout adds on top of hbm_bytes: the incidence-slot index of every
    member (4 per member) and the reduce's node lists and offsets (about 12 per node)."""
    return 4 * nnz + 12 * n


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 20 ms in the background."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 8:
                for nm, v in zip(names, r[4:8]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# the sources the FP32 Bernoulli kernel is compiled from (its translation unit and headers)
BERN_KERNEL_SOURCES = ("s3_bern.cuh", "s3_bern_f32.cu", "s3_series.cuh", "s3_kernels.h")


def csrc_digest(names=None):
    """sha256 over the library's sources (names and contents): all of them, or the given ones."""
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2311_08595_gb300", "csrc")
    paths = sorted(glob.glob(os.path.join(csrc, "*"))) if names is None else [os.path.join(csrc, n) for n in names]
    for p in paths:
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_workload(n=None):
    """The power-law workload (n nodes, 5n edges; default the full size) and its x."""
    import s3synth
    n = n or WORKLOAD["n"]
    m = WORKLOAD["m"] * n // WORKLOAD["n"]
    hg = s3synth.config_powerlaw(n=n, m=m, rank=WORKLOAD["rank"], seed=WORKLOAD["seed"])
    # a centrality-like positive vector (degree^(1/(N-1)) jittered, max 1)
    return hg, s3synth.x_degree_like(hg, seed=5)


# ------------------------------------------------------------ CPU oracle ---

def host_cores():
    """Host threads this process may run on (its CPU affinity): the oracle is timed on all of them."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(hg, x, budget_s=12.0, seed=0):
    """Time the FP64 CPU oracle (Algorithm 2) on a bounded random node sample.

    Returns (members/s, cores, sample description).  A 'member' is one
    (edge, node) contribution, the unit of the GPU metric."""
    import oracle
    cores = host_cores()
    deg = hg.degrees()
    rng = np.random.default_rng(seed)
    perm = rng.permutation(hg.n)
    # grow the sample (x2) until a run takes >= budget_s / 3; the timed run uses twice that
    # (each call also rebuilds the oracle's node->edge incidence, a fixed cost it amortises)
    k = 4000
    while k < hg.n:
        t0 = time.perf_counter()
        oracle.ttsv1(hg, x, nodes=perm[:k], nthreads=cores)
        if time.perf_counter() - t0 >= budget_s / 3:
            break
        k *= 2
    k = int(min(hg.n, 2 * k))
    nodes = perm[:k]
    t0 = time.perf_counter()
    oracle.ttsv1(hg, x, nodes=nodes, nthreads=cores)
    dt = time.perf_counter() - t0
    members = int(deg[nodes].sum())
    return members / dt, cores, f"{k} random nodes, {members} (edge,node) contributions, {dt:.1f} s"


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    hg, x = make_workload()
    import oracle
    cores = host_cores()
    deg = hg.degrees()
    rng = np.random.default_rng(1)
    nodes = rng.permutation(hg.n)[:20000]
    members = int(deg[nodes].sum())
    for _ in range(args.warmup):
        oracle.ttsv1(hg, x, nodes=nodes[:2000], nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.ttsv1(hg, x, nodes=nodes, nthreads=cores)
    dt = (time.perf_counter() - t0) / args.steps
    v = members / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, sample="20000 random nodes per step"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"20000 random nodes ({members} contributions) per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU ---

def run_gpu(args):
    import torch

    import paper_2311_08595_gb300 as s3
    from paper_2311_08595_gb300 import build as s3build
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    s3build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    hg, x_np = make_workload(args.n or None)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    info = s3.s3_graph_query(g)
    N, nnz, n = info["rank"], info["nnz"], info["n"]
    x = torch.tensor(x_np, dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(max(args.warmup, 3)):
        s3.s3_sttsvc(g, x, y)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(args.steps):
            s3.s3_sttsvc(g, x, y)
        stop.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = start.elapsed_time(stop) / args.steps
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = nnz * ws / (ms * 1e-3)
    launches = s3.s3_sttsvc_profile(g, x, y)["launches"]

    # phase split (device events inside the library), averaged
    prof = [s3.s3_sttsvc_profile(g, x, y) for _ in range(20)]
    edge_ms = float(np.mean([p["edge_ms"] for p in prof]))
    reduce_ms = float(np.mean([p["reduce_ms"] for p in prof]))
    bern_ms = float(np.mean([p["bern_ms"] for p in prof]))
    closed = s3.s3_closed_form_query(g)
    bern = s3.s3_bernoulli_query(g)
    flops, fmas = algorithmic_counts(info["edges_per_size"], N, closed["f32"], bern["f32"])
    bflops = bernoulli_flops(info["edges_per_size"], N, bern["f32"])
    peaks, peak_kind = measured_peaks()
    clocks = clk.summary()
    # measured FMA peaks of this device (FP32, FP64), clocks sampled while they run
    with ClockSampler(local) as pclk:
        p32 = s3.s3_fma_peak(fp64=False, reps=50)
        p64 = s3.s3_fma_peak(fp64=True, reps=20)
    pclocks = pclk.summary()
    achieved_tflops = flops / (edge_ms * 1e-3) / 1e12
    bytes_call = hbm_bytes(nnz, n)
    # DRAM traffic of one Bernoulli launch, from the committed ncu capture of that kernel on a
    # smaller case of the same recipe, scaled by the members the launch processes -- only while
    # the kernel sources are the ones it was taken with
    traffic, traffic_note = None, None
    bern_members = int(sum(info["edges_per_size"][s_] * s_ for s_ in bern["f32"]))
    tp = os.path.join(ROOT, "profiles", "edge_bern_traffic.json")
    if os.path.exists(tp):
        try:
            tj = json.load(open(tp))
            if tj.get("kernel_digest") == csrc_digest(BERN_KERNEL_SOURCES):
                traffic = tj["bytes_per_member"] * bern_members
                traffic_note = ("dram__bytes_read.sum + dram__bytes_write.sum of edge_bern_kernel<float> on "
                                + tj["workload"] + f" ({tj['members']} members), scaled to {bern_members} members")
        except Exception:
            traffic = None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD, n=n, m=info["m"], x="degree^(1/24) jittered, max 1",
                       reduce="segmented (deterministic)",
                       l2="inputs larger than L2: ids+slots+buffer = 16 bytes x members" if nnz > 8_000_000
                       else "inputs smaller than L2 (reduced workload)",
                       nnz=nnz, parallelism=f"replicas x{ws}"),
        "roofline": {"bound": "alu", "kernel": "edge_bern_kernel<float> (one launch per call: edge sizes "
                     + f"{min(bern['f32'])}-{max(bern['f32'])}, the Bernoulli form)" if bern["f32"] else "none",
                     "achieved": bflops / (bern_ms * 1e-3) / 1e12 if bern_ms > 0 else None,
                     "peak": p32["tflops"], "unit": "TFLOP/s",
                     "frac": bflops / (bern_ms * 1e-3) / 1e12 / p32["tflops"] if bern_ms > 0 else None,
                     "traffic": traffic, "traffic_note": traffic_note,
                     "algorithmic_bytes_per_launch": bern_members * 8 + n * 4,
                     "peak_note": "of measured: FP32 FMA-chain probe (s3_fma_peak) on this device, "
                                  f"{p32['sm_count']} SMs, median SM clock {pclocks['sm_mhz']} MHz during the probe",
                     "algorithmic_flops_per_launch": bflops, "launch_ms": bern_ms,
                     "launch_ms_note": "CUDA events around the launch on the stream it runs on, mean of 20 calls"},
        "edge_phase": {"bound": "alu", "kernels": "all per-edge kernels of one call (closed form for sizes "
                       + ",".join(map(str, closed["f32"])) + ", Bernoulli form for "
                       + (f"{min(bern['f32'])}-{max(bern['f32'])}" if bern["f32"] else "none") + ", series otherwise)",
                       "achieved": achieved_tflops, "peak": p32["tflops"], "unit": "TFLOP/s",
                       "frac": achieved_tflops / p32["tflops"], "algorithmic_flops_per_call": flops,
                       "edge_ms": edge_ms, "reduce_ms": reduce_ms,
                       "edge_ms_x_sm_mhz": edge_ms * (clocks["sm_mhz"] or 0.0)},
        "hbm": {"algorithmic_bytes_per_call": bytes_call, "achieved_gbs": bytes_call / (ms * 1e-3) / 1e9,
                "peak_gbs": peaks["hbm_gbs"], "frac": bytes_call / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                "peak_kind": peak_kind, "layout_bytes_per_call": layout_bytes(nnz, n),
                "count": "4 B ids per member + x and y + 8 B per member buffer write+read (deterministic mode)"},
        "fma_peaks": {"fp32_tflops": p32["tflops"], "fp64_tflops": p64["tflops"], "sm_count": p32["sm_count"],
                      "threads_per_sm": p32["threads_per_sm"], "rated_clock_mhz": p32["clock_mhz"],
                      "clocks_during_probe": pclocks},
        "clocks": clocks, "gpu_launches": launches * args.steps,
    }
    # FP64 S^3TTVc (event-timed over 20 calls), with its roofline against the FP64 FMA peak
    x64, y64 = x.double(), torch.empty(n, dtype=torch.float64, device=dev)
    with ClockSampler(local) as c64:   # clocks under sustained FP64 load (about 0.2 s)
        ms64 = _time_calls(g, x64, y64, 100)
    prof64 = [s3.s3_sttsvc_profile(g, x64, y64) for _ in range(3)]
    edge64 = float(np.mean([p["edge_ms"] for p in prof64]))
    flops64, _ = algorithmic_counts(info["edges_per_size"], N, closed["f64"], bern["f64"], "powersum")
    out["fp64"] = {"value": nnz / (ms64 * 1e-3), "unit": UNIT, "ms_per_call": ms64, "calls_timed": 100,
                   "fp32_speedup": ms64 / ms, "clocks": c64.summary(),
                   "roofline": {"bound": "alu", "achieved": flops64 / (edge64 * 1e-3) / 1e12, "peak": p64["tflops"],
                                "unit": "TFLOP/s", "frac": flops64 / (edge64 * 1e-3) / 1e12 / p64["tflops"],
                                "edge_ms": edge64, "closed_form_sizes": closed["f64"], "bernoulli_sizes": bern["f64"],
                                "peak_note": "of measured: FP64 FMA-chain probe (s3_fma_peak)"},
                   "bernoulli_kernel": _bern64_roofline(prof64, info["edges_per_size"], N, bern["f64"], p64["tflops"]),
                   "hbm_bytes_per_call": hbm_bytes(nnz, n, esz=8)}
    # FP64 in and out with the series in double-float (pairs of FP32)
    ydf = torch.empty_like(y64)
    msdf = _time_calls(g, x64, ydf, 20, df=True)
    a, b = ydf.cpu().numpy(), y64.cpu().numpy()
    nz = b != 0
    out["df64"] = {"value": nnz / (msdf * 1e-3), "unit": UNIT, "ms_per_call": msdf, "calls_timed": 20,
                   "speedup_vs_fp64": ms64 / msdf,
                   "max_rel_diff_vs_fp64": float(np.max(np.abs(a[nz] - b[nz]) / np.abs(b[nz])))}
    # end to end through the host-buffer entry point
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    s3.s3_sttsvc_host(g, xh, yh)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s3.s3_sttsvc_host(g, xh, yh)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    out["e2e"] = {"value": nnz * ws / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
                  "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n}
    if rank == 0 and ws == 1 and not args.skip_extras:
        out["small_fp64"] = small_config(dev)
        out["atomic_mode"] = atomic_mode(hg, x, ms)

    if rank == 0 and ws == 1 and (args.batched or not args.skip_extras):
        out["batched"] = batched(dev, scale=args.batched_scale)
    if rank == 0 and ws == 1 and not args.skip_extras:
        out["large_rank"] = large_rank(dev)
        out["layouts"] = layouts(dev)
        out["cpu_comparators"] = cpu_comparators(dev)
        out["centrality"] = centrality(hg, dev)
        rate, cores, sample = time_oracle(hg, x_np)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    s3.s3_destroy(g)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def atomic_mode(hg, x, ms_segmented):
    """The same FP32 call with y scattered by warp-aggregated atomics (FP32 two-sum
    compensation) instead of the deterministic segmented reduce: event-timed over 50 calls."""
    import torch

    import paper_2311_08595_gb300 as s3
    ga = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members, reduce=s3.S3_REDUCE_ATOMIC)
    y = torch.empty_like(x)
    ms = _time_calls(ga, x, y, 50)
    s3.s3_destroy(ga)
    return {"reduce": "atomic (warp-aggregated, FP32 two-sum compensation)", "ms_per_call": ms,
            "value": hg.nnz / (ms * 1e-3), "unit": UNIT, "vs_segmented": ms / ms_segmented}


def batched(dev, scale=1.0, nvec=16, reps=3):
    """64 power-law hypergraphs (n log-uniform in [10k, 500k], m = 5n, Zipf(2.5) sizes on
    {2..r_i}, r_i uniform in {8..32}) with 16 x-vectors each: one batched call (persistent
    kernels replayed from a CUDA graph, autotuned) against 1024 single s3_sttsvc calls."""
    import torch

    import paper_2311_08595_gb300 as s3
    import s3synth
    t0 = time.perf_counter()
    hgs = s3synth.config_batched(count=64, scale=scale, seed=4)
    gs = [s3.s3_build_format(h.n, h.edge_ptr, h.members) for h in hgs]
    t_build = time.perf_counter() - t0
    nnz = sum(h.nnz for h in hgs)
    xs, ys = [], []
    for gi, h in enumerate(hgs):
        base = torch.rand(h.n, device=dev, generator=torch.Generator(device=dev).manual_seed(gi)) * 0.5 + 0.5
        for v in range(nvec):
            xs.append((base * (1.0 + 0.01 * v)).float().contiguous())
            ys.append(torch.empty(h.n, dtype=torch.float32, device=dev))
    b = s3.s3_batch_create(gs, nvec)
    tune = s3.s3_batch_autotune(b, xs, ys)
    for _ in range(2):
        s3.s3_sttsvc_batched(b, xs, ys)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        s3.s3_sttsvc_batched(b, xs, ys)
    e1.record(st)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / reps
    # the same work as 1024 single calls
    ref = [torch.empty_like(y) for y in ys]
    for j, x in enumerate(xs):
        s3.s3_sttsvc(gs[j // nvec], x, ref[j])
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        for j, x in enumerate(xs):
            s3.s3_sttsvc(gs[j // nvec], x, ref[j])
    e1.record(st)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1) / reps
    err = max(float(((y - r).abs() / r.abs().clamp_min(1e-30)).max()) for y, r in zip(ys, ref))
    members = nnz * nvec
    s3.s3_batch_destroy(b)
    return {"workload": f"64 power-law hypergraphs x {nvec} vectors (scale {scale})", "nnz_per_vector": nnz,
            "batched_ms": ms_b, "single_calls_ms": ms_s, "speedup": ms_s / ms_b,
            "batched_members_per_s": members / (ms_b * 1e-3), "single_members_per_s": members / (ms_s * 1e-3),
            "autotune": {k: tune[k] for k in ("block_threads", "edges_per_thread", "thread_max_w", "tried")},
            "max_rel_diff_vs_single": err, "build_s": t_build}


WARM_WEIGHTS = os.path.join(ROOT, "paper_2311_08595_gb300", "data", "warmstart_500x50k.npy")


def warm_start(lcc, dev, graphs=48, n=50000, epochs=20):
    """Learned warm start on the workload's largest component: NQZ to 1e-8 from the uniform start
    vs from the network's prediction (features + MLP time included).  The network is the one the
    package ships (trained by `python -m paper_2311_08595_gb300.warmstart --graphs 500 --n 50000`
    on 500 power-law hypergraphs of n = 50k, the recipe of the workload); without that file it is
    trained here on `graphs` such hypergraphs."""
    import s3synth
    from paper_2311_08595_gb300 import s3_mlp_create
    from paper_2311_08595_gb300 import warmstart as ws
    out = {}
    if os.path.exists(WARM_WEIGHTS):
        model = s3_mlp_create(params=np.load(WARM_WEIGHTS))
        out["weights"] = "shipped: 500 training hypergraphs of n = 50k (warmstart.py)"
    else:
        rng = np.random.default_rng(2024)
        t0 = time.perf_counter()
        hgs = [s3synth.largest_component(s3synth.config_powerlaw(n=n, m=5 * n, seed=int(rng.integers(1 << 30))))[0]
               for _ in range(graphs)]
        feat, tgt = ws.build_dataset(hgs)
        t_data = time.perf_counter() - t0
        t0 = time.perf_counter()
        model, hist = ws.train(feat, tgt, epochs=epochs, batch=65536, lr=2e-3)
        out.update({"weights": f"trained here: {graphs} hypergraphs of n = {n}", "train_nodes": int(feat.shape[0]),
                    "epochs": epochs, "loss_first": hist[0][1], "loss_last": hist[-1][1], "data_s": t_data,
                    "train_s": time.perf_counter() - t0})
    for name, prec in (("fp64", 0), ("fp32_mixed", 1), ("fp32_then_double_float", 2), ("double_float", 3)):
        out[name] = ws.evaluate(lcc, model, tol=1e-8, precision=prec)
    out["start_cost"] = ws.start_cost(lcc, model)
    return out


def _bern64_roofline(prof, edges_per_size, N, sizes, peak):
    """The FP64 Bernoulli launch (power-sum form) against the FP64 FMA peak."""
    ms = float(np.mean([p["bern_ms"] for p in prof]))
    fl = bernoulli_flops(edges_per_size, N, sizes, "powersum")
    if ms <= 0 or not sizes:
        return None
    return {"kernel": "edge_bern_kernel<double>", "launch_ms": ms, "algorithmic_flops_per_launch": fl,
            "achieved": fl / (ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": fl / (ms * 1e-3) / 1e12 / peak}


def _time_calls(g, x, y, reps, df=False):
    """Device time per s3_sttsvc call (CUDA events on the current stream), after one warm-up call."""
    import torch

    import paper_2311_08595_gb300 as s3
    s3.s3_sttsvc(g, x, y, df=df)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        s3.s3_sttsvc(g, x, y, df=df)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def small_config(dev, calls=2000):
    """The small single-call case: n=1000, m=5000, sizes U{2..5} (rank 5), x ~ U(0,1), FP64,
    one S^3TTVc call at a time (launch-latency bound); event-timed over `calls` calls, and the
    result against the CPU oracle on every node."""
    import torch

    import oracle
    import paper_2311_08595_gb300 as s3
    import s3synth
    hg = s3synth.config_small(seed=1)
    x_np = s3synth.x_uniform(hg.n, 0.0, 1.0, 1)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    x = torch.tensor(x_np, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    ms = _time_calls(g, x, y, calls)
    info = s3.s3_graph_query(g)
    want = oracle.ttsv1(hg, x_np)
    err = float(np.max(np.abs(y.cpu().numpy() - want) / np.abs(want)))
    out = {"workload": "small n=1000 m=5000 sizes U{2..5} rank 5, x~U(0,1), FP64", "nnz": hg.nnz,
           "ms_per_call": ms, "members_per_s": hg.nnz / (ms * 1e-3), "calls_timed": calls,
           "launches_per_call": s3.s3_sttsvc_profile(g, x, y)["launches"],
           "max_rel_err_vs_oracle": err, "hbm_bytes_per_call": hbm_bytes(hg.nnz, hg.n, esz=8),
           "edges_per_size": info["edges_per_size"][:6]}
    s3.s3_destroy(g)
    return out


def large_rank(dev, sample=300):
    """Rank-100 stress workload: n=200k, m=1M, Geometric(0.1) sizes on {2..100}, x ~ U(0.5,1.5).
    FP32 and FP64 throughput; FP32 error per node against the GPU FP64 result, and the FP64
    result against the CPU oracle on sampled nodes."""
    import torch

    import oracle
    import paper_2311_08595_gb300 as s3
    import s3synth
    hg = s3synth.config_large_rank()
    x_np = s3synth.x_uniform(hg.n, 0.5, 1.5, 3)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    x64 = torch.tensor(x_np, dtype=torch.float64, device=dev)
    x32 = x64.float()
    y64, y32 = torch.empty_like(x64), torch.empty_like(x32)
    ms32 = _time_calls(g, x32, y32, 20)
    ms64 = _time_calls(g, x64, y64, 20)
    a, b = y32.double().cpu().numpy(), y64.cpu().numpy()
    d = hg.degrees()
    rel = np.abs(a - b)[d > 0] / np.abs(b)[d > 0]
    nodes = np.random.default_rng(0).choice(np.nonzero(d > 0)[0], size=sample, replace=False)
    want = oracle.ttsv1(hg, x_np, nodes=nodes, nthreads=host_cores())
    e64 = float(np.max(np.abs(b[nodes] - want) / np.abs(want)))
    s3.s3_destroy(g)
    return {"workload": "largerank n=200k m=1M geometric(0.1) sizes on 2..100, x~U(0.5,1.5)", "nnz": hg.nnz,
            "fp32_ms": ms32, "fp64_ms": ms64, "calls_timed": 20, "fp32_members_per_s": hg.nnz / (ms32 * 1e-3),
            "fp64_members_per_s": hg.nnz / (ms64 * 1e-3), "fp32_speedup": ms64 / ms32,
            "fp32_rel_err_per_node": {"max": float(rel.max()), "median": float(np.median(rel)),
                                      "p99": float(np.quantile(rel, 0.99))},
            "fp64_vs_oracle_max_rel_err": e64, "oracle_sample_nodes": sample}


def layouts(dev):
    """Edge layout (per-edge prefix/suffix products) vs the level-by-level CCSS forest, FP32, on a
    power-law graph (n=100k, m=500k, rank 25) and on nested edge families (Fig. 3)."""
    import torch

    import paper_2311_08595_gb300 as s3
    import s3synth
    out = {}
    cases = {"powerlaw_n100k": s3synth.config_powerlaw(n=100000, m=500000, seed=8),
             "nested_4000x6": s3synth.nested(chains=4000, length=6, start=5, step=5, n=200000)}
    for name, hg in cases.items():
        g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members, build_ccss=1)
        info = s3.s3_graph_query(g)
        x = torch.tensor(s3synth.x_uniform(hg.n, 0.5, 1.5, 1), dtype=torch.float32, device=dev)
        ye, yc = torch.empty_like(x), torch.empty_like(x)
        ms_e = _time_calls(g, x, ye, 5)
        s3.s3_sttsvc_layout(g, s3.S3_LAYOUT_CCSS, x, yc)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(5):
            s3.s3_sttsvc_layout(g, s3.S3_LAYOUT_CCSS, x, yc)
        e1.record(st)
        torch.cuda.synchronize()
        ms_c = e0.elapsed_time(e1) / 5
        sizes = np.bincount(hg.sizes(), minlength=hg.rank + 1)
        edge_products = int(sum(c * max(2 * s - 5, 0) for s, c in enumerate(sizes)))
        diff = float(((yc - ye).abs() / ye.abs().clamp_min(1e-30)).max())
        out[name] = {"nnz": hg.nnz, "edge_ms": ms_e, "ccss_ms": ms_c, "ccss_forest_nodes": info["ccss_nodes"],
                     "ccss_products": info["ccss_products"], "edge_layout_products": edge_products,
                     "max_rel_diff": diff}
        s3.s3_destroy(g)
    return out


def cpu_comparators(dev, budget_s=8.0):
    """The paper's own CPU algorithms (Algorithm 4, memoised DFS on the CCSS forest; Algorithm 3,
    its naive leaf-to-root baseline) in FP64 on all host cores, next to the GPU library on the
    same hypergraphs: the power-law recipe at n=200k, m=1M (rank 25), the sunflower and nested
    structures of Fig. 3, and the Table I style rank family (sizes 5, 10, .., r).  Each CPU
    algorithm runs on a bounded sample of whole trees (roots) of the forest, grown until one
    run takes about budget_s / 4; members/s counts the special leaves (edge, node) processed."""
    import torch

    import baseline
    import paper_2311_08595_gb300 as s3
    import s3synth
    cores = host_cores()
    cases = {"powerlaw_n200k_m1M_r25": s3synth.config_powerlaw(n=200000, m=1000000, rank=25, seed=9),
             "nested_4000x6": s3synth.nested(chains=4000, length=6, start=5, step=5, n=200000),
             "sunflower_20000x12_core8": s3synth.sunflower(petals=20000, k=12, core=8, n=100000)}
    for r in (15, 25, 35):
        cases[f"s_family_r{r}"] = s3synth.paper_s_family(r, n=100000, m=100000, seed=r)
    out = {"cores": cores}
    for name, hg in cases.items():
        x = s3synth.x_uniform(hg.n, 0.5, 1.5, 17)
        t0 = time.perf_counter()
        f = baseline.Forest(hg)
        t_build = time.perf_counter() - t0
        res = {"n": hg.n, "m": hg.m, "nnz": hg.nnz, "rank": hg.rank, "forest_nodes": f.nodes,
               "products_alg3": f.products3, "products_alg4": f.products4, "forest_build_s": t_build}
        for alg in ("alg4", "alg3"):
            run = getattr(f, alg)
            k = max(1, f.roots // 256)
            while True:
                t0 = time.perf_counter()
                run(x, nthreads=cores, roots=(0, k))
                dt = time.perf_counter() - t0
                if dt >= budget_s / 4 or k >= f.roots:
                    break
                k = min(f.roots, k * 4)
            leaves = f.leaves_in_roots(0, k)
            res[alg] = {"members_per_s": leaves / dt, "sample": f"{k} of {f.roots} trees, {leaves} members",
                        "seconds": dt}
        g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members, build_ccss=1)
        for dt_name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
            xd = torch.tensor(x, dtype=dt, device=dev)
            yd = torch.empty_like(xd)
            ms = _time_calls(g, xd, yd, 20)
            res[f"gpu_{dt_name}_members_per_s"] = hg.nnz / (ms * 1e-3)
        xd = torch.tensor(x, dtype=torch.float64, device=dev)
        yc = torch.empty_like(xd)
        s3.s3_sttsvc_layout(g, s3.S3_LAYOUT_CCSS, xd, yc)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(5):
            s3.s3_sttsvc_layout(g, s3.S3_LAYOUT_CCSS, xd, yc)
        e1.record(st)
        torch.cuda.synchronize()
        res["gpu_ccss_fp64_members_per_s"] = hg.nnz / (e0.elapsed_time(e1) / 5 * 1e-3)
        res["gpu_fp64_vs_alg4"] = res["gpu_fp64_members_per_s"] / res["alg4"]["members_per_s"]
        res["alg4_vs_alg3"] = res["alg4"]["members_per_s"] / res["alg3"]["members_per_s"]
        s3.s3_destroy(g)
        del f
        out[name] = res
    return out


def centrality(hg, dev):
    """NQZ to 1e-8 on the largest connected component: plain FP64 vs FP32 series with an FP64 or a
    double-float finish, and double-float throughout (each after one untimed run)."""
    import torch

    import paper_2311_08595_gb300 as s3
    import s3synth
    lcc, _ = s3synth.largest_component(hg)
    g = s3.s3_build_format(lcc.n, lcc.edge_ptr, lcc.members)
    res = {}
    xs = {}
    for name, prec in (("fp64", 0), ("fp32_mixed", 1), ("fp32_then_double_float", 2), ("double_float", 3)):
        s3.s3_hcentrality(g, tol=1e-8, precision=prec, raise_on_noconv=False)   # untimed: scratch, graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xo, r = s3.s3_hcentrality(g, tol=1e-8, precision=prec, raise_on_noconv=False)
        torch.cuda.synchronize()
        r["wall_s"] = time.perf_counter() - t0
        xs[name] = xo.cpu().numpy()
        res[name] = {k: r[k] for k in ("iters", "iters_fp32", "seconds", "wall_s", "lambda_min", "lambda_max",
                                       "converged", "status")}
    res["n_lcc"] = lcc.n
    res["speedup_fp32_mixed"] = res["fp64"]["wall_s"] / res["fp32_mixed"]["wall_s"]
    res["max_rel_diff_x"] = float(np.max(np.abs(xs["fp32_mixed"] - xs["fp64"]) / xs["fp64"]))
    for name in ("fp32_then_double_float", "double_float"):
        res[name]["speedup_vs_fp64"] = res["fp64"]["wall_s"] / res[name]["wall_s"]
        res[name]["max_rel_diff_x"] = float(np.max(np.abs(xs[name] - xs["fp64"]) / xs["fp64"]))
    s3.s3_destroy(g)
    if WARM_GRAPHS > 0:
        res["learned_warm_start"] = warm_start(lcc, dev, graphs=WARM_GRAPHS)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--skip-extras", action="store_true", help="skip centrality and CPU-baseline legs")
    ap.add_argument("--batched", action="store_true", help="also time 64 graphs x 16 vectors batched vs single")
    ap.add_argument("--batched-scale", type=float, default=1.0)
    ap.add_argument("--warm-graphs", type=int, default=48, help="training hypergraphs of the warm start (0 = skip)")
    ap.add_argument("--n", type=int, default=0, metavar="N",
                    help="nodes of the power-law workload (5N edges; default 1,000,000)")
    args = ap.parse_args()
    global WARM_GRAPHS
    WARM_GRAPHS = args.warm_graphs
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
