#!/usr/bin/env python
"""Benchmark of the biharmonic field extension on GB300: extension solves/s at relative residual
1e-8.

Workloads (seeded synthetic inputs shaped like the paper's test problems):
  batch  : (default) 256 uneven grids (sides drawn from {128,192,256,384,512}, wobbly interfaces,
           field known inside, extend out, symmetric edges) solved together with the tensor-core
           (mixed BF16) preconditioner; a step is the whole batch.  The plain FP32 single-solve
           path is timed on a sample of the same grids for the comparison.
  single : one 1024x1024 extension (six-lobed star, field known outside, extend in, periodic
           edges); a step is one complete solve (set-up, PCG to 1e-8, output).
  serve  : a bounded sample of the serving workload: Poisson arrivals of requests with
           log-uniform sides, star or multi-circle interfaces, random direction and edges;
           reports p50/p99 latency beside throughput.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle (assembled sparse matrix and
SuperLU direct solve, which reaches a residual far below 1e-8) on the same workload instead.

Timing: inputs resident in HBM, CUDA events on the library's stream around each step, a 256 MiB
L2 flush between steps (outside the events); the whole loop bracketed by barrier + synchronize.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
CSRC = os.path.join(ROOT, "paper_1704_08897_gb300", "csrc")

# FP32 CUDA-core peak of a GB300 derived from unit counts and clock:
# 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz.
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch", choices=["single", "batch", "serve"])
    ap.add_argument("--requests", type=int, default=400, help="serve: requests per step")
    ap.add_argument("--rate", type=float, default=500.0, help="serve: arrivals per second")
    ap.add_argument("--plain-sample", type=int, default=16, help="batch: grids timed on the plain path")
    ap.add_argument("--instances", type=int, default=256,
                    help="batch: number of grids (256 = the benchmark workload; fewer for profiling)")
    ap.add_argument("--prec", default=None, help="fp32 | mixed_fp16 | mixed_bf16")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=48,
                    help="batch: requests of the serving leg (config-4 shape); 0 skips it")
    ap.add_argument("--peanut3d", default="64,128,256",
                    help="batch: sides of the three-dimensional Example 2 leg ('' skips it)")
    ap.add_argument("--low-modes", type=int, default=None,
                    help="low-mode correction of the mixed preconditioner: 1 on, 0 off (library default)")
    ap.add_argument("--fold", type=int, default=None,
                    help="mirror-class transforms of the mixed preconditioner: 1 on, 0 off (library default)")
    args = ap.parse_args()
    if args.low_modes is not None:
        _OPTION_OVERRIDES["low_modes"] = args.low_modes
    if args.fold is not None:
        _OPTION_OVERRIDES["fold"] = args.fold
    return args


_OPTION_OVERRIDES = {}


def _options(prec, **kw):
    """Solver options of every context the bench creates, with the command line's overrides."""
    from paper_1704_08897_gb300 import ext
    kw = {**kw, **_OPTION_OVERRIDES}
    return ext.options(prec, **kw)


# ----------------------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------------------
def make_workload(name, rank, args=None):
    from paper_1704_08897_gb300 import synth
    if name == "single":
        p = synth.single_star_case(1024)
        return [p], {"workload": "star1024_periodic_extend_in", "grid": "1024x1024",
                     "instances": 1, "prec": "fp32"}
    if name == "serve":
        reqs = synth.serving_stream(count=args.requests, rate=args.rate,
                                    seed=synth.BASE_SEED + 1000 * rank, side_lo=64, side_hi=512)
        probs = [r.problem for r in reqs]
        return probs, {"workload": f"serve{args.requests}_poisson{args.rate:g}per_s_sides64-512",
                       "instances": len(probs), "arrivals": [r.arrival_s for r in reqs],
                       "prec": "mixed_bf16"}
    count = args.instances if args is not None else 256
    probs = synth.batch_case(count, seed=synth.BASE_SEED + 1000 * rank)
    nodes = sum(p.nx * p.ny for p in probs)
    return probs, {"workload": f"batch{count}_sides128-512_wobbly_extend_out", "instances": count,
                   "nodes": nodes, "prec": "mixed_bf16"}


# Slice products the tensor cores execute per useful product in the mixed modes (four slices per
# operand, orders 0..3: 1 + 2 + 3 + 4), and the tile granularity the operands are padded to.
TC_PRODUCTS = 10
TC_PAD = 128


# The low-mode products use six slices per operand: orders 0..5, 21 products per useful product,
# with k padded to 64 in the inverse product.
TC_LOW_PRODUCTS = 21


def mirror_classes(n, fold=True):
    """Node counts of one axis's transform problems in the mixed preconditioner: two mirror
    classes of ceil(n/2) nodes where both, padded to 128, fit in the padded axis, else the axis."""
    pad = lambda m: -(-m // TC_PAD) * TC_PAD
    h = (n + 1) // 2
    return [h, h] if fold and 2 * pad(h) <= pad(n) else [n]


def issued_tensor_flop(probs, kind, fold=None):
    """Flops the tensor cores execute in one launch of transform stage `kind` (mixed modes), over
    the transform problems (mirror classes) of every instance."""
    fold = _fold_default() if fold is None else fold
    pad = lambda n: -(-n // TC_PAD) * TC_PAD
    fl = 0
    for p in probs:
        for cx in mirror_classes(p.nx, fold):
            for cy in mirror_classes(p.ny, fold):
                if kind == "low_fwd":
                    fl += 2 * TC_LOW_PRODUCTS * pad(cy) * 32 * pad(cx)
                elif kind == "low_inv":
                    fl += 2 * TC_LOW_PRODUCTS * pad(cx) * pad(cy) * 64
                else:
                    s = int(kind[-1])
                    fl += 2 * TC_PRODUCTS * pad(cx) * pad(cy) * pad(cx if s in (0, 2) else cy)
    return fl


def _fold_default():
    return bool(_OPTION_OVERRIDES.get("fold", 1))


def algorithmic_cost(probs, kind, low=False):
    """(amount, unit) per launch of one kernel kind over the workload's instances; low: the
    low-mode correction ran (the residual is then cut into six slices instead of four)."""
    if kind in ("low_fwd", "low_inv"):
        # the lowest 32 modes of one axis against the whole grid: 2 * nx * ny * 32 flop
        return sum(2 * p.nx * p.ny * min(32, p.nx) for p in probs), "flop"
    if kind.startswith("prec_stage"):
        # stage k contracts one axis: 2 * nx * ny * (length of that axis) flop
        s = int(kind[-1])
        fl = 0
        for p in probs:
            fl += 2 * p.nx * p.ny * (p.nx if s in (0, 2) else p.ny)
        return fl, "flop"
    # CG vectors are double-float pairs of FP32 planes: 8 bytes per node each
    if kind == "stencil":   # read z, p_old (8 + 8), mask (1); write p, q (8 + 8)
        return sum(33 * p.nx * p.ny for p in probs), "byte"
    if kind == "update":    # read x, p, q, r; write x, r (8 bytes each)
        return sum(48 * p.nx * p.ny for p in probs), "byte"
    if kind in ("split", "fold"):  # read r (8); write four (six) 16-bit slices: unfolded / folded
        f = kind == "fold"
        per_node = 8 + 2 * (6 if low else 4)
        return sum(per_node * p.nx * p.ny for p in probs
                   if (len(mirror_classes(p.nx, _fold_default())) > 1 or
                       len(mirror_classes(p.ny, _fold_default())) > 1) == f), "byte"
    if kind == "unfold":    # read the classes' g (8), r (8), mask (1); write z (8); q (8) is read
        return sum(25 * p.nx * p.ny for p in probs), "byte"  # only for the flexible beta
    return None, None


# ----------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------------------------
# our implementation
# ----------------------------------------------------------------------------------------------
def kernel_hash(kind, prec="fp32"):
    if kind.startswith("prec") or kind in ("split", "fold", "unfold") or kind.startswith("low"):
        f = "kernels_gemm_simt.cu" if prec == "fp32" else "kernels_gemm_tc.cu"
    else:
        f = "kernels_grid.cu"
    with open(os.path.join(CSRC, f), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def reduce_over_ranks(value, op, device):
    """Max or sum of a per-rank number over all ranks (torch.distributed initialised)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_1704_08897_gb300 import ext

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    ext.load()
    probs, cfg = make_workload(args.workload, rank, args)
    arrivals = cfg.pop("arrivals", None)
    prec = args.prec or cfg["prec"]
    cfg["prec"] = prec
    stream = torch.cuda.Stream()
    # hard extend-out grids need up to ~10 n iterations at 1e-8 in FP32 arithmetic
    maxit = 40 * max(max(p.nx, p.ny) for p in probs)
    ctx = ext.ext_create(_options(prec, rtol=1e-8, maxit=maxit), stream=stream)
    dprobs = [ext.problem_of(p) for p in probs]
    phis = [torch.from_numpy(p.phi).cuda() for p in probs]
    fs = [torch.from_numpy(p.f).cuda() for p in probs]
    outs = [torch.empty_like(x) for x in phis]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2

    serve_stats = []

    def step():
        if args.workload == "serve":
            # requests arrive on their Poisson schedule while earlier ones are on the GPU
            t0 = time.perf_counter()
            tickets = []
            for k in range(len(probs)):
                while time.perf_counter() - t0 < arrivals[k]:
                    time.sleep(5e-5)
                tickets.append(ext.ext_submit(ctx, dprobs[k], phis[k], fs[k], outs[k]))
            ext.ext_drain(ctx)
            wall = time.perf_counter() - t0
            res = [ext.ext_poll(ctx, t) for t in tickets]
            serve_stats.append({"wall_s": wall,
                                "lat_ms": [r["ms_queue"] + r["ms_solve"] for r in res]})
            return res
        if len(probs) == 1:
            r = ext.ext_solve(ctx, dprobs[0], phis[0], fs[0], outs[0])
            return [r]
        rc, res = ext.ext_solve_batch(ctx, dprobs, phis, fs, outs, check=False)
        return res

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = ext.ext_launch_count(ctx)
    step_ms, results = [], None
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        results = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = ext.ext_launch_count(ctx) - launches0
    tile = ext.ext_stencil_tile(ctx)
    # answers of the last timed step, for the error against the oracle (later passes reuse outs)
    answers = [o.cpu().numpy() for o in outs[:32]]
    clk = clocks.stop()
    total_ms = sum(step_ms)
    converged = sum(1 for r in results if r.get("status", 0) == 0)
    if world > 1:
        # the job's time is the slowest rank's; its work is every rank's converged solves
        total_ms = reduce_over_ranks(total_ms, "max", "cuda")
        converged = reduce_over_ranks(converged, "sum", "cuda")
        torch.distributed.barrier()
    solves = converged * args.steps
    value = solves / (total_ms / 1e3)
    serving = None
    if serve_stats:
        lat = sorted(x for st in serve_stats for x in st["lat_ms"])
        wall = sum(st["wall_s"] for st in serve_stats)
        value = solves / wall  # arrivals pace the step: throughput over wall time
        serving = {"p50_ms": round(lat[len(lat) // 2], 3), "p99_ms": round(lat[int(0.99 * (len(lat) - 1))], 3),
                   "requests": len(lat), "offered_rate_per_s": args.rate}
    iters = [r["iters"] for r in results]
    nodes = sum(p.nx * p.ny for p in probs)
    pt_its = sum(p.nx * p.ny * r["iters"] for p, r in zip(probs, results))

    # the same sample of the workload's grids through the four combinations of path and launch
    # (FP32 / mixed, one ext_solve per grid / one ext_solve_batch), so that the gain of batching
    # and the gain of the tensor-core preconditioner are reported separately; the plain FP32
    # single-solve path is the comparison the batched and served paths are measured against
    plain, same_grids, sample_answers, sample_iters = None, None, {}, {}
    if args.workload != "single" and args.plain_sample > 0:
        k = min(args.plain_sample, len(probs))
        same_grids = {"sample": f"first {k} grids of the workload", "grids": k}
        for pname in ("fp32", "mixed_bf16"):
            cctx = ext.ext_create(_options(pname, rtol=1e-8, maxit=maxit), stream=stream)
            for mode in ("single", "batched"):
                # warm: plans and workspaces of these shapes
                if mode == "single":
                    for j in range(k):
                        ext.ext_solve(cctx, dprobs[j], phis[j], fs[j], outs[j], check=False)
                else:
                    ext.ext_solve_batch(cctx, dprobs[:k], phis[:k], fs[:k], outs[:k], check=False)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if mode == "single":
                    rr = [ext.ext_solve(cctx, dprobs[j], phis[j], fs[j], outs[j], check=False)
                          for j in range(k)]
                else:
                    _, rr = ext.ext_solve_batch(cctx, dprobs[:k], phis[:k], fs[:k], outs[:k],
                                                check=False)
                e1.record(stream)
                e1.synchronize()
                el = e0.elapsed_time(e1) / 1e3
                its = [r["iters"] for r in rr]
                same_grids[f"{pname}_{mode}"] = {
                    "value": round(k / el, 4), "unit": "solves/s",
                    "iterations_median": statistics.median(its),
                    "all_converged": all(r["rc"] == 0 if "rc" in r else r["status"] == 0 for r in rr)}
                sample_answers[f"{pname}_{mode}"] = [o.cpu().numpy() for o in outs[:k]]
                sample_iters[f"{pname}_{mode}"] = its
            ext.ext_destroy(cctx)
        plain = dict(same_grids["fp32_single"],
                     sample=f"first {k} grids of the workload, one ext_solve each, FP32 path")

    # end to end through the public API with host (pinned) buffers
    e2e = None
    if not args.no_e2e and args.workload != "serve":
        hphis = [torch.from_numpy(p.phi).pin_memory() for p in probs]
        hfs = [torch.from_numpy(p.f).pin_memory() for p in probs]
        houts = [torch.empty(p.phi.shape, dtype=torch.float32).pin_memory() for p in probs]
        if len(probs) == 1:
            ext.ext_solve(ctx, dprobs[0], hphis[0], hfs[0], houts[0])
        else:
            ext.ext_solve_batch(ctx, dprobs, hphis, hfs, houts, check=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            if len(probs) == 1:
                ext.ext_solve(ctx, dprobs[0], hphis[0], hfs[0], houts[0])
            else:
                ext.ext_solve_batch(ctx, dprobs, hphis, hfs, houts, check=False)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e = {"value": len(probs) * args.steps * world / el, "unit": "solves/s",
               "h2d_bytes_per_step": sum(8 * p.nx * p.ny for p in probs),
               "d2h_bytes_per_step": sum(4 * p.nx * p.ny for p in probs)}

    # per-kernel CUDA-event durations of the same workload (a profiled pass: no graphs)
    roofline, kernels, kernels_hbm = None, None, None
    if not args.no_profile and rank == 0:
        # profiled pass: the first 100 iterations, during which every instance is still iterating,
        # so each launch processes the whole workload (the algorithmic cost per launch holds)
        pctx = ext.ext_create(_options(prec, rtol=1e-8, maxit=100, profile=1), stream=stream)
        if args.workload == "serve":
            ext.ext_solve_batch(pctx, dprobs, phis, fs, outs, check=False)
        elif len(probs) == 1:
            ext.ext_solve(pctx, dprobs[0], phis[0], fs[0], outs[0], check=False)
        else:
            ext.ext_solve_batch(pctx, dprobs, phis, fs, outs, check=False)
        prof = ext.ext_profile_read(pctx)
        ext.ext_destroy(pctx)
        tot = sum(ms for ms, n in prof.values())
        kernels = {k: {"ms_total": round(ms, 3), "launches": n, "share": round(ms / tot, 4) if tot else 0,
                       "us_per_launch": round(1e3 * ms / n, 3) if n else None}
                   for k, (ms, n) in prof.items() if n}
        dom = max(prof, key=lambda k: prof[k][0])
        ms, n = prof[dom]
        amount, unit = algorithmic_cost(probs, dom, low="low_fwd" in kernels)
        if amount is not None and n:
            per_launch_s = ms / n / 1e3
            if unit == "flop" and prec != "fp32":
                # tensor-core stage: algorithmic flops (2 n^3-type, unpadded) against the measured
                # sustained dense BF16 peak; the MMAs actually issued (ten slice products over
                # padded tiles) are reported beside it
                achieved = amount / per_launch_s / 1e12
                with open(PEAKS_FILE) as fh:
                    peak = json.load(fh)["bf16_tflops_sustained"]
                bound, u = "tensor", "TFLOP/s"
                peak_src = "measured bf16_tflops_sustained"
            elif unit == "flop":
                achieved = amount / per_launch_s / 1e12
                peak, bound, u = FP32_ALU_PEAK_TFLOPS, "alu", "TFLOP/s"
                peak_src = "derived: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz"
            else:
                achieved = amount / per_launch_s / 1e9
                with open(PEAKS_FILE) as fh:
                    peak = json.load(fh)["hbm_gbs"]
                bound, u, peak_src = "hbm", "GB/s", "measured hbm_gbs"
            traffic = None
            if os.path.exists(TRAFFIC_FILE):
                with open(TRAFFIC_FILE) as fh:
                    tr = json.load(fh)
                ent = tr.get(f"{dom}:{prec}:{cfg['workload']}")
                if ent and ent.get("source_hash") == kernel_hash(dom, prec):
                    traffic = ent.get("bytes_per_launch")
            roofline = {"kernel": dom, "bound": bound, "achieved": round(achieved, 3),
                        "peak": round(peak, 3), "unit": u, "frac": round(achieved / peak, 4),
                        "traffic": traffic, "peak_source": peak_src,
                        "algorithmic_per_launch": amount, "algorithmic_unit": unit}
            # the memory-bound kernels against the measured copy bandwidth, from the same pass
            with open(PEAKS_FILE) as fh:
                hbm_peak = json.load(fh)["hbm_gbs"]
            hbm = {}
            for kd in ("stencil", "update", "split", "fold", "unfold"):
                amt, un = algorithmic_cost(probs, kd, low="low_fwd" in kernels)
                if kd in prof and prof[kd][1] and un == "byte":
                    gbs = amt / (prof[kd][0] / prof[kd][1] / 1e3) / 1e9
                    hbm[kd] = {"achieved_gbs": round(gbs, 1), "frac": round(gbs / hbm_peak, 4),
                               "bytes_per_launch": amt}
            kernels_hbm = hbm
            if bound == "tensor":
                # what the tensor pipe actually executes: the exact slice products on padded tiles
                issued = issued_tensor_flop(probs, dom) / per_launch_s / 1e12
                roofline["issued"] = {"achieved": round(issued, 3), "frac": round(issued / peak, 4),
                                      "products_per_useful_product":
                                          TC_LOW_PRODUCTS if dom.startswith("low") else TC_PRODUCTS,
                                      "pad": TC_PAD}

    ext.ext_destroy(ctx)
    out = {"metric": "extension solves/s at rel-res 1e-8", "value": round(value, 4),
           "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded; paper-shaped interfaces and fields)",
           "config": dict(cfg, l2="flushed between steps (256 MiB write)",
                          parallelism="replicas" if world > 1 else "single",
                          low_modes=_options(cfg["prec"]).low_modes,
                          # whether the profiled pass ran the low-mode kernels (None: not profiled)
                          low_modes_active=None if kernels is None else "low_fwd" in kernels,
                          fold=_options(cfg["prec"]).fold),
           "iterations": iters if len(iters) <= 4 else
           {"min": min(iters), "median": statistics.median(iters), "max": max(iters)},
           "iterations_per_grid": iters[:32],
           "grid_point_iterations_per_s": round(pt_its * args.steps * world / (total_ms / 1e3), 1),
           "relres_true_max": max(r["relres_true"] for r in results),
           "all_converged": all(r.get("status", 0) == 0 for r in results),
           "plain_fp32_single_solve": plain, "same_grids": same_grids, "serving": serving,
           "e2e": e2e, "roofline": roofline, "hbm_kernels": kernels_hbm, "kernels": kernels,
           "stencil_tile": {"x": tile[0], "y": tile[1], "chosen_by": "autotuner"},
           "gpu_launches": launches, "clocks": clk}
    return out, probs, answers, (sample_answers, sample_iters)


def oracle_solve(p):
    import numpy as np

    from oracle import biharmonic as ob
    return ob.extend(p.phi.astype(np.float64), p.f.astype(np.float64), p.direction, p.bc_x,
                     p.bc_y, p.hx, p.hy, method="direct")


def cpu_baseline(args, probs, budget_s=30.0):
    """The oracle, as it stands, on a bounded sample of the workload (whole problems only).
    Returns the timing record and the oracle's answers."""
    t0 = time.perf_counter()
    done, refs = 0, []
    for p in probs:
        refs.append(oracle_solve(p)[0])
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": round(done / el, 5), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} of {len(probs)} problem(s) of the workload solved completely by the "
                      f"FP64 oracle (sparse assembly + SuperLU), {el:.1f} s",
            "host_cores_available": os.cpu_count()}, refs


def error_vs_oracle(probs, answers, refs, prec, at="rel-res 1e-8, answers of the last timed step"):
    """Max-norm relative error (max over unknowns of |x - x*| / max |out*|) of the GPU answers
    of the timed run against the oracle's direct solves, over the problems the oracle solved."""
    import numpy as np

    from oracle import biharmonic as ob
    errs = []
    for p, a, r in zip(probs, answers, refs):
        known = ob.known_mask(p.phi.astype(np.float64), p.direction)
        errs.append(ob.max_rel_error(a, r, known))
    bound = 1e-6 if prec == "fp32" else 1e-5
    return {"max_rel": float(max(errs)), "median_rel": float(np.median(errs)),
            "problems": len(errs), "bound": bound, "within": bool(max(errs) <= bound),
            "at": at}


# The paper's Example 2 table (three-dimensional peanut, periodic): n -> (iterations, error)
PAPER_EXAMPLE2 = {32: (21, 1.08e-01), 64: (46, 3.42e-02), 128: (112, 1.07e-02), 256: (276, 2.84e-03)}


def peanut3d_leg(sides=(64, 128, 256)):
    """The three-dimensional extension (Sec. 3 Example 2): the peanut on [-pi, pi]^3, periodic,
    extend out, through ext_solve3d, on the FP32 path (CUDA-core transforms) and, for sides that
    are multiples of 128, the mixed path (tensor-core transforms).  Per side and path: time and
    iterations at rel-res 1e-8 and at the paper's 1e-6 (beside the printed iterations), and the
    max error within one grid cell of the interface against the analytic field."""
    import numpy as np
    import torch
    from paper_1704_08897_gb300 import ext
    out = {"workload": "Example 2 peanut, [-pi, pi]^3, periodic, extend out; FP32 path, and mixed "
                       "(tensor-core transforms) for sides that are multiples of 128",
           "note": "paper errors match the one-cell band (its caption says four cells)", "sides": {}}
    for n in sides:
        h = 2 * np.pi / n
        xs = -np.pi + (np.arange(n) + 0.5) * h
        Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
        phi = np.minimum(np.sqrt((X - 0.8) ** 2 + Y ** 2 + Z ** 2) - 1,
                         np.sqrt((X + 0.8) ** 2 + Y ** 2 + Z ** 2) - 1).astype(np.float32)
        f = (np.cos(X) * np.sin(Y) * np.sin(np.pi / 4 - Z)).astype(np.float32)
        band = np.abs(phi) <= h
        dphi, dfv = torch.from_numpy(phi).cuda(), torch.from_numpy(f).cuda()
        o = torch.empty_like(dphi)
        prob = ext.problem3(n, n, n, "periodic", "periodic", "periodic", "out", h)
        row = {}
        for prec in ("fp32", "mixed_bf16") if n % 128 == 0 else ("fp32",):
            for rtol in (1e-8, 1e-6):
                c = ext.ext_create(_options(prec, rtol=rtol))
                try:
                    if rtol == 1e-8:
                        ext.ext_solve3d(c, prob, dphi, dfv, o)    # warm-up (plans, code)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    res = ext.ext_solve3d(c, prob, dphi, dfv, o)
                    torch.cuda.synchronize()
                    dt = time.perf_counter() - t0
                finally:
                    ext.ext_destroy(c)
                err = float(np.abs(o.cpu().numpy() - f)[band].max())
                row[f"{prec}_rtol_{rtol:g}"] = {"iterations": res["iters"], "s_per_solve": round(dt, 4),
                                                "relres_true": res["relres_true"], "error_1cell": err}
        if n in PAPER_EXAMPLE2:
            row["paper"] = {"iterations": PAPER_EXAMPLE2[n][0], "error": PAPER_EXAMPLE2[n][1]}
        # the six dense transform products dominate the FP32 path: 2 n^4 multiply-adds each
        it = row["fp32_rtol_1e-08"]["iterations"]
        row["fp32_transform_fma_per_s"] = (6 * 2 * n ** 4 * (it + 1)) / row["fp32_rtol_1e-08"]["s_per_solve"]
        out["sides"][str(n)] = row
    return out


def serving_leg(count=48, seed=None, side_lo=64, side_hi=2048, plain_budget_s=20.0):
    """A bounded sample of the serving workload (config-4 shape): `count` requests with sides
    log-uniform in [side_lo, side_hi], star or multi-circle interfaces, extend in or out and
    symmetric or periodic edges at random, served by ext_submit / ext_poll with the mixed BF16
    path.  Plans of every shape are built first (an all-known solve per shape); then the stream
    is offered (1) all at once (saturation: the throughput is the capacity C) and (2) as Poisson
    arrivals at 0.5 C (below saturation), each reporting p50/p99 latency (arrival to result) and
    solves/s over wall time.  The serial plain FP32 path is timed on the same requests in arrival
    order within a time budget."""
    import numpy as np
    import torch

    from paper_1704_08897_gb300 import ext, synth
    seed = synth.BASE_SEED if seed is None else seed
    reqs = synth.serving_stream(count=count, rate=1.0, seed=seed, side_lo=side_lo, side_hi=side_hi)
    probs = [r.problem for r in reqs]
    unit_t = [r.arrival_s for r in reqs]  # arrivals at 1 request/s; scaled per offered rate
    maxit = 40 * max(p.nx for p in probs)
    ctx = ext.ext_create(_options("mixed_bf16", rtol=1e-8, maxit=maxit))
    dprobs = [ext.problem_of(p) for p in probs]
    phis = [torch.from_numpy(p.phi).cuda() for p in probs]
    fs = [torch.from_numpy(p.f).cuda() for p in probs]
    outs = [torch.empty_like(x) for x in phis]
    seen = set()
    for p, dp, f in zip(probs, dprobs, fs):
        key = (p.nx, p.bc_x)
        if key in seen:
            continue
        seen.add(key)
        allk = torch.full((p.ny, p.nx), -1.0 if p.direction == "out" else 1.0, device="cuda")
        ext.ext_solve(ctx, dp, allk, f, torch.empty_like(allk), check=False)

    def offer(times):
        t0 = time.perf_counter()
        tickets = []
        for k in range(len(probs)):
            while time.perf_counter() - t0 < times[k]:
                time.sleep(5e-5)
            tickets.append(ext.ext_submit(ctx, dprobs[k], phis[k], fs[k], outs[k]))
        ext.ext_drain(ctx)
        wall = time.perf_counter() - t0
        res = [ext.ext_poll(ctx, t) for t in tickets]
        lat = sorted(r["ms_queue"] + r["ms_solve"] for r in res)
        ok = sum(1 for r in res if r["rc"] == 0)
        return {"solves_per_s": round(ok / wall, 3), "p50_ms": round(lat[len(lat) // 2], 2),
                "p99_ms": round(lat[int(0.99 * (len(lat) - 1))], 2), "requests": len(res),
                "converged": ok, "wall_s": round(wall, 2),
                "iterations_median": statistics.median(r["iters"] for r in res)}

    sat = offer([0.0] * len(probs))
    cap = sat["solves_per_s"]
    low_rate = 0.5 * cap
    low = offer([t / low_rate for t in unit_t])
    ext.ext_destroy(ctx)
    # the serial plain FP32 path on the same requests (those with sides up to 512: a single
    # large request alone takes the path a minute), in arrival order, within a time budget
    pctx = ext.ext_create(_options("fp32", rtol=1e-8, maxit=maxit))
    done, t0 = 0, time.perf_counter()
    for p, dp, ph, f, o in zip(probs, dprobs, phis, fs, outs):
        if p.nx > 512:
            continue
        ext.ext_solve(pctx, dp, ph, f, o, check=False)
        done += 1
        if time.perf_counter() - t0 > plain_budget_s:
            break
    el = time.perf_counter() - t0
    ext.ext_destroy(pctx)
    sides = sorted(p.nx for p in probs)
    return {"workload": f"serve{count}_poisson_sides{side_lo}-{side_hi}_star_or_circles_mixed_bf16",
            "sides": {"min": sides[0], "median": sides[len(sides) // 2], "max": sides[-1]},
            "saturated": dict(sat, offered="all requests at once"),
            "below_saturation": dict(low, offered_rate_per_s=round(low_rate, 3),
                                     offered="Poisson arrivals at half the saturated throughput"),
            "p50_ms": low["p50_ms"], "p99_ms": low["p99_ms"],
            "serial_plain_fp32": {"solves_per_s": round(done / el, 4), "requests": done,
                                  "sample": f"first {done} requests with sides up to 512 in "
                                            f"arrival order, one ext_solve each, FP32 path "
                                            f"({el:.1f} s)"}}


def oracle_pcg_iterations(probs, batched_iters, sample_iters, count=3, budget_s=20.0):
    """Iterations of the oracle's FP64 PCG (the same fast Poisson preconditioner and
    Fletcher-Reeves beta, rel-res 1e-8) beside the GPU's on the first grids of the workload."""
    import numpy as np

    from oracle import biharmonic as ob
    rows, t0 = [], time.perf_counter()
    for j, p in enumerate(probs[:count]):
        _, info = ob.extend(p.phi.astype(np.float64), p.f.astype(np.float64), p.direction, p.bc_x,
                            p.bc_y, p.hx, p.hy, method="pcg", rtol=1e-8)
        row = {"grid": f"{p.nx}x{p.ny}", "oracle_fp64_pcg": info["iters"]}
        if batched_iters is not None and j < len(batched_iters):
            row["timed_run"] = batched_iters[j]
        for key, its in sample_iters.items():
            if j < len(its):
                row[key] = its[j]
        rows.append(row)
        if time.perf_counter() - t0 > budget_s:
            break
    return rows


def run_reference(args, rank, world):
    """The FP64 oracle (sparse assembly + SuperLU) timed on the host cores; each step solves a
    bounded sample of the workload's problems completely."""
    probs, cfg = make_workload(args.workload, rank, args)
    cfg.pop("arrivals", None)
    if args.prec:
        cfg["prec"] = args.prec
    cfg = dict(cfg, l2="flushed between steps (256 MiB write)",
               parallelism="replicas" if world > 1 else "single")
    sample = probs[:1] if len(probs) == 1 else probs[:4]
    for _ in range(args.warmup):
        oracle_solve(sample[0])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for p in sample:
            oracle_solve(p)
    el = time.perf_counter() - t0
    value = len(sample) * args.steps / el
    desc = (f"{len(sample)} complete oracle solve(s) per step (the first {len(sample)} problems of "
            f"the workload; FP64, SuperLU, single-threaded)")
    return {"impl": "reference", "metric": "extension solves/s at rel-res 1e-8",
            "value": round(value, 5), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * el / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded; paper-shaped interfaces and fields)", "config": cfg,
            "cpu_baseline": {"value": round(value, 5), "unit": "solves/s", "cores": 1,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": round(value, 5), "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)))
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    out, probs, answers, (sample_answers, sample_iters) = run_ours(args, rank, world)
    if rank == 0 and args.workload == "batch" and args.serve_requests > 0:
        out["serving"] = serving_leg(count=args.serve_requests)
    if rank == 0 and args.workload == "batch" and args.peanut3d:
        out["peanut3d"] = peanut3d_leg(tuple(int(v) for v in args.peanut3d.split(",")))
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"], refs = cpu_baseline(args, probs)
            prec = out["config"]["prec"]
            acc = {"rtol_1e-08": error_vs_oracle(probs, answers, refs, prec)}
            # every path and launch of the same-grid comparison, against the same direct solves
            for key, ans in sample_answers.items():
                acc[f"rtol_1e-08_{key}"] = error_vs_oracle(
                    probs, ans, refs, "fp32" if key.startswith("fp32") else "mixed",
                    at=f"rel-res 1e-8, {key.replace('_', ' ')} answers of the same-grid sample")
            out["iterations_vs_oracle_pcg"] = oracle_pcg_iterations(
                probs, out.get("iterations_per_grid"), sample_iters)
            out["error_vs_oracle"] = acc
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
