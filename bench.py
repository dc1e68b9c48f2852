#!/usr/bin/env python
"""Benchmark of the coupled electroconvection step (arXiv:1812.05711) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the single large channel run -- 2048 x 1680 nodes, FP32 compute on
shifted FP32 populations, T ~ U[150, 250] (seeded), C = 10, M = 10, Fe = 4000,
Lambda = 1/4, random Eq. 29 modes of amplitude 1e-4 u_ion.  One benchmark step
is one whole coupled step: fused collide-and-stream of f and g with the
electric force and drift, wall fluxes, and the FFT / tridiagonal Poisson solve
of the new charge.  Metric: GLUPS = lattice node updates per second / 1e9
(whole job; with N GPUs each rank advances its own run: weak scaling, no
collective on the data path).

Prints one JSON line.  Inputs (the 495 MB population state) are larger than
the 129 MB L2, so no L2 flush is needed between steps.
"""
from __future__ import annotations

import argparse
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

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

METRIC = "coupled-step GLUPS"
UNIT = "GLUPS"
# kernels per coupled step: collide-stream (march form, writes the charge),
# forward row FFT, mean mode (side stream), wavenumber systems, inverse row FFT
LAUNCHES_PER_STEP = 5
# algorithmic bytes per node of the fused collide-stream kernel: 9 f + 9 g
# loaded, 9 f + 9 g stored, one potential value loaded, one charge density
# stored (both in the compute precision: FP64 for f64 storage, else FP32)
K4_BYTES_PER_NODE = {"f32": 36 * 4 + 8, "f64": 36 * 8 + 16, "bf16": 36 * 2 + 8, "f16": 36 * 2 + 8}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the fused step kernel, from an ncu capture of the 2048 x 1680 FP32 channel
# in the steady state of this bench (no cache flush between launches: the
# mean of three consecutive launches); keyed by a hash of the kernel's sources
# so that it reads null once the kernel has changed since the capture.
NCU_TRAFFIC = {("f32", "b117d667c207899e"): (245.364736e6 + 241.394688e6 + 241.035008e6) / 3
               + (262.903808e6 + 260.883456e6 + 260.696832e6) / 3}


def _kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for name in ("k_march.cu", "ehd_dev.cuh"):
        with open(os.path.join(ROOT, "paper_1812_05711_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the run."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        maxmhz = max(r[1] for r in rows)
        busy = [r[0] for r in rows if r[2] > 200.0] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": maxmhz, "reasons": reasons,
                "samples": len(rows), "samples_under_load": len(busy)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1, 0
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    import torch
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return dist, rank, ws, local


def _weak_value(ws: int, cells: int, steps: int, ms_max: float) -> float:
    """Whole-job GLUPS: every rank advances its own channel of `cells` nodes
    (weak scaling), timed by the slowest rank."""
    return ws * cells * steps / (ms_max * 1e-3) / 1e9


def _max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_glups(w: wl.Workload, budget_s: float, max_steps: int | None = None):
    """The FP64 CPU oracle as it stands (one thread) on the given channel."""
    import oracle as o
    p = o.setup(*w.args())
    s = o.init_state(p, w.amp, w.phase)
    t0 = time.perf_counter()
    o.step(s, 1)  # warm-up step, also sizes the timed sample
    est = time.perf_counter() - t0
    n = max(1, int(budget_s / max(est, 1e-6)))
    if max_steps is not None:
        n = min(n, max_steps)
    t0 = time.perf_counter()
    o.step(s, n)
    el = time.perf_counter() - t0
    return w.Nx * w.Ny * n / el / 1e9, n, el


def _cpu_baseline(w: wl.Workload, budget_s: float, what: str) -> dict:
    """The oracle timed twice on a bounded sample of the workload: its one-
    thread build, and its OpenMP build (rows, wavenumbers and nodes shared
    among all host cores; bitwise the same states).  The line's value is the
    all-cores figure; the one-thread figure sits beside it."""
    import oracle as o
    v1, n1, el1 = _oracle_glups(w, budget_s)
    out = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{n1} oracle steps of {what} in {el1:.1f} s (one thread)"}
    threads = o.use_threads(os.cpu_count())
    try:
        if threads > 1:
            vn, nn, eln = _oracle_glups(w, budget_s)
            out = {"value": vn, "unit": UNIT, "cores": threads, "kind": "oracle",
                   "sample": f"{nn} oracle steps of {what} in {eln:.1f} s ({threads} OpenMP threads over rows, "
                             f"wavenumbers and nodes)",
                   "one_thread": {"value": v1, "cores": 1, "sample": f"{n1} steps in {el1:.1f} s"}}
    finally:
        o.use_one_thread()
    out["cpu_model"] = _cpu_model()
    out["host_cores"] = os.cpu_count()
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed on the host cores.  Under
    torchrun only rank 0 works; the other ranks exit at once (no process
    group is formed: the arm has no collective)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    import oracle as o
    threads = max(1, o.use_threads(os.cpu_count()))  # the oracle's OpenMP build on every host core
    full = wl.large_channel()
    # each benchmark step: one oracle step of a 512 x 416 channel with the same
    # groups and perturbation recipe (1/16 of the 2048 x 1680 nodes)
    w = wl.Workload("channel-512x416-sample", 512, 416, full.T, amp=full.amp, phase=full.phase)
    p = o.setup(*w.args())
    s = o.init_state(p, w.amp, w.phase)
    o.step(s, args.warmup)
    t0 = time.perf_counter()
    o.step(s, args.steps)
    el = time.perf_counter() - t0
    val = w.Nx * w.Ny * args.steps / el / 1e9
    sample = (f"oracle steps of a 512x416 channel (same T, C, M, Fe, Lambda and Eq. 29 modes as the "
              f"2048x1680 workload); {args.steps} steps in {el:.2f} s on {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "channel-2048x1680 (sampled as 512x416)", "Nx": w.Nx, "Ny": w.Ny,
                       "T": w.T, "C": w.C, "M": w.M, "Fe": w.Fe, "Lambda": w.Lambda},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu_model": _cpu_model()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    import paper_1812_05711_gb300 as ehd

    dist, rank, ws, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    clk = Clocks(local) if rank == 0 else None
    storage = args.storage
    w = wl.large_channel()
    cells = w.Nx * w.Ny
    pert = 1 if getattr(args, "perturbation", False) else 0
    if pert and storage == "f64":
        raise SystemExit("--perturbation takes FP32 compute (storage f32, bf16 or f16)")
    run = ehd.Run(*w.args(), storage=storage, amp=w.amp, phase=w.phase, perturbation=pert)
    h = run.handle
    stream = torch.cuda.ExternalStream(ehd.ehd_stream(h))
    f0, g0 = run.save()  # initial state, kept for the end-to-end leg

    # warm-up: builds the CUDA graphs of the step and pages everything in
    run.step(max(args.warmup, 16) if args.steps >= 16 else args.warmup)
    run.sync()

    # ---- device-resident timed region: K coupled steps through ehd_step
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    ms_max = _max_over_ranks(dist, ms)
    value = _weak_value(ws, cells, args.steps, ms_max)
    run.sync()

    # ---- per-kernel timing (events around each kernel on the run's stream)
    prof = ehd.ehd_step_profile(h, args.steps)
    k4_ms = prof["collide_stream_ms"] / args.steps
    bytes_k4 = K4_BYTES_PER_NODE[storage] * cells
    peak, peak_kind = _peaks()
    achieved = bytes_k4 / (k4_ms * 1e-3) / 1e9
    # whole coupled step: the step kernel's bytes plus phi read and rho_c written
    # once more by the Poisson chain's transforms (160 B per node in FP32)
    step_bytes = (K4_BYTES_PER_NODE[storage] + 8) * cells
    step_achieved = step_bytes / (ms_max / args.steps * 1e-3) / 1e9

    # ---- end to end through the C ABI with host buffers (pinned)
    pin_f = torch.empty(f0.shape, dtype=torch.float64, pin_memory=True).numpy()
    pin_g = torch.empty(g0.shape, dtype=torch.float64, pin_memory=True).numpy()
    pin_f[...] = f0
    pin_g[...] = g0
    mask = ehd.FIELD_BITS["rho"] | ehd.FIELD_BITS["ux"] | ehd.FIELD_BITS["uy"] | ehd.FIELD_BITS["rho_c"]
    out = torch.empty((4, w.Ny, w.Nx), dtype=torch.float64, pin_memory=True).numpy()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ehd.ehd_load(h, pin_f, pin_g)
    ehd.ehd_step(h, args.steps)
    ehd.ehd_fields(h, mask, out)
    e2e_s = time.perf_counter() - t0
    e2e_s = _max_over_ranks(dist, e2e_s)
    e2e = _weak_value(ws, cells, args.steps, e2e_s * 1e3)
    h2d = (pin_f.nbytes + pin_g.nbytes) / args.steps
    d2h = out.nbytes / args.steps
    diag = run.diagnostics()
    clocks = clk.stop() if clk else None

    if rank != 0:
        run.close()
        return 0

    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(w, args.cpu_seconds, "the full 2048x1680 channel")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if storage != "f64" else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "Nx": w.Nx, "Ny": w.Ny, "T": round(w.T, 6), "C": w.C, "M": w.M,
                   "Fe": w.Fe, "Lambda": w.Lambda, "storage": storage, "compute": "f32" if storage != "f64" else "f64",
                "form": "perturbation" if pert else ("shifted" if storage != "f64" else "plain"),
                   "per_rank": "one independent run", "l2": "state 495 MB > 129 MB L2, no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": NCU_TRAFFIC.get((storage, _kernel_hash())) if w.name == "channel-2048x1680" and not pert else None,
                     "traffic_unit": "bytes per launch, ncu dram read + write", "kernel": "k_march2 (fused collide-stream)",
                     "bytes_per_node": K4_BYTES_PER_NODE[storage], "kernel_ms": k4_ms,
                     "peak_kind": f"{peak_kind} hbm_gbs", "poisson_ms": prof["poisson_ms"] / args.steps,
                     "charge_ms": prof["charge_ms"] / args.steps,
                     "profiled_step_ms": prof["step_ms"] / args.steps,
                     "whole_step": {"bytes_per_node": K4_BYTES_PER_NODE[storage] + 8, "achieved": step_achieved,
                                    "frac": step_achieved / peak}},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": (LAUNCHES_PER_STEP + 2 * pert) * args.steps,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "check": {"mass": diag["mass"], "charge": diag["charge"], "max_u": diag["max_u"]},
    }
    print(json.dumps(line), flush=True)
    run.close()
    return 0


def _cells(w):
    return w.Nx * w.Ny


def run_batch(args):
    """64 runs of uneven sizes advanced together (FP32), launch shapes from the
    autotuner; metric: aggregate GLUPS over all runs."""
    import torch

    import paper_1812_05711_gb300 as ehd
    from paper_1812_05711_gb300 import autotune

    torch.cuda.set_device(0)
    ws = wl.batch_workloads(seed=4, n=64)
    K = args.steps
    max_nx, max_ny = 512, wl.ny_for(512)
    # tune on a throwaway copy of the batch (tuning consumes step budget)
    tb = ehd.Batch(len(ws), max_nx, max_ny)
    truns = [ehd.Run(*w.args(), storage="f32", amp=w.amp, phase=w.phase) for w in ws]
    for r in truns:
        tb.add(r, 10 ** 9)
    rec = autotune.tune(tb, steps=8, ticks=3, use_cache=False)
    params = rec["params"]
    tb.close()
    for r in truns:
        r.close()
    batch = ehd.Batch(len(ws), max_nx, max_ny)
    batch.tune(**params)
    runs = [ehd.Run(*w.args(), storage="f32", amp=w.amp, phase=w.phase) for w in ws]
    inits = [r.save() for r in runs]
    for r in runs:
        batch.add(r, K + args.warmup * args.tick)
    stream = torch.cuda.ExternalStream(ehd.ehd_batch_stream(batch.handle))
    for _ in range(args.warmup):
        batch.tick(args.tick)
    batch.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ticks = (K + args.tick - 1) // args.tick
    e0.record(stream)
    for _ in range(ticks):
        batch.tick(args.tick)
    e1.record(stream)
    batch.sync()
    ms = e0.elapsed_time(e1)
    cells = sum(_cells(w) for w in ws)
    value = cells * K / (ms * 1e-3) / 1e9
    # end to end: host initial states in, K steps, four fields of every run out
    for r in runs:
        batch.remove(r)
    pins = []
    for f0, g0 in inits:
        pf = torch.empty(f0.shape, dtype=torch.float64, pin_memory=True).numpy()
        pg = torch.empty(g0.shape, dtype=torch.float64, pin_memory=True).numpy()
        pf[...] = f0
        pg[...] = g0
        pins.append((pf, pg))
    outs = [torch.empty((4, w.Ny, w.Nx), dtype=torch.float64, pin_memory=True).numpy() for w in ws]
    mask = ehd.FIELD_BITS["rho"] | ehd.FIELD_BITS["ux"] | ehd.FIELD_BITS["uy"] | ehd.FIELD_BITS["rho_c"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r, (pf, pg) in zip(runs, pins):
        ehd.ehd_load(r.handle, pf, pg)
        batch.add(r, K)
    for _ in range(ticks):
        batch.tick(args.tick)
    batch.sync()
    for r, o in zip(runs, outs):
        ehd.ehd_fields(r.handle, mask, o)
    e2e_s = time.perf_counter() - t0
    h2d = sum(pf.nbytes + pg.nbytes for pf, pg in pins) / K
    d2h = sum(o.nbytes for o in outs) / K
    cpu = None
    if not args.no_cpu_baseline:
        cpu = _cpu_baseline(ws[0], args.cpu_seconds, f"member 0 ({ws[0].Nx}x{ws[0].Ny})")
    sizes = {}
    for w in ws:
        sizes[f"{w.Nx}x{w.Ny}"] = sizes.get(f"{w.Nx}x{w.Ny}", 0) + 1
    line = {"metric": "batched coupled-step GLUPS", "value": value, "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / ticks / args.tick, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch-64-uneven", "runs": len(ws), "sizes": sizes, "tick": args.tick,
                       "tuning": params, "tuner_us_per_step": rec["us_per_step"]},
            "roofline": None,
            "e2e": {"value": cells * K / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": 5 * ticks * args.tick, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    batch.close()
    return 0


def run_serve(args):
    """Poisson-arrival stream of stability-sweep requests through the
    continuous-batching server; the plain FP64 one-at-a-time path serves a
    bounded prefix of the same stream for comparison."""
    import torch

    from paper_1812_05711_gb300 import serve

    torch.cuda.set_device(0)
    stream = wl.serving_stream(seed=5, n=args.requests, rate=20.0)
    reqs = [serve.Request(k, w.Nx, w.Ny, w.T, w.C, w.M, w.Fe, w.Lambda, w.steps, w.amp, w.phase, arrival=t)
            for k, (t, w) in enumerate(stream)]
    budget = int(args.hbm_gb * 1e9)
    srv = serve.Server(budget, max_runs=256, tick_steps=args.tick, max_nx=1024, max_ny=wl.ny_for(1024))
    res = srv.serve(reqs, realtime=True)
    srv.close()
    cells = {r.rid: r.Nx * r.Ny for r in reqs}
    summ = serve.summarize(res, cells_of=lambda r: cells[r.rid])
    # comparison: plain FP64, one run at a time, on the first requests of the
    # same stream (bounded by time); the server again on the same prefix
    prefix = reqs[:args.fp64_requests]
    base = serve.summarize(serve.serve_plain_fp64(prefix, realtime=True), cells_of=lambda r: cells[r.rid])
    srv2 = serve.Server(budget, max_runs=256, tick_steps=args.tick, max_nx=1024, max_ny=wl.ny_for(1024))
    pref = serve.summarize(srv2.serve([serve.Request(**{**q.__dict__}) for q in prefix], realtime=True),
                           cells_of=lambda r: cells[r.rid])
    srv2.close()
    line = {"metric": "served runs/s", "value": summ["runs_per_s"], "unit": "runs/s", "n_gpus": 1,
            "steps": int(sum(q.steps for q in reqs)), "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serve-poisson-{args.requests}req-20per_s", "tick": args.tick,
                       "hbm_budget_gb": args.hbm_gb},
            "latency": {"p50_s": summ["p50_s"], "p99_s": summ["p99_s"], "mean_s": summ["mean_s"]},
            "served_glups": summ.get("glups"), "makespan_s": summ["makespan_s"],
            "prefix_compare": {"requests": len(prefix), "batched_fp32": pref, "plain_fp64_one_at_a_time": base},
            "roofline": None, "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


def run_fp64(args):
    """Plain FP64 single run (128x104, T = 200, 10,000 steps) on the GPU and
    the FP64 oracle on the host, same steps."""
    import torch

    import paper_1812_05711_gb300 as ehd

    torch.cuda.set_device(0)
    w = wl.plain_fp64_channel()
    K = args.steps
    run = ehd.Run(*w.args(), storage="f64", amp=w.amp, phase=w.phase)
    run.step(args.warmup)
    run.sync()
    stream = torch.cuda.ExternalStream(ehd.ehd_stream(run.handle))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run.step(K)
    e1.record(stream)
    run.sync()
    ms = e0.elapsed_time(e1)
    value = _cells(w) * K / (ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        cpu = _cpu_baseline(w, args.cpu_seconds, "the 128x104 channel")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "Nx": w.Nx, "Ny": w.Ny, "storage": "f64", "compute": "f64"},
            "roofline": None, "e2e": None, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def run_ysolve(args):
    """The two y solves of the Poisson equation side by side: the
    per-wavenumber tridiagonal and the literal odd-extension transform of
    Eqs. 21-25, on the 2048x1680 FP32 channel (NE = 3360) and the 1024x840
    plain FP64 channel (NE = 1680).  Whole graph-launched steps (CUDA events
    on the run's stream) and, from ehd_step_profile, the Poisson solve and its
    m >= 1 part.  The line's value is the odd-extension FP32 channel."""
    import torch

    import paper_1812_05711_gb300 as ehd

    torch.cuda.set_device(0)
    out = {}
    value = ms_value = None
    for w, st, K in ((wl.large_channel(), "f32", args.steps), (wl.precision_channel(), "f64", max(args.steps // 10, 20))):
        run = ehd.Run(*w.args(), storage=st, amp=w.amp, phase=w.phase)
        stream = torch.cuda.ExternalStream(ehd.ehd_stream(run.handle))
        res = {}
        for ys, name in ((0, "tridiagonal"), (1, "odd_extension")):
            ehd.ehd_tune(run.handle, "y_solver", ys)
            run.step(args.warmup)
            run.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run.step(K)
            e1.record(stream)
            run.sync()
            ms = e0.elapsed_time(e1) / K
            prof = ehd.ehd_step_profile(run.handle, min(K, 200))
            n = prof["steps"]
            res[name] = {"glups": _cells(w) / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                         "poisson_us": 1e3 * prof["poisson_ms"] / n, "y_solve_us": 1e3 * prof["modes_ms"] / n,
                         "fft_x_us": 1e3 * (prof["fft_fwd_ms"] + prof["fft_inv_ms"]) / n}
            if st == "f32" and ys == 1:
                value, ms_value = res[name]["glups"], ms
        run.close()
        out[f"{w.name}-{st}"] = res
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "channel-2048x1680-oddext", "Nx": 2048, "Ny": 1680, "storage": "f32",
                       "compute": "f32", "y_solver": "odd_extension"},
            "y_solvers": out, "roofline": None, "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


def run_variants(args):
    """The step variants on the 2048x1680 FP32 channel, graph-launched steps
    timed with CUDA events on the run's stream: the default (Lambda = 1/4,
    spectral x symbol, central-difference E_x), Lambda = 1/12 and 3/16, the
    SRT limit Lambda = (tau+ - 1/2)^2, the 3-point x symbol, and spectral
    E_x.  The line's value is the spectral-E_x run."""
    import torch

    import paper_1812_05711_gb300 as ehd

    torch.cuda.set_device(0)
    w = wl.large_channel()
    cases = [("default", {}, 0.25), ("lambda_1_12", {}, 1.0 / 12.0), ("lambda_3_16", {}, 3.0 / 16.0),
             ("srt", {}, None), ("x_symbol_3pt", {"x_symbol": 1}, 0.25), ("ex_spectral", {"ex_spectral": 1}, 0.25)]
    out = {}
    K = args.steps
    tau_p = None
    for name, kw, lam in cases:
        if lam is None:  # SRT limit: tau- = tau+ (tau+ does not depend on Lambda)
            lam = (tau_p - 0.5) ** 2
        run = ehd.Run(w.Nx, w.Ny, w.T, w.C, w.M, w.Fe, lam, storage="f32", amp=w.amp, phase=w.phase, **kw)
        if tau_p is None:
            tau_p = run.params()["tau_p"]
        stream = torch.cuda.ExternalStream(ehd.ehd_stream(run.handle))
        run.step(args.warmup)
        run.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run.step(K)
        e1.record(stream)
        run.sync()
        ms = e0.elapsed_time(e1) / K
        prof = ehd.ehd_step_profile(run.handle, min(K, 200))
        n = prof["steps"]
        out[name] = {"glups": _cells(w) / (ms * 1e-3) / 1e9, "ms_per_step": ms, "Lambda": lam,
                     "profile_us": {"collide_stream": 1e3 * prof["collide_stream_ms"] / n,
                                    "poisson": 1e3 * prof["poisson_ms"] / n,
                                    "fft_inv": 1e3 * prof["fft_inv_ms"] / n, "step": 1e3 * prof["step_ms"] / n}}
        run.close()
    line = {"metric": METRIC, "value": out["ex_spectral"]["glups"], "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": out["ex_spectral"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "channel-2048x1680-ex-spectral", "Nx": w.Nx, "Ny": w.Ny, "storage": "f32",
                       "compute": "f32", "ex_spectral": 1},
            "variants": out, "roofline": None, "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args):
    """1024x840, T = 170: every storage (FP64 / FP32 / BF16 / FP16, FP32
    compute) against the plain FP64 GPU path after K steps; GLUPS of each.
    (Their agreement with the FP64 oracle is a parity test,
    tests/test_gpu_parity.py::test_storage_variants_vs_oracle_1024x840.)"""
    import torch

    import paper_1812_05711_gb300 as ehd

    torch.cuda.set_device(0)
    w = wl.precision_channel()
    K = args.steps
    ref = ehd.Run(*w.args(), storage="f64", amp=w.amp, phase=w.phase)
    par = ref.params()
    u_ion = 2e-3  # the runs' default lattice ion drift speed
    scale = {"rho": 1.0, "ux": u_ion, "uy": u_ion, "rho_c": par["rho0"], "phi": 1.0, "Ex": 1.0 / w.Ny,
             "Ey": 1.0 / w.Ny}

    def err(a, b):
        return {k: float(np.abs(a[k] - b[k]).max() / scale[k]) for k in a}

    ref.step(K)
    ref_long = ref.fields()
    ref.close()
    rows = {}
    for st in ("f64", "f32", "bf16", "f16"):
        r = ehd.Run(*w.args(), storage=st, compute="f32", amp=w.amp, phase=w.phase)
        r.step(args.warmup)
        stream = torch.cuda.ExternalStream(ehd.ehd_stream(r.handle))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.step(K - args.warmup)
        e1.record(stream)
        r.sync()
        ms = e0.elapsed_time(e1)
        rows[st] = {"glups": _cells(w) * (K - args.warmup) / (ms * 1e-3) / 1e9,
                    f"scaled_err_vs_gpu_fp64_at_{K}": err(r.fields(), ref_long)}
        r.close()
    line = {"metric": METRIC, "value": rows["f32"]["glups"], "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "Nx": w.Nx, "Ny": w.Ny, "compute": "f32"},
            "precision": rows, "roofline": None, "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


def _table2():
    rows = {}
    with open(os.path.join(ROOT, "tests", "golden", "table2_hydrostatic.txt")) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                C, ra, ya, eE, erc = map(float, ln.split())
                rows[C] = {"rho_a": ra, "y_a": ya, "eL2_Ey": eE, "eL2_rhoc": erc}
    return rows


def run_hydrostatic(args):
    """Sec. V.1: the no-flow steady state at NY = 100, Fe = 4000 against Eqs.
    27-28 for a sweep of the injection strength C (Table II prints C = 0.1
    and 10); plain FP64 path."""
    import time as _t

    import torch

    from paper_1812_05711_gb300 import studies

    torch.cuda.set_device(0)
    tab = _table2()
    rows = []
    t0 = _t.perf_counter()
    for C in (0.1, 0.3, 1.0, 3.0, 10.0):
        r = studies.hydrostatic(C)
        rows.append({"C": C, "eL2_Ey": r["eL2_Ey"], "eL2_rhoc": r["eL2_rhoc"], "rho_a": r["rho_a"],
                     "y_a": r["y_a"], "paper": tab.get(C)})
    el = _t.perf_counter() - t0
    line = {"metric": "hydrostatic e_L2 vs Eqs. 27-28", "value": rows[0]["eL2_Ey"], "unit": "relative L2",
            "n_gpus": 1, "steps": 30000, "warmup": 0, "ms_per_step": None, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "hydrostatic-16x100-Fe4000", "u_ion": 0.01, "seconds": el},
            "table": rows, "roofline": None, "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


def run_bifurcation(args):
    """Sec. V.2 (FIG. 3): electric Nusselt number Ne(T) on the branch that
    starts from a small roll and on the branch continued downwards from a
    finite-amplitude state; T_c and T_f by linear interpolation."""
    import time as _t

    import torch

    from paper_1812_05711_gb300 import studies

    torch.cuda.set_device(0)
    Ts = [100.0 + 5.0 * k for k in range(17)] + [190.0, 200.0, 220.0]
    Nx = args.grid
    Ny = wl.ny_for(Nx)
    steps = 200000 * Nx // 64  # the same number of ion transits on every grid
    t0 = _t.perf_counter()
    # every sweep point is a request to the continuous-batching server: the
    # reference and the lower branch advance together, the upper branch is a
    # chain of continuations admitted beside them
    r = studies.nusselt_sweep_served(Ts, Nx=Nx, Ny=Ny, u_ion=5e-3, steps=steps, window=steps // 5)
    el = _t.perf_counter() - t0

    def crossing(branch, level, rising):
        pts = sorted(branch)
        for (t0_, n0), (t1_, n1) in zip(pts, pts[1:]):
            if (n0 - level) * (n1 - level) <= 0 and n0 != n1:
                return t0_ + (t1_ - t0_) * (level - n0) / (n1 - n0)
        return None

    Tc = crossing(r["lower"], 1.01, True)
    Tf = crossing(r["upper"], 1.01, False)
    lat = [q.latency for q in r["results"].values()]
    line = {"metric": "Ne(T) thresholds", "value": Tc, "unit": "T", "n_gpus": 1, "steps": steps, "warmup": 0,
            "ms_per_step": None, "higher_is_better": None, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"bifurcation-{Nx}x{Ny}", "u_ion": 5e-3, "steps_per_T": steps, "seconds": el,
                       "path": "served (continuous batching; upper branch by continuation requests)",
                       "requests": len(r["results"]), "max_latency_s": max(lat)},
            "T_c_onset": Tc, "T_f": Tf, "paper": {"T_c": 163.4, "T_f": 108.7},
            "lower": r["lower"], "upper": r["upper"], "I_h": r["I_h"],
            "roofline": None, "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f64", "bf16", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--perturbation", action="store_true",
                    help="channel: the FP32 perturbation form (charge populations as departures from an FP64 "
                         "x-uniform base state)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="channel",
                    choices=["channel", "batch", "serve", "fp64", "precision", "hydrostatic", "bifurcation",
                             "ysolve", "variants"],
                    help="channel: 2048x1680 headline (default); batch: 64 uneven runs; serve: request stream; "
                         "fp64: 128x104 plain FP64; precision: 1024x840 storage variants; "
                         "hydrostatic: Table II e_L2 for a C sweep; bifurcation: Ne(T) both branches; "
                         "ysolve: tridiagonal vs odd-extension y solve of the Poisson equation; "
                         "variants: Lambda, SRT, x symbol and spectral E_x on the headline channel")
    ap.add_argument("--tick", type=int, default=100, help="steps per batch tick (batch / serve)")
    ap.add_argument("--requests", type=int, default=600, help="requests in the serving stream")
    ap.add_argument("--fp64-requests", type=int, default=32, help="prefix served by the plain FP64 path")
    ap.add_argument("--hbm-gb", type=float, default=200.0, help="HBM budget of the server")
    ap.add_argument("--grid", type=int, default=64, help="bifurcation: Nx of the channel (Ny = 0.82 Nx)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "channel" and int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit(f"--workload {args.workload} runs on one GPU; use the channel workload under torchrun")
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "fp64":
        return run_fp64(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "hydrostatic":
        return run_hydrostatic(args)
    if args.workload == "bifurcation":
        return run_bifurcation(args)
    if args.workload == "ysolve":
        return run_ysolve(args)
    if args.workload == "variants":
        return run_variants(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
