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
# algorithmic bytes per node of the fused collide-stream kernel (FP32
# storage): 9 f + 9 g loaded, 9 f + 9 g stored, one potential value loaded
# kernels per coupled step: collide-stream (march form, writes the charge),
# forward row FFT, FP64 mean mode, wavenumber systems, inverse row FFT
LAUNCHES_PER_STEP = 5
K4_BYTES_PER_NODE = {"f32": 36 * 4 + 4, "f64": 36 * 8 + 8, "bf16": 36 * 2 + 4, "f16": 36 * 2 + 4}


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


def _max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed on the host cores."""
    dist, rank, ws, _ = _dist()
    if rank != 0:
        return 0
    import oracle as o
    full = wl.large_channel()
    # each benchmark step: one oracle step of a 256 x 208 channel with the same
    # groups and perturbation recipe (1/66 of the 2048 x 1680 nodes)
    w = wl.Workload("channel-256x208-sample", 256, 208, full.T, amp=full.amp, phase=full.phase)
    p = o.setup(*w.args())
    s = o.init_state(p, w.amp, w.phase)
    o.step(s, args.warmup)
    t0 = time.perf_counter()
    o.step(s, args.steps)
    el = time.perf_counter() - t0
    val = w.Nx * w.Ny * args.steps / el / 1e9
    sample = (f"oracle steps of a 256x208 channel (same T, C, M, Fe, Lambda and Eq. 29 modes as the "
              f"2048x1680 workload); {args.steps} steps in {el:.2f} s")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "channel-2048x1680 (sampled as 256x208)", "Nx": w.Nx, "Ny": w.Ny,
                       "T": w.T, "C": w.C, "M": w.M, "Fe": w.Fe, "Lambda": w.Lambda},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
    run = ehd.Run(*w.args(), storage=storage, amp=w.amp, phase=w.phase)
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
    value = ws * cells * args.steps / (ms_max * 1e-3) / 1e9
    run.sync()

    # ---- per-kernel timing (events around each kernel on the run's stream)
    prof = ehd.ehd_step_profile(h, args.steps)
    k4_ms = prof["collide_stream_ms"] / args.steps
    bytes_k4 = K4_BYTES_PER_NODE[storage] * cells
    peak, peak_kind = _peaks()
    achieved = bytes_k4 / (k4_ms * 1e-3) / 1e9

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
    e2e = ws * cells * args.steps / e2e_s / 1e9
    h2d = (pin_f.nbytes + pin_g.nbytes) / args.steps
    d2h = out.nbytes / args.steps
    diag = run.diagnostics()
    clocks = clk.stop() if clk else None

    if rank != 0:
        run.close()
        return 0

    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        v, n, el = _oracle_glups(w, budget_s=args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} oracle steps of the full 2048x1680 channel in {el:.1f} s (one thread)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if storage != "f64" else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "Nx": w.Nx, "Ny": w.Ny, "T": round(w.T, 6), "C": w.C, "M": w.M,
                   "Fe": w.Fe, "Lambda": w.Lambda, "storage": storage, "compute": "f32" if storage != "f64" else "f64",
                   "per_rank": "one independent run", "l2": "state 495 MB > 129 MB L2, no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_march (fused collide-stream)",
                     "bytes_per_node": K4_BYTES_PER_NODE[storage], "kernel_ms": k4_ms,
                     "peak_kind": f"{peak_kind} hbm_gbs", "poisson_ms": prof["poisson_ms"] / args.steps,
                     "charge_ms": prof["charge_ms"] / args.steps,
                     "profiled_step_ms": prof["step_ms"] / args.steps},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "check": {"mass": diag["mass"], "charge": diag["charge"], "max_u": diag["max_u"]},
    }
    print(json.dumps(line), flush=True)
    run.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f64", "bf16", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
