"""Autotuner of the batch launch shapes.

For a batch whose members are fixed, time a small grid of candidate launch
shapes -- rows per march warp item and the CTA counts of the persistent
march, row-FFT and wavenumber kernels -- with CUDA events on the batch
stream, keep the fastest, and cache the choice in a JSON file keyed by the
multiset of member grid sizes and the GPU's SM count.  The candidates only
change how work is cut, never the results (members stay bitwise equal to
their solo runs).
"""
from __future__ import annotations

import json
import os
import time

from . import ehd_batch_stream, ehd_batch_tune, ehd_batch_tune_get

# the launch shapes the tuner times (the batch's other settings stay as they are)
SHAPES = ("slab_rows", "march_ctas", "row_ctas", "tile_ctas")
CACHE = os.environ.get("EHD_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ehd_gb300_tune.json"))


def _key(batch, sms: int) -> str:
    sizes = sorted((r.Nx, r.Ny) for r in batch.members.values())
    return f"sms{sms}:" + ",".join(f"{nx}x{ny}" for nx, ny in sizes)


def _load():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(db):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(db, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def time_ticks(batch, ticks: int, steps: int) -> float:
    """Milliseconds per step of `ticks` ticks, CUDA events on the batch stream."""
    import torch
    stream = torch.cuda.ExternalStream(ehd_batch_stream(batch.handle))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batch.tick(steps)  # captures the graph for this shape
    batch.sync()
    e0.record(stream)
    for _ in range(ticks):
        batch.tick(steps)
    e1.record(stream)
    batch.sync()
    return e0.elapsed_time(e1) / (ticks * steps)


def tune(batch, steps: int = 8, ticks: int = 4, use_cache: bool = True, verbose: bool = False) -> dict:
    """Pick launch shapes for the current membership.  The members' step
    budgets are consumed by the timing ticks; tune a batch whose members have
    budget to spare (or add them afterwards with fresh budgets)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    key = _key(batch, sms)
    db = _load() if use_cache else {}
    if use_cache and key in db:
        for k, v in db[key]["params"].items():
            ehd_batch_tune(batch.handle, k, v)
        return db[key]
    base = {k: ehd_batch_tune_get(batch.handle, k) for k in SHAPES}
    auto_rows = base["slab_rows"]
    cands = []
    for rows in sorted({max(4, auto_rows // 2), auto_rows, auto_rows * 2, 8, 12, 16, 24, 0}):
        for mf in (0.5, 1.0, 2.0):
            for rf in (0.5, 1.0, 1.25):
                cands.append({"slab_rows": rows, "march_ctas": max(1, int(base["march_ctas"] * mf)),
                              "row_ctas": max(1, int(base["row_ctas"] * rf)), "tile_ctas": base["tile_ctas"]})
    # wavenumber-tile CTAs: the default (as many per SM as fit, up to four) and half of it
    cands += [dict(c, tile_ctas=max(1, base["tile_ctas"] // 2)) for c in cands if c["march_ctas"] == base["march_ctas"]
              and c["row_ctas"] == base["row_ctas"]]
    best, best_ms, t0 = None, float("inf"), time.perf_counter()
    for c in cands:
        for k, v in c.items():
            ehd_batch_tune(batch.handle, k, v)
        ms = time_ticks(batch, ticks, steps)
        if verbose:
            print(f"  {c} -> {ms * 1e3:.1f} us/step")
        if ms < best_ms:
            best, best_ms = c, ms
    for k, v in best.items():
        ehd_batch_tune(batch.handle, k, v)
    rec = {"params": best, "us_per_step": best_ms * 1e3, "candidates": len(cands),
           "seconds": time.perf_counter() - t0}
    if use_cache:
        db[key] = rec
        _store(db)
    return rec
