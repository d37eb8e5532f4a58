"""Autotuner of the batched persistent step.

Times a short batched run for each candidate configuration -- persistent
blocks per SM (how many work items run side by side) and particles per
readout work item (the chunking of the fused readout-kick-drift phase) --
on scratch copies of the particle state, keeps the fastest, and caches the
choice in a JSON file keyed by GPU name and the batch's size mix.
"""
from __future__ import annotations

import itertools
import json
import os
import time
from typing import Dict, List, Optional

CACHE = os.environ.get("FPM_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "fpm_gb300", "batch_autotune.json"))
CANDIDATES = {"blocks_per_sm": [1, 2, 3], "readout_chunks": [1, 2, 4]}


def _key(batch, nsteps: int) -> str:
    import torch
    sizes: Dict[int, int] = {}
    for p in batch.plans:
        sizes[p.nc] = sizes.get(p.nc, 0) + 1
    mix = "+".join(f"{n}x{c}" for c, n in sorted(sizes.items()))
    return f"{torch.cuda.get_device_name()}|{mix}|steps{nsteps}"


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(batch, dxs: List, ps: List, a, reps: int = 2, use_cache: bool = True) -> dict:
    """Pick (blocks_per_sm, readout_chunks) for `batch` by timing runs on
    copies of (dxs, ps); configure the batch with the winner and return
    {"config": ..., "timings_ms": ..., "cached": bool}."""
    import torch
    key = _key(batch, len(a) - 1)
    cache = _load() if use_cache else {}
    if key in cache:
        cfg = cache[key]["config"]
        batch.configure(cfg["blocks_per_sm"], cfg["readout_chunks"])
        return {"config": cfg, "timings_ms": cache[key].get("timings_ms", {}), "cached": True}
    dx_s = [x.clone() for x in dxs]
    p_s = [x.clone() for x in ps]
    timings = {}
    best: Optional[tuple] = None
    for bps, roc in itertools.product(CANDIDATES["blocks_per_sm"], CANDIDATES["readout_chunks"]):
        batch.configure(bps, roc)
        for x, y, x0, y0 in zip(dx_s, p_s, dxs, ps):
            x.copy_(x0)
            y.copy_(y0)
        batch.kdk(dx_s, p_s, a)                    # capture + warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            batch.kdk(dx_s, p_s, a)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        timings[f"bps{bps}_roc{roc}"] = ms
        if best is None or ms < best[0]:
            best = (ms, bps, roc)
    cfg = {"blocks_per_sm": best[1], "readout_chunks": best[2]}
    batch.configure(cfg["blocks_per_sm"], cfg["readout_chunks"])
    if use_cache:
        cache[key] = {"config": cfg, "timings_ms": timings, "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
        try:
            os.makedirs(os.path.dirname(CACHE), exist_ok=True)
            with open(CACHE, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return {"config": cfg, "timings_ms": timings, "cached": False}
