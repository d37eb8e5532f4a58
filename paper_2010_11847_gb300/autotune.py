"""Autotuner of the batched persistent step.

Times short batched runs on scratch copies of the particle state and keeps
the fastest configuration of

  * the launch: persistent blocks per SM (how many work items run side by
    side) and particles per work item of the chunked readout;
  * per mesh size: the fused readout's traversal (chunks of consecutive
    particles, or Lagrangian bricks of 4 x 32 x 32 / 4 x 16 x 64 particles),
    the paint tile shape (8^3 or 16^3 cells: the particles are bucketed and
    painted by tiles of that edge) and the FFT plan of the power-of-two
    passes (8 or 16 points per thread, i.e. twice the lines per block).

The search is coordinate descent from the library's defaults: the launch
knobs jointly, then each per-size knob in turn with the others held, until
a sweep changes nothing.  No knob changes a result bit, so the choice is a
matter of time alone.  The winner is cached in a JSON file keyed by GPU
name, the batch's size mix and the number of steps.
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
SIZE_KNOBS = {"readout": [0, 1, 2], "paint_tile": [16, 8], "fft_slots": [8, 16]}
MAX_SWEEPS = 2


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


def _default_size_config(batch) -> Dict[str, Dict[str, int]]:
    """The library's defaults per mesh size (bricks where the lattice allows)."""
    out = {}
    for p in batch.plans:
        if str(p.nc) in out:
            continue
        f4 = p.nc in (16, 32, 64, 128, 256, 512)
        rd = 2 if (f4 and p.np % 64 == 0) else (1 if (f4 and p.np % 32 == 0) else 0)
        out[str(p.nc)] = {"readout": rd, "paint_tile": 16, "fft_slots": 8}
    return out


def apply(batch, cfg: dict):
    """Configure `batch` with a configuration returned by ``tune``."""
    batch.configure(cfg["blocks_per_sm"], cfg["readout_chunks"])
    for nc, knobs in cfg.get("sizes", {}).items():
        for knob, value in knobs.items():
            batch.tune(int(nc), knob, value)


def _valid(batch, nc: int, knob: str, value: int) -> bool:
    from .binding import FpmError
    try:
        batch.tune(nc, knob, value)
        return True
    except FpmError:
        return False


def tune(batch, dxs: List, ps: List, a, reps: int = 2, use_cache: bool = True) -> dict:
    """Pick the launch knobs and, per mesh size, the readout traversal, the
    paint tile shape and the FFT plan of `batch` by timing runs on copies of
    (dxs, ps); configure the batch with the winner and return {"config": ...,
    "timings_ms": ..., "cached": bool}."""
    import torch
    key = _key(batch, len(a) - 1)
    cache = _load() if use_cache else {}
    if key in cache:
        cfg = cache[key]["config"]
        apply(batch, cfg)
        return {"config": cfg, "timings_ms": cache[key].get("timings_ms", {}), "cached": True}
    dx_s = [x.clone() for x in dxs]
    p_s = [x.clone() for x in ps]
    timings: Dict[str, float] = {}

    def measure(label: str) -> float:
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
        timings[label] = ms
        return ms

    sizes = _default_size_config(batch)
    for nc, knobs in sizes.items():
        for knob in list(knobs):
            if _valid(batch, int(nc), knob, knobs[knob]):
                continue
            if knob == "readout" and _valid(batch, int(nc), knob, 0):
                knobs[knob] = 0
            else:
                del knobs[knob]                  # not a knob of this mesh (e.g. FFT slots of 96^3)
    # launch knobs jointly
    best: Optional[tuple] = None
    for bps, roc in itertools.product(CANDIDATES["blocks_per_sm"], CANDIDATES["readout_chunks"]):
        batch.configure(bps, roc)
        ms = measure(f"bps{bps}_roc{roc}")
        if best is None or ms < best[0]:
            best = (ms, bps, roc)
    best_ms, bps, roc = best
    batch.configure(bps, roc)
    # per-size knobs, coordinate descent
    for _ in range(MAX_SWEEPS):
        changed = False
        for nc in sorted(sizes, key=int):
            for knob, values in SIZE_KNOBS.items():
                if knob not in sizes[nc]:
                    continue
                current = sizes[nc][knob]
                for v in values:
                    if v == current or not _valid(batch, int(nc), knob, v):
                        continue
                    ms = measure(f"nc{nc}_{knob}{v}")
                    if ms < best_ms:
                        best_ms, current, changed = ms, v, True
                batch.tune(int(nc), knob, current)
                sizes[nc][knob] = current
        if not changed:
            break
    cfg = {"blocks_per_sm": bps, "readout_chunks": roc, "sizes": sizes, "ms": best_ms}
    apply(batch, cfg)
    if use_cache:
        cache[key] = {"config": cfg, "timings_ms": timings, "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
        try:
            os.makedirs(os.path.dirname(CACHE), exist_ok=True)
            with open(CACHE, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return {"config": cfg, "timings_ms": timings, "cached": False}
