#!/usr/bin/env python
"""Throughput of the GB300-native FastPM particle-mesh loop.

One bench step is one whole simulation of the workload: FP64 coefficients,
the linear field and 2LPT initial conditions at a = 0.1, every KDK step to
a = 1 (readout + kick + drift, sort, paint, r2c FFT, force transfer, three
c2r FFTs) and the final paint and power spectrum.  The metric is
particle-steps/s = particles x KDK steps / time; ms per PM step is the step
time divided by the number of KDK steps (initial conditions included).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fpm|reference]

N > 1 (under torchrun) runs independent replicas, one simulation per rank
with its own seed: weak scaling, no data-path collective.
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
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s and ms/PM-step at 512³ (fwd, fwd+adjoint), % of HBM roofline"
ROOFLINE_CLASS = "kdk_readout_kick_drift"     # the kernel class the roofline line reports
UNIT = "particle-steps/s"

# Algorithmic (compulsory) device bytes per launch of each kernel class, as
# (bytes per particle, bytes per mesh cell): each input read once and each
# output written once.  Half spectra count (nc/2+1)/nc * 8 B per cell.
def _alg_bytes(cls, N, M, nc):
    h = 8.0 * (nc // 2 + 1) / nc            # bytes per cell of a half spectrum
    table = {
        "kdk_readout_kick_drift": 24 + 24 + 12 * M / N,       # dx,p r/w, F read (keys: build overhead)
        "cell_keys": 12 + 4,
        "tile_scan": 0.0,
        "tile_scatter": 4 + 4,                         # key read, item write
        "paint_tiles": 4 + 12 + 4 * M / N,            # item, dx gather, rho write
        "paint_halo": 4 * M / N * 0.176,
        "fft_z_r2c": (4 + h) * M / N,
        "fft_y_fwd": 2 * h * M / N,
        "fft_x_green": (h + 3 * h) * M / N,
        "fft_y_inv": 6 * h * M / N,
        "fft_z_c2r": (3 * h + 12) * M / N,
        "pot_fft_fwd_zy": (4 + h) * M / N,           # rho read, half spectrum written once
        "pot_fft_x_green": 2 * h * M / N,
        "pot_fft_inv_yz": (h + 4) * M / N,           # half spectrum read, phi written once
        "pot_gradient": (4 + 16) * M / N,            # phi read, float4 force mesh written
    }
    v = table.get(cls)
    return None if v is None else v * N


# The same, counting what the implementation's structure adds on top of the
# method's bytes (not the roofline's numerator): the readout also writes the
# next cell keys (4 B/particle) and reads the force mesh as float4 (16 B/cell).
def _build_bytes(cls, N, M, nc):
    if cls == "kdk_readout_kick_drift":
        return (24 + 24 + 4 + 16 * M / N) * N
    return _alg_bytes(cls, N, M, nc)


def step_algorithmic_bytes(N, M):
    """Method minimum per PM step (60 B per particle + 44 B per cell)."""
    return 60.0 * N + 44.0 * M


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["fpm", "reference"], default="fpm")
    ap.add_argument("--workload", choices=["large", "eighth", "medium", "small"], default="large")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-simulation batched measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the forward+adjoint measurements")
    ap.add_argument("--profile-json", default=None, help="write the per-class timing here")
    return ap.parse_args()


def workload(name):
    from paper_2010_11847_gb300 import inputs
    return {"large": inputs.LARGE, "eighth": inputs.LARGE_EIGHTH, "medium": inputs.MEDIUM,
            "small": inputs.SMALL}[name]


def dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- replicas (N > 1)
# Every rank runs its own simulation (its own seed): no data-path collective;
# the only exchange is the max of the per-rank times.
def rank_seed(seed, rank):
    return seed + rank


def max_over_ranks(x, world, device="cpu"):
    """Largest value of x over all ranks (x itself when world == 1)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, particles, pm_steps, seconds):
    """Whole-job particle-steps/s: every rank advanced `particles` for
    `pm_steps` steps; the job took the slowest rank's time."""
    return world * particles * pm_steps / seconds


def shard(items, rank, world):
    """Items (e.g. the simulations of a batch) assigned to one rank."""
    return items[rank::world]


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, enabled=True):
        self.gpu, self.proc, self.path = gpu_index, None, None
        self.enabled = enabled

    def start(self):
        if not self.enabled:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        self.proc.wait(timeout=10)
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        mx = max(num(r[2]) for r in rows)
        load = [s for s, r in zip(sm, rows) if num(r[3]) > 200.0] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- CPU oracle sample
def oracle_sample(steps=4, full_runs=True):
    """The FP64 oracle's KDK steps (paint, force, readout, kick, drift) on a
    128^3-particle, 128^3-mesh sub-box of the 512^3 workload (same cell size
    1000/512 Mpc/h and particle density): one continuous call over `steps`
    steps (steps + 1 force evaluations), about 10 s of CPU work."""
    import numpy as np
    from oracle import fpm_oracle as O
    from paper_2010_11847_gb300 import inputs
    n = 128
    box = 1000.0 * n / 512
    wl = inputs.LARGE
    lk = O.linear_field(inputs.white_noise(n, 7), box, wl.cosmo)
    dx, p = O.lpt(lk, n, wl.a0, wl.cosmo)
    stages = wl.stages()
    t = time.perf_counter()
    O.kdk(dx, p, stages[:steps + 1], n, n, wl.cosmo["omega_m"])
    ms = 1e3 * (time.perf_counter() - t) / steps
    threads = int(os.environ.get("OMP_NUM_THREADS", "0")) or os.cpu_count()
    out = {"value": n ** 3 / (ms / 1e3), "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{steps} KDK steps ({steps + 1} force evaluations) of the FP64 numpy/scipy oracle in one "
                     f"call on a 128^3-particle 128^3-mesh sub-box (250 Mpc/h, same cell size and density as "
                     f"512^3/1000 Mpc/h): {ms:.0f} ms per step; scipy.fft may use all host cores",
           "ms_per_pm_step": ms}
    if not full_runs:
        return out
    # the same sample, two steps, with one FFT thread (paint and readout are single-threaded anyway)
    O.FFT_WORKERS = 1
    t = time.perf_counter()
    O.kdk(dx, p, stages[:3], n, n, wl.cosmo["omega_m"])
    out["ms_per_pm_step_one_thread"] = 1e3 * (time.perf_counter() - t) / 2
    O.FFT_WORKERS = -1
    # whole simulations (linear field, 2LPT, all KDK steps, final paint) of the small configurations
    runs = {}
    for w in (inputs.SMALL, inputs.DIFFERENTIABLE):
        t = time.perf_counter()
        O.simulate(inputs.white_noise(w.np_, w.seed), w.nc, w.box, w.cosmo, w.stages())
        runs[w.name] = {"ms_per_simulation": 1e3 * (time.perf_counter() - t), "kdk_steps": w.nsteps}
    out["full_runs"] = runs
    return out


def run_reference(args):
    rank, world, _ = dist()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import fpm_oracle as O
    from paper_2010_11847_gb300 import inputs
    n = 128
    box = 1000.0 * n / 512
    wl = inputs.LARGE
    lk = O.linear_field(inputs.white_noise(n, 7), box, wl.cosmo)
    dx, p = O.lpt(lk, n, wl.a0, wl.cosmo)
    stages = wl.stages()
    om = wl.cosmo["omega_m"]
    # continuous KDK calls (a call of m steps evaluates m + 1 forces), at most
    # the workload's 40 steps per call
    w0 = min(args.warmup, wl.nsteps)
    if w0:
        dx, p = O.kdk(dx, p, stages[:w0 + 1], n, n, om)
    t0 = time.perf_counter()
    done, j = 0, w0
    while done < args.steps:
        if j >= wl.nsteps:
            j = 0
        m = min(args.steps - done, wl.nsteps - j)
        dx, p = O.kdk(dx, p, stages[j:j + m + 1], n, n, om)
        done += m
        j += m
    dt = time.perf_counter() - t0
    ms = 1e3 * dt / args.steps
    value = n ** 3 * args.steps / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "sample": "one oracle KDK step per bench step on a 128^3/128^3 "
                       "sub-box at the 512^3 workload's resolution, the timed steps in continuous calls",
                       "np": n, "nc": n, "box_mpc_h": box},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "FP64 numpy/scipy oracle, 128^3 sub-box, one KDK step per bench step "
                                       "(continuous calls: a call of m steps evaluates m + 1 forces)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def kernel_source_hash(files):
    """Hash of the code (comments and whitespace runs removed) of the CUDA
    sources a kernel class is built from."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2010_11847_gb300", "csrc")
    for f in sorted(files):
        text = open(os.path.join(csrc, f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(re.sub(r"\s+", " ", text).strip().encode())
    return h.hexdigest()[:16]


def ncu_traffic(cls):
    """DRAM bytes per full-size launch of kernel class `cls` from the committed
    ncu summary, when it was taken on the current sources of that kernel."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        e = json.load(open(path)).get("kernels", {}).get(cls)
    except ValueError:
        return None
    if not e or e.get("source_hash") != kernel_source_hash(e.get("files", [])):
        return None
    return e.get("dram_bytes_per_launch_full_size")


def measure_batched(reps=3, peak=None):
    """64 simulations (meshes 32/64/96/128, 16 each, own cosmologies, 10 KDK
    steps) by the persistent batched step, autotuned, against the same 64 runs
    launched one by one.  Each run starts from its own 2LPT initial state."""
    import torch
    from paper_2010_11847_gb300 import inputs, autotune
    from paper_2010_11847_gb300.binding import Plan, Batch
    wls = inputs.batched_workloads()
    plans, d0, p0 = [], [], []
    for wl in wls:
        pl = Plan(wl.np_, wl.nc, wl.box, wl.cosmo)
        lk = pl.linear_field(torch.from_numpy(inputs.white_noise(wl.np_, wl.seed)).cuda())
        dx, p = pl.lpt(lk, wl.a0, 2)
        plans.append(pl)
        d0.append(dx)
        p0.append(p)
    a = wls[0].stages()
    dxs = [x.clone() for x in d0]
    ps = [x.clone() for x in p0]
    b = Batch(plans)
    tuned = autotune.tune(b, dxs, ps, a)

    def reset():
        for x, y, x0, y0 in zip(dxs, ps, d0, p0):
            x.copy_(x0)
            y.copy_(y0)

    def timed(fn):
        ts = []
        for _ in range(reps):
            reset()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    b.phase_times()                              # reset the per-phase clocks
    t_batch = timed(lambda: b.kdk(dxs, ps, a))
    assert b.status() == 0
    nsteps = wls[0].nsteps
    phases = {k: v / (reps * nsteps) for k, v in b.phase_times().items() if v > 0}
    t_one = timed(lambda: [pl.kdk(x, y, a) for pl, x, y in zip(plans, dxs, ps)])
    nps = sum(wl.np_ ** 3 for wl in wls) * wls[0].nsteps
    info = b.info()
    alg = sum(step_algorithmic_bytes(wl.np_ ** 3, wl.nc ** 3) for wl in wls) * wls[0].nsteps
    roof = None
    if peak:
        roof = {"bound": "hbm", "alg_bytes": alg, "peak": peak, "unit": "GB/s",
                "achieved_batched": alg / (t_batch / 1e3) / 1e9, "frac_batched": alg / (t_batch / 1e3) / 1e9 / peak,
                "achieved_one_by_one": alg / (t_one / 1e3) / 1e9, "frac_one_by_one": alg / (t_one / 1e3) / 1e9 / peak,
                "bytes_model": "per simulation and PM step 60 B/particle + 44 B/cell"}
    return {"roofline": roof, "workload": "batch64_mixed_32_64_96_128_10step", "sims": len(wls), "kdk_steps": wls[0].nsteps,
            "ms_per_batched_run": t_batch, "ms_per_one_by_one_run": t_one, "speedup": t_one / t_batch,
            "particle_steps_per_s_batched": nps / (t_batch / 1e3),
            "launches_per_step": 1, "graph_captured": info["graph_captured"], "grid_blocks": info["grid_blocks"],
            "autotune": tuned["config"], "autotune_cached": tuned["cached"],
            "ms_per_step_by_phase": phases}


def adjoint_algorithmic_bytes(N, M, nsteps):
    """Method bytes of a forward + adjoint run: the forward's per-step bytes
    and, per reverse step, about twice as many (8 transforms, 3 cotangent
    paints and the position terms), i.e. 3x the forward per PM step."""
    return 3.0 * step_algorithmic_bytes(N, M) * nsteps


def measure_fwd_adjoint(wl, reps=1, peak=None):
    """Forward + hand-written adjoint (d chi^2 / d white) of workload wl,
    with dx checkpointed at every stage; ms per iteration and per PM step,
    the roofline fraction of the method's bytes and the per-class device
    time of one forward + adjoint (CUDA events around each launcher)."""
    import numpy as np
    import torch
    from paper_2010_11847_gb300 import inputs
    from paper_2010_11847_gb300.binding import Plan
    from paper_2010_11847_gb300.autograd import chi2_of_final_density
    pl = Plan(wl.np_, wl.nc, wl.box, wl.cosmo)
    stages = wl.stages()
    w = torch.from_numpy(inputs.white_noise(wl.np_, wl.seed)).cuda()
    target = torch.zeros(wl.nc, wl.nc, wl.nc, device="cuda")

    def fwd_only():
        lk = pl.linear_field(w)
        dx, p = pl.lpt(lk, float(stages[0]), 2)
        pl.kdk(dx, p, stages)
        return pl.paint(dx)

    def fwd_adj():
        wt = w.clone().requires_grad_(True)
        loss = chi2_of_final_density(wt, target, pl, stages)
        loss.backward()
        return wt.grad

    out = {}
    for name, fn in (("fwd", fwd_only), ("fwd_adj", fwd_adj)):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        out[name] = 1e3 * (time.perf_counter() - t0) / reps
    pl.profile(True)
    fwd_adj()
    prof = pl.profile_read()
    pl.profile(False)
    pl.close()
    N, M = wl.np_ ** 3, wl.nc ** 3
    alg = adjoint_algorithmic_bytes(N, M, wl.nsteps)
    res = {"workload": wl.name, "ms_fwd": out["fwd"], "ms_fwd_adj": out["fwd_adj"],
           "ms_per_pm_step_fwd_adj": out["fwd_adj"] / wl.nsteps, "ratio_fwd_adj_to_fwd": out["fwd_adj"] / out["fwd"],
           "particle_steps_per_s_fwd_adj": N * wl.nsteps / (out["fwd_adj"] / 1e3),
           "breakdown_fwd_adj": {k: {"ms": v[0], "launches": v[1]} for k, v in sorted(prof.items())}}
    if peak:
        gbs = alg / (out["fwd_adj"] / 1e3) / 1e9
        res["roofline"] = {"bound": "hbm", "alg_bytes": alg, "achieved": gbs, "peak": peak, "unit": "GB/s",
                           "frac": gbs / peak,
                           "bytes_model": "forward 60 B/particle + 44 B/cell per PM step, adjoint twice that per "
                                          "reverse step (3x the forward in all)"}
    return res


def measure_force_variants(wl, reps=10):
    """Cost of the force variants (naive / Eq. 4 Green's function x Eq. 5 /
    exact gradient) at workload wl's mesh: CUDA-event ms of one fpm_force
    (density -> three force meshes) and of one PM step inside a 5-step
    fpm_kdk from 2LPT initial conditions."""
    import numpy as np
    import torch
    from paper_2010_11847_gb300 import inputs
    from paper_2010_11847_gb300.binding import Plan
    pl = Plan(wl.np_, wl.nc, wl.box, wl.cosmo)
    rho = torch.from_numpy((1.0 + 0.5 * inputs.random_field(wl.nc, 11)).astype(np.float32)).cuda()
    F = torch.empty(3, wl.nc, wl.nc, wl.nc, device="cuda")
    lk = pl.linear_field(torch.from_numpy(inputs.white_noise(wl.np_, wl.seed)).cuda())
    stages = np.linspace(wl.a0, 1.0, 6)
    dx0, p0 = pl.lpt(lk, float(stages[0]), 2)
    out = {}
    for green in ("naive", "discrete"):
        for grad in ("fd4", "exact"):
            pl.set_force_kernel(green, grad)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for _ in range(3):
                pl.force(rho, F)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                pl.force(rho, F)
            e1.record()
            torch.cuda.synchronize()
            ms_force = e0.elapsed_time(e1) / reps
            dx, p = dx0.clone(), p0.clone()
            pl.kdk(dx, p, stages)
            dx, p = dx0.clone(), p0.clone()
            torch.cuda.synchronize()
            e0.record()
            pl.kdk(dx, p, stages)
            e1.record()
            torch.cuda.synchronize()
            assert pl.status() == 0
            out[f"{green}/{grad}"] = {"ms_force": ms_force, "ms_per_pm_step": e0.elapsed_time(e1) / 5}
    pl.set_force_kernel("naive", "fd4")
    pl.close()
    return {"workload": wl.name, "variants": out}


def measure_pyramid(levels=2, split=2, halo=16):
    """The multi-grid pyramid force (Algorithms 2-3) against the plain force
    in the accuracy configuration (128^3 on 128^3, 400 Mpc/h, 10 KDK steps
    from 1LPT at a = 0.1), for each reading of Algorithm 3 (band-pass per
    padded block or on the assembled mesh; coarse operator matched to the
    fine mesh or Eq. 5 in coarse cells): residual of the final density
    contrast, transfer function and cross-correlation of the two (Eqs.
    10-11), and the cost of one force evaluation (CUDA events) here and on
    the 512^3 mesh with the default reading."""
    import math
    import numpy as np
    import torch
    from paper_2010_11847_gb300 import inputs
    from paper_2010_11847_gb300.binding import Plan
    wl = inputs.ACCURACY_10STEP
    pl = Plan(wl.np_, wl.nc, wl.box, wl.cosmo)
    stages = wl.stages()
    lk = pl.linear_field(torch.from_numpy(inputs.white_noise(wl.np_, wl.seed)).cuda())
    dx0, p0 = pl.lpt(lk, float(stages[0]), 1)

    def timed(fn, reps):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def final_delta():
        dx, p = dx0.clone(), p0.clone()
        pl.kdk(dx, p, stages)
        return pl.paint(dx) - 1.0

    pl.set_pyramid(0)
    dm = final_delta()
    rho_m = dm + 1.0
    out = {"workload": wl.name, "levels": levels, "split": split, "halo": halo,
           "block_mesh": wl.nc // split + 2 * halo, "coarse_mesh": wl.nc >> levels,
           "ms_force_plain": timed(lambda: pl.force(rho_m), 10), "readings": {}}
    k, pb, _ = pl.power(dm)
    low = k < 0.5 * math.pi * wl.nc / wl.box
    for bandpass, kernel in (("block", "matched"), ("global", "coarse"), ("block", "coarse"), ("global", "matched")):
        pl.set_pyramid_reading(bandpass, kernel)
        pl.set_pyramid(levels, split, halo)
        dp = final_delta()
        assert pl.status() == 0
        _, pa, _ = pl.power(dp)
        _, pab, _ = pl.power(dp, dm)
        tf = np.sqrt(pa / pb)
        rc = pab / np.sqrt(pa * pb)
        out["readings"][f"{bandpass}/{kernel}"] = {
            "ms_force_pyramid": timed(lambda: pl.force(rho_m), 10),
            "field_residual_rms": float((dp - dm).pow(2).mean().sqrt() / dm.pow(2).mean().sqrt()),
            "projected_residual_rms": float((dp - dm).sum(2).pow(2).mean().sqrt() / dm.sum(2).pow(2).mean().sqrt()),
            "max_abs_tf_minus_1": float(np.abs(tf - 1).max()),
            "max_abs_tf_minus_1_below_half_nyquist": float(np.abs(tf[low] - 1).max()),
            "max_1_minus_rc": float((1 - rc).max()),
            "max_1_minus_rc_below_half_nyquist": float((1 - rc[low]).max())}
        pl.set_pyramid(0)
    pl.close()
    big = inputs.LARGE
    pb_ = Plan(128, big.nc, big.box, big.cosmo)
    rho = torch.from_numpy((1.0 + 0.5 * inputs.random_field(big.nc, 12)).astype(np.float32)).cuda()
    out["ms_force_plain_512"] = timed(lambda: pb_.force(rho), 5)
    pb_.set_pyramid(2, 4, 32)
    out["ms_force_pyramid_512"] = timed(lambda: pb_.force(rho), 5)
    out["pyramid_512"] = {"levels": 2, "split": 4, "halo": 32, "block_mesh": 192, "coarse_mesh": 128,
                          "reading": "block/matched"}
    pb_.close()
    return out


def measure_cufft_reference(reps=10):
    """Reference only: cuFFT through torch.fft (rfftn + irfftn of one field)
    at 512^3, against this library's forward + Green + inverse passes of the
    potential (one field) from its own per-class CUDA events."""
    import numpy as np
    import torch
    from paper_2010_11847_gb300 import inputs
    from paper_2010_11847_gb300.binding import Plan
    n = inputs.LARGE.nc
    rho = torch.from_numpy(inputs.random_field(n, 13)).cuda()
    spec = torch.fft.rfftn(rho)
    back = torch.fft.irfftn(spec, s=(n, n, n))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        spec = torch.fft.rfftn(rho)
        back = torch.fft.irfftn(spec, s=(n, n, n))
    e1.record()
    torch.cuda.synchronize()
    cufft = e0.elapsed_time(e1) / reps
    del spec, back
    pl = Plan(128, n, inputs.LARGE.box, inputs.LARGE.cosmo)
    F = torch.empty(3, n, n, n, device="cuda")
    pl.force(rho + 1.0, F)
    pl.profile(True)
    for _ in range(reps):
        pl.force(rho + 1.0, F)
    prof = pl.profile_read()
    pl.profile(False)
    pl.close()
    ours = sum(prof[k][0] for k in ("pot_fft_fwd_zy", "pot_fft_x_green", "pot_fft_inv_yz") if k in prof) / reps
    return {"mesh": n, "ms_cufft_rfftn_plus_irfftn": cufft, "ms_ours_fwd_green_inv": ours,
            "note": "reference only: cuFFT is a library transform pair without the Green's function"}


def measure_reconstruction(iters=10, warmup=2):
    """Adam iterations of the Sec. 7.1 reconstruction (forward with checkpoints,
    adjoint, fused Adam + prior) at 128^3 particles on 128^3 cells, 400 Mpc/h,
    5 KDK steps, against a target density from another seed."""
    import torch
    from paper_2010_11847_gb300 import inputs
    from paper_2010_11847_gb300.binding import Plan
    from paper_2010_11847_gb300.reconstruct import Reconstruction
    wl = inputs.DIFFERENTIABLE
    stages = wl.stages()
    pl = Plan(wl.np_, wl.nc, wl.box, wl.cosmo)
    wt = torch.from_numpy(inputs.white_noise(wl.np_, wl.seed + 1)).cuda()
    lk = pl.linear_field(wt)
    dx, p = pl.lpt(lk, float(stages[0]), 2)
    pl.kdk(dx, p, stages)
    target = pl.paint(dx) - 1.0
    rec = Reconstruction(pl, target, stages, torch.zeros_like(wt), lr=0.01)
    first = rec.step()
    for _ in range(warmup - 1):
        rec.step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(iters):
        last = rec.step()
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0) / iters
    pl.close()
    return {"workload": wl.name, "ms_per_iteration": ms, "iterations": iters,
            "neg_log_posterior_first": first, "neg_log_posterior_last": last,
            "paper_context": "about 1.1 s per iteration on one V100 (another machine; context only)"}


def run_fpm(args):
    import numpy as np
    import torch
    import torch.distributed as tdist
    rank, world, local = dist()
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl")
    from paper_2010_11847_gb300 import build, inputs
    build.build()
    from paper_2010_11847_gb300.binding import Plan, launch_count

    wl = workload(args.workload)
    N, M = wl.np_ ** 3, wl.nc ** 3
    stages = wl.stages()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    plan = Plan(wl.np_, wl.nc, wl.box, wl.cosmo)
    white_h = torch.from_numpy(inputs.white_noise(wl.np_, rank_seed(wl.seed, rank))).pin_memory()
    white = white_h.to(dev)
    lin_k = torch.empty(plan.spectrum_shape(), dtype=torch.complex64, device=dev)
    dx = torch.empty(3, N, device=dev)
    p = torch.empty(3, N, device=dev)
    rho = torch.empty(wl.nc, wl.nc, wl.nc, device=dev)

    def one_sim(w):
        plan.linear_field(w, lin_k)
        plan.lpt(lin_k, float(stages[0]), 2, dx, p)
        plan.kdk(dx, p, stages)
        plan.paint(dx, rho)
        return plan.power(rho)

    def barrier():
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 0)):
        one_sim(white)
    st = plan.status()
    assert st == 0, f"device error flag set during warm-up (status {st})"

    # the fused readout (the kernel class with the largest share) is timed by
    # CUDA events over the timed region; the other classes are not
    # bracketed there (their per-class times come from one more simulation
    # after it)
    clocks = Clocks(local, enabled=not args.no_clocks and rank == 0)
    plan.profile(True, only=ROOFLINE_CLASS)
    barrier()
    launches0 = launch_count()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one_sim(white)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = launch_count() - launches0
    prof_timed = plan.profile_read()
    # per-class device time of every class from one more simulation, outside
    # the timed region (an event pair around every launcher)
    plan.profile(True)
    one_sim(white)
    prof = plan.profile_read()
    plan.profile(False)
    ms_total = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_step = ms_total / args.steps
    pm_steps = wl.nsteps
    value = job_value(world, N, pm_steps, ms_step / 1e3)
    st = plan.status()
    assert st == 0, f"device error flag set during the timed run (status {st})"

    # end to end: host white noise in, density and P(k) out, every step.  The
    # next simulation's white noise is uploaded and the previous density read
    # back on a copy stream while the current simulation runs (double
    # buffers); every copy is inside the timed region.
    e2e = None
    if not args.no_e2e:
        rho_h = [torch.empty(wl.nc, wl.nc, wl.nc).pin_memory() for _ in range(2)]
        rho_d = [rho, torch.empty_like(rho)]
        w_d = [torch.empty_like(white), torch.empty_like(white)]
        copy = torch.cuda.Stream(device=dev)
        up = [torch.cuda.Event(), torch.cuda.Event()]
        sim_done = [torch.cuda.Event(), torch.cuda.Event()]
        down = [torch.cuda.Event(), torch.cuda.Event()]

        def sim_into(w, r):
            plan.linear_field(w, lin_k)
            plan.lpt(lin_k, float(stages[0]), 2, dx, p)
            plan.kdk(dx, p, stages)
            plan.paint(dx, r)
            return plan.power(r)

        barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(copy):
            w_d[0].copy_(white_h, non_blocking=True)
            up[0].record(copy)
        for k in range(args.steps):
            j = k % 2
            if k + 1 < args.steps:
                with torch.cuda.stream(copy):
                    if k >= 1:
                        copy.wait_event(sim_done[1 - j])        # simulation k-1 has read w_d[1-j]
                    w_d[1 - j].copy_(white_h, non_blocking=True)
                    up[1 - j].record(copy)
            if k >= 2:
                down[j].synchronize()                          # rho_d[j], rho_h[j] free again
            stream.wait_event(up[j])
            sim_into(w_d[j], rho_d[j])
            sim_done[j].record(stream)
            with torch.cuda.stream(copy):
                copy.wait_event(sim_done[j])
                rho_h[j].copy_(rho_d[j], non_blocking=True)
                down[j].record(copy)
        copy.synchronize()
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": job_value(world, N, pm_steps * args.steps, dt), "unit": UNIT,
               "h2d_bytes_per_step": int(white_h.numel() * 4),
               "d2h_bytes_per_step": int(rho_h[0].numel() * 4 + 3 * 8 * (wl.nc // 2))}

    if rank != 0:
        if world > 1:
            tdist.destroy_process_group()
        return 0

    # roofline of the dominant kernel class (device time inside the timed region)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    dominant = max((k for k in prof if _alg_bytes(k, N, M, wl.nc) is not None), key=lambda k: prof[k][0])
    if dominant != ROOFLINE_CLASS:
        print(f"warning: the largest class is {dominant}, not {ROOFLINE_CLASS}", file=sys.stderr)
    dominant = ROOFLINE_CLASS
    dms, dn = prof_timed[dominant]
    per_launch_ms = dms / dn
    alg = _alg_bytes(dominant, N, M, wl.nc)
    achieved = alg / (per_launch_ms / 1e3) / 1e9
    step_ms = ms_step / pm_steps
    step_alg = step_algorithmic_bytes(N, M)
    build = _build_bytes(dominant, N, M, wl.nc)
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src, "traffic": ncu_traffic(dominant),
                "alg_bytes_per_launch": alg, "ms_per_launch": per_launch_ms,
                "build_bytes_per_launch": build,
                "build_frac": build / (per_launch_ms / 1e3) / 1e9 / peak}
    cpu = None if args.no_cpu_baseline else oracle_sample()
    extra = {}
    if not args.no_adjoint and args.workload == "large":
        plan.close()
        del dx, p, rho, lin_k
        torch.cuda.empty_cache()
        from paper_2010_11847_gb300 import inputs as _in
        extra["fwd_adjoint"] = measure_fwd_adjoint(wl, peak=peak)
        extra["reconstruction"] = measure_reconstruction()
        torch.cuda.empty_cache()
        extra["force_variants"] = measure_force_variants(wl)
        torch.cuda.empty_cache()
        extra["pyramid"] = measure_pyramid()
        torch.cuda.empty_cache()
        extra["cufft_reference"] = measure_cufft_reference()
        # the paper's reconstruction iteration (5-step 128^3, 400 Mpc/h) is this config:
        # ~1.1 s/iter on one V100 for forward + gradient + Adam (context only)
        extra["fwd_adjoint_128"] = measure_fwd_adjoint(_in.DIFFERENTIABLE, reps=5, peak=peak)
        torch.cuda.empty_cache()
    if not args.no_batch:
        extra["batched"] = measure_batched(peak=peak)
    breakdown = {k: {"ms_per_sim": v[0], "launches_per_sim": v[1]} for k, v in prof.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "np": wl.np_, "nc": wl.nc, "box_mpc_h": wl.box, "kdk_steps": pm_steps,
                   "a0": wl.a0, "lpt_order": 2, "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "inputs larger than L2 (working set several GB)",
                   "bench_step": "one whole simulation: coefficients, linear field, 2LPT, all KDK steps, "
                                 "final paint and P(k)"},
        "ms_per_pm_step": step_ms,
        "step_roofline": {"alg_bytes_per_pm_step": step_alg, "achieved_gbs": step_alg / (step_ms / 1e3) / 1e9,
                          "frac_of_measured": step_alg / (step_ms / 1e3) / 1e9 / peak,
                          "frac_of_8tbs_nominal": step_alg / (step_ms / 1e3) / 1e9 / 8000.0},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "breakdown": breakdown,
    }
    line.update(extra)
    if args.profile_json:
        json.dump(line, open(args.profile_json, "w"), indent=1)
    print(json.dumps(line))
    if world > 1:
        tdist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_fpm(args)


if __name__ == "__main__":
    sys.exit(main())
