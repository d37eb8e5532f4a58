"""Batched persistent step: every simulation must give exactly the bits of
its own one-by-one fpm_kdk run (the kernels and their arithmetic are the
same; the paint is deterministic), and a barrier that runs out of spins must
report FPM_ETIMEOUT instead of hanging."""
import numpy as np
import pytest

from paper_2010_11847_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod(cuda):
    import torch
    return torch


def _setup(workloads, torch):
    from paper_2010_11847_gb300.binding import Plan
    plans, dxs, ps = [], [], []
    for wl in workloads:
        pl = Plan(wl.np_, wl.nc, wl.box, wl.cosmo)
        w = torch.from_numpy(inputs.white_noise(wl.np_, wl.seed)).cuda()
        lk = pl.linear_field(w)
        dx, p = pl.lpt(lk, wl.a0, 2)
        plans.append(pl)
        dxs.append(dx)
        ps.append(p)
    return plans, dxs, ps


def _mix(n_each, nsteps, seed0=300):
    wls = inputs.batched_workloads(seed0)
    out = []
    for size in (32, 64, 96, 128):
        out += [w for w in wls if w.nc == size][:n_each]
    import dataclasses
    return [dataclasses.replace(w, nsteps=nsteps) for w in out]


def test_batch_matches_one_by_one_bitwise(torch_mod):
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Batch
    wls = _mix(2, 3)
    plans, dxs, ps = _setup(wls, torch)
    ref_dx = [x.clone() for x in dxs]
    ref_p = [x.clone() for x in ps]
    a = wls[0].stages()
    for pl, x, y in zip(plans, ref_dx, ref_p):
        pl.kdk(x, y, a)
    b = Batch(plans)
    b.kdk(dxs, ps, a)
    torch.cuda.synchronize()
    assert b.status() == 0
    info = b.info()
    assert info["grid_blocks"] > 0
    for i in range(len(plans)):
        assert torch.equal(dxs[i], ref_dx[i]), (i, wls[i].nc)
        assert torch.equal(ps[i], ref_p[i]), (i, wls[i].nc)


def test_batch_graph_replay_is_reproducible(torch_mod):
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Batch
    wls = _mix(1, 2, seed0=500)
    plans, dxs, ps = _setup(wls, torch)
    d0 = [x.clone() for x in dxs]
    p0 = [x.clone() for x in ps]
    b = Batch(plans)
    a = wls[0].stages()
    b.kdk(dxs, ps, a)
    first = [x.clone() for x in dxs]
    for x, y, x0, y0 in zip(dxs, ps, d0, p0):
        x.copy_(x0)
        y.copy_(y0)
    b.kdk(dxs, ps, a)            # replays the captured graph
    torch.cuda.synchronize()
    assert b.status() == 0
    for x, y in zip(dxs, first):
        assert torch.equal(x, y)


def test_barrier_timeout_is_reported_not_hung(torch_mod):
    """A spin limit of one iteration makes the grid barrier give up: the run
    ends early with FPM_ETIMEOUT, and the batch works again afterwards."""
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Batch, FPM_ETIMEOUT
    wls = _mix(1, 1, seed0=700)
    plans, dxs, ps = _setup(wls, torch)
    b = Batch(plans)
    b.configure(spin_limit=1)
    b.kdk(dxs, ps, wls[0].stages())
    torch.cuda.synchronize()
    assert b.status() == FPM_ETIMEOUT
    for pl in plans:
        pl.status()                       # clear any flag left by the truncated run
    b.configure(spin_limit=1 << 22)
    plans2, dxs2, ps2 = _setup(wls, torch)
    b2 = Batch(plans2)
    b2.kdk(dxs2, ps2, wls[0].stages())
    torch.cuda.synchronize()
    assert b2.status() == 0


def test_full_batched_config_runs(torch_mod):
    """64 simulations, meshes 32/64/96/128 (16 each), 10 KDK steps."""
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Batch
    wls = inputs.batched_workloads()
    plans, dxs, ps = _setup(wls, torch)
    check = [0, 17, 34, 63]
    ref = {}
    a = wls[0].stages()
    for i in check:
        x, y = dxs[i].clone(), ps[i].clone()
        plans[i].kdk(x, y, a)
        ref[i] = (x, y)
    b = Batch(plans)
    b.kdk(dxs, ps, a)
    torch.cuda.synchronize()
    assert b.status() == 0
    for i in check:
        assert torch.equal(dxs[i], ref[i][0]) and torch.equal(ps[i], ref[i][1])
    assert all(bool(torch.isfinite(x).all()) for x in dxs)


# every value of every per-size knob of the batched step: bricks of both
# shapes or chunks for the readout, 8^3 or 16^3 paint tiles, 8 or 16 FFT
# points per thread (96 has no power-of-two passes)
KNOB_SETTINGS = [
    {"readout": 0, "paint_tile": 8, "fft_slots": 16},
    {"readout": 1, "paint_tile": 8, "fft_slots": 8},
    {"readout": 2, "paint_tile": 16, "fft_slots": 16},
]


@pytest.mark.parametrize("knobs", KNOB_SETTINGS)
def test_batch_knobs_keep_the_bits(torch_mod, knobs):
    """The autotuner's per-size knobs change the layout, never a result bit:
    the batch stays equal to one-by-one runs under each setting."""
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Batch, FpmError
    wls = _mix(1, 3, seed0=900)
    plans, dxs, ps = _setup(wls, torch)
    ref_dx = [x.clone() for x in dxs]
    ref_p = [x.clone() for x in ps]
    a = wls[0].stages()
    for pl, x, y in zip(plans, ref_dx, ref_p):
        pl.kdk(x, y, a)
    b = Batch(plans)
    applied = 0
    for nc in (32, 64, 96, 128):
        for knob, value in knobs.items():
            try:
                b.tune(nc, knob, value)
                applied += 1
            except FpmError:
                assert (knob == "fft_slots" and nc == 96) or (knob == "readout" and value == 2 and nc in (32, 96)) \
                    or (knob == "readout" and nc == 96)
    assert applied >= 8
    b.kdk(dxs, ps, a)
    torch.cuda.synchronize()
    assert b.status() == 0
    for i in range(len(plans)):
        assert torch.equal(dxs[i], ref_dx[i]), (i, wls[i].nc, knobs)
        assert torch.equal(ps[i], ref_p[i]), (i, wls[i].nc, knobs)


def test_autotuner_picks_per_size_plans(torch_mod, tmp_path, monkeypatch):
    """The autotuner reports, for every mesh size of the batch, the readout
    traversal, the paint tile edge and the FFT plan it chose, caches them,
    and the tuned batch keeps the bits."""
    torch = torch_mod
    from paper_2010_11847_gb300 import autotune
    from paper_2010_11847_gb300.binding import Batch
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    wls = _mix(1, 2, seed0=950)
    plans, dxs, ps = _setup(wls, torch)
    a = wls[0].stages()
    ref_dx = [x.clone() for x in dxs]
    for pl, x, y in zip(plans, ref_dx, [y.clone() for y in ps]):
        pl.kdk(x, y, a)
    b = Batch(plans)
    r = autotune.tune(b, dxs, ps, a, reps=1)
    assert not r["cached"]
    sizes = r["config"]["sizes"]
    assert sorted(sizes, key=int) == ["32", "64", "96", "128"]
    for nc, k in sizes.items():
        assert k["paint_tile"] in (8, 16) and k["readout"] in (0, 1, 2)
        assert k["fft_slots"] in (8, 16) if nc != "96" else "fft_slots" not in k   # 96^3: no power-of-two passes
    assert len(r["timings_ms"]) > 9
    again = autotune.tune(Batch(plans), dxs, ps, a)
    assert again["cached"] and again["config"] == r["config"]
    b.kdk(dxs, ps, a)
    torch.cuda.synchronize()
    assert b.status() == 0
    for i in range(len(plans)):
        assert torch.equal(dxs[i], ref_dx[i])
