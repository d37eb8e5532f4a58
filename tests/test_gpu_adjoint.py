"""Adjoint (reverse-mode) CUDA path against the FP64 oracle's adjoint.

Per primitive: relative L2 <= 1e-5 (fixed positions, linear maps); reverse
KDK and 2LPT <= 1e-4; the full gradient of chi^2 with respect to the white
noise at 128^3 / 128^3, 400 Mpc/h, 5 steps: vector-norm relative error over
32 random voxels <= 1e-3 against the oracle adjoint and against the FP64
oracle's central finite differences at eps = 1e-4 (converged), <= 1e-2
against those at eps = 1e-3 (which carry the CIC kinks crossed within the
step); the FP32 GPU forward's own differences (all-voxel directional and
per voxel) are printed with their noise and checked at their measured
level.
"""
import json
import os

import numpy as np
import pytest

from oracle import fpm_oracle as O
from paper_2010_11847_gb300 import inputs

pytestmark = pytest.mark.gpu

COSMO = dict(inputs.COSMO_DEFAULT)
FULL_EPS = (3e-4, 1e-3, 3e-3)
VOXEL_FD_BOUND = 3e-2
OM = COSMO["omega_m"]


def rel_l2(a, b):
    dt = np.complex128 if (np.iscomplexobj(a) or np.iscomplexobj(b)) else np.float64
    a = np.asarray(a, dtype=dt)
    b = np.asarray(b, dtype=dt)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_mod(cuda):
    import torch
    return torch


def plan(np_, nc, box=100.0, cosmo=COSMO):
    from paper_2010_11847_gb300.binding import Plan
    return Plan(np_, nc, box, cosmo)


def dev(x, torch):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_force_adj_matches_oracle(torch_mod):
    torch = torch_mod
    n = 64
    pl = plan(32, n)
    gF = np.stack([inputs.random_field(n, 60 + d) for d in range(3)])
    got = pl.force_adj(dev(gF, torch)).cpu().numpy()
    assert rel_l2(got, O.force_adj(gF.astype(np.float64), OM)) < 1e-5


# (32, 32), (32, 64): the three cotangent channels painted by one launch;
# (64, 256): one launch per channel (meshes of more than 512 tiles)
@pytest.mark.parametrize("np_,nc", [(32, 32), (32, 64), (64, 256)])
def test_paint_and_readout_adj_match_oracle(torch_mod, np_, nc):
    torch = torch_mod
    pl = plan(np_, nc)
    dx = inputs.random_displacements(np_, 3.0, 70 + nc)
    g_rho = inputs.random_field(nc, 71)
    got = pl.paint_adj(dev(dx, torch), dev(g_rho, torch)).cpu().numpy()
    assert rel_l2(got, O.paint_adj(g_rho.astype(np.float64), dx, np_, nc)) < 1e-5
    F = np.stack([inputs.random_field(nc, 72 + d) for d in range(3)])
    gf = inputs.random_displacements(np_, 1.0, 73)
    gF, gdx = pl.readout_adj(dev(F, torch), dev(dx, torch), dev(gf, torch))
    rF, rdx = O.readout_adj(F.astype(np.float64), dx, gf.astype(np.float64), np_, nc)
    assert rel_l2(gF.cpu().numpy(), rF) < 1e-5
    assert rel_l2(gdx.cpu().numpy(), rdx) < 1e-5


def test_readout_adj_is_deterministic(torch_mod):
    torch = torch_mod
    pl = plan(32, 64)
    dx = dev(inputs.random_displacements(32, 5.0, 3), torch)
    F = dev(np.stack([inputs.random_field(64, 5 + d) for d in range(3)]), torch)
    gf = dev(inputs.random_displacements(32, 1.0, 4), torch)
    a, _ = pl.readout_adj(F, dx, gf)
    b, _ = pl.readout_adj(F, dx, gf)
    assert torch.equal(a, b)


@pytest.mark.parametrize("order", [1, 2])
def test_lpt_and_linear_field_adj_match_oracle(torch_mod, order):
    torch = torch_mod
    n, nc, box = 32, 64, 100.0
    pl = plan(n, nc, box)
    w = inputs.white_noise(n, 90)
    lk = O.linear_field(w, box, COSMO)
    gdx = inputs.random_displacements(n, 1.0, 91)
    gp = inputs.random_displacements(n, 1.0, 92)
    lk_dev = dev(np.ascontiguousarray(lk.transpose(0, 2, 1)).astype(np.complex64), torch)
    G = pl.lpt_adj(lk_dev, 0.1, dev(gdx, torch), dev(gp, torch), order)
    rG = O.lpt_adj(lk, nc, 0.1, COSMO, gdx, gp, order)
    assert rel_l2(G.permute(0, 2, 1).cpu().numpy(), rG) < 1e-4
    gw = pl.linear_field_adj(dev(np.ascontiguousarray(rG.transpose(0, 2, 1)).astype(np.complex64), torch))
    assert rel_l2(gw.cpu().numpy(), O.linear_field_adj(rG, box, COSMO)) < 1e-5


# 32^3: the velocity cotangents stored by a drift-kick kernel; 64^3 (a
# lattice of whole 4 x 16 x 64 bricks): read as K g_p by the paint and the
# gather, which also applies the next step's drift and kick transposes
@pytest.mark.parametrize("n,nc,box", [(32, 32, 100.0), (64, 64, 200.0)])
def test_kdk_adj_matches_oracle_given_the_same_checkpoints(torch_mod, n, nc, box):
    torch = torch_mod
    stages = np.linspace(0.1, 0.7, 4)
    pl = plan(n, nc, box)
    lk = O.linear_field(inputs.white_noise(n, 5), box, COSMO)
    dx0, p0 = O.lpt(lk, nc, stages[0], COSMO)
    rec = []
    dxn, _ = O.kdk(dx0, p0, stages, n, nc, OM, record=rec)
    xs = [x.astype(np.float32) for x, _ in rec] + [dxn.astype(np.float32)]
    gdx = inputs.random_displacements(n, 1.0, 6)
    gp = inputs.random_displacements(n, 1.0, 7)
    rx, rp = O.kdk_adj(xs, stages, gdx, gp, n, nc, OM)
    ckpt = dev(np.stack(xs), torch)
    g_dx = dev(gdx, torch).clone()
    g_dx, g_p = pl.kdk_adj(ckpt, stages, g_dx, g_p_in=dev(gp, torch))
    assert rel_l2(g_dx.cpu().numpy(), rx) < 1e-4
    assert rel_l2(g_p.cpu().numpy(), rp) < 1e-4
    # without a momentum cotangent (a loss on the density alone)
    rx0, rp0 = O.kdk_adj(xs, stages, gdx, np.zeros_like(gdx), n, nc, OM)
    g_dx = dev(gdx, torch).clone()
    g_dx, g_p = pl.kdk_adj(ckpt, stages, g_dx)
    assert rel_l2(g_dx.cpu().numpy(), rx0) < 1e-4
    assert rel_l2(g_p.cpu().numpy(), rp0) < 1e-4


def test_differentiable_config_gradient(torch_mod):
    """128^3 particles on 128^3, 400 Mpc/h, 2LPT at a=0.1 + 5 KDK steps;
    chi^2 against the final density contrast of a second seed (sigma = 1)."""
    torch = torch_mod
    from paper_2010_11847_gb300.autograd import chi2_of_final_density
    wl = inputs.DIFFERENTIABLE
    stages = wl.stages()
    w = inputs.white_noise(wl.np_, wl.seed)
    ref_t = O.simulate(inputs.white_noise(wl.np_, wl.seed + 1), wl.nc, wl.box, wl.cosmo, stages)
    target = (ref_t["rho"] - 1.0).astype(np.float32)
    pl = plan(wl.np_, wl.nc, wl.box, wl.cosmo)
    wt = dev(w, torch).requires_grad_(True)
    tt = dev(target, torch)
    loss = chi2_of_final_density(wt, tt, pl, stages)
    loss.backward()
    g = wt.grad.detach().cpu().numpy().reshape(-1)
    L_ref, g_ref = O.chi2_and_grad(w, target.astype(np.float64), wl.nc, wl.box, wl.cosmo, stages)
    assert abs(float(loss.detach()) / L_ref - 1) < 1e-4
    idx = np.random.default_rng(2024).choice(w.size, size=32, replace=False)
    ad, ref = g[idx], g_ref.reshape(-1)[idx]
    vec = np.linalg.norm(ad - ref) / np.linalg.norm(ref)
    per_voxel = np.abs(ad - ref) / np.maximum(np.abs(ref), 1e-30)
    print(f"adjoint vs oracle adjoint: vector rel {vec:.2e}, per-voxel median {np.median(per_voxel):.2e}, "
          f"max {per_voxel.max():.2e}")
    assert vec < 1e-3
    assert rel_l2(g, g_ref.reshape(-1)) < 1e-3

    # FP64 central differences of the oracle's forward (FP64 positions) at the
    # same 32 voxels, written by tests/golden/make_fd_gradient_128.py: at
    # eps = 1e-4 they have converged to the gradient (the chi^2 is piecewise
    # smooth: a CIC weight's derivative jumps where a particle crosses a cell
    # face); at eps = 1e-3 they still carry the kinks crossed within the
    # step (the oracle's own FP64 adjoint is 3.9e-3 from them)
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fd_gradient_128.json")))
    assert gold["voxels"] == [int(i) for i in idx]
    assert gold["eps"] == 1e-3 and gold["eps_converged"] == 1e-4
    fd3, fd4 = np.asarray(gold["fd"]), np.asarray(gold["fd_converged"])
    vec3 = np.linalg.norm(ad - fd3) / np.linalg.norm(fd3)
    vec4 = np.linalg.norm(ad - fd4) / np.linalg.norm(fd4)
    print(f"adjoint vs FP64 central differences, 32 voxels: eps=1e-4 vector rel {vec4:.2e} "
          f"(per-voxel max {np.max(np.abs(ad - fd4) / np.abs(fd4)):.2e}); eps=1e-3 vector rel {vec3:.2e}")
    assert vec4 < 1e-3
    assert vec3 < 1e-2

    def gpu_loss(wv):
        with torch.no_grad():
            return float(chi2_of_final_density(wv, tt, pl, stages))

    # FP32 GPU forward, central directional derivative along a direction that
    # spans every voxel (unit variance per voxel): its signal 2 eps g.u grows
    # like sqrt(N) over a single voxel's; at small eps the FP32 rounding of
    # the loss and at large eps the CIC kinks crossed by the moving particles
    # bound the agreement (measured 1e-3..3e-3 at eps = 3e-4, 1e-2..2e-2 at 1e-3)
    u = np.random.default_rng(7).standard_normal(w.size).astype(np.float32)
    ut = torch.from_numpy(u).cuda().view(w.shape)
    exact = float(g.astype(np.float64) @ u.astype(np.float64))
    full = {}
    for eps in FULL_EPS:
        full[eps] = (gpu_loss(wt.detach() + eps * ut) - gpu_loss(wt.detach() - eps * ut)) / (2 * eps)
        print(f"FP32 directional derivative over all voxels eps={eps:g}: rel error "
              f"{abs(full[eps] - exact) / abs(exact):.2e}")
    assert abs(full[3e-4] - exact) < 1e-2 * abs(exact)

    # FP32 central differences voxel by voxel: the loss's FP32 rounding noise
    # (printed, implied by |fd - ad| 2 eps) swamps 2 eps dchi2/dw at small
    # eps, and at eps = 3e-2 the kinks crossed within the step dominate (the
    # FP64 differences are 3.9e-3 off already at a 30x smaller step)
    fds = {}
    for eps in (1e-3, 3e-3, 3e-2):
        out = []
        for i in idx:
            e = torch.zeros(w.size, device="cuda")
            e[int(i)] = eps
            e = e.view(w.shape)
            out.append((gpu_loss(wt.detach() + e) - gpu_loss(wt.detach() - e)) / (2 * eps))
        fds[eps] = np.array(out)
    for eps, fd in fds.items():
        print(f"FP32 central differences eps={eps:g}: vector rel error vs adjoint "
              f"{np.linalg.norm(fd - ad) / np.linalg.norm(ad):.2e}, implied loss noise "
              f"{np.median(np.abs(fd - ad)) * 2 * eps:.2e}")
    assert np.linalg.norm(fds[3e-2] - ad) / np.linalg.norm(ad) < VOXEL_FD_BOUND


@pytest.mark.parametrize("np_,nc,reverse", [(32, 64, True), (32, 32, True), (64, 64, True), (48, 96, False)])
def test_force_checkpoints_give_the_same_bits(torch_mod, np_, nc, reverse):
    """Keeping the forward's force meshes and tile buckets (fckpt) changes
    nothing but the work: the same forward state and checkpoints (float4 and
    planar force meshes) as without them and as without any checkpoint, and
    the same cotangents as the reverse pass that recomputes the forces and
    buckets (the reverse pass runs on power-of-two meshes)."""
    torch = torch_mod
    stages = np.linspace(0.1, 0.7, 4)
    pl = plan(np_, nc)
    lk = pl.linear_field(dev(inputs.white_noise(np_, 9), torch))
    dx, p = pl.lpt(lk, float(stages[0]), 2)
    dx2, p2 = dx.clone(), p.clone()
    dx3, p3 = dx.clone(), p.clone()
    ck = torch.empty(len(stages), 3, pl.N, device="cuda")
    ck2 = torch.empty_like(ck)
    fck = torch.empty(len(stages), pl.force_ckpt_floats, device="cuda")
    pl.kdk(dx, p, stages, ckpt=ck)
    pl.kdk(dx2, p2, stages, ckpt=ck2, fckpt=fck)
    pl.kdk(dx3, p3, stages)                     # no checkpoints: the steps run on dx itself
    assert torch.equal(dx, dx2) and torch.equal(p, p2) and torch.equal(ck, ck2)
    assert torch.equal(dx, dx3) and torch.equal(p, p3)
    assert torch.equal(ck[-1], dx3)              # the closing kick does not move the particles
    if not reverse:
        return
    gdx = dev(inputs.random_displacements(np_, 1.0, 6), torch)
    gp = dev(inputs.random_displacements(np_, 1.0, 7), torch)
    r1 = pl.kdk_adj(ck, stages, gdx.clone(), g_p_in=gp.clone())
    r2 = pl.kdk_adj(ck, stages, gdx.clone(), g_p_in=gp.clone(), fckpt=fck)
    torch.cuda.synchronize()
    assert pl.status() == 0
    assert torch.equal(r1[0], r2[0]) and torch.equal(r1[1], r2[1])
