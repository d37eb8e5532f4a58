"""Force variants through the C ABI against the oracle's variants (Sec. 2):
Eq. 4's discrete-Laplacian Green's function and the exact i k gradient,
each combined with the default naive Green's function / Eq. 5 difference.

Tolerances as for the default force: force meshes and their transposes
relative L2 <= 1e-5; positions and momenta after a 4-step run <= 1e-4.
Power-of-two meshes with Eq. 5's gradient go through the potential form,
the exact gradient through three spectral fields; 96^3 takes the
shared-memory passes.
"""
import numpy as np
import pytest

from oracle import fpm_oracle as O
from paper_2010_11847_gb300 import inputs

pytestmark = pytest.mark.gpu

COSMO = dict(inputs.COSMO_DEFAULT)
OM = COSMO["omega_m"]
VARIANTS = [("naive", "fd4"), ("naive", "exact"), ("discrete", "fd4"), ("discrete", "exact")]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_mod(cuda):
    import torch
    return torch


def plan(np_, nc, box=100.0, green="naive", gradient="fd4"):
    from paper_2010_11847_gb300.binding import Plan
    pl = Plan(np_, nc, box, COSMO)
    pl.set_force_kernel(green, gradient)
    return pl


def dev(x, torch):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("green,gradient", VARIANTS)
@pytest.mark.parametrize("nc", [64, 96, 128])
def test_variant_force_matches_oracle(torch_mod, green, gradient, nc):
    torch = torch_mod
    pl = plan(nc // 2, nc, green=green, gradient=gradient)
    rho = (1.0 + 0.5 * inputs.random_field(nc, 300 + nc)).astype(np.float32)
    F = pl.force(dev(rho, torch)).cpu().numpy()
    ref = O.force(rho.astype(np.float64), OM, green, gradient)
    for d in range(3):
        assert rel_l2(F[d], ref[d]) < 1e-5, (d, rel_l2(F[d], ref[d]))


@pytest.mark.parametrize("green,gradient", VARIANTS)
def test_variant_force_adj_matches_oracle(torch_mod, green, gradient):
    torch = torch_mod
    n = 64
    pl = plan(32, n, green=green, gradient=gradient)
    gF = np.stack([inputs.random_field(n, 360 + d) for d in range(3)])
    got = pl.force_adj(dev(gF, torch)).cpu().numpy()
    assert rel_l2(got, O.force_adj(gF.astype(np.float64), OM, green, gradient)) < 1e-5


@pytest.mark.parametrize("green,gradient", VARIANTS[1:])
def test_variant_kdk_matches_oracle(torch_mod, green, gradient):
    """Four KDK steps from the oracle's 2LPT at a = 0.1, 32^3 on 64^3
    (the interleaved force mesh of the fused readout)."""
    torch = torch_mod
    n, nc, box = 32, 64, 100.0
    stages = np.linspace(0.1, 0.5, 5)
    lk = O.linear_field(inputs.white_noise(n, 21), box, COSMO)
    dx0, p0 = O.lpt(lk, nc, stages[0], COSMO)
    dx0 = dx0.astype(np.float32)
    p0 = p0.astype(np.float32)
    rdx, rp = O.kdk(dx0, p0, stages, n, nc, OM, green=green, gradient=gradient)
    pl = plan(n, nc, box, green, gradient)
    dx, p = dev(dx0, torch), dev(p0, torch)
    pl.kdk(dx, p, stages)
    torch.cuda.synchronize()
    assert pl.status() == 0
    assert rel_l2(dx.cpu().numpy(), rdx) < 1e-4
    assert rel_l2(p.cpu().numpy(), rp) < 1e-4


def test_switching_back_gives_the_default_bits(torch_mod):
    torch = torch_mod
    nc = 64
    rho = dev((1.0 + 0.5 * inputs.random_field(nc, 390)).astype(np.float32), torch)
    ref = plan(32, nc).force(rho)
    pl = plan(32, nc, green="discrete", gradient="exact")
    other = pl.force(rho)
    pl.set_force_kernel("naive", "fd4")
    again = pl.force(rho)
    torch.cuda.synchronize()
    assert not torch.equal(other, ref)
    assert torch.equal(again, ref)


def test_batch_takes_the_green_variant_and_refuses_the_exact_gradient(torch_mod):
    """A batch built from plans with Eq. 4's Green's function gives the bits
    of their one-by-one runs; the exact gradient is not batched."""
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Batch, FpmError
    a = np.linspace(0.1, 0.3, 3)
    plans, dxs, ps = [], [], []
    for i, (n, nc) in enumerate([(32, 32), (96, 96), (64, 64)]):
        pl = plan(n, nc, green="discrete")
        lk = pl.linear_field(dev(inputs.white_noise(n, 400 + i), torch))
        dx, p = pl.lpt(lk, float(a[0]), 2)
        plans.append(pl)
        dxs.append(dx)
        ps.append(p)
    ref = [(x.clone(), y.clone()) for x, y in zip(dxs, ps)]
    for pl, (x, y) in zip(plans, ref):
        pl.kdk(x, y, a)
    b = Batch(plans)
    b.kdk(dxs, ps, a)
    torch.cuda.synchronize()
    assert b.status() == 0
    for i in range(len(plans)):
        assert torch.equal(dxs[i], ref[i][0]) and torch.equal(ps[i], ref[i][1]), i
    b.close()
    plans[0].set_force_kernel("naive", "exact")
    with pytest.raises(FpmError):
        Batch(plans)
