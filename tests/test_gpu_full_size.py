"""The bench workload's sizes (512^3 particles on a 512^3 mesh), in the
launch configuration the bench times, against the FP64 oracle element by
element: the force meshes of a density field (every slab-ordered FFT pass,
the x pass with the Green's function and the Eq. 5 stencil) and the
deterministic paint (cube-aggregated bucketing, tile paint, face sums),
plus bitwise run-to-run equality of the paint.  Each oracle call takes
tens of seconds and a few tens of GB of host memory."""
import numpy as np
import pytest

from oracle import fpm_oracle as O
from paper_2010_11847_gb300 import inputs

pytestmark = pytest.mark.gpu

COSMO = dict(inputs.COSMO_DEFAULT)
N = 512


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_mod(cuda):
    import torch
    return torch


def test_force_at_512_matches_oracle(torch_mod):
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Plan
    pl = Plan(N, N, 1000.0, COSMO)
    rho = (1.0 + 0.5 * inputs.random_field(N, 612)).astype(np.float32)
    F = pl.force(torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    assert pl.status() == 0
    F = F.cpu().numpy()
    pl.close()
    ref = O.force(rho.astype(np.float64), COSMO["omega_m"])
    for d in range(3):
        assert rel_l2(F[d], ref[d]) < 1e-5, (d, rel_l2(F[d], ref[d]))


def test_paint_at_512_matches_oracle_and_is_bitwise_reproducible(torch_mod):
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Plan
    pl = Plan(N, N, 1000.0, COSMO)
    dx = inputs.random_displacements(N, 6.0, 613)
    d = torch.from_numpy(dx).cuda()
    rho = pl.paint(d)
    again = pl.paint(d)
    torch.cuda.synchronize()
    assert pl.status() == 0
    assert torch.equal(rho, again)
    rho = rho.cpu().numpy()
    pl.close()
    del d, again
    ref = O.paint(dx, N, N)
    assert rel_l2(rho, ref) < 1e-5
    assert abs(rho.astype(np.float64).sum() / N ** 3 - 1) < 1e-6


def test_one_kdk_step_at_512_on_sampled_particles(torch_mod):
    """One KDK step of the bench workload's configuration (512^3 on 512^3,
    2LPT at a = 0.1, first step of 40) through fpm_kdk, checked on 2000
    sampled particles: the oracle reads out its FP64 forces of the GPU's
    densities before and after the drift (the full-size paint is checked
    above) and applies the FastPM kick and drift factors in FP64."""
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Plan
    wl = inputs.LARGE
    stages = wl.stages()[:2]
    pl = Plan(N, N, wl.box, wl.cosmo)
    lk = pl.linear_field(torch.from_numpy(inputs.white_noise(N, wl.seed)).cuda())
    dx, p = pl.lpt(lk, float(stages[0]), 2)
    del lk
    rho0 = pl.paint(dx).cpu().numpy()
    dx0, p0 = dx.cpu().numpy(), p.cpu().numpy()
    pl.kdk(dx, p, stages)
    rho1 = pl.paint(dx).cpu().numpy()
    torch.cuda.synchronize()
    assert pl.status() == 0
    dx1, p1 = dx.cpu().numpy(), p.cpu().numpy()
    pl.close()
    del dx, p
    om = wl.cosmo["omega_m"]
    k1, dr, k2 = (v[0] for v in O.fastpm_factors(stages, om))
    idx = np.random.default_rng(512).choice(N ** 3, size=2000, replace=False)

    def sampled_force(rho, x):
        F = O.force(rho.astype(np.float64), om)
        cell, t = O.cic_cells(x, N, N)
        return O.readout_cells(F, cell[:, idx], t[:, idx])

    f0 = sampled_force(rho0, dx0)
    del rho0
    f1 = sampled_force(rho1, dx1)
    ph = p0[:, idx].astype(np.float64) + k1 * f0
    want_dx = dx0[:, idx].astype(np.float64) + dr * ph
    want_p = ph + k2 * f1
    assert rel_l2(dx1[:, idx] - dx0[:, idx], want_dx - dx0[:, idx]) < 1e-4
    assert rel_l2(p1[:, idx], want_p) < 1e-4
