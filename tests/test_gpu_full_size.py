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
