"""Multi-grid pyramid force (Algorithms 2-3) through the C ABI against the
oracle's ``pyramid_force``: force meshes relative L2 <= 1e-5 for coarse and
block meshes on both FFT paths (power-of-two potential form, shared-memory
passes) under the four readings (band-pass per padded block or on the
assembled mesh, coarse operator matched to the fine mesh or in coarse
cells), KDK positions and momenta <= 1e-4, the reading and off switches,
and the refusals (bad sizes, adjoint, batch)."""
import numpy as np
import pytest

from oracle import fpm_oracle as O
from paper_2010_11847_gb300 import inputs

pytestmark = pytest.mark.gpu

COSMO = dict(inputs.COSMO_DEFAULT)
OM = COSMO["omega_m"]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_mod(cuda):
    import torch
    return torch


def plan(np_, nc, box=100.0):
    from paper_2010_11847_gb300.binding import Plan
    return Plan(np_, nc, box, COSMO)


def dev(x, torch):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# (nc, levels, split, halo): coarse mesh nc >> levels, blocks nc/split + 2 halo
CASES = [(64, 2, 2, 16), (128, 2, 2, 16), (64, 1, 4, 8), (96, 1, 2, 24), (128, 2, 4, 16)]


READINGS = [("block", "matched"), ("global", "coarse"), ("block", "coarse"), ("global", "matched")]


@pytest.mark.parametrize("reading", READINGS)
@pytest.mark.parametrize("nc,levels,split,halo", CASES)
def test_pyramid_force_matches_oracle(torch_mod, nc, levels, split, halo, reading):
    torch = torch_mod
    pl = plan(nc // 2, nc)
    pl.set_pyramid_reading(*reading)
    pl.set_pyramid(levels, split, halo)
    rho = (1.0 + 0.5 * inputs.random_field(nc, 500 + nc)).astype(np.float32)
    F = pl.force(dev(rho, torch)).cpu().numpy()
    torch.cuda.synchronize()
    assert pl.status() == 0
    ref = O.pyramid_force(rho.astype(np.float64), OM, levels, split, halo, bandpass=reading[0],
                          coarse_kernel=reading[1])
    for d in range(3):
        assert rel_l2(F[d], ref[d]) < 1e-5, (d, rel_l2(F[d], ref[d]))


def test_pyramid_kdk_matches_oracle(torch_mod):
    """Four KDK steps from the oracle's 2LPT at a = 0.1, 32^3 on 64^3, two
    levels, 2^3 blocks with a 16-cell halo (interleaved force mesh)."""
    torch = torch_mod
    n, nc, box = 32, 64, 100.0
    stages = np.linspace(0.1, 0.5, 5)
    lk = O.linear_field(inputs.white_noise(n, 23), box, COSMO)
    dx0, p0 = O.lpt(lk, nc, stages[0], COSMO)
    dx0 = dx0.astype(np.float32)
    p0 = p0.astype(np.float32)
    pyr = dict(levels=2, split=2, halo=16)
    rdx, rp = O.kdk(dx0, p0, stages, n, nc, OM, pyramid=pyr)
    pl = plan(n, nc, box)
    pl.set_pyramid(**pyr)
    dx, p = dev(dx0, torch), dev(p0, torch)
    pl.kdk(dx, p, stages)
    torch.cuda.synchronize()
    assert pl.status() == 0
    assert rel_l2(dx.cpu().numpy(), rdx) < 1e-4
    assert rel_l2(p.cpu().numpy(), rp) < 1e-4


def test_pyramid_reading_switch_rebuilds_the_pyramid(torch_mod):
    """Changing the reading of a set pyramid rebuilds it: the force follows
    the new reading, and switching back gives the first bits again."""
    torch = torch_mod
    nc = 64
    rho = dev((1.0 + 0.5 * inputs.random_field(nc, 530)).astype(np.float32), torch)
    pl = plan(32, nc)
    pl.set_pyramid(2, 2, 16)
    a = pl.force(rho).clone()
    pl.set_pyramid_reading("global", "coarse")
    b = pl.force(rho).clone()
    pl.set_pyramid_reading("block", "matched")
    c = pl.force(rho)
    torch.cuda.synchronize()
    assert not torch.equal(a, b) and torch.equal(a, c)
    ref = O.pyramid_force(rho.cpu().numpy().astype(np.float64), OM, 2, 2, 16, bandpass="global", coarse_kernel="coarse")
    assert rel_l2(b.cpu().numpy(), ref) < 1e-5


def test_switching_the_pyramid_off_gives_the_default_bits(torch_mod):
    torch = torch_mod
    nc = 64
    rho = dev((1.0 + 0.5 * inputs.random_field(nc, 520)).astype(np.float32), torch)
    ref = plan(32, nc).force(rho)
    pl = plan(32, nc)
    pl.set_pyramid(2, 2, 16)
    other = pl.force(rho)
    pl.set_pyramid(0)
    again = pl.force(rho)
    torch.cuda.synchronize()
    assert not torch.equal(other, ref)
    assert torch.equal(again, ref)


def test_pyramid_refusals(torch_mod):
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Batch, FpmError, FPM_EINVAL, FPM_ENOTIMPL
    pl = plan(32, 64)
    for bad in [(3, 2, 16), (2, 3, 16), (2, 2, 5), (1, 2, -1)]:
        with pytest.raises(FpmError) as e:
            pl.set_pyramid(*bad)
        assert e.value.code == FPM_EINVAL
    pl.set_pyramid(2, 2, 16)
    gF = dev(np.zeros((3, 64, 64, 64), np.float32), torch)
    with pytest.raises(FpmError) as e:
        pl.force_adj(gF)
    assert e.value.code == FPM_ENOTIMPL
    bp = plan(64, 64)
    bp.set_pyramid(2, 2, 16)
    with pytest.raises(FpmError) as e:
        Batch([bp])
    assert e.value.code == FPM_ENOTIMPL
