"""Reconstruction (Sec. 7.1, Eq. 12) on the GPU against the oracle: the fused
Adam + prior kernel element by element, and three Adam iterations of the
whole posterior (forward, adjoint, update) on a small problem."""
import numpy as np
import pytest

from oracle import fpm_oracle as O
from paper_2010_11847_gb300 import inputs

pytestmark = pytest.mark.gpu

COSMO = dict(inputs.COSMO_DEFAULT)


@pytest.fixture(scope="module")
def torch_mod(cuda):
    import torch
    return torch


def test_adam_kernel_matches_oracle(torch_mod):
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Plan
    pl = Plan(16, 16, 100.0, COSMO)
    r = np.random.default_rng(5)
    n = 100_003                                   # ragged against the block size
    x, g = r.standard_normal(n).astype(np.float32), r.standard_normal(n).astype(np.float32)
    m = (0.1 * r.standard_normal(n)).astype(np.float32)
    v = (0.01 * r.random(n) + 1e-4).astype(np.float32)
    X, G, Mm, V = (torch.from_numpy(a.copy()).cuda() for a in (x, g, m, v))
    prior = pl.adam_step(X, G, Mm, V, 3, lr=0.01, gscale=0.5, pscale=1.0)
    rx, rm, rv = O.adam_step(x.astype(np.float64), 0.5 * g.astype(np.float64) + x.astype(np.float64), m, v, 3)
    assert prior == pytest.approx(0.5 * float((x.astype(np.float64) ** 2).sum()), rel=1e-12)
    np.testing.assert_allclose(Mm.cpu().numpy(), rm, rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(V.cpu().numpy(), rv, rtol=2e-6, atol=1e-9)
    np.testing.assert_allclose(X.cpu().numpy(), rx, rtol=0, atol=2e-6)


def test_three_iterations_match_oracle(torch_mod):
    torch = torch_mod
    from paper_2010_11847_gb300.binding import Plan
    from paper_2010_11847_gb300.reconstruct import Reconstruction
    n, box = 32, 100.0
    a = np.linspace(0.1, 1.0, 4)
    truth = O.simulate(inputs.white_noise(n, 11), n, box, COSMO, a)
    target = (truth["rho"] - 1.0).astype(np.float32)
    w0 = (0.5 * inputs.white_noise(n, 12)).astype(np.float32)
    pl = Plan(n, n, box, COSMO)
    rec = Reconstruction(pl, torch.from_numpy(target).cuda(), a, torch.from_numpy(w0).cuda(), sigma=1.0, lr=0.01)
    w, m, v = w0.astype(np.float64), np.zeros(w0.shape), np.zeros(w0.shape)
    for t in range(1, 4):
        got = rec.step()
        ref, g = O.posterior_and_grad(w.astype(np.float32), target.astype(np.float64), n, box, COSMO, a)
        w, m, v = O.adam_step(w, g, m, v, t)
        assert got == pytest.approx(ref, rel=1e-3), t
    wg = rec.w.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(wg - w) / np.linalg.norm(w) < 1e-3
