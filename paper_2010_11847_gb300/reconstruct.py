"""MAP reconstruction of the initial conditions from a final density field
(Sec. 7.1): Adam on Eq. 12's negative log-posterior

    -log p(w | delta_e) = chi^2(delta_m(w), delta_e) / 2 + w^T w / 2,

with the white noise w as the variable (s = L w, S = L L^dagger, so that
s^dagger S^-1 s = w^T w).  Each iteration is one forward simulation with
checkpoints, the hand-written adjoint, and one fused Adam + prior update,
all in libfpm's kernels.
"""
from __future__ import annotations

import numpy as np

from .autograd import chi2_of_final_density
from .binding import Plan


class Reconstruction:
    def __init__(self, plan: Plan, target_delta, a, w0, sigma: float = 1.0, lr: float = 0.01,
                 betas=(0.9, 0.999), eps: float = 1e-8, order: int = 2):
        import torch
        self.plan, self.target, self.a = plan, target_delta.contiguous(), np.asarray(a, dtype=np.float64)
        self.sigma, self.lr, self.betas, self.eps, self.order = float(sigma), float(lr), betas, float(eps), order
        self.w = w0.detach().clone().contiguous()
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.t = 0

    def step(self) -> float:
        """One Adam iteration; returns -log p at the white noise it started from."""
        w = self.w.detach().requires_grad_(True)
        chi2 = chi2_of_final_density(w, self.target, self.plan, self.a, self.sigma, self.order)
        chi2.backward()
        self.t += 1
        prior = self.plan.adam_step(self.w, w.grad, self.m, self.v, self.t, lr=self.lr, betas=self.betas,
                                    eps=self.eps, gscale=0.5, pscale=1.0)
        return 0.5 * float(chi2.detach()) + prior
