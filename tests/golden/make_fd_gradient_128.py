"""Write fd_gradient_128.json: central finite differences of chi^2 with
respect to the white noise at 32 voxels of the differentiable configuration
(128^3 particles on 128^3 cells, 400 Mpc/h, 2LPT at a = 0.1, 5 KDK steps),
at steps eps = 1e-3 and 1e-4, computed by the FP64 oracle alone with FP64
positions (no rounding of the positions to float32 anywhere, so the
differences carry no rounding noise).

chi^2 = sum (delta_final - delta_target)^2 (sigma = 1), delta_target the
float32 final density contrast of the oracle run from the next seed: the
loss of the differentiable configuration.  The loss is piecewise smooth (a
CIC weight's derivative jumps where a particle crosses a cell face), so
the differences at eps = 1e-3 still carry the kinks that particles cross
within the step; at 1e-4 they have converged to the gradient.  The GPU
adjoint is compared to these stored differences.

Usage: python tests/golden/make_fd_gradient_128.py [workers]  (about 130
oracle simulations at 128^3, spread over worker processes).
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
EPS = (1e-3, 1e-4)
NVOX = 32
VOXEL_SEED = 2024

_state = {}


def _setup(fft_threads):
    sys.path.insert(0, ROOT)
    from oracle import fpm_oracle as O
    from paper_2010_11847_gb300 import inputs
    O.FFT_WORKERS = fft_threads
    O.POSITIONS_FP32 = False      # FP64 positions in every paint and readout
    wl = inputs.DIFFERENTIABLE
    stages = wl.stages()
    ref_t = O.simulate(inputs.white_noise(wl.np_, wl.seed + 1), wl.nc, wl.box, wl.cosmo, stages)
    _state.update(O=O, wl=wl, stages=stages, w=inputs.white_noise(wl.np_, wl.seed).astype(np.float64),
                  target=(ref_t["rho"] - 1.0).astype(np.float32).astype(np.float64))


def _loss(wv):
    O, wl, stages = _state["O"], _state["wl"], _state["stages"]
    lk = O.linear_field(wv, wl.box, wl.cosmo)
    dx0, p0 = O.lpt(lk, wl.nc, stages[0], wl.cosmo)
    dx, _ = O.kdk(dx0, p0, stages, wl.np_, wl.nc, wl.cosmo["omega_m"], round_to_float32=False)
    return O.chi2(O.paint(dx, wl.np_, wl.nc), _state["target"])[0]


def _job(args):
    i, eps = args
    w = _state["w"]
    e = np.zeros(w.size)
    e[i] = eps
    e = e.reshape(w.shape)
    return i, eps, (_loss(w + e) - _loss(w - e)) / (2 * eps)


def _base_loss(_):
    return _loss(_state["w"])


def main():
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else 4
    n = 128 ** 3
    idx = [int(i) for i in np.random.default_rng(VOXEL_SEED).choice(n, size=NVOX, replace=False)]
    threads = max(1, (os.cpu_count() or 4) // workers)
    t0 = time.time()
    with mp.get_context("spawn").Pool(workers, initializer=_setup, initargs=(threads,)) as pool:
        L0 = pool.map(_base_loss, [0])[0]
        res = pool.map(_job, [(i, eps) for eps in EPS for i in idx])
    fd = {eps: [v for (i, e, v) in res if e == eps] for eps in EPS}
    out = {"config": "pm_128p_128m_400mpc_5step_adjoint", "voxel_seed": VOXEL_SEED, "voxels": idx, "loss": L0,
           "eps": EPS[0], "fd": fd[EPS[0]], "eps_converged": EPS[1], "fd_converged": fd[EPS[1]],
           "made_by": "tests/golden/make_fd_gradient_128.py (FP64 oracle, FP64 positions)"}
    with open(os.path.join(HERE, "fd_gradient_128.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(f"done in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
