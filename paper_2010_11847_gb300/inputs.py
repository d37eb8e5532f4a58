"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds no arithmetic of the particle-mesh method: it only draws
the random numbers the method consumes (the white-noise field of the initial
conditions, Algorithm 4's first step) and spells out the workload
configurations.  Both sides receive the same arrays as inputs.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

# Planck-2015 parameters; omega_b and t_cmb are not stated by the paper and
# complete the set that matches the given omega_m, h, n_s and sigma8.
COSMO_DEFAULT = dict(omega_m=0.3075, omega_b=0.0486, h=0.6774, n_s=0.9667,
                     sigma8=0.8159, t_cmb=2.7255)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One simulation: np^3 particles on an nc^3 mesh in a periodic box."""
    name: str
    np_: int
    nc: int
    box: float              # Mpc/h
    nsteps: int
    a0: float = 0.1
    a1: float = 1.0
    seed: int = 1
    omega_m: float = COSMO_DEFAULT["omega_m"]
    sigma8: float = COSMO_DEFAULT["sigma8"]

    @property
    def cosmo(self) -> dict:
        c = dict(COSMO_DEFAULT)
        c["omega_m"] = self.omega_m
        c["sigma8"] = self.sigma8
        return c

    def stages(self) -> np.ndarray:
        """Scale factors of the KDK steps, linear in a from a0 to a1."""
        return np.linspace(self.a0, self.a1, self.nsteps + 1)


SMALL = Workload("pm_32p_32m_100mpc_5step", 32, 32, 100.0, 5)
MEDIUM = Workload("pm_128p_256m_400mpc_10step", 128, 256, 400.0, 10)
LARGE = Workload("pm_512p_512m_1000mpc_40step", 512, 512, 1000.0, 40)
# 1/8 of LARGE at the same cell size and particle density (profiling case)
LARGE_EIGHTH = Workload("pm_256p_256m_500mpc_40step", 256, 256, 500.0, 40)
DIFFERENTIABLE = Workload("pm_128p_128m_400mpc_5step_adjoint", 128, 128, 400.0, 5)
# accuracy configuration of the mesh / pyramid comparison (1LPT initial conditions)
ACCURACY_10STEP = Workload("pm_128p_128m_400mpc_10step_1lpt", 128, 128, 400.0, 10)


def batched_workloads(seed0: int = 100) -> List[Workload]:
    """64 independent simulations: meshes 32/64/96/128 (16 each), particles
    equal to mesh, boxes 100-400 Mpc/h, omega_m in [0.25, 0.35], sigma8 in
    [0.7, 0.9], distinct seeds, 10 KDK steps from a=0.1."""
    rng = np.random.default_rng(seed0)
    out = []
    sizes = [32, 64, 96, 128]
    for j in range(64):
        n = sizes[j % 4]
        box = float(100.0 * n / 32.0)            # 100, 200, 300, 400 Mpc/h
        om = float(rng.uniform(0.25, 0.35))
        s8 = float(rng.uniform(0.7, 0.9))
        out.append(Workload(f"batch{j:02d}_{n}", n, n, box, 10, seed=seed0 + 1 + j,
                            omega_m=om, sigma8=s8))
    return out


def white_noise(n: int, seed: int) -> np.ndarray:
    """Standard-normal white noise on an n^3 grid, float32, C order [x][y][z]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n, n, n), dtype=np.float32)


def random_displacements(np_: int, scale: float, seed: int) -> np.ndarray:
    """Smooth-free random displacements dx[3][np^3] (float32, mesh cells) for
    unit tests of paint/readout that need no initial-condition physics."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.standard_normal((3, np_ ** 3), dtype=np.float32) * np.float32(scale))


def random_field(n: int, seed: int) -> np.ndarray:
    """A generic float32 real field on an n^3 grid (uniform in [-1, 1))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.random((n, n, n), dtype=np.float32) * 2 - 1).astype(np.float32)
