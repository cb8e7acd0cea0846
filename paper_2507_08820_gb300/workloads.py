"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no lattice-Boltzmann arithmetic: it only draws random numbers and
evaluates the macroscopic fields of the flows the paper's tests use (a fluid at rest
and the Taylor-Green vortex). Both the CUDA path and the FP64 oracle take their inputs
from here; each side then builds its own populations from these fields.

Conventions (shared with the C ABI):
  * a periodic box of nx*ny*nz sites, site index s = x + nx*(y + ny*z), x fastest;
  * scalar fields are arrays of shape (N,), vector fields (3, N) (x, y, z rows).

The workloads follow the paper's tests (Sec. III: periodic cubic boxes, rho normalised
to 1, thermal energies of order 1e-4): there is no dataset, every input is drawn here.
"""
from __future__ import annotations

import numpy as np


def generator(seed: int) -> np.random.Generator:
    """The one random source of every synthetic input (PCG64, fixed seed)."""
    return np.random.default_rng(int(seed))


def site_coords(nx: int, ny: int, nz: int):
    """Integer coordinates (x, y, z) of every site, each of shape (N,)."""
    s = np.arange(nx * ny * nz, dtype=np.int64)
    return s % nx, (s // nx) % ny, s // (nx * ny)


def taylor_green_fields(nx: int, ny: int, nz: int, u0: float, rho0: float = 1.0,
                        cs2: float = 1.0 / 3.0):
    """Density and velocity of the 2-D Taylor-Green vortex in the x-y plane.

    u_x = -u0 cos(k x) sin(k y), u_y = u0 sin(k x) cos(k y), u_z = 0 with k = 2 pi / nx
    (nx == ny), and the pressure of the incompressible solution expressed through the
    isothermal equation of state p = cs2 * rho:
    rho = rho0 - rho0 u0^2 (cos 2kx + cos 2ky) / (4 cs2).
    """
    if nx != ny:
        raise ValueError("Taylor-Green workload needs nx == ny")
    x, y, _ = site_coords(nx, ny, nz)
    k = 2.0 * np.pi / nx
    u = np.zeros((3, x.size))
    u[0] = -u0 * np.cos(k * x) * np.sin(k * y)
    u[1] = u0 * np.sin(k * x) * np.cos(k * y)
    rho = rho0 - rho0 * u0 * u0 * (np.cos(2 * k * x) + np.cos(2 * k * y)) / (4.0 * cs2)
    return rho, u


def random_fields(nx: int, ny: int, nz: int, seed: int, drho: float = 1e-2,
                  du: float = 1e-2, rho0: float = 1.0):
    """Uncorrelated random density and velocity per site (uniform perturbations)."""
    g = generator(seed)
    n = nx * ny * nz
    rho = rho0 * (1.0 + drho * g.uniform(-1.0, 1.0, n))
    u = du * g.uniform(-1.0, 1.0, (3, n))
    return rho, u


def population_perturbation(n_sites: int, seed: int, amp: float = 1e-4, q: int = 27):
    """Independent standard normals times amp, shape (q, n_sites): a non-equilibrium
    perturbation added on top of an equilibrium state to exercise every mode."""
    return amp * generator(seed).standard_normal((q, n_sites))


def sample_sites(n_sites: int, n_samples: int, seed: int):
    """Sorted distinct site indices for sampled comparisons at large sizes; the first
    and last site are always included so that both periodic edges are covered."""
    g = generator(seed)
    k = min(n_samples, n_sites)
    s = g.choice(n_sites, size=k, replace=False)
    s = np.unique(np.concatenate([s, [0, n_sites - 1]]))
    return s.astype(np.int64)


def replica_ensemble(n_replicas: int = 64, seed: int = 0):
    """The batched-ensemble workload: independent boxes with edges uniform in
    {16,24,32,48,64,96}, seeds 1..n, kT log-uniform in [1e-5, 1e-3] and tau uniform in
    [0.55, 1.2], all drawn from one host generator with the given seed."""
    g = generator(seed)
    edges = g.choice(np.array([16, 24, 32, 48, 64, 96]), size=n_replicas)
    kts = 10.0 ** g.uniform(-5.0, -3.0, n_replicas)
    taus = g.uniform(0.55, 1.2, n_replicas)
    return [dict(nx=int(e), ny=int(e), nz=int(e), tau=float(t), kT=float(k),
                 rho0=1.0, seed=i + 1) for i, (e, k, t) in enumerate(zip(edges, kts, taus))]
