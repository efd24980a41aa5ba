"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds data only: grid coordinates, sensor sets, right-hand sides
and the parameter table of the synthetic heat-equation Hessians.  It contains
none of the method's arithmetic (no operator, no tree, no sampling), so that
the oracle and the CUDA path can both consume the same inputs without sharing
any computational code.  `workloads.advdiff` generates the second family's
input data (the factor of an advection-diffusion misfit Hessian, from a sparse
solve of its PDE): the operator's data, again none of the hierarchical method.

The workload stands in for the PDE-constrained Hessians of the paper
(Section 4): a 2-D initial-condition inversion for the heat equation on the
unit square, with sensor-limited data (cf. the sensor-count study of
Section 4.2), KD-tree leaves of 64 points (Section 4.2, Appendix A.1) and a
construction tolerance of 1e-6 (Section 4.1).
"""
from __future__ import annotations

import dataclasses

import numpy as np

ADM_WEAK = 0
ADM_STRONG = 1


@dataclasses.dataclass(frozen=True)
class HeatProblem:
    """Parameters of one synthetic heat-equation Hessian H = F O^T O F / sigma^2."""

    n: int                 # grid is n x n interior nodes, N = n*n unknowns
    m: int                 # number of sensor nodes
    kappa: float           # diffusivity
    T: float               # final time
    sigma: float           # noise level
    sensor_seed: int

    @property
    def N(self) -> int:
        return self.n * self.n


@dataclasses.dataclass(frozen=True)
class BuildParams:
    """Construction parameters (tree, admissibility, truncation, probing)."""

    leaf: int
    adm: int
    eta: float
    tol: float
    kmax: int
    q0: int                # initial probe count per level (fixed count when adaptive is False)
    b_inc: int             # probe increment of the adaptive range finder
    q_max: int             # probe cap per level
    adaptive: bool
    seed: int              # seed of the counter-based probe generator


def grid_coords(n: int) -> np.ndarray:
    """Interior nodes (i h, j h), i, j = 1..n, h = 1/(n+1), row-major index p = (i-1) n + (j-1)."""
    h = 1.0 / (n + 1)
    i, j = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    return np.ascontiguousarray(np.stack([i.ravel() * h, j.ravel() * h], axis=1).astype(np.float64))


def sensor_indices(N: int, m: int, seed: int) -> np.ndarray:
    """m distinct grid nodes drawn uniformly without replacement (sorted)."""
    if not 0 <= m <= N:
        raise ValueError("sensor count out of range")
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N, size=m, replace=False)).astype(np.int64)


def sensor_mask(N: int, m: int, seed: int) -> np.ndarray:
    mask = np.zeros(N, dtype=np.float64)
    mask[sensor_indices(N, m, seed)] = 1.0
    return mask


def rhs(N: int, nrhs: int, seed: int, dtype=np.float64) -> np.ndarray:
    """N(0,1) right-hand sides, column-major (Fortran) N x nrhs."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nrhs, N)).T
    return np.asfortranarray(x.astype(dtype))


# ---------------------------------------------------------------------------
# Workload table.  Sizes follow the configurations the library is measured on.
# ---------------------------------------------------------------------------

SMALL_N32 = dict(
    name="heat2d_n32_weak_fixed64",
    problem=HeatProblem(n=32, m=200, kappa=0.01, T=0.5, sigma=0.01, sensor_seed=1001),
    build=BuildParams(leaf=32, adm=ADM_WEAK, eta=0.7, tol=1e-6, kmax=16, q0=64, b_inc=16,
                      q_max=64, adaptive=False, seed=7),
    nrhs=(16,),
    rhs_seed=11,
)

MEDIUM_N256 = dict(
    name="heat2d_n256_strong_adaptive",
    problem=HeatProblem(n=256, m=4096, kappa=0.01, T=0.5, sigma=0.01, sensor_seed=1002),
    build=BuildParams(leaf=64, adm=ADM_STRONG, eta=0.7, tol=1e-6, kmax=32, q0=32, b_inc=16,
                      q_max=256, adaptive=True, seed=7),
    nrhs=(1, 32, 256),
    rhs_seed=12,
)

LARGE_N512 = dict(
    name="heat2d_n512_strong_adaptive",
    problem=HeatProblem(n=512, m=16384, kappa=0.005, T=0.5, sigma=0.01, sensor_seed=1003),
    build=BuildParams(leaf=64, adm=ADM_STRONG, eta=0.7, tol=1e-6, kmax=48, q0=32, b_inc=16,
                      q_max=256, adaptive=True, seed=7),
    nrhs=(1024,),
    rhs_seed=13,
)


def batch_problems(count: int = 64, seed: int = 2024, n_lo: int = 64, n_hi: int = 256):
    """Uneven batch of heat Hessians: n ~ U{n_lo..n_hi}, kappa ~ U[0.002, 0.05], m/N ~ U[0.05, 0.20]."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        kappa = float(rng.uniform(0.002, 0.05))
        frac = float(rng.uniform(0.05, 0.20))
        m = max(1, int(round(frac * n * n)))
        out.append(HeatProblem(n=n, m=m, kappa=kappa, T=0.5, sigma=0.01, sensor_seed=5000 + b))
    return out
