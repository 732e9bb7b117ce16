"""Seeded synthetic inputs and the named workloads.

This module holds no arithmetic of the method: it only draws seeded random
arrays and names the lattice sizes and parameters of the workloads.  It is
the one place both the CUDA path's tests and the oracle get their inputs from.

Input recipe (states fed through ``set_state``): the paper's phi^4 benchmark
starts from Gaussian white noise (Sec. 4); here every field is a homogeneous
value plus independent N(0, sigma^2) noise per site, momenta likewise.
``init_fluctuations`` states (Gaussian random fields with power A/(2 omega_k))
are drawn inside the library and the oracle from a seed, not here.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Sequence, Tuple

import numpy as np


def white_noise_state(N: int, nf: int, seed: int, phi0: Sequence[float] = (1.0, 0.0, 0.0),
                      sigma_phi: float = 1e-2, pi0: Sequence[float] = (0.0, 0.0, 0.0),
                      sigma_pi: float = 1e-2, dtype=np.float64) -> Tuple[np.ndarray, np.ndarray]:
    """(phi, pi), each shaped [nf, N, N, N] (z, y, x; x fastest), in ``dtype``."""
    rng = np.random.default_rng(seed)
    phi = np.empty((nf, N, N, N), dtype=np.float64)
    pi = np.empty((nf, N, N, N), dtype=np.float64)
    for f in range(nf):
        phi[f] = phi0[f] + sigma_phi * rng.standard_normal((N, N, N))
        pi[f] = pi0[f] + sigma_pi * rng.standard_normal((N, N, N))
    return phi.astype(dtype), pi.astype(dtype)


def plane_wave(N: int, n: Sequence[int], amp: float = 1.0) -> np.ndarray:
    """amp * cos(2 pi (n . i)/N) on the [z, y, x] grid: one Fourier mode."""
    i = np.arange(N)
    iz, iy, ix = np.meshgrid(i, i, i, indexing="ij")
    return amp * np.cos(2.0 * np.pi * (n[0] * ix + n[1] * iy + n[2] * iz) / N)


def sample_sites(N: int, count: int, seed: int) -> np.ndarray:
    """``count`` distinct random site coordinates [count, 3] as (z, y, x)."""
    rng = np.random.default_rng(seed)
    flat = rng.choice(N ** 3, size=min(count, N ** 3), replace=False)
    z, rem = np.divmod(flat, N * N)
    y, x = np.divmod(rem, N)
    return np.stack([z, y, x], axis=1)


def random_su2_links(N: int, seed: int, amp: float) -> np.ndarray:
    """Random SU(2) links as unit quaternions, component-major [3, 4, N, N, N]
    (direction, component, z, y, x): q = (1, amp xi1, amp xi2, amp xi3) with xi
    standard normal, divided by its norm."""
    rng = np.random.default_rng(seed)
    q = np.empty((3, 4, N, N, N))
    q[:, 0] = 1.0
    q[:, 1:] = amp * rng.standard_normal((3, 3, N, N, N))
    return q / np.sqrt(np.sum(q * q, axis=1, keepdims=True))


def random_su2_gauge(N: int, seed: int) -> np.ndarray:
    """A random SU(2) element per site as a unit quaternion [4, N, N, N]."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((4, N, N, N))
    return q / np.sqrt(np.sum(q * q, axis=0, keepdims=True))


@dataclass(frozen=True)
class Workload:
    """One named synthetic workload (sizes and model parameters only)."""
    name: str
    N: int
    nf: int
    kIR: float
    expanding: bool
    alpha: float
    lam: float
    q: float
    m2: Tuple[float, float, float]
    dt: float
    steps: int
    integrator: str               # "leapfrog" | "verlet" | "yoshida4"
    dtype: str                    # "f64" | "f32"
    A: float = 1e-10
    meff2: Tuple[float, float, float] = (3.0, 0.0, 0.0)
    phi0: Tuple[float, float, float] = (1.0, 0.0, 0.0)
    seed: int = 1
    fstar_over_mp: float = 1.0


# phi^4 in a static box: 32^3, kIR = 0.5, dt = 0.05, 400 leapfrog steps, FP64.
PHI4_STATIC_32 = Workload("phi4-static-32^3-f64-leapfrog", 32, 1, 0.5, False, 0.0, 1.0, 0.0,
                          (0.0, 0.0, 0.0), 0.05, 400, "leapfrog", "f64")
# free field m = 1 on the same box (single plane wave, exact discrete solution)
FREE_STATIC_32 = Workload("free-static-32^3-f64-leapfrog", 32, 1, 0.5, False, 0.0, 0.0, 0.0,
                          (1.0, 0.0, 0.0), 0.05, 400, "leapfrog", "f64")
# phi^4 through parametric resonance, expanding (alpha = 1): 256^3, VV, dt = 0.01
PHI4_EXPANDING_256 = Workload("phi4-expanding-256^3-verlet", 256, 1, 0.1, True, 1.0, 1.0, 0.0,
                              (0.0, 0.0, 0.0), 0.01, 3000, "verlet", "f64")
# two fields phi^4 + (q/2) phi^2 chi^2, q = 100: 1024^3, Yoshida-4, dt = 0.005, FP32
TWO_FIELD_1024 = Workload("phi4-chi-q100-expanding-1024^3-f32-yoshida4", 1024, 2, 0.05, True, 1.0,
                          1.0, 100.0, (0.0, 0.0, 0.0), 0.005, 500, "yoshida4", "f32",
                          meff2=(3.0, 100.0, 0.0))

WORKLOADS = {w.name: w for w in (PHI4_STATIC_32, FREE_STATIC_32, PHI4_EXPANDING_256, TWO_FIELD_1024)}
