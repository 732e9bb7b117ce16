"""Langevin phi^4 (the paper's Sec. 2 example) on the GPU against the oracle.
The noise is Philox-2x64-10 + Box-Muller computed independently on each side
from the generator's definition, so the two trajectories coincide."""
import numpy as np
import pytest

import oracle as o
from paper_2607_24908_gb300 import tl as T
from paper_2607_24908_gb300.workloads import plane_wave, white_noise_state

pytestmark = pytest.mark.gpu


def gpu_langevin(N, dtype, phi0, n_calls, steps, dt, lam, m2, noise, seed, kIR=0.5):
    npd = np.float32 if dtype == "f32" else np.float64
    with T.Lattice(N, kIR, 1, dtype) as lat:
        lat.set_state(phi0[None].astype(npd), np.zeros((1, N, N, N), npd))
        for _ in range(n_calls):
            lat.langevin(steps // n_calls, dt, lam, m2, noise, seed)
        return lat.get(0, 0)


@pytest.mark.parametrize("dtype,N,tol", [("f64", 24, 1e-12), ("f32", 40, 1e-5), ("f64", 36, 1e-12)])
def test_langevin_matches_oracle(dtype, N, tol):
    dt, steps, lam, m2, noise, seed = 0.01, 100, 1.0, 0.5, 1.0, 2024
    phi0, _ = white_noise_state(N, 1, seed=N, phi0=(0.5,), sigma_phi=0.2)
    npd = np.float32 if dtype == "f32" else np.float64
    phi0 = phi0[0].astype(npd).astype(np.float64)
    g = gpu_langevin(N, dtype, phi0, 1, steps, dt, lam, m2, noise, seed)
    ref = o.langevin_run(N, 0.5, phi0, dt, steps, lam, m2, noise, seed)
    assert np.max(np.abs(g - ref)) / np.max(np.abs(ref)) < tol


def test_langevin_split_calls_are_bitwise_one_call_and_noiseless_closed_form():
    N, dt = 32, 0.01
    phi0, _ = white_noise_state(N, 1, seed=1, phi0=(0.3,), sigma_phi=0.1)
    a = gpu_langevin(N, "f64", phi0[0], 1, 60, dt, 1.0, 0.2, 0.7, 99)
    b = gpu_langevin(N, "f64", phi0[0], 3, 60, dt, 1.0, 0.2, 0.7, 99)
    assert np.array_equal(a, b)
    p = o.Params(N=N, kIR=0.5)
    w2 = 0.5 + sum((2.0 / p.dx * np.sin(p.kIR * c * p.dx / 2.0)) ** 2 for c in (1, 2, 3))
    pw = plane_wave(N, (1, 2, 3))
    g = gpu_langevin(N, "f64", pw, 1, 50, 0.02, 0.0, 0.5, 0.0, 1)
    assert np.max(np.abs(g - pw * (1.0 - 0.02 * w2) ** 50)) < 1e-13
