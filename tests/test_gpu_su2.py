"""SU(2) Yang-Mills (the paper's Sec. 4 benchmark workload) on the GPU
against the FP64 oracle, plus Gauss's law and energy conservation on the
device."""
import numpy as np
import pytest

import oracle.su2 as Y
from paper_2607_24908_gb300 import tl as T
from paper_2607_24908_gb300.workloads import random_su2_links

pytestmark = pytest.mark.gpu


# N = 8-12 run z-chunks of one plane; N = 40 (FP32: 2-plane chunks, the last ragged) and N = 64
# (FP64: 8-plane chunks) run the kernel's plane pipeline over several planes per CTA.
@pytest.mark.parametrize("dtype,N,tol", [("f64", 8, 1e-12), ("f64", 12, 1e-12), ("f32", 10, 1e-5),
                                         ("f32", 40, 1e-5), ("f64", 64, 1e-12)])
def test_su2_leapfrog_matches_oracle(dtype, N, tol):
    dt, steps = 0.05, 20 if N <= 40 else 6
    U0 = random_su2_links(N, seed=N, amp=0.6)
    rng = np.random.default_rng(1)
    E0 = 0.2 * rng.standard_normal((3, 3, N, N, N))
    npd = np.float32 if dtype == "f32" else np.float64
    U0, E0 = U0.astype(npd), E0.astype(npd)
    with T.SU2(N, dtype) as lat:
        lat.set_state(U0, E0)
        lat.step(steps, dt)
        U, E = lat.get_state()
        m = lat.measure()
    oU, oE = Y.step(U0.astype(np.float64), E0.astype(np.float64), dt, steps)
    assert np.max(np.abs(U - oU)) < tol
    assert np.max(np.abs(E - oE)) / np.max(np.abs(oE)) < tol
    el, mag = Y.electric_energy(oE), Y.plaquette_energy(oU)
    assert abs(m[0] - el) / el < tol * 10 and abs(m[1] - mag) / mag < tol * 10
    G = Y.gauss(oU, oE)
    assert abs(m[2] - np.max(np.sqrt(np.sum(G * G, axis=0)))) < max(tol, 1e-12) * 100


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_su2_large_rotation_angles_match_oracle(dtype, tol):
    """dt = 0.25 with |e| ~ 2.4: per-step drift angles dt |e| on both sides of the
    kernel's small-angle cut (series below, sincos above), against the oracle's sincos."""
    N, dt, steps = 8, 0.25, 4
    U0 = random_su2_links(N, seed=3, amp=0.6)
    E0 = 1.5 * np.random.default_rng(2).standard_normal((3, 3, N, N, N))
    theta = dt * np.sqrt(np.sum(E0 * E0, axis=1))
    assert np.mean(theta < 0.25) > 0.02 and np.mean(theta > 0.5) > 0.3
    npd = np.float32 if dtype == "f32" else np.float64
    U0, E0 = U0.astype(npd), E0.astype(npd)
    with T.SU2(N, dtype) as lat:
        lat.set_state(U0, E0)
        lat.step(steps, dt)
        U, E = lat.get_state()
    oU, oE = Y.step(U0.astype(np.float64), E0.astype(np.float64), dt, steps)
    assert np.max(np.abs(U - oU)) < tol
    assert np.max(np.abs(E - oE)) / np.max(np.abs(oE)) < tol


def test_su2_gauss_law_and_energy_on_device():
    """From random links and E = 0, Gauss's law stays at rounding level; the
    energy measured with the leapfrog's half-step E deviates at O(dt), so the
    largest deviation over a fixed time halves with dt."""
    N, T_end = 16, 2.0
    worst = []
    for dt in (0.02, 0.01):
        with T.SU2(N, "f64") as lat:
            lat.init_random(seed=5, amp=0.8)
            U0, E0 = lat.get_state()
            assert np.max(np.abs(E0)) == 0.0
            assert np.max(np.abs(np.sum(U0 * U0, axis=1) - 1.0)) < 1e-14
            m0 = lat.measure()
            assert m0[2] == 0.0 and m0[0] == 0.0 and m0[1] > 0.1
            H0 = m0[0] + m0[1]
            devs = []
            chunk = int(round(0.2 / dt))
            for _ in range(int(round(T_end / 0.2))):
                lat.step(chunk, dt)
                m = lat.measure()
                devs.append(abs(m[0] + m[1] - H0) / H0)
                assert m[2] < 1e-11  # Gauss's law is preserved by both updates
            assert m[0] > 0.01 * m[1]  # energy moved into the electric field
            worst.append(max(devs))
    assert worst[1] < 0.02
    assert 1.6 < worst[0] / worst[1] < 2.5, worst
