"""Pins of the SU(2) Yang-Mills oracle (Sec. 4 benchmark workload): exact
Gauss-law preservation, O(dt^2) energy conservation, gauge covariance,
unitarity, and the abelian (compact U(1)) reduction written independently
with angles."""
import numpy as np

import oracle.su2 as Y
from paper_2607_24908_gb300.workloads import random_su2_gauge, random_su2_links


def hamiltonian_integer_time(U, E_half, dt):
    """E at the integer time from the half-step field: E_n = E_{n-1/2} + dt/2 F(U_n)."""
    En = E_half + 0.5 * dt * Y.force(U)
    return Y.electric_energy(En) + Y.plaquette_energy(U)


def test_gauss_law_preserved_exactly():
    U = random_su2_links(6, seed=1, amp=0.6)
    E = np.zeros((3, 3, 6, 6, 6))
    assert np.max(np.abs(Y.gauss(U, E))) == 0.0
    U1, E1 = Y.step(U, E, 0.05, 60)
    assert np.max(np.abs(E1)) > 0.1
    assert np.max(np.abs(Y.gauss(U1, E1))) < 1e-12


def test_energy_conserved_second_order():
    U = random_su2_links(6, seed=2, amp=0.5)
    E0 = np.zeros((3, 3, 6, 6, 6))
    devs = []
    for dt in (0.04, 0.02):
        # start the half-step field from E_0 = 0: E_{-1/2} = -dt/2 F(U_0)
        U, E = U.copy(), E0 - 0.5 * dt * Y.force(U)
        H0 = hamiltonian_integer_time(U, E, dt)
        dev = 0.0
        Uc, Ec = U, E
        for _ in range(int(round(2.0 / dt))):
            Uc, Ec = Y.step(Uc, Ec, dt)
            dev = max(dev, abs(hamiltonian_integer_time(Uc, Ec, dt) - H0) / H0)
        devs.append(dev)
        U = random_su2_links(6, seed=2, amp=0.5)
    assert devs[1] < 1e-3
    assert 3.3 < devs[0] / devs[1] < 4.7, devs


def test_gauge_covariance():
    N, dt = 5, 0.05
    U = random_su2_links(N, seed=3, amp=0.7)
    E = Y.force(U) * 0.3  # any E; covariance does not need Gauss's law
    Om = random_su2_gauge(N, seed=4)

    def transform(U, E):
        Ut = np.stack([Y.qmul(Y.qmul(Om, U[i]), Y.qadj(Y.shift(Om, i, 1))) for i in range(3)])
        Et = []
        for i in range(3):
            Eq = np.concatenate([np.zeros((1, N, N, N)), E[i]])
            Et.append(Y.qmul(Y.qmul(Om, Eq), Y.qadj(Om))[1:])
        return Ut, np.stack(Et)

    a = transform(*Y.step(U, E, dt, 20))
    b = Y.step(*transform(U, E), dt, 20)
    assert np.max(np.abs(a[0] - b[0])) < 1e-12 and np.max(np.abs(a[1] - b[1])) < 1e-12
    assert abs(Y.plaquette_energy(U) - Y.plaquette_energy(transform(U, E)[0])) < 1e-13


def test_links_stay_unitary():
    U = random_su2_links(6, seed=5, amp=1.0)
    U1, _ = Y.step(U, np.zeros((3, 3, 6, 6, 6)), 0.05, 100)
    assert np.max(np.abs(np.sum(U1 * U1, axis=1) - 1.0)) < 1e-13


def test_abelian_reduction_is_compact_u1():
    """Links exp(i theta s3), fields along s3: the dynamics is compact U(1),
    e_i -= 2 dt sum_j [sin F_ij(x) - sin F_ij(x - j)], theta_i += dt e_i, with
    F_ij(x) = theta_i(x) + theta_j(x+i) - theta_i(x+j) - theta_j(x)."""
    N, dt, steps = 6, 0.05, 40
    rng = np.random.default_rng(6)
    th = 0.8 * rng.standard_normal((3, N, N, N))
    e = 0.3 * rng.standard_normal((3, N, N, N))
    sh = lambda f, d, s: np.roll(f, -s, axis=f.ndim - 1 - d)
    U = np.zeros((3, 4, N, N, N))
    U[:, 0] = np.cos(th)
    U[:, 3] = np.sin(th)
    E = np.zeros((3, 3, N, N, N))
    E[:, 2] = e
    U1, E1 = Y.step(U, E, dt, steps)
    for _ in range(steps):
        F = {(i, j): th[i] + sh(th[j], i, 1) - sh(th[i], j, 1) - th[j] for i in range(3) for j in range(3) if i != j}
        for i in range(3):
            e[i] = e[i] - 2.0 * dt * sum(np.sin(F[i, j]) - sh(np.sin(F[i, j]), j, -1) for j in range(3) if j != i)
        th = th + dt * e
    assert np.max(np.abs(E1[:, 2] - e)) < 1e-12 and np.max(np.abs(E1[:, :2])) < 1e-14
    assert np.max(np.abs(U1[:, 0] - np.cos(th))) < 1e-12 and np.max(np.abs(U1[:, 3] - np.sin(th))) < 1e-12
