"""Oracle for classical SU(2) Yang-Mills on the lattice in temporal gauge
(the paper's benchmark workload, Sec. 4): plain numpy, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Representation: an SU(2) link U = u0 + i (u1 s1 + u2 s2 + u3 s3) is the unit
quaternion (u0, u1, u2, u3); an electric field E = i (e1 s1 + e2 s2 + e3 s3)
is the 3-vector e.  Products: (a0 + i a.s)(b0 + i b.s) = (a0 b0 - a.b) +
i (a0 b + b0 a - a x b).s; the adjoint negates the vector part.  Arrays are
component-major: U[i, c, z, y, x] (i = direction, c = 0..3), E[i, c, z, y, x].

Dynamics (lattice units, dx = 1), with H = sum_{x,i} |e_i|^2/2 +
sum_{x, i<j} 2 (1 - Re P_ij(x)), P_ij(x) = U_i(x) U_j(x+i) U_i(x+j)^+ U_j(x)^+:
  kick   e_i(x) <- e_i(x) - 2 dt sum_{j != i} Im[U_i(x) S_ij(x)]
         S_ij(x) = U_j(x+i) U_i(x+j)^+ U_j(x)^+ + U_j(x+i-j)^+ U_i(x-j)^+ U_j(x-j)
         (the paper's E+ = E - dt sum_j (P_ij - P_ij^+): for SU(2),
         P - P^+ = 2 i Im P);
  drift  U_i(x) <- exp(dt E_i(x)) U_i(x),  exp(i e.s dt) = cos(dt|e|) + i sin(dt|e|) e/|e|.
Leapfrog as in the paper: each step a kick then a drift (E at half steps).
Gauss law G(x) = sum_i [E_i(x) - U_i(x-i)^+ E_i(x-i) U_i(x-i)] is preserved
by both updates.
"""
from __future__ import annotations

import numpy as np


def qmul(a, b):
    """Quaternion (SU(2)) product of arrays shaped [4, ...]."""
    a0, av = a[0], a[1:]
    b0, bv = b[0], b[1:]
    r0 = a0 * b0 - np.sum(av * bv, axis=0)
    rv = a0 * bv + b0 * av - np.cross(av, bv, axis=0)
    return np.concatenate([r0[None], rv], axis=0)


def qadj(a):
    return np.concatenate([a[:1], -a[1:]], axis=0)


def shift(f, d, s):
    """f(x + s d-hat) on the periodic grid; d = 0, 1, 2 is x, y, z (array axes -1, -2, -3)."""
    return np.roll(f, -s, axis=f.ndim - 1 - d)


def staples(U, i, j):
    Ui, Uj = U[i], U[j]
    fwd = qmul(qmul(shift(Uj, i, 1), qadj(shift(Ui, j, 1))), qadj(Uj))
    Ujm = shift(Uj, j, -1)
    bwd = qmul(qmul(qadj(shift(Ujm, i, 1)), qadj(shift(Ui, j, -1))), Ujm)
    return fwd + bwd


def force(U):
    """-2 sum_{j != i} Im[U_i S_ij] for every link: array [3, 3, ...]."""
    F = np.zeros((3, 3) + U.shape[2:])
    for i in range(3):
        S = sum(staples(U, i, j) for j in range(3) if j != i)
        F[i] = -2.0 * qmul(U[i], S)[1:]
    return F


def qexp(e, dt):
    """exp(i dt e.s) for e shaped [3, ...]."""
    n = np.sqrt(np.sum(e * e, axis=0))
    th = dt * n
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.where(n > 0, np.sin(th) / np.where(n > 0, n, 1.0), dt)
    return np.concatenate([np.cos(th)[None], s * e], axis=0)


def step(U, E, dt, n=1):
    """n leapfrog steps (kick, then drift) of copies of (U, E)."""
    U = np.array(U, dtype=np.float64, copy=True)
    E = np.array(E, dtype=np.float64, copy=True)
    for _ in range(n):
        E = E + dt * force(U)
        for i in range(3):
            U[i] = qmul(qexp(E[i], dt), U[i])
    return U, E


def plaquette_energy(U):
    """sum over sites and planes of 2 (1 - Re P_ij), per site (mean)."""
    tot = 0.0
    for i in range(3):
        for j in range(i + 1, 3):
            P = qmul(qmul(qmul(U[i], shift(U[j], i, 1)), qadj(shift(U[i], j, 1))), qadj(U[j]))
            tot = tot + np.mean(2.0 * (1.0 - P[0]))
    return float(tot)


def electric_energy(E):
    return float(np.mean(0.5 * np.sum(E * E, axis=(0, 1))))


def gauss(U, E):
    """G(x) = sum_i [E_i(x) - U_i(x-i)^+ E_i(x-i) U_i(x-i)] as su(2) vectors [3, ...]."""
    G = np.zeros(E.shape[1:])
    for i in range(3):
        Ei = np.concatenate([np.zeros((1,) + E.shape[2:]), E[i]], axis=0)  # pure quaternion
        Um, Em = shift(U[i], i, -1), shift(Ei, i, -1)
        G = G + E[i] - qmul(qmul(qadj(Um), Em), Um)[1:]
    return G
