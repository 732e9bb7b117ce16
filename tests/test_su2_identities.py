"""Host checks of the two identities the SU(2) kernel is built on (no GPU).

1. The force in plaquette form.  With P_ij(x) = U_i(x) U_j(x+i) U_i(x+j)^+ U_j(x)^+
   and V_ij = Im P_ij, the kick's Im[U_i S_i] (staples of Sec. 4, as the oracle
   writes them) equals sum_{j != i} V_ij(x) - R(W^+) V_ij(x-j) with W = U_j(x-j),
   where R(W^+) v = Im(W^+ (0, v) W) = (w^2 - |u|^2) v + 2 (u.v) u + 2 w (u x v)
   for W = w + i u.s, and = v + 2 w (u x v) + 2 u x (u x v) for a unit W.  The
   backward identity needs W^+ W = 1: the links must be unit quaternions.
2. The drift's small-angle series.  sin(t)/t and cos(t) truncated as in the
   kernel (FP32: terms to t^8 below t = 1/2; FP64: to t^10 and t^12 below
   t = 1/4) stay within a few units in the last place of the exact values.
"""
import numpy as np
import pytest

import oracle.su2 as Y
from paper_2607_24908_gb300.workloads import random_su2_links


def _plaquette_im(U, i, j):
    a, b, c, d = U[i], Y.shift(U[j], i, 1), Y.shift(U[i], j, 1), U[j]
    return Y.qmul(Y.qmul(a, b), Y.qmul(Y.qadj(c), Y.qadj(d)))[1:]


def _force_plaquette_form(U, unit_form):
    V = {}
    for i in range(3):
        for j in range(i + 1, 3):
            V[(i, j)] = _plaquette_im(U, i, j)
            V[(j, i)] = -V[(i, j)]
    F = np.zeros((3, 3) + U.shape[2:])
    for i in range(3):
        acc = 0.0
        for j in range(3):
            if j == i:
                continue
            W = Y.shift(U[j], j, -1)
            w, u = W[0], W[1:]
            v = Y.shift(V[(i, j)], j, -1)
            c = np.cross(u, v, axis=0)
            if unit_form:
                rot = v + 2 * w * c + 2 * np.cross(u, c, axis=0)
            else:
                rot = (w * w - np.sum(u * u, axis=0)) * v + 2 * np.sum(u * v, axis=0) * u + 2 * w * c
            acc = acc + V[(i, j)] - rot
        F[i] = -2.0 * acc
    return F


@pytest.mark.parametrize("unit_form", [False, True])
def test_plaquette_form_equals_staple_force(unit_form):
    U = random_su2_links(6, seed=3, amp=0.8).astype(np.float64)
    Fo = Y.force(U)
    F = _force_plaquette_form(U, unit_form)
    assert np.max(np.abs(F - Fo)) < 1e-13 * np.max(np.abs(Fo))


def test_plaquette_form_needs_unit_links():
    """The backward identity U_i b_ij = W^+ P_ij(x-j)^+ W uses W^+ W = 1: with links
    scaled by 1.01 both rotation forms leave the staple force by O(|W|^2 - 1)."""
    U = random_su2_links(5, seed=4, amp=0.7).astype(np.float64) * 1.01
    Fo = Y.force(U)
    for unit_form in (False, True):
        assert np.max(np.abs(_force_plaquette_form(U, unit_form) - Fo)) > 1e-3 * np.max(np.abs(Fo))


def _series(t2, dtype, fp64):
    t2 = t2.astype(dtype)
    f = lambda c: dtype(c)  # noqa: E731
    if fp64:
        sc = f(-1.0 / 39916800.0)
        for c in (1.0 / 362880.0, -1.0 / 5040.0, 1.0 / 120.0, -1.0 / 6.0):
            sc = sc * t2 + f(c)
        cc = f(1.0 / 479001600.0)
        for c in (-1.0 / 3628800.0, 1.0 / 40320.0, -1.0 / 720.0, 1.0 / 24.0, -1.0 / 2.0):
            cc = cc * t2 + f(c)
    else:
        sc = f(1.0 / 362880.0)
        for c in (-1.0 / 5040.0, 1.0 / 120.0, -1.0 / 6.0):
            sc = sc * t2 + f(c)
        cc = f(1.0 / 40320.0)
        for c in (-1.0 / 720.0, 1.0 / 24.0, -1.0 / 2.0):
            cc = cc * t2 + f(c)
    return sc * t2 + f(1.0), cc * t2 + f(1.0)


@pytest.mark.parametrize("fp64", [False, True])
def test_small_angle_series_within_a_few_ulp(fp64):
    dtype = np.float64 if fp64 else np.float32
    cut = 0.25 if fp64 else 0.5
    t = np.linspace(0.0, cut, 200001)[:-1]
    sinc, cos = _series(t * t, dtype, fp64)
    # exact values in extended precision where available, else float64 (enough for the FP32 case)
    te = t.astype(np.longdouble)
    ex_sinc = np.where(te > 0, np.sin(te) / np.where(te > 0, te, 1), 1)
    ex_cos = np.cos(te)
    eps = np.finfo(dtype).eps
    assert np.max(np.abs(sinc.astype(np.longdouble) - ex_sinc)) < 4 * eps
    assert np.max(np.abs(cos.astype(np.longdouble) - ex_cos)) < 4 * eps
