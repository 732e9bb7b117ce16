"""Parity tolerances shared by the GPU tests (see tests/test_gpu_parity.py).

Fields are compared normwise, max|x_gpu - x_oracle| / max|x_oracle|.  FP32
momenta get a bound derived from the storage arithmetic: each pass rounds
phi ~ 1 to FP32 (unit roundoff u = 2^-24), a per-site white error that
random-walks as u sqrt(passes) and that the lattice turns into momentum error
through its highest frequency omega_max = sqrt(12/dx^2 + max V''); the bound
allows 3 times that, and never less than 1e-5."""
import math

import numpy as np

TOL = {"f64": 1e-12, "f32": 1e-5}


def normwise(x, ref):
    return float(np.max(np.abs(np.asarray(x, np.float64) - ref)) / np.max(np.abs(ref)))


def f32_pi_tol(p, passes, phimax, pimax):
    """3 u sqrt(passes) omega_max max|phi| / max|pi|, at least 1e-5."""
    u = 2.0 ** -24
    w2 = 12.0 / p.dx ** 2 + 3.0 * p.lam * phimax ** 2 + p.q * phimax ** 2 + max(p.m2)
    return max(1e-5, 3.0 * u * math.sqrt(passes) * math.sqrt(w2) * phimax / pimax)


def check_hubble(p, R, E, a, b, oE, oa, ob):
    """The device's Hubble residual R = |1 - a^(2 alpha) mu2 rho/(3 H^2)| (with
    its energies E = [K.., G.., V], a and a' = b) is the constraint evaluated on
    those values (to rounding), and it differs from the oracle's by what the
    relative errors of a, a' and rho propagate to it: to first order
    dR = (1 - R)((2 alpha + 2) da + drho - 2 db), bounded here by 1.25 (1 + R)
    times the sum of magnitudes.  A gate of the residual's own size
    (R ~ 1e-8 ... 1e-4; FP32 bound ~1e-8)."""
    import oracle as o
    E = np.ascontiguousarray(E, dtype=np.float64)
    assert abs(R - o.hubble_residual(p, E, a, b)) < 1e-13
    oR = o.hubble_residual(p, oE, oa, ob)
    rho = float(np.sum(oE))
    da, db = abs(a - oa) / oa, abs(b - ob) / abs(ob)
    drho = abs(float(np.sum(E)) - rho) / rho
    bound = 1.25 * (1.0 + oR) * ((2.0 * p.alpha + 2.0) * da + drho + 2.0 * db) + 1e-13
    assert abs(R - oR) < bound, (R, oR, bound)
