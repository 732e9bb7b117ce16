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
