"""Oracle: plain double-precision CPU reference for the lattice stepper.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library; the two meet only through the seeded
input generators in ``paper_2607_24908_gb300.workloads`` (which hold none of
the method's arithmetic) and through the C-ABI calls the tests make.

Contents
  * ``tlo.c`` (compiled here with gcc into ``liboracle.so``): the literal
    velocity-Verlet, leapfrog and Yoshida-4 steppers, forces, energies, the
    scale-factor acceleration and Hubble residual, and Philox-2x64-10.
  * this module: ctypes wrappers, the Gaussian random initial state
    (Philox-drawn modes with power A/(2 omega_k), inverse DFT via numpy.fft)
    and the binned power spectrum (forward DFT via numpy.fft).

Paper passages followed: the phi^4 kick/drift leapfrog and 7-point stencil
(Sec. 4, Benchmarks); Gaussian random fields from counter-based Philox
(Sec. 2, Interface); Fourier-space views for state preparation and
measurement (Sec. 2 and Sec. 3.5, Fourier Transformations).  The expanding
background, alpha time variable, Yoshida-4 and spectrum conventions are not
printed in the paper; the readings used are stated in the C file's header and
in the functions below.

Parity pins: see tests/test_oracle_pins.py and tests/test_golden.py.
``philox2x64`` is pinned to the published known-answer vectors of
Philox-2x64-10 (Random123's kat_vectors rows), to its round structure by exact
inversion of its ten rounds, and statistically.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "tlo.c")

LEAPFROG, VERLET, YOSHIDA4 = 0, 1, 2
MAX_FIELDS = 3


def build(force: bool = False) -> str:
    """Compile tlo.c into liboracle.so next to it (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("nf", ctypes.c_int), ("expanding", ctypes.c_int),
                ("pad_", ctypes.c_int), ("kIR", ctypes.c_double), ("alpha", ctypes.c_double),
                ("mu2", ctypes.c_double), ("lam", ctypes.c_double), ("q", ctypes.c_double),
                ("m2", ctypes.c_double * MAX_FIELDS)]


@dataclass
class Params:
    """Lattice, background and potential of one run (program variables)."""
    N: int
    nf: int = 1
    kIR: float = 0.5
    expanding: bool = False
    alpha: float = 0.0
    fstar_over_mp: float = 1.0
    lam: float = 1.0
    q: float = 0.0
    m2: Sequence[float] = field(default_factory=lambda: (0.0, 0.0, 0.0))

    @property
    def dx(self) -> float:
        return 2.0 * math.pi / (self.kIR * self.N)

    @property
    def L(self) -> float:
        return 2.0 * math.pi / self.kIR

    def c(self) -> _Params:
        m2 = list(self.m2) + [0.0] * (MAX_FIELDS - len(self.m2))
        return _Params(self.N, self.nf, int(bool(self.expanding)), 0, self.kIR, self.alpha,
                       self.fstar_over_mp ** 2, self.lam, self.q,
                       (ctypes.c_double * MAX_FIELDS)(*m2[:MAX_FIELDS]))


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        L.tlo_force.argtypes = [pp, dp, ctypes.c_double, dp]
        L.tlo_energies.argtypes = [pp, dp, dp, ctypes.c_double, dp]
        L.tlo_fb.argtypes = [pp, dp, ctypes.c_double]
        L.tlo_fb.restype = ctypes.c_double
        L.tlo_hubble_residual.argtypes = [pp, dp, ctypes.c_double, ctypes.c_double]
        L.tlo_hubble_residual.restype = ctypes.c_double
        L.tlo_run.argtypes = [pp, dp, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        L.tlo_run.restype = ctypes.c_int
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.tlo_philox2x64.argtypes = [ctypes.c_size_t, u64p, ctypes.c_uint64, ctypes.c_uint64, u64p]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fields(x, p: Params) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if a.shape != (p.nf, p.N, p.N, p.N):
        raise ValueError(f"expected shape {(p.nf, p.N, p.N, p.N)}, got {a.shape}")
    return a


def force(p: Params, phi, a: float = 1.0) -> np.ndarray:
    """F_f = a^(1+alpha) Lap phi_f - a^(3+alpha) dV/dphi_f (field equation for pi)."""
    phi = _fields(phi, p)
    F = np.empty_like(phi)
    pc = p.c()
    lib().tlo_force(ctypes.byref(pc), _dp(phi), a, _dp(F))
    return F


def energies(p: Params, phi, pi, a: float = 1.0) -> np.ndarray:
    """[K_0..K_{nf-1}, G_0..G_{nf-1}, V] volume averages at scale factor a."""
    phi = _fields(phi, p)
    pi = _fields(pi, p)
    out = np.zeros(2 * p.nf + 1)
    pc = p.c()
    lib().tlo_energies(ctypes.byref(pc), _dp(phi), _dp(pi), a, _dp(out))
    return out


def scale_accel(p: Params, E, a: float) -> float:
    """a'' from the Friedmann equations in alpha time."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    pc = p.c()
    return lib().tlo_fb(ctypes.byref(pc), _dp(E), a)


def hubble_residual(p: Params, E, a: float, b: float) -> float:
    E = np.ascontiguousarray(E, dtype=np.float64)
    pc = p.c()
    return lib().tlo_hubble_residual(ctypes.byref(pc), _dp(E), a, b)


def run(p: Params, phi, pi, a: float, b: float, dt: float, nsteps: int, integrator: int = VERLET):
    """Advance a copy of (phi, pi, a, b) by nsteps steps; returns (phi, pi, a, b)."""
    phi = _fields(phi, p).copy()
    pi = _fields(pi, p).copy()
    ab = np.array([a, b], dtype=np.float64)
    pc = p.c()
    rc = lib().tlo_run(ctypes.byref(pc), _dp(phi), _dp(pi), _dp(ab), dt, int(nsteps), int(integrator))
    if rc != 0:
        raise ValueError(f"unknown integrator {integrator}")
    if not p.expanding:
        ab[:] = (1.0, 0.0)
    return phi, pi, float(ab[0]), float(ab[1])


def philox2x64(c0, c1: int, key: int) -> np.ndarray:
    """Philox-2x64-10 of counters (c0[i], c1) under key; returns uint64 [n, 2]."""
    c0 = np.ascontiguousarray(np.asarray(c0, dtype=np.uint64).ravel())
    out = np.empty((c0.size, 2), dtype=np.uint64)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib().tlo_philox2x64(c0.size, c0.ctypes.data_as(u64p), ctypes.c_uint64(c1 & (2**64 - 1)),
                         ctypes.c_uint64(key & (2**64 - 1)), out.ctypes.data_as(u64p))
    return out


# ---- Gaussian random initial state ------------------------------------------

@dataclass
class InitSpec:
    """Homogeneous values plus vacuum-like Gaussian fluctuations.

    Reading of the workload's "power spectrum A/(2 omega_k)": every mode n with
    0 < |n| < N/2 (k = kIR |n|) gets a complex amplitude with
    <|d(n)|^2> = P(k)/L^3, P = A/(2 omega_k), omega_k^2 = k^2 + meff2, so that
    <dphi^2> approximates the integral of P over d^3k/(2 pi)^3.  Modulus is
    Rayleigh (sqrt(-ln u1)), phase 2 pi u2: a Gaussian field; with
    ``fixed_modulus`` every mode gets the modulus sqrt(P/L^3) exactly and a
    random phase (same mean power).  With ``fluct_pi`` the momenta get an
    independent draw with P = A omega_k/2, scaled by a0^(3-alpha).
    """
    A: float = 1e-10
    meff2: Sequence[float] = (3.0, 0.0, 0.0)
    phi0: Sequence[float] = (1.0, 0.0, 0.0)
    pi0: Sequence[float] = (0.0, 0.0, 0.0)
    fluct_pi: bool = False
    a0: float = 1.0
    fixed_modulus: bool = False


def _mode_grid(N: int):
    n = np.rint(np.fft.fftfreq(N, 1.0 / N)).astype(np.int64)
    nz, ny, nx = np.meshgrid(n, n, n, indexing="ij")
    return nz, ny, nx


def _uniforms(words: np.ndarray):
    two53 = float(2 ** 53)
    u1 = ((words[:, 0] >> np.uint64(11)).astype(np.float64) + 1.0) / two53  # (0, 1]
    u2 = (words[:, 1] >> np.uint64(11)).astype(np.float64) / two53          # [0, 1)
    return u1, u2


def gaussian_modes(N: int, kIR: float, power, seed: int, stream: int, fixed_modulus: bool = False) -> np.ndarray:
    """Complex Hermitian mode array d(n) (full N^3, numpy FFT order [z, y, x]).

    Each pair (n, -n) is drawn once, at the member that is canonical: nx > 0,
    or nx == 0 and ny > 0, or nx == ny == 0 and nz > 0.  Its Philox counter is
    (index of that member in the [z, y, x] array, stream) under key seed; the
    partner gets the complex conjugate."""
    nz, ny, nx = _mode_grid(N)
    r = np.sqrt((nx * nx + ny * ny + nz * nz).astype(np.float64))
    live = (r > 0) & (r < N / 2)
    canon = (nx > 0) | ((nx == 0) & (ny > 0)) | ((nx == 0) & (ny == 0) & (nz > 0))
    own = (np.mod(nz, N) * N + np.mod(ny, N)) * N + np.mod(nx, N)
    partner = (np.mod(-nz, N) * N + np.mod(-ny, N)) * N + np.mod(-nx, N)
    rep = np.where(canon, own, partner)
    words = philox2x64(rep[live], stream, seed)
    u1, u2 = _uniforms(words)
    L = 2.0 * math.pi / kIR
    P = power(kIR * r[live])
    amp = np.sqrt(P / L ** 3) * (1.0 if fixed_modulus else np.sqrt(-np.log(u1)))
    ph = 2.0 * math.pi * u2
    sgn = np.where(canon[live], 1.0, -1.0)
    d = np.zeros((N, N, N), dtype=np.complex128)
    d[live] = amp * (np.cos(ph) + 1j * sgn * np.sin(ph))
    return d


def modes_to_field(d: np.ndarray) -> np.ndarray:
    """dphi(x) = sum_n d(n) exp(i k.x): unnormalised inverse DFT, real part."""
    N = d.shape[0]
    return np.real(np.fft.ifftn(d)) * float(N) ** 3


def init_fluctuations(p: Params, seed: int, spec: InitSpec):
    """Initial (phi, pi, a0, b0).  b0 = a0^(1+alpha) sqrt(mu2 rho0/3) with rho0
    the lattice-averaged K+G+V of the initial state (expanding runs)."""
    N = p.N
    phi = np.empty((p.nf, N, N, N))
    pi = np.empty((p.nf, N, N, N))
    for f in range(p.nf):
        m2 = spec.meff2[f]
        d = gaussian_modes(N, p.kIR, lambda k: spec.A / (2.0 * np.sqrt(k * k + m2)), seed, f,
                           spec.fixed_modulus)
        phi[f] = spec.phi0[f] + modes_to_field(d)
        pi[f] = spec.pi0[f]
        if spec.fluct_pi:
            scale = spec.a0 ** (3.0 - p.alpha) if p.expanding else 1.0
            dp = gaussian_modes(N, p.kIR, lambda k: spec.A * np.sqrt(k * k + m2) / 2.0, seed, 8 + f,
                                spec.fixed_modulus)
            pi[f] += scale * modes_to_field(dp)
    a0, b0 = 1.0, 0.0
    if p.expanding:
        a0 = spec.a0
        E = energies(p, phi, pi, a0)
        b0 = a0 ** (1.0 + p.alpha) * math.sqrt(p.fstar_over_mp ** 2 * float(np.sum(E)) / 3.0)
    return phi, pi, a0, b0


# ---- binned power spectrum ---------------------------------------------------

def n_bins(N: int) -> int:
    return int(math.ceil(math.sqrt(3.0) * N / 2.0)) + 1


def spectrum(p: Params, f3: np.ndarray):
    """Shell-binned spectrum of one real N^3 array.

    d(n) = N^-3 sum_x f(x) exp(-i k.x); bin b = floor(|n| + 1/2);
    P_b = L^3 mean_{n in b} |d(n)|^2, k_b = kIR mean_{n in b} |n|.
    Returns (k_b, P_b, count_b); empty bins give k = P = 0."""
    N = p.N
    d = np.fft.fftn(np.asarray(f3, dtype=np.float64)) / float(N) ** 3
    pw = (d.real ** 2 + d.imag ** 2).ravel()
    nz, ny, nx = _mode_grid(N)
    r = np.sqrt((nx * nx + ny * ny + nz * nz).astype(np.float64)).ravel()
    b = np.floor(r + 0.5).astype(np.int64)
    nb = n_bins(N)
    cnt = np.bincount(b, minlength=nb)
    ps = np.bincount(b, weights=pw, minlength=nb)
    rs = np.bincount(b, weights=r, minlength=nb)
    nz_ = cnt > 0
    P = np.zeros(nb)
    k = np.zeros(nb)
    P[nz_] = p.L ** 3 * ps[nz_] / cnt[nz_]
    k[nz_] = p.kIR * rs[nz_] / cnt[nz_]
    return k, P, cnt.astype(np.int64)


# ---- one step at sampled sites (full-size parity) ------------------------------

def _dV_np(p: Params, v):
    """dV/dphi_f for stacked site values v[..., f] (same potential as tlo.c)."""
    out = np.empty_like(v)
    others = np.sum(v[..., 1:] ** 2, axis=-1) if p.nf > 1 else 0.0
    out[..., 0] = p.m2[0] * v[..., 0] + p.lam * v[..., 0] ** 3 + p.q * v[..., 0] * others
    for f in range(1, p.nf):
        out[..., f] = p.m2[f] * v[..., f] + p.q * v[..., 0] ** 2 * v[..., f]
    return out


def _patch_force(p: Params, ph):
    """F on the interior of a patch ph[S, nf, n, n, n] -> [S, nf, n-2, n-2, n-2] (a == 1)."""
    c = ph[:, :, 1:-1, 1:-1, 1:-1]
    lap = ((ph[:, :, 1:-1, 1:-1, 2:] + ph[:, :, 1:-1, 1:-1, :-2] - 2.0 * c)
           + (ph[:, :, 1:-1, 2:, 1:-1] + ph[:, :, 1:-1, :-2, 1:-1] - 2.0 * c)
           + (ph[:, :, 2:, 1:-1, 1:-1] + ph[:, :, :-2, 1:-1, 1:-1] - 2.0 * c)) / p.dx ** 2
    dv = np.moveaxis(_dV_np(p, np.moveaxis(c, 1, -1)), -1, 1)
    return lap - dv


def vv_step_at_sites(p: Params, phi, pi, sites, dt: float):
    """One velocity-Verlet step in a static background, evaluated only at the
    given sites (z, y, x): the same operator sequence as tlo.c on the 5^3
    periodic neighbourhood each output depends on.  phi, pi: [nf, N, N, N]
    arrays (any float dtype; promoted to FP64).  Returns (phi1, pi1) as
    [S, nf]."""
    if p.expanding:
        raise ValueError("site-local evaluation needs a static background")
    N = p.N
    sites = np.asarray(sites)
    o = np.arange(-2, 3)
    iz = (sites[:, 0:1] + o) % N
    iy = (sites[:, 1:2] + o) % N
    ix = (sites[:, 2:3] + o) % N
    sel = (iz[:, :, None, None], iy[:, None, :, None], ix[:, None, None, :])
    ph = np.stack([np.asarray(phi[f])[sel].astype(np.float64) for f in range(p.nf)], axis=1)
    pp = np.stack([np.asarray(pi[f])[sel].astype(np.float64) for f in range(p.nf)], axis=1)
    F0 = _patch_force(p, ph)                              # 3^3
    pih = pp[:, :, 1:-1, 1:-1, 1:-1] + 0.5 * dt * F0       # 3^3
    ph1 = ph[:, :, 1:-1, 1:-1, 1:-1] + dt * pih            # 3^3
    F1 = _patch_force(p, ph1)                             # centre
    pi1 = pih[:, :, 1, 1, 1] + 0.5 * dt * F1[:, :, 0, 0, 0]
    return ph1[:, :, 1, 1, 1], pi1


# ---- Langevin phi^4 (Sec. 2, Eq. 1) -------------------------------------------------

LANGEVIN_STREAM = 1 << 63  # high bit of the second Philox counter word marks Langevin noise


def langevin_noise(N: int, seed: int, step: int) -> np.ndarray:
    """Unit Gaussian per site for one step: the sites with dense indices 2k and
    2k + 1 share Philox-2x64-10 of counter (k, 2^63 + step) under key seed;
    Box-Muller on the two words (u1 in (0, 1], u2 in [0, 1)) gives the pair of
    independent Gaussians sqrt(-2 ln u1) (cos, sin)(2 pi u2), the cosine for
    site 2k and the sine for site 2k + 1."""
    w = philox2x64(np.arange(N ** 3 // 2, dtype=np.uint64), LANGEVIN_STREAM + int(step), seed)
    u1, u2 = _uniforms(w)
    r = np.sqrt(-2.0 * np.log(u1))
    xi = np.empty(N ** 3)
    xi[0::2] = r * np.cos(2.0 * math.pi * u2)
    xi[1::2] = r * np.sin(2.0 * math.pi * u2)
    return xi.reshape(N, N, N)


def langevin_run(N: int, kIR: float, phi, dt: float, nsteps: int, lam: float, m2: float, noise: float,
                 seed: int, step0: int = 0) -> np.ndarray:
    """Euler-Maruyama for d phi/dt = Lap phi - m^2 phi - (lam/2) phi^3 + noise * eta,
    <eta eta> = delta(t - t') per site:  phi += dt (Lap phi - m^2 phi - lam/2 phi^3)
    + noise sqrt(dt) xi_n  (the update of the paper's Langevin listing, Sec. 2,
    where eta is drawn per site and rescaled by 1/sqrt(dt)).  Steps are numbered
    from step0 for the noise counters."""
    dx = 2.0 * math.pi / (kIR * N)
    f = np.array(phi, dtype=np.float64, copy=True).reshape(N, N, N)
    for n in range(nsteps):
        lap = sum(np.roll(f, 1, ax) + np.roll(f, -1, ax) - 2.0 * f for ax in range(3)) / dx ** 2
        drift = lap - m2 * f - 0.5 * lam * f ** 3
        xi = langevin_noise(N, seed, step0 + n) if noise != 0.0 else 0.0
        f = f + dt * drift + noise * math.sqrt(dt) * xi
    return f
