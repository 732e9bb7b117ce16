"""GPU path (libtl.so through the C ABI) against the FP64 oracle.

Tolerances (fields normwise: max|x_gpu - x_oracle| / max|x_oracle|; energy
components relative to the total energy density K+G+V; a, b relative):
FP64 <= 1e-12; FP32 <= 1e-5 on phi, the energies, a and b (linear regime,
<= 400 steps).  FP32 momenta get the bound ``f32_pi_tol`` derived from the
storage arithmetic: each pass rounds phi ~ 1 to FP32 (unit roundoff
u = 2^-24), a per-site white error that random-walks as u sqrt(passes) and
that the lattice turns into momentum error through its highest frequency
omega_max = sqrt(12/dx^2 + max V''); the test allows 3 times that.  Inputs are
seeded white-noise or Philox-drawn states from paper_2607_24908_gb300.workloads
and the oracle; nothing the oracle consumes comes from the GPU.
"""
import math

import numpy as np
import pytest

import oracle as o
from paper_2607_24908_gb300 import tl as T
from paper_2607_24908_gb300.workloads import plane_wave, sample_sites, white_noise_state
from _tol import TOL, check_hubble, f32_pi_tol, normwise

pytestmark = pytest.mark.gpu

OINT = {"leapfrog": o.LEAPFROG, "verlet": o.VERLET, "yoshida4": o.YOSHIDA4}


def make(p: o.Params, dtype: str) -> T.Lattice:
    lat = T.Lattice(p.N, p.kIR, p.nf, dtype, p.expanding, p.alpha, p.fstar_over_mp, 1.0)
    lat.set_potential(p.lam, p.q, p.m2)
    return lat


def oracle_b0(p, phi, pi):
    E = o.energies(p, phi, pi, 1.0)
    return math.sqrt(p.fstar_over_mp ** 2 * float(np.sum(E)) / 3.0)


def compare_run(p, dtype, phi0, pi0, dt, n, integ, tol=None, calls=1):
    """Same input on both sides (the dtype-rounded state), n steps, compare."""
    tol = tol or TOL[dtype]
    npd = np.float32 if dtype == "f32" else np.float64
    phi0 = phi0.astype(npd)
    pi0 = pi0.astype(npd)
    b0 = oracle_b0(p, phi0, pi0) if p.expanding else 0.0
    with make(p, dtype) as lat:
        lat.set_state(phi0, pi0, 1.0, 0.0, b_from_constraint=p.expanding)
        if p.expanding:
            assert abs(lat.energies().b - b0) / b0 < TOL[dtype] * 10
        for _ in range(calls):
            lat.step(n // calls, dt, integ)
        E = lat.energies()
        phi, pi = lat.get_all()
    ophi, opi, oa, ob = o.run(p, phi0, pi0, 1.0, b0, dt, n, OINT[integ])
    oE = o.energies(p, ophi, opi, oa)
    rho = float(np.sum(oE))
    passes = n * (3 if integ == "yoshida4" else 1) + calls
    tol_pi = tol if dtype == "f64" else f32_pi_tol(p, passes, np.max(np.abs(ophi)), np.max(np.abs(opi)))
    assert normwise(phi, ophi) < tol, normwise(phi, ophi)
    assert normwise(pi, opi) < tol_pi, (normwise(pi, opi), tol_pi)
    assert np.max(np.abs(E.vector() - oE)) / rho < tol, (E.vector(), oE)
    assert E.step == n
    if p.expanding:
        assert abs(E.a - oa) / oa < tol and abs(E.b - ob) / abs(ob) < tol, (E.a, oa, E.b, ob)
        check_hubble(p, E.hubble_resid, E.vector(), E.a, E.b, oE, oa, ob)
    return E


def init_tol_abs(dtype, phi, dphi):
    """Largest admissible |phi_gpu - phi_oracle| of a drawn initial field
    phi = phi0 + dphi: the fluctuation dphi to 1e-12 of its size (both sides
    draw the same Philox modes and differ only in FFT and libm rounding), plus
    the rounding of phi0 + dphi to the storage precision (FP64 one ulp of
    |phi|, since the two sides add in a different order; FP32 half an ulp of
    the stored value)."""
    u = 2.0 ** -52 if dtype == "f64" else 2.0 ** -24
    return u * float(np.max(np.abs(phi))) + 1e-12 * float(np.max(np.abs(dphi)))


# --- closed form ---------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_plane_wave_exact_discrete_solution(dtype):
    """Free field m = 1 on 32^3, kIR = 0.5, dt = 0.05, 400 leapfrog steps:
    phi_n = cos(k.x) cos(n W dt) with cos(W dt) = 1 - dt^2 w_lat^2/2."""
    N, n, dt, steps = 32, (1, 2, 3), 0.05, 400
    p = o.Params(N=N, nf=1, kIR=0.5, lam=0.0, m2=(1.0, 0, 0))
    phi0 = plane_wave(N, n)[None]
    with make(p, dtype) as lat:
        lat.set_state(phi0, np.zeros_like(phi0))
        lat.step(steps, dt, "leapfrog")
        phi, pi = lat.get_all()
    w2 = 1.0 + sum((2.0 / p.dx * math.sin(p.kIR * c * p.dx / 2.0)) ** 2 for c in n)
    Wdt = math.acos(1.0 - dt * dt * w2 / 2.0)
    assert np.max(np.abs(phi - phi0 * math.cos(steps * Wdt))) < TOL[dtype]
    assert np.max(np.abs(pi + phi0 * math.sin(steps * Wdt) * math.sin(Wdt) / dt)) < TOL[dtype] * 2


# --- static phi^4, 32^3, initial Gaussian field, 400 leapfrog steps -------------

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_phi4_static_32_init_and_400_leapfrog_steps(dtype):
    p = o.Params(N=32, nf=1, kIR=0.5, lam=1.0)
    spec = o.InitSpec(A=1e-10, meff2=(3.0, 0, 0), phi0=(1.0, 0, 0))
    ophi0, opi0, _, _ = o.init_fluctuations(p, 1, spec)
    with make(p, dtype) as lat:
        lat.init_fluctuations(1, A=1e-10, meff2=(3.0, 0, 0), phi0=(1.0, 0, 0))
        gphi0, gpi0 = lat.get_all()
    # initial fluctuations: to rounding in FP64, to the storage rounding of phi ~ 1 in FP32
    err = float(np.max(np.abs(gphi0.astype(np.float64) - ophi0)))
    assert err <= init_tol_abs(dtype, ophi0, ophi0 - 1.0), err
    assert np.max(np.abs(gpi0)) == 0.0
    compare_run(p, dtype, ophi0, opi0, 0.05, 400, "leapfrog")


# --- expanding backgrounds, ragged tiles, several fields --------------------------

@pytest.mark.parametrize("dtype,N,nf,integ,steps", [
    ("f64", 72, 1, "verlet", 100),
    ("f64", 40, 2, "yoshida4", 40),
    ("f64", 24, 3, "leapfrog", 60),
    ("f32", 72, 2, "yoshida4", 100),
    ("f32", 40, 1, "verlet", 100),
    ("f32", 28, 3, "verlet", 50),
])
def test_expanding_parity(dtype, N, nf, integ, steps):
    p = o.Params(N=N, nf=nf, kIR=0.5, expanding=True, alpha=1.0, lam=1.0, q=100.0 if nf > 1 else 0.0,
                 m2=(0.0, 0.1, 0.2))
    phi0, pi0 = white_noise_state(N, nf, seed=100 + N + nf, phi0=(1.0, 0.0, 0.0), sigma_phi=1e-3,
                                  sigma_pi=1e-3)
    compare_run(p, dtype, phi0, pi0, 0.01 if integ != "yoshida4" else 0.005, steps, integ)


def test_static_three_fields_alpha_ignored():
    p = o.Params(N=32, nf=3, kIR=0.5, lam=1.0, q=10.0, m2=(0.0, 0.5, 1.0))
    phi0, pi0 = white_noise_state(32, 3, seed=9, phi0=(1.0, 0.3, 0.2), sigma_phi=1e-2, sigma_pi=1e-2)
    compare_run(p, "f64", phi0, pi0, 0.02, 100, "verlet")


def test_split_step_calls_match_single_call():
    """step(n) = prologue + n P - 1 merged passes + closing; two calls of n/2
    resynchronise in between, which only changes rounding."""
    p = o.Params(N=32, nf=2, kIR=0.5, expanding=True, alpha=1.0, lam=1.0, q=100.0)
    phi0, pi0 = white_noise_state(32, 2, seed=21, phi0=(1.0, 0.0), sigma_phi=1e-3, sigma_pi=1e-3)
    compare_run(p, "f64", phi0, pi0, 0.005, 40, "yoshida4", calls=4)


# --- init and spectrum ------------------------------------------------------------------

@pytest.mark.parametrize("dtype,fixed", [("f64", False), ("f32", False), ("f64", True)])
def test_init_fluctuations_two_fields_parity(dtype, fixed):
    """N = 48 (non-power-of-two FFT), two fields, momentum fluctuations on,
    expanding: fields, b0 from the constraint (Rayleigh or fixed modulus)."""
    p = o.Params(N=48, nf=2, kIR=0.05, expanding=True, alpha=1.0, lam=1.0, q=100.0)
    spec = o.InitSpec(A=1e-10, meff2=(3.0, 100.0, 0), phi0=(1.0, 0.0, 0), fluct_pi=True, fixed_modulus=fixed)
    ophi, opi, oa, ob = o.init_fluctuations(p, 77, spec)
    with make(p, dtype) as lat:
        lat.init_fluctuations(77, A=1e-10, meff2=(3.0, 100.0, 0), phi0=(1.0, 0, 0), fluct_pi=True,
                              fixed_modulus=fixed)
        gphi, gpi = lat.get_all()
        E = lat.energies()
    err = float(np.max(np.abs(gphi[0].astype(np.float64) - ophi[0])))
    assert err <= init_tol_abs(dtype, ophi[0], ophi[0] - 1.0), err
    # chi and the momenta carry the fluctuations alone: relative to rounding in FP64
    assert normwise(gphi[1], ophi[1]) < (1e-12 if dtype == "f64" else 1e-6)
    assert normwise(gpi, opi) < (1e-12 if dtype == "f64" else 1e-6)
    assert abs(E.b - ob) / ob < (1e-12 if dtype == "f64" else 1e-6)
    assert E.hubble_resid < 1e-12


def test_inits_on_two_streams_share_one_plan():
    """tl_init_fluctuations only enqueues work; lattices of one size on two
    streams share one cuFFT plan (and its workspace), each execution ordered
    after the previous one by the plan's event.  Four inits enqueued back to
    back, alternating streams, then a spectrum of each: bitwise the results of
    one lattice at a time."""
    import torch
    N, seeds = 96, (31, 32, 33, 34)

    def run(lat, seed):
        lat.set_potential(1.0, 10.0, (0.0, 0.0, 0.0))
        lat.init_fluctuations(seed, A=1e-8, meff2=(3.0, 10.0, 0.0), phi0=(1.0, 0.0, 0.0))

    ref = []
    for sd in seeds:
        with T.Lattice(N, 0.5, 2, "f64", True, 1.0, 1.0, 1.0) as lat:
            run(lat, sd)
            ref.append((lat.get_all(), lat.spectrum(1, 1)[1]))
    streams = [torch.cuda.Stream() for _ in range(2)]
    lats = [T.Lattice(N, 0.5, 2, "f64", True, 1.0, 1.0, 1.0, stream=streams[i % 2].cuda_stream)
            for i in range(len(seeds))]
    try:
        for lat, sd in zip(lats, seeds):
            run(lat, sd)
        spectra = [lat.spectrum(1, 1)[1] for lat in lats]
        for lat, P, ((rphi, rpi), rP) in zip(lats, spectra, ref):
            phi, pi = lat.get_all()
            assert np.array_equal(phi, rphi) and np.array_equal(pi, rpi)
            assert np.array_equal(P, rP)
    finally:
        for lat in lats:
            lat.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_spectrum_parity(dtype):
    p = o.Params(N=48, nf=1, kIR=0.1)
    npd = np.float32 if dtype == "f32" else np.float64
    phi0, pi0 = white_noise_state(48, 1, seed=5, phi0=(0.5,), sigma_phi=0.1, sigma_pi=0.2)
    phi0, pi0 = phi0.astype(npd), pi0.astype(npd)
    with make(p, dtype) as lat:
        lat.set_state(phi0, pi0)
        for which, arr in ((0, phi0), (1, pi0)):
            k, P, c = lat.spectrum(0, which)
            ok, oP, oc = o.spectrum(p, arr[0].astype(np.float64))
            assert np.array_equal(c, oc)
            assert np.max(np.abs(k - ok)) < 1e-12
            assert np.max(np.abs(P - oP) / np.maximum(oP, 1e-300)) < 1e-10


# --- properties of the GPU path ---------------------------------------------------------

def test_reversibility_on_gpu():
    p = o.Params(N=32, nf=2, kIR=0.5, expanding=True, alpha=1.0, lam=1.0, q=50.0)
    phi0, pi0 = white_noise_state(32, 2, seed=33, phi0=(1.0, 0.1), sigma_phi=1e-2, sigma_pi=1e-2)
    with make(p, "f64") as lat:
        lat.set_state(phi0, pi0, 1.0, 0.0, b_from_constraint=True)
        b0 = lat.energies().b
        lat.step(50, 0.01, "yoshida4")
        assert lat.energies().a > 1.1
        lat.step(50, -0.01, "yoshida4")
        phi, pi = lat.get_all()
        E = lat.energies()
    assert normwise(phi, phi0) < 1e-12 and normwise(pi, pi0) < 1e-11
    assert abs(E.a - 1.0) < 1e-13 and abs(E.b - b0) / b0 < 1e-12


def test_bitwise_determinism_and_leapfrog_equals_verlet():
    p = o.Params(N=40, nf=2, kIR=0.5, expanding=True, alpha=1.0, lam=1.0, q=100.0)
    phi0, pi0 = white_noise_state(40, 2, seed=44, phi0=(1.0, 0.0), sigma_phi=1e-2, sigma_pi=1e-2)
    outs = []
    for integ in ("verlet", "verlet", "leapfrog"):
        with make(p, "f32") as lat:
            lat.set_state(phi0.astype(np.float32), pi0.astype(np.float32), 1.0, 0.0, True)
            lat.step(30, 0.01, integ)
            outs.append((*lat.get_all(), lat.energies()))
    for other in outs[1:]:
        assert np.array_equal(outs[0][0], other[0]) and np.array_equal(outs[0][1], other[1])
        assert np.array_equal(outs[0][2].vector(), other[2].vector())
        assert outs[0][2].a == other[2].a and outs[0][2].b == other[2].b


def test_nonfinite_state_reports_unstable():
    p = o.Params(N=16, nf=1, kIR=0.5, lam=1.0)
    phi0, pi0 = white_noise_state(16, 1, seed=1)
    phi0[0, 3, 4, 5] = np.inf
    with make(p, "f64") as lat:
        lat.set_state(phi0, pi0)
        lat.step(2, 0.01, "verlet")
        with pytest.raises(T.TLError) as e:
            lat.energies()
        assert e.value.code == T.EUNSTABLE


def test_argument_errors():
    with pytest.raises(T.TLError) as e:
        T.Lattice(30, 0.5, 1, "f64")
    assert e.value.code == T.EINVAL
    with pytest.raises(T.TLError) as e:
        T.Lattice(32, 0.5, 4, "f64")
    assert e.value.code == T.EINVAL
    with T.Lattice(16, 0.5, 1, "f64") as lat:
        with pytest.raises(T.TLError) as e:
            lat.step(1, 0.01)
        assert e.value.code == T.ESTATE
        lat.set_potential(1.0)
        with pytest.raises(T.TLError) as e:
            lat.step(1, 0.01)
        assert e.value.code == T.ESTATE
        with pytest.raises(T.TLError) as e:
            T.tl_get_state(lat.h, 1, 0, np.empty((16, 16, 16)))
        assert e.value.code == T.EINVAL
        with pytest.raises(T.TLError) as e:
            T.tl_get_state(lat.h, 0, 0, np.empty((16, 16, 15)))
        assert e.value.code == T.EINVAL
        with pytest.raises(T.TLError) as e:
            T.tl_step(lat.h, 1, 0.01, 7)
        assert e.value.code in (T.EINVAL, T.ESTATE)


# --- full size: 1024^3 x 2 fields FP32 (the benchmark's kernel and geometry) -------------

def _host_ram_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


@pytest.mark.slow
def test_full_size_1024_two_fields_sampled():
    """Energies of the input state (one reduction over 2^31 site-fields) and
    one Verlet step at 4096 sampled sites, against the oracle evaluated at
    those sites (static background: each output depends on a 5^3
    neighbourhood only)."""
    if _host_ram_gb() < 80:
        pytest.skip("needs ~64 GB of host memory for the FP64 oracle arrays")
    N, nf, dt = 1024, 2, 0.005
    p = o.Params(N=N, nf=nf, kIR=0.05, lam=1.0, q=100.0)
    rng = np.random.default_rng(2024)
    phi0 = np.empty((nf, N, N, N), np.float32)
    pi0 = np.empty((nf, N, N, N), np.float32)
    for f in range(nf):
        phi0[f] = rng.standard_normal((N, N, N), dtype=np.float32) * np.float32(1e-2) + np.float32(1.0 - f)
        pi0[f] = rng.standard_normal((N, N, N), dtype=np.float32) * np.float32(1e-2)
    sites = sample_sites(N, 4096, seed=7)
    with make(p, "f32") as lat:
        lat.set_state(phi0, pi0)
        E0 = lat.energies()
        lat.step(1, dt, "verlet")
        buf = np.empty((N, N, N), np.float32)
        g = np.empty((2, len(sites), nf))
        for f in range(nf):
            for w in range(2):
                T.tl_get_state(lat.h, f, w, buf)
                g[w, :, f] = buf[sites[:, 0], sites[:, 1], sites[:, 2]]
        del buf
    ophi1, opi1 = o.vv_step_at_sites(p, phi0, pi0, sites, dt)
    assert normwise(g[0], ophi1) < 1e-5
    assert np.max(np.abs(g[1] - opi1)) / np.max(np.abs(opi1)) < 1e-5
    oE0 = o.energies(p, phi0.astype(np.float64), pi0.astype(np.float64), 1.0)
    assert np.max(np.abs(E0.vector() - oE0)) / np.sum(oE0) < 1e-5
    for i in range(len(oE0)):  # every component, relative to itself
        assert abs(E0.vector()[i] - oE0[i]) / abs(oE0[i]) < 1e-4, (i, E0.vector()[i], oE0[i])


# --- chaotic nonlinear regime: volume averages and spectra within 1% ----------------------

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_chaotic_regime_energies_and_spectra_within_one_percent(dtype):
    """Strongly nonlinear two-field state (white noise sigma 0.3 on phi = 1,
    q = 10), 2000 Verlet steps: the dynamics is chaotic (on the oracle alone a
    1e-7 perturbation of the input grows to ~3e-3 in the fields by then), yet
    volume averages and shell spectra must stay within 1% (bins with >= 100
    modes and P_b >= 1e-6 max)."""
    N, nf, dt, steps = 48, 2, 0.02, 2000
    p = o.Params(N=N, nf=nf, kIR=0.5, lam=1.0, q=10.0, m2=(0.0, 0.5, 0.0))
    npd = np.float32 if dtype == "f32" else np.float64
    phi0, pi0 = white_noise_state(N, nf, seed=99, phi0=(1.0, 0.5), sigma_phi=0.3, sigma_pi=0.3)
    phi0, pi0 = phi0.astype(npd), pi0.astype(npd)
    with make(p, dtype) as lat:
        lat.set_state(phi0, pi0)
        lat.step(steps, dt, "verlet")
        E = lat.energies()
        spec = [lat.spectrum(f, 0) for f in range(nf)]
    ophi, opi, _, _ = o.run(p, phi0, pi0, 1.0, 0.0, dt, steps, o.VERLET)
    oE = o.energies(p, ophi, opi)
    # nonlinear: the potential and gradient energies are of the same order as the kinetic
    assert min(oE[:2 * nf]) > 1e-3 * max(oE)
    assert np.max(np.abs(E.vector() - oE) / np.abs(oE)) < 0.01, (E.vector(), oE)
    for f in range(nf):
        k, P, c = spec[f]
        ok, oP, oc = o.spectrum(p, ophi[f])
        sel = (oc >= 100) & (oP >= 1e-6 * oP.max())
        assert sel.sum() > 10
        assert np.max(np.abs(P[sel] - oP[sel]) / oP[sel]) < 0.01


# --- padded layout: caller-owned buffers, ghosts kept current ---------------------------

@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_caller_buffers_and_ghost_cells(dtype):
    """tl_lattice_create_with_buffers on torch-allocated padded arrays: after
    init and several passes every ghost row equals its periodic image (the
    reserved x-edge elements are not kept), and the results are bitwise those
    of a library-allocated lattice."""
    import torch
    N, nf = 24, 2
    esz = 4 if dtype == "f32" else 8
    tdt = torch.float32 if dtype == "f32" else torch.float64
    elems, P, PP, origin = T.tl_array_layout(N, T.DTYPES[dtype])
    bufs = [torch.zeros(elems, dtype=tdt, device="cuda") for _ in range(4 * nf)]
    ex = T.tl_expansion(1, 1.0, 1.0, 1.0)
    h = T.tl_lattice_create_with_buffers(N, 0.5, nf, T.DTYPES[dtype], ex, 0, [b.data_ptr() for b in bufs])
    try:
        T.tl_set_potential(h, 1.0, 100.0, (0.0, 0.0, 0.0))
        T.tl_init_fluctuations(h, 5, 1e-4, (3.0, 100.0, 0.0), (1.0, 0.0, 0.0))
        T.tl_step(h, 7, 0.005, T.YOSHIDA4)
        T.tl_energies(h)
        torch.cuda.synchronize()
        for f in range(nf):
            for which in range(2):
                ptr = T.tl_state_device_ptr(h, f, which)
                b = next(b for b in bufs if b.data_ptr() + origin * esz == ptr)
                a = b.view(N, N + 2, P)  # [z][row incl. ghost rows][padded row]
                L0 = origin - P  # x = 0 within a padded row
                inner = a[:, 1:N + 1, L0:L0 + N]
                assert torch.equal(a[:, 0, L0:L0 + N], inner[:, N - 1, :])              # row above
                assert torch.equal(a[:, N + 1, L0:L0 + N], inner[:, 0, :])              # row below
                out = np.empty((N, N, N), np.float32 if dtype == "f32" else np.float64)
                T.tl_get_state(h, f, which, out)
                assert np.array_equal(out, inner.cpu().numpy())
        with T.Lattice(N, 0.5, nf, dtype, True, 1.0, 1.0, 1.0) as lat:
            lat.set_potential(1.0, 100.0, (0.0, 0.0, 0.0))
            lat.init_fluctuations(5, A=1e-4, meff2=(3.0, 100.0, 0.0), phi0=(1.0, 0.0, 0.0))
            lat.step(7, 0.005, "yoshida4")
            for f in range(nf):
                ref = lat.get(f, 0)
                out = np.empty_like(ref)
                T.tl_get_state(h, f, 0, out)
                assert np.array_equal(out, ref)
    finally:
        T.tl_lattice_destroy(h)
