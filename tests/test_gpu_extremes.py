"""Edge cases of the lattice path on the GPU: the smallest lattice under
every launch shape, a zero-step call, a state written on the device and
committed (tl_commit_state), the largest lattice the ABI accepts (2048^3),
checked through a property that holds at any size (a homogeneous state
evolves exactly like the same state on the smallest lattice), and a device
wait made to run out (TL_ETIMEOUT, then recovery)."""
import math

import numpy as np
import pytest

import oracle as o
from paper_2607_24908_gb300 import tl as T
from paper_2607_24908_gb300.workloads import white_noise_state
from _tol import f32_pi_tol, normwise

pytestmark = pytest.mark.gpu

SHAPES = [dict(kind="stream"), dict(kind="stream", threads=512), dict(kind="stream", tile_x=8, z_chunk=5),
          dict(kind="tma"), dict(kind="tma", warps=15), dict(kind="tma", stages=3, z_chunk=3)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "-".join(f"{k}{v}" for k, v in s.items()))
def test_smallest_lattice_every_shape(dtype, shape):
    """N = 8 (the smallest N accepted), two fields, expanding, 10 Verlet steps, against the oracle."""
    N, nf, dt, steps = 8, 2, 0.01, 10
    npd = np.float32 if dtype == "f32" else np.float64
    phi0, pi0 = white_noise_state(N, nf, seed=21, phi0=(1.0, 0.0), sigma_phi=1e-2, sigma_pi=1e-2)
    phi0, pi0 = phi0.astype(npd), pi0.astype(npd)
    p = o.Params(N=N, nf=nf, kIR=0.5, expanding=True, alpha=1.0, lam=1.0, q=10.0, m2=(0.0, 0.2, 0.0))
    with T.Lattice(N, 0.5, nf, dtype, True, 1.0, 1.0, 1.0) as lat:
        lat.set_pass_config(**shape)
        lat.set_potential(1.0, 10.0, (0.0, 0.2, 0.0))
        lat.set_state(phi0, pi0, 1.0, 0.0, b_from_constraint=True)
        lat.step(steps, dt, "verlet")
        phi, pi = lat.get_all()
        E = lat.energies()
    ph64, pi64 = phi0.astype(np.float64), pi0.astype(np.float64)
    b0 = math.sqrt(float(np.sum(o.energies(p, ph64, pi64, 1.0))) / 3.0)
    ophi, opi, oa, ob = o.run(p, ph64, pi64, 1.0, b0, dt, steps, o.VERLET)
    if dtype == "f64":
        assert normwise(phi, ophi) < 1e-12 and normwise(pi, opi) < 1e-12
        assert abs(E.a - oa) / oa < 1e-12 and abs(E.b - ob) / ob < 1e-12
    else:
        assert normwise(phi, ophi) < 1e-5
        tol = f32_pi_tol(p, steps + 1, float(np.max(np.abs(ophi))), float(np.max(np.abs(opi))))
        assert normwise(pi, opi) < tol
        assert abs(E.a - oa) / oa < 1e-5 and abs(E.b - ob) / ob < 1e-5


def test_zero_steps_is_a_noop():
    phi0, pi0 = white_noise_state(16, 1, seed=2)
    with T.Lattice(16, 0.5, 1, "f64", True, 1.0, 1.0, 1.0) as lat:
        lat.set_potential(1.0, 0.0, (0.0, 0.0, 0.0))
        lat.set_state(phi0, pi0, 1.0, 0.0, b_from_constraint=True)
        E0 = lat.energies()
        lat.step(0, 0.01, "yoshida4")
        phi, pi = lat.get_all()
        E1 = lat.energies()
    assert np.array_equal(phi, phi0) and np.array_equal(pi, pi0)
    assert np.array_equal(E0.vector(), E1.vector()) and E1.step == 0 and E1.a == E0.a and E1.b == E0.b


def padded_views(buf, N, P, origin):
    """[z][y][x] view of the interior of a padded array held in a flat torch tensor."""
    L0 = origin - P
    return buf.view(N, N + 2, P)[:, 1:N + 1, L0:L0 + N]


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_commit_state_equals_set_state(dtype):
    """Arrays written on the device into caller buffers and committed give bitwise the
    results of the same arrays passed through tl_set_state."""
    import torch
    N, nf = 20, 2
    tdt = torch.float32 if dtype == "f32" else torch.float64
    npd = np.float32 if dtype == "f32" else np.float64
    phi0, pi0 = white_noise_state(N, nf, seed=8, phi0=(1.0, 0.0), sigma_phi=1e-2, sigma_pi=1e-2)
    phi0, pi0 = phi0.astype(npd), pi0.astype(npd)
    elems, P, PP, origin = T.tl_array_layout(N, T.DTYPES[dtype])
    bufs = [torch.zeros(elems, dtype=tdt, device="cuda") for _ in range(4 * nf)]
    for f in range(nf):  # pointer order per field: phi, pi of the current state, then the other pair
        padded_views(bufs[4 * f], N, P, origin).copy_(torch.from_numpy(phi0[f]))
        padded_views(bufs[4 * f + 1], N, P, origin).copy_(torch.from_numpy(pi0[f]))
    torch.cuda.synchronize()
    ex = T.tl_expansion(1, 1.0, 1.0, 1.0)
    h = T.tl_lattice_create_with_buffers(N, 0.5, nf, T.DTYPES[dtype], ex, 0, [b.data_ptr() for b in bufs])
    try:
        T.tl_set_potential(h, 1.0, 10.0, (0.0, 0.3, 0.0))
        T.tl_commit_state(h)
        T.tl_set_background(h, 1.0, 0.0, True)
        T.tl_step(h, 5, 0.01, T.YOSHIDA4)
        E = T.tl_energies(h)
        got = []
        for f in range(nf):
            for which in range(2):
                out = np.empty((N, N, N), npd)
                T.tl_get_state(h, f, which, out)
                got.append(out)
    finally:
        T.tl_lattice_destroy(h)
    with T.Lattice(N, 0.5, nf, dtype, True, 1.0, 1.0, 1.0) as lat:
        lat.set_potential(1.0, 10.0, (0.0, 0.3, 0.0))
        lat.set_state(phi0, pi0, 1.0, 0.0, b_from_constraint=True)
        lat.step(5, 0.01, "yoshida4")
        ref = [lat.get(f, w) for f in range(nf) for w in range(2)]
        Er = lat.energies()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    assert E.a == Er.a and E.b == Er.b


def test_largest_lattice_homogeneous_state():
    """N = 2048 (the largest N accepted), one FP32 field in caller buffers (4 x 35.5 GB),
    homogeneous phi = 1, pi = 0, expanding: after 6 Verlet steps under three launch shapes (the
    streaming kernel, TMA 7+1 warps, and the default at this size, TMA 15+1 warps with 92-plane chunks)
    a, b, K and V equal the oracle's run of the same homogeneous state on 8^3 (1e-5) and
    the gradient energy is exactly zero."""
    import torch
    N = 2048
    elems, P, PP, origin = T.tl_array_layout(N, T.F32)
    need = 4 * elems * 4
    free, _ = torch.cuda.mem_get_info()
    if free < need + (8 << 30):
        pytest.skip(f"needs {need / 2**30:.0f} GiB of free device memory")
    dt, steps = 0.01, 6
    p = o.Params(N=8, nf=1, kIR=0.05, expanding=True, alpha=1.0, lam=1.0, q=0.0, m2=(0.0, 0.0, 0.0))
    ph, pi = np.ones((1, 8, 8, 8)), np.zeros((1, 8, 8, 8))
    b0 = math.sqrt(float(np.sum(o.energies(p, ph, pi, 1.0))) / 3.0)
    _, _, oa, ob = o.run(p, ph, pi, 1.0, b0, dt, steps, o.VERLET)
    oE = o.energies(p, *o.run(p, ph, pi, 1.0, b0, dt, steps, o.VERLET)[:2], oa)
    bufs = [torch.empty(elems, dtype=torch.float32, device="cuda") for _ in range(4)]
    try:
        for shape in (dict(kind="stream"), dict(kind="tma"), dict(kind="tma", warps=15, z_chunk=92)):
            bufs[0].fill_(1.0)
            bufs[1].fill_(0.0)
            torch.cuda.synchronize()
            ex = T.tl_expansion(1, 1.0, 1.0, 1.0)
            h = T.tl_lattice_create_with_buffers(N, 0.05, 1, T.F32, ex, 0, [b.data_ptr() for b in bufs])
            try:
                T.tl_set_pass_config(h, T.PASS_KINDS[shape["kind"]], shape.get("warps", 0), 0, shape.get("z_chunk", 0))
                T.tl_set_potential(h, 1.0, 0.0, (0.0, 0.0, 0.0))
                T.tl_commit_state(h)
                T.tl_set_background(h, 1.0, 0.0, True)
                T.tl_step(h, steps, dt, T.VERLET)
                E = T.tl_energies(h)
            finally:
                T.tl_lattice_destroy(h)
            assert abs(E.a - oa) / oa < 1e-5 and abs(E.b - ob) / ob < 1e-5, shape
            assert abs(E.K[0] - oE[0]) / oE[0] < 1e-5 and abs(E.V - oE[2]) / oE[2] < 1e-5, shape
            assert E.G[0] == 0.0, shape
    finally:
        del bufs
        torch.cuda.empty_cache()


def test_expired_device_wait_reports_etimeout_and_recovers(monkeypatch):
    """Failure detection without a fault: the host encodes the TMA boxes one row short
    (TL_TEST_STALL_TMA), so the ring's stages never complete; the kernel's bounded waits
    give up after about a second, record TL_ETIMEOUT and return, the context stays usable,
    and a fresh state on re-encoded maps steps bitwise like the streaming shape."""
    import time
    N, nf = 24, 2
    phi0, pi0 = white_noise_state(N, nf, seed=31, phi0=(1.0, 0.0), sigma_phi=1e-2, sigma_pi=1e-2)
    phi0, pi0 = phi0.astype(np.float32), pi0.astype(np.float32)
    monkeypatch.setenv("TL_TEST_STALL_TMA", "1")
    with T.Lattice(N, 0.5, nf, "f32") as lat:
        lat.set_pass_config("tma")
        lat.set_potential(1.0, 10.0, (0.0, 0.2, 0.0))
        lat.set_state(phi0, pi0)
        t0 = time.perf_counter()
        lat.step(1, 0.01, "verlet")
        with pytest.raises(T.TLError) as e:
            lat.energies()
        assert e.value.code == T.ETIMEOUT
        assert 0.9 < time.perf_counter() - t0 < 120.0
        monkeypatch.delenv("TL_TEST_STALL_TMA")
        lat.set_pass_config("tma")  # re-encodes the tensor maps
        lat.set_state(phi0, pi0)    # resets the status word
        lat.step(3, 0.01, "verlet")
        phi, pi = lat.get_all()
        lat.energies()
    with T.Lattice(N, 0.5, nf, "f32") as ref:
        ref.set_pass_config("stream")
        ref.set_potential(1.0, 10.0, (0.0, 0.2, 0.0))
        ref.set_state(phi0, pi0)
        ref.step(3, 0.01, "verlet")
        rphi, rpi = ref.get_all()
    assert np.array_equal(phi, rphi) and np.array_equal(pi, rpi)
