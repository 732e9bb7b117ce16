"""tl_step's CUDA-graph replay on the GPU.

A repeated tl_step call (same n, dt, integrator and buffer parity) replays a
captured graph of its passes instead of launching them one by one; it must
give bitwise the results of direct launches (TL_STEP_GRAPHS=0), and anything a
captured pass bakes in (launch shape, potential, buffer assignment after a
Langevin step) must drop the captured graphs."""
import numpy as np
import pytest

from paper_2607_24908_gb300 import tl as T
from paper_2607_24908_gb300.workloads import white_noise_state

pytestmark = pytest.mark.gpu


def new(N, nf, dtype, expanding, shape=None, seed=3):
    npd = np.float32 if dtype == "f32" else np.float64
    phi, pi = white_noise_state(N, nf, seed=seed, phi0=(1.0, 0.0, 0.0)[:nf], sigma_phi=1e-2, sigma_pi=1e-2)
    lat = T.Lattice(N, 0.5, nf, dtype, expanding, 1.0, 1.0, 1.0)
    if shape:
        lat.set_pass_config(**shape)
    lat.set_potential(1.0, 10.0, (0.0, 0.2, 0.0))
    lat.set_state(phi.astype(npd), pi.astype(npd), 1.0, 0.0, b_from_constraint=expanding)
    return lat


def calls(lat, monkeypatch, graphs, script):
    if graphs:
        monkeypatch.delenv("TL_STEP_GRAPHS", raising=False)
    else:
        monkeypatch.setenv("TL_STEP_GRAPHS", "0")
    for op in script:
        op(lat)
    phi, pi = lat.get_all()
    return phi, pi, lat.energies()


@pytest.mark.parametrize("N,nf,dtype,shape", [(192, 2, "f32", dict(kind="tma")), (40, 2, "f64", None),
                                              (36, 1, "f32", dict(kind="stream", threads=512))])
@pytest.mark.parametrize("integ", ["verlet", "yoshida4"])
def test_replay_is_bitwise_direct(N, nf, dtype, shape, integ, monkeypatch):
    # 4 calls of 5 steps: the second captures, the third and fourth replay (both parities for
    # Yoshida's 16 passes per call are even, Verlet's 6 too; one odd call flips the parity)
    script = [lambda l: l.step(5, 0.01, integ)] * 4 + [lambda l: l.step(2, 0.01, "leapfrog")] + \
             [lambda l: l.step(5, 0.01, integ)] * 3
    with new(N, nf, dtype, True, shape) as a, new(N, nf, dtype, True, shape) as b:
        ra = calls(a, monkeypatch, True, script)
        rb = calls(b, monkeypatch, False, script)
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
    assert np.array_equal(ra[2].vector(), rb[2].vector()) and ra[2].a == rb[2].a and ra[2].b == rb[2].b
    assert ra[2].step == 37


def test_potential_change_drops_captured_graphs(monkeypatch):
    def script():
        return [lambda l: l.step(4, 0.01, "verlet")] * 3 + [lambda l: l.set_potential(1.0, 50.0, (0.0, 0.5, 0.0))] + \
               [lambda l: l.step(4, 0.01, "verlet")] * 3
    with new(192, 2, "f32", False) as a, new(192, 2, "f32", False) as b:
        ra = calls(a, monkeypatch, True, script())
        rb = calls(b, monkeypatch, False, script())
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
    assert np.array_equal(ra[2].vector(), rb[2].vector())


def test_langevin_buffer_swap_keeps_tma_path_correct(monkeypatch):
    """A Langevin step trades phi_0's two buffers; the TMA pass must then use
    tensor maps of the new assignment.  On a static background both launch
    shapes give bitwise the same fields, and the streaming shape uses no maps."""
    def script():
        return [lambda l: l.step(3, 0.01, "verlet")] * 2 + [lambda l: l.langevin(1, 0.01, 1.0, 0.5, 0.3, 11)] + \
               [lambda l: l.step(3, 0.01, "verlet")] * 3
    monkeypatch.delenv("TL_STEP_GRAPHS", raising=False)
    with new(192, 2, "f32", False, dict(kind="tma")) as a, new(192, 2, "f32", False, dict(kind="stream")) as b:
        ra = calls(a, monkeypatch, True, script())
        rb = calls(b, monkeypatch, True, script())
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
