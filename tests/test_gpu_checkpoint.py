"""Checkpoint and resume: a lattice restored from a checkpoint (state at an
integer time, a, a', the clock, the potential and the pass shape, written to
an .npz file and read back) continues bitwise as the lattice it was taken
from under the same tl_step calls: fields, energies, a, a', the Hubble
residual and the clock.  Langevin runs resume their noise stream too."""
import numpy as np
import pytest

from paper_2607_24908_gb300 import tl as T

pytestmark = pytest.mark.gpu

CASES = [
    # N, fields, dtype, integrator, pass shape (None: the library default)
    (24, 2, "f64", "verlet", None),
    (32, 3, "f64", "yoshida4", None),
    (32, 1, "f32", "leapfrog", None),
    (48, 2, "f32", "yoshida4", {"kind": "stream", "z_chunk": 8, "tile_x": 16}),
    (192, 2, "f32", "verlet", None),  # the TMA pass by default
]


def _lattice(N, nf, dtype):
    return T.Lattice(N, 0.5, nf, dtype, True, 1.0, 1.0, 1.0)


def _snapshot(lat):
    E = lat.energies()
    phi, pi = lat.get_all()
    return phi, pi, E, lat.clock()


@pytest.mark.parametrize("N,nf,dtype,integ,shape", CASES)
def test_resumed_run_is_bitwise_the_uninterrupted_one(tmp_path, N, nf, dtype, integ, shape):
    with _lattice(N, nf, dtype) as lat:
        if shape:
            lat.set_pass_config(**shape)
        lat.set_potential(1.0, 100.0, (0.0, 0.1, 0.0))
        lat.init_fluctuations(seed=17, A=1e-4, meff2=(3.0, 100.0, 100.0), phi0=(1.0, 0.0, 0.0))
        lat.step(7, 0.01, integ)
        T.save_checkpoint(tmp_path / "ck.npz", lat.checkpoint())
        lat.step(9, 0.01, integ)
        phi, pi, E, clk = _snapshot(lat)
    with _lattice(N, nf, dtype) as res:
        res.restore(T.load_checkpoint(tmp_path / "ck.npz"))
        assert res.clock()["step"] == 7
        res.step(9, 0.01, integ)
        rphi, rpi, rE, rclk = _snapshot(res)
    assert np.array_equal(rphi, phi) and np.array_equal(rpi, pi)
    assert np.array_equal(rE.vector(), E.vector())
    assert (rE.a, rE.b, rE.hubble_resid) == (E.a, E.b, E.hubble_resid)
    assert rclk == clk and clk["step"] == 16 and rE.step == 16 and rE.time == E.time


def test_langevin_resumes_its_noise_stream(tmp_path):
    with T.Lattice(32, 0.5, 1, "f32") as lat:
        lat.set_potential(1.0, 0.0, (0.0, 0.0, 0.0))
        lat.init_fluctuations(seed=3, A=1e-3, meff2=(1.0, 0.0, 0.0), phi0=(0.5, 0.0, 0.0))
        lat.langevin(6, 0.01, 1.0, 0.1, 0.5, seed=99)
        ck = lat.checkpoint()
        assert ck["langevin_steps"] == 6
        T.save_checkpoint(tmp_path / "lv.npz", ck)
        lat.langevin(6, 0.01, 1.0, 0.1, 0.5, seed=99)
        phi = lat.get(0, 0)
    with T.Lattice(32, 0.5, 1, "f32") as res:
        res.restore(T.load_checkpoint(tmp_path / "lv.npz"))
        res.langevin(6, 0.01, 1.0, 0.1, 0.5, seed=99)
        assert np.array_equal(res.get(0, 0), phi)
        assert res.clock()["langevin_steps"] == 12


def test_restore_refuses_a_mismatched_lattice(tmp_path):
    with _lattice(16, 1, "f64") as lat:
        lat.set_potential(1.0, 0.0, (0.0, 0.0, 0.0))
        lat.init_fluctuations(seed=1, A=1e-4)
        ck = lat.checkpoint()
    for args in ((16, 1, "f32"), (16, 2, "f64"), (20, 1, "f64")):
        with _lattice(*args) as other:
            with pytest.raises(ValueError):
                other.restore(ck)
    with _lattice(16, 1, "f64") as other:  # counters need a state, and are checked
        with pytest.raises(T.TLError):
            other.set_clock(3, 0.1)
        other.restore(ck)
        for bad in ((-1, 0.0, 0), (0, float("nan"), 0), (0, 0.0, -2)):
            with pytest.raises(T.TLError):
                other.set_clock(*bad)
