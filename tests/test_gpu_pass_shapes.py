"""Launch shapes of the fused pass (tl_set_pass_config) on the GPU.

Every shape computes each site with the same operations in the same order, so
on a static background the fields after any number of steps are bitwise the
same whichever shape ran them; only the energy sums (whose order follows the
CTA tiles) differ, by rounding.  The sizes are chosen for ragged tiles: rows
of 25 or 11 threads that straddle warps, last tile rows past the lattice edge
(whole warps with nothing to do in the TMA ring), several z-chunks."""
import numpy as np
import pytest

import oracle as o
from paper_2607_24908_gb300 import tl as T
from paper_2607_24908_gb300.workloads import white_noise_state

pytestmark = pytest.mark.gpu

SHAPES = [
    dict(kind="stream"),
    dict(kind="stream", threads=512),
    dict(kind="stream", tile_x=8, z_chunk=5),
    dict(kind="tma"),
    dict(kind="tma", warps=15),
    dict(kind="tma", warps=7, stages=3, z_chunk=7),
    dict(kind="tma", warps=15, stages=8, z_chunk=1),
]


def run(N, nf, dtype, shape, steps, integ="verlet", expanding=False, seed=5):
    npd = np.float32 if dtype == "f32" else np.float64
    phi, pi = white_noise_state(N, nf, seed=seed, phi0=(1.0, 0.0, 0.0)[:nf], sigma_phi=1e-2, sigma_pi=1e-2)
    lat = T.Lattice(N, 0.5, nf, dtype, expanding, 1.0, 1.0, 1.0)
    try:
        lat.set_pass_config(**shape)
        lat.set_potential(1.0, 10.0, (0.0, 0.2, 0.1))
        lat.set_state(phi.astype(npd), pi.astype(npd), 1.0, 0.0, b_from_constraint=expanding)
        lat.step(steps, 0.01, integ)
        return (*lat.get_all(), lat.energies(), lat.pass_config())
    finally:
        lat.close()


@pytest.mark.parametrize("N,nf,dtype", [(100, 2, "f32"), (44, 3, "f32"), (36, 1, "f64"), (52, 2, "f64"),
                                        (24, 2, "f32"), (128, 1, "f32")])
def test_fields_bitwise_equal_across_shapes(N, nf, dtype):
    ref = None
    for shape in SHAPES:
        phi, pi, E, cfg = run(N, nf, dtype, shape, steps=6)
        assert cfg["kind"] == shape["kind"]
        if shape.get("warps"):
            assert cfg["warps"] == shape["warps"]
        if ref is None:
            ref = (phi, pi, E)
            continue
        assert np.array_equal(phi, ref[0]), shape
        assert np.array_equal(pi, ref[1]), shape
        tol = 1e-5 if dtype == "f32" else 1e-12
        assert np.max(np.abs(E.vector() - ref[2].vector())) <= tol * np.sum(np.abs(ref[2].vector())), shape


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "-".join(f"{k}{v}" for k, v in s.items()))
def test_each_shape_against_oracle_expanding_fp64(shape):
    """Expanding FP64 run of 5 Yoshida steps on a 40^3 lattice with two fields
    (ragged in y for every TMA tiling) against the oracle to 1e-12."""
    N, nf, steps, dt = 40, 2, 5, 0.01
    phi0, pi0 = white_noise_state(N, nf, seed=9, phi0=(1.0, 0.0), sigma_phi=1e-2, sigma_pi=1e-2)
    p = o.Params(N=N, nf=nf, kIR=0.5, expanding=True, alpha=1.0, lam=1.0, q=10.0, m2=(0.0, 0.2, 0.0))
    lat = T.Lattice(N, 0.5, nf, "f64", True, 1.0, 1.0, 1.0)
    try:
        lat.set_pass_config(**shape)
        lat.set_potential(1.0, 10.0, (0.0, 0.2, 0.0))
        lat.set_state(phi0, pi0, 1.0, 0.0, b_from_constraint=True)
        E0 = lat.energies()
        lat.step(steps, dt, "yoshida4")
        phi, pi = lat.get_all()
        E = lat.energies()
    finally:
        lat.close()
    b0 = np.sqrt(np.sum(o.energies(p, phi0, pi0, 1.0)) / 3.0)
    assert abs(E0.b - b0) / b0 < 1e-12
    ophi, opi, oa, ob = o.run(p, phi0, pi0, 1.0, b0, dt, steps, o.YOSHIDA4)
    assert np.max(np.abs(phi - ophi)) / np.max(np.abs(ophi)) < 1e-12
    assert np.max(np.abs(pi - opi)) / np.max(np.abs(opi)) < 1e-12
    assert abs(E.a - oa) / oa < 1e-12 and abs(E.b - ob) / ob < 1e-12


def test_default_shape_and_errors():
    with T.Lattice(192, 0.5, 2, "f32") as big, T.Lattice(128, 0.5, 2, "f32") as small:
        cfg = big.pass_config()
        assert cfg["kind"] == "tma" and cfg["warps"] == 7 and 3 <= cfg["stages"] <= 8 and cfg["z_chunk"] == 48
        assert small.pass_config()["kind"] == "stream"
        with T.Lattice(256, 0.5, 1, "f32") as one:  # FP32 from 192: TMA, 64-plane chunks below 512
            c1 = one.pass_config()
            assert (c1["kind"], c1["warps"], c1["z_chunk"]) == ("tma", 7, 64)
        with T.Lattice(512, 0.5, 1, "f32") as mid:  # 15 + 1 warps, 160-plane chunks around 512
            c3 = mid.pass_config()
            assert (c3["kind"], c3["warps"], c3["z_chunk"]) == ("tma", 15, 160)
        with T.Lattice(384, 0.5, 1, "f32") as mid:  # 7 + 1 warps, 56-plane chunks around 384
            c5 = mid.pass_config()
            assert (c5["kind"], c5["warps"], c5["z_chunk"]) == ("tma", 7, 56)
        with T.Lattice(256, 0.5, 2, "f64") as f64:  # FP64: the streaming pass, 32-plane chunks from 128
            c4 = f64.pass_config()
            assert (c4["kind"], c4["z_chunk"]) == ("stream", 32)
        bad = [dict(kind="tma", warps=8), dict(kind="tma", stages=2), dict(kind="tma", stages=9),
               dict(kind="tma", tile_x=16), dict(kind="stream", warps=7), dict(kind="stream", tile_x=12),
               dict(kind="stream", threads=128), dict(kind="stream", z_chunk=193)]
        for shape in bad:
            with pytest.raises(T.TLError) as e:
                big.set_pass_config(**shape)
            assert e.value.code == T.EINVAL, shape
        assert big.pass_config() == cfg  # a refused change leaves the shape alone
        big.set_pass_config("stream", tile_x=16, threads=512, z_chunk=32)
        c2 = big.pass_config()
        assert (c2["kind"], c2["tile_x"], c2["threads"], c2["z_chunk"]) == ("stream", 16, 512, 32)


def test_batch_moves_members_to_the_batch_shape():
    N, nf = 128, 2
    phi, pi = white_noise_state(N, nf, seed=4, phi0=(1.0, 0.0), sigma_phi=1e-2, sigma_pi=1e-2)

    def new():
        lat = T.Lattice(N, 0.5, nf, "f32", False, 1.0, 1.0, 1.0)
        lat.set_potential(1.0, 10.0, (0.0, 0.2, 0.0))
        lat.set_state(phi.astype(np.float32), pi.astype(np.float32))
        return lat

    with new() as ref:  # alone, on the batch shape
        ref.set_pass_config(**T.batch_pass_config(N, nf, "f32"))
        ref.step(10, 0.01, "verlet")
        rphi, rpi = ref.get_all()
        rE = ref.energies().vector()
    lats = [new(), new()]
    for lat in lats:
        lat.set_pass_config("tma")
    with T.Batch(lats) as b:
        with pytest.raises(T.TLError) as e:
            lats[0].set_pass_config("tma")
        assert e.value.code == T.ESTATE
        b.step(10, 0.01, "verlet")
    want = T.batch_pass_config(N, nf, "f32")  # the untuned rule (streaming, 32-plane chunks) unless tuned
    for lat in lats:
        cfg = lat.pass_config()
        assert cfg["kind"] == want["kind"] and cfg["z_chunk"] == want["z_chunk"]
        p, q = lat.get_all()
        assert np.array_equal(p, rphi) and np.array_equal(q, rpi)
        assert np.array_equal(lat.energies().vector(), rE)
        lat.close()


def test_ragged_at_scale_tma_default_equals_stream():
    """N = 500, two FP32 fields: TMA shapes with ragged tiles in every direction (x tiles
    of 128 with a last one of 116 sites; 7 + 1 warps: y tiles of 7 rows with a last one
    of 3, z-chunks of 64 planes with a last one of 52; the default 15 + 1 warps: y tiles
    of 15 rows with a last one of 5, z-chunks of 96 with a last one of 20); two Verlet
    steps give bitwise the fields of the streaming kernel."""
    N, nf = 500, 2
    rng = np.random.default_rng(17)
    phi = (rng.standard_normal((nf, N, N, N), dtype=np.float32) * np.float32(1e-2)
           + np.array([1.0, 0.0], np.float32)[:, None, None, None])
    pi = rng.standard_normal((nf, N, N, N), dtype=np.float32) * np.float32(1e-2)
    out = []
    for shape in (None, dict(kind="tma", warps=7, z_chunk=64), dict(kind="stream")):
        with T.Lattice(N, 0.1, nf, "f32") as lat:
            if shape:
                lat.set_pass_config(**shape)
            else:
                cfg = lat.pass_config()
                assert (cfg["kind"], cfg["warps"], cfg["z_chunk"]) == ("tma", 15, 96)
            lat.set_potential(1.0, 10.0, (0.0, 0.2, 0.0))
            lat.set_state(phi, pi)
            lat.step(2, 0.01, "verlet")
            out.append(lat.get_all())
    for o in out[:2]:
        assert np.array_equal(o[0], out[2][0]) and np.array_equal(o[1], out[2][1])


def test_every_reported_shape_can_be_set_again():
    """tl_get_pass_config's resolved shape (automatic values filled in, a row
    narrower than the requested tile width reported as its own width) is
    accepted by tl_set_pass_config and gives the same shape: what a checkpoint
    restores."""
    for N, dtype in ((16, "f32"), (48, "f32"), (100, "f32"), (256, "f32"), (12, "f64"), (40, "f64"), (96, "f64")):
        for shape in [None] + SHAPES:
            with T.Lattice(N, 0.5, 2, dtype) as lat:
                if shape is not None:
                    lat.set_pass_config(**shape)
                cfg = lat.pass_config()
            with T.Lattice(N, 0.5, 2, dtype) as other:
                other.set_pass_config(**cfg)
                assert other.pass_config() == cfg, (N, dtype, shape, cfg, other.pass_config())



@pytest.mark.parametrize("N,nf,dtype", [(300, 2, "f32"), (136, 2, "f64"), (72, 1, "f64")])
def test_tma_interior_and_edge_tiles_equal_stream(N, nf, dtype):
    """Lattices with tiles inside the lattice and at both x-edges, the last one
    ragged (FP32 300 = 128 + 128 + 44 sites, FP64 136 = 64 + 64 + 8 and
    72 = 64 + 8): the edge tiles' halo columns (the periodic image beyond each
    edge) give bitwise the fields of the streaming kernel, under the default
    and a 15 + 1 warp TMA shape, in a static and an expanding background."""
    rng = np.random.default_rng(N)
    npd = np.float32 if dtype == "f32" else np.float64
    phi = (rng.standard_normal((nf, N, N, N)) * 1e-2 + np.array([1.0, 0.0][:nf])[:, None, None, None]).astype(npd)
    pi = (rng.standard_normal((nf, N, N, N)) * 1e-2).astype(npd)
    for expanding in (False, True):
        out = []
        for shape in (dict(kind="stream"), dict(kind="tma"), dict(kind="tma", warps=15, z_chunk=40)):
            with T.Lattice(N, 0.3, nf, dtype, expanding, 1.0, 1.0, 1.0) as lat:
                lat.set_pass_config(**shape)
                lat.set_potential(1.0, 10.0, (0.0, 0.2, 0.0))
                lat.set_state(phi, pi, 1.0, 0.0, b_from_constraint=expanding)
                lat.step(3, 0.01, "verlet")
                out.append((*lat.get_all(), lat.energies()))
        for o in out[1:]:
            if not expanding:  # fields do not depend on the reduction order
                assert np.array_equal(o[0], out[0][0]) and np.array_equal(o[1], out[0][1])
            else:  # a, a' do (energy sums per tile): agree to rounding
                tol = 1e-5 if dtype == "f32" else 1e-12
                assert np.max(np.abs(o[0] - out[0][0])) <= tol * np.max(np.abs(out[0][0]))
                assert abs(o[2].a - out[0][2].a) <= tol * out[0][2].a
