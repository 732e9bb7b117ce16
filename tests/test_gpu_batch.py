"""Batched ensembles (tl_batch_*) and the autotuners on the GPU.

A batch advances lattices of uneven N, 1-2 fields, different couplings,
backgrounds and seeds with one persistent launch per pass (per field count)
replayed as a CUDA graph; each lattice runs on the batch launch shape
(tl_batch_pass_config), so the results must be bitwise those of tl_step on
the lattice alone on that shape."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as o
from paper_2607_24908_gb300 import tl as T
from paper_2607_24908_gb300.workloads import white_noise_state

pytestmark = pytest.mark.gpu

JOBS = [  # N, fields, q, expanding, dtype seed
    (32, 1, 0.0, True, 11), (48, 2, 10.0, True, 12), (24, 2, 100.0, False, 13),
    (40, 1, 0.0, False, 14), (64, 2, 100.0, True, 15), (16, 1, 0.0, True, 16),
]


def make(N, nf, q, expanding, dtype):
    lat = T.Lattice(N, 0.5, nf, dtype, expanding, 1.0, 1.0, 1.0)
    lat.set_pass_config(**T.batch_pass_config(N, nf, dtype))  # the shape a batch gives it
    lat.set_potential(1.0, q, (0.0, 0.1, 0.0))
    return lat


def fill(lat, N, nf, seed, dtype):
    npd = np.float32 if dtype == "f32" else np.float64
    phi, pi = white_noise_state(N, nf, seed=seed, phi0=(1.0, 0.0), sigma_phi=1e-3, sigma_pi=1e-3)
    lat.set_state(phi.astype(npd), pi.astype(npd), 1.0, 0.0, b_from_constraint=lat.expanding)
    return phi.astype(npd), pi.astype(npd)


@pytest.mark.parametrize("dtype,integ,steps", [("f32", "verlet", 40), ("f64", "yoshida4", 10)])
def test_batch_is_bitwise_the_single_lattice_path(dtype, integ, steps):
    alone, batched = [], []
    for N, nf, q, ex, seed in JOBS:
        a = make(N, nf, q, ex, dtype)
        fill(a, N, nf, seed, dtype)
        a.step(steps, 0.01, integ)
        alone.append((*a.get_all(), a.energies()))
        a.close()
    lats = [make(N, nf, q, ex, dtype) for N, nf, q, ex, _ in JOBS]
    for lat, (N, nf, q, ex, seed) in zip(lats, JOBS):
        fill(lat, N, nf, seed, dtype)
    with T.Batch(lats) as b:
        b.step(steps // 2, 0.01, integ)
        b.step(steps - steps // 2, 0.01, integ)  # second call reuses the captured graph when n repeats
    # the reference ran one call of `steps`; rerun alone with the same split for bitwise comparison
    alone2 = []
    for N, nf, q, ex, seed in JOBS:
        a = make(N, nf, q, ex, dtype)
        fill(a, N, nf, seed, dtype)
        a.step(steps // 2, 0.01, integ)
        a.step(steps - steps // 2, 0.01, integ)
        alone2.append((*a.get_all(), a.energies()))
        a.close()
    for lat, ref, ref1 in zip(lats, alone2, alone):
        phi, pi = lat.get_all()
        E = lat.energies()
        assert np.array_equal(phi, ref[0]) and np.array_equal(pi, ref[1])
        assert np.array_equal(E.vector(), ref[2].vector()) and E.a == ref[2].a and E.b == ref[2].b
        assert E.step == steps
        # one call vs two calls differ only by rounding of the resynchronisation
        assert np.max(np.abs(phi.astype(np.float64) - ref1[0])) <= 1e-5 * np.max(np.abs(ref1[0]))
    for lat in lats:
        lat.close()


def test_batch_against_oracle_fp64():
    dt, steps = 0.01, 20
    lats, inputs = [], []
    for N, nf, q, ex, seed in JOBS[:4]:
        lat = make(N, nf, q, ex, "f64")
        inputs.append(fill(lat, N, nf, seed, "f64"))
        lats.append(lat)
    with T.Batch(lats) as b:
        b.step(steps, dt, "verlet")
    for lat, (phi0, pi0), (N, nf, q, ex, seed) in zip(lats, inputs, JOBS[:4]):
        p = o.Params(N=N, nf=nf, kIR=0.5, expanding=ex, alpha=1.0, lam=1.0, q=q, m2=(0.0, 0.1, 0.0))
        b0 = math.sqrt(float(np.sum(o.energies(p, phi0, pi0, 1.0))) / 3.0) if ex else 0.0
        ophi, opi, oa, ob = o.run(p, phi0, pi0, 1.0, b0, dt, steps, o.VERLET)
        phi, pi = lat.get_all()
        assert np.max(np.abs(phi - ophi)) / np.max(np.abs(ophi)) < 1e-12
        assert np.max(np.abs(pi - opi)) / np.max(np.abs(opi)) < 1e-12
        if ex:
            E = lat.energies()
            assert abs(E.a - oa) / oa < 1e-12 and abs(E.b - ob) / ob < 1e-12
        lat.close()


def test_autotune_keeps_state_and_parity(tmp_path, monkeypatch):
    monkeypatch.setenv("TL_TUNE_FILE", str(tmp_path / "tune.txt"))
    N, nf = 64, 2
    p = o.Params(N=N, nf=nf, kIR=0.5, expanding=True, alpha=1.0, lam=1.0, q=100.0)
    phi0, pi0 = white_noise_state(N, nf, seed=3, phi0=(1.0, 0.0), sigma_phi=1e-3, sigma_pi=1e-3)
    lat = make(N, nf, 100.0, True, "f64")
    lat.set_potential(1.0, 100.0, (0.0, 0.0, 0.0))
    lat.set_state(phi0, pi0, 1.0, 0.0, True)
    E0 = lat.energies()
    ms = lat.autotune()
    assert ms > 0
    phi, pi = lat.get_all()
    assert np.array_equal(phi, phi0) and np.array_equal(pi, pi0)  # identity passes
    E1 = lat.energies()
    assert E1.a == E0.a and E1.b == E0.b
    lat.step(10, 0.005, "yoshida4")
    b0 = math.sqrt(float(np.sum(o.energies(p, phi0, pi0, 1.0))) / 3.0)
    ophi, opi, oa, ob = o.run(p, phi0, pi0, 1.0, b0, 0.005, 10, o.YOSHIDA4)
    phi, pi = lat.get_all()
    assert np.max(np.abs(phi - ophi)) / np.max(np.abs(ophi)) < 1e-12
    lat.close()
    # the cache file: JSON lines, and a fresh process takes the entry instead of re-timing
    rec = json.loads((tmp_path / "tune.txt").read_text().strip().splitlines()[-1])
    assert (rec["N"], rec["fields"], rec["dtype"]) == (64, 2, T.F64) and rec["variant"] in (0, 1)
    assert abs(rec["ms"] - ms) < 1e-5
    code = ("from paper_2607_24908_gb300 import tl as T; import numpy as np\n"
            "lat = T.Lattice(64, 0.5, 2, 'f64', True, 1.0, 1.0, 1.0)\n"
            "lat.set_potential(1.0, 100.0, (0.0, 0.0, 0.0))\n"
            "lat.set_state(np.ones((2, 64, 64, 64)), np.zeros((2, 64, 64, 64)), 1.0, 1.0)\n"
            "print(repr(lat.autotune())); lat.close()\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, TL_TUNE_FILE=str(tmp_path / "tune.txt")))
    assert out.returncode == 0, out.stderr[-2000:]
    assert float(out.stdout.strip().splitlines()[-1]) == rec["ms"]
    assert len((tmp_path / "tune.txt").read_text().strip().splitlines()) == 1  # nothing re-timed or appended


def test_ensemble_recipe_fp32_batch_against_oracle():
    """The batched-ensemble recipe (FP32 storage with FP64 reductions, expanding with alpha 1, kIR 0.5,
    V = phi^4/4 + (q/2) phi^2 chi^2, Philox vacuum fluctuations A = 1e-10 drawn by the oracle, Verlet
    dt 0.01): 8 jobs with N in {32, 48}, 1-2 fields, q in {0, 10, 100}, own seeds, 100 steps in one
    batch; every job against the oracle run from the same FP32-rounded state."""
    from _tol import f32_pi_tol, normwise
    rng = np.random.default_rng(4242)
    jobs = [(int(rng.choice([32, 48])), int(rng.integers(1, 3)), float(rng.choice([0.0, 10.0, 100.0])), 100 + k)
            for k in range(8)]
    dt, steps = 0.01, 100
    lats, refs = [], []
    for N, nf, q, seed in jobs:
        p = o.Params(N=N, nf=nf, kIR=0.5, expanding=True, alpha=1.0, lam=1.0, q=q, m2=(0.0, 0.0, 0.0))
        phi, pi, _, _ = o.init_fluctuations(p, seed, o.InitSpec(A=1e-10, meff2=(3.0, q, 0.0), phi0=(1.0, 0.0, 0.0)))
        phi32, pi32 = phi.astype(np.float32), pi.astype(np.float32)
        lat = T.Lattice(N, 0.5, nf, "f32", True, 1.0, 1.0, 1.0)
        lat.set_potential(1.0, q, (0.0, 0.0, 0.0))
        lat.set_state(phi32, pi32, 1.0, 0.0, b_from_constraint=True)
        lats.append(lat)
        ph64, pi64 = phi32.astype(np.float64), pi32.astype(np.float64)
        b0 = math.sqrt(float(np.sum(o.energies(p, ph64, pi64, 1.0))) / 3.0)
        refs.append((p, o.run(p, ph64, pi64, 1.0, b0, dt, steps, o.VERLET)))
    with T.Batch(lats) as b:
        b.step(steps, dt, "verlet")
    for lat, (p, (ophi, opi, oa, ob)), job in zip(lats, refs, jobs):
        phi, pi = lat.get_all()
        E = lat.energies()
        assert normwise(phi, ophi) < 1e-5, job
        tol = f32_pi_tol(p, steps + 1, float(np.max(np.abs(ophi))), float(np.max(np.abs(opi))))
        assert normwise(pi, opi) < tol, (job, normwise(pi, opi), tol)
        assert abs(E.a - oa) / oa < 1e-5 and abs(E.b - ob) / ob < 1e-5, job
        lat.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_autotune_keeps_state_and_steps_bitwise_like_each_member_alone(dtype, tmp_path, monkeypatch):
    """tl_batch_autotune times member shapes and batch options with identity passes: it leaves
    every state untouched; the tuned batch then steps each member bitwise like tl_step on the
    member alone on its tuned shape (tl_batch_pass_config reports it); the shapes and options
    go to the cache file; and FP64 members still match the oracle to 1e-12."""
    monkeypatch.setenv("TL_TUNE_FILE", str(tmp_path / "tune.txt"))
    dt, steps = 0.01, 12
    # the shapes the members start on (their b0 from the constraint is reduced under them)
    before = {(N, nf): T.batch_pass_config(N, nf, dtype) for N, nf, _, _, _ in JOBS}
    lats, inputs = [], []
    for N, nf, q, ex, seed in JOBS:
        lat = make(N, nf, q, ex, dtype)
        inputs.append(fill(lat, N, nf, seed, dtype))
        lats.append(lat)
    E0 = [lat.energies() for lat in lats]
    with T.Batch(lats) as b:
        ms = b.autotune()
        assert ms > 0
        opts = b.options()
        assert opts["prefetch"] in (0, 3) and opts["split"] in (0, 1) and opts["share"] in (0, 1)
        for lat, (phi0, pi0), e0 in zip(lats, inputs, E0):
            phi, pi = lat.get_all()
            assert np.array_equal(phi, phi0) and np.array_equal(pi, pi0)
            e1 = lat.energies()
            assert e1.a == e0.a and e1.b == e0.b
        b.step(steps, dt, "verlet")
    recs = [json.loads(line) for line in (tmp_path / "tune.txt").read_text().strip().splitlines()]
    shapes = {(r["batch_shape"]["N"], r["batch_shape"]["fields"]): r["batch_shape"] for r in recs
              if "batch_shape" in r}
    assert set(shapes) == {(N, nf) for N, nf, _, _, _ in JOBS}
    assert sum("batch_options" in r for r in recs) == 1
    for lat, (N, nf, q, ex, seed), (phi0, pi0) in zip(lats, JOBS, inputs):
        cfg = T.batch_pass_config(N, nf, dtype)
        assert cfg["z_chunk"] == shapes[(N, nf)]["z_chunk"] == lat.pass_config()["z_chunk"]
        # the twin replays the member's history: state and b0 on the starting shape, then the tuned one
        twin = T.Lattice(N, 0.5, nf, dtype, ex, 1.0, 1.0, 1.0)
        twin.set_pass_config(**before[(N, nf)])
        twin.set_potential(1.0, q, (0.0, 0.1, 0.0))
        fill(twin, N, nf, seed, dtype)
        twin.set_pass_config(**cfg)
        twin.step(steps, dt, "verlet")
        phi, pi = lat.get_all()
        tphi, tpi = twin.get_all()
        E, tE = lat.energies(), twin.energies()
        assert np.array_equal(phi, tphi) and np.array_equal(pi, tpi), (N, nf)
        assert np.array_equal(E.vector(), tE.vector()) and E.a == tE.a and E.b == tE.b
        twin.close()
        if dtype == "f64":
            p = o.Params(N=N, nf=nf, kIR=0.5, expanding=ex, alpha=1.0, lam=1.0, q=q, m2=(0.0, 0.1, 0.0))
            b0 = math.sqrt(float(np.sum(o.energies(p, phi0, pi0, 1.0))) / 3.0) if ex else 0.0
            ophi, opi, oa, ob = o.run(p, phi0, pi0, 1.0, b0, dt, steps, o.VERLET)
            assert np.max(np.abs(phi - ophi)) / np.max(np.abs(ophi)) < 1e-12
            assert np.max(np.abs(pi - opi)) / np.max(np.abs(opi)) < 1e-12
            if ex:
                assert abs(E.a - oa) / oa < 1e-12 and abs(E.b - ob) / ob < 1e-12
        lat.close()


_TMA_GROUP_SCRIPT = r"""
import json, math, os, sys
import numpy as np
import torch
sys.path.insert(0, os.getcwd())
import oracle as o
from paper_2607_24908_gb300 import tl as T
from paper_2607_24908_gb300.workloads import white_noise_state
jobs = json.loads(sys.argv[1])
sms = torch.cuda.get_device_properties(0).multi_processor_count
path = sys.argv[2]
with open(path, "w") as fh:  # batch shapes on the TMA pass for every class, read at the first batch call
    for dt in (0, 1):
        for N, nf, q, ex, seed, zc in jobs:
            fh.write(json.dumps({"batch_shape": {"N": N, "fields": nf, "dtype": dt, "sms": sms, "variant": 1,
                                                 "z_chunk": zc, "tile_x": 0, "prefetch": 0}}) + "\n")
os.environ["TL_TUNE_FILE"] = path
out = {}
for dtype in ("f32", "f64"):
    npd = np.float32 if dtype == "f32" else np.float64
    def make(N, nf, q, ex):
        lat = T.Lattice(N, 0.5, nf, dtype, ex, 1.0, 1.0, 1.0)
        cfg = T.batch_pass_config(N, nf, dtype)
        assert cfg["kind"] == "tma", cfg
        lat.set_pass_config(**cfg)
        lat.set_potential(1.0, q, (0.0, 0.1, 0.0))
        return lat
    def fill(lat, N, nf, seed, ex):
        phi, pi = white_noise_state(N, nf, seed=seed, phi0=(1.0, 0.0, 0.0), sigma_phi=1e-3, sigma_pi=1e-3)
        lat.set_state(phi.astype(npd), pi.astype(npd), 1.0, 0.0, b_from_constraint=ex)
        return phi.astype(npd), pi.astype(npd)
    lats, inputs = [], []
    for N, nf, q, ex, seed, zc in jobs:
        lat = make(N, nf, q, ex); inputs.append(fill(lat, N, nf, seed, ex)); lats.append(lat)
    with T.Batch(lats) as b:
        b.step(6, 0.01, "verlet")
        b.step(6, 0.01, "verlet")  # the second call replays the captured graph
    worst = 0.0
    for lat, (N, nf, q, ex, seed, zc), (phi0, pi0) in zip(lats, jobs, inputs):
        assert lat.pass_config()["kind"] == "tma"
        twin = make(N, nf, q, ex); fill(twin, N, nf, seed, ex)
        twin.step(6, 0.01, "verlet"); twin.step(6, 0.01, "verlet")
        phi, pi = lat.get_all(); tphi, tpi = twin.get_all()
        E, tE = lat.energies(), twin.energies()
        assert np.array_equal(phi, tphi) and np.array_equal(pi, tpi), (dtype, N, nf)
        assert np.array_equal(E.vector(), tE.vector()) and E.a == tE.a and E.b == tE.b, (dtype, N, nf)
        twin.close()
        if dtype == "f64":
            p = o.Params(N=N, nf=nf, kIR=0.5, expanding=ex, alpha=1.0, lam=1.0, q=q, m2=(0.0, 0.1, 0.0))
            b0 = math.sqrt(float(np.sum(o.energies(p, phi0, pi0, 1.0))) / 3.0) if ex else 0.0
            ophi, opi, oa, ob = o.run(p, phi0, pi0, 1.0, b0, 0.01, 12, o.VERLET)
            worst = max(worst, float(np.max(np.abs(phi - ophi)) / np.max(np.abs(ophi))),
                        float(np.max(np.abs(pi - opi)) / np.max(np.abs(opi))))
            if ex:
                worst = max(worst, abs(E.a - oa) / oa, abs(E.b - ob) / ob)
        lat.close()
    out[dtype] = worst
print("RESULT " + json.dumps(out))
"""


def test_tma_group_is_bitwise_the_single_lattice_tma_pass(tmp_path):
    """Members whose batch shape is the TMA pass (here from TL_TUNE_FILE entries, read by a fresh
    process) run through the grouped TMA kernel (one CTA per item, each job's tensor maps in global
    memory): fields, energies, a and a' bitwise those of each member alone on the same shape, across a
    graph replay; FP64 members against the oracle to 1e-12."""
    jobs = [(N, nf, q, ex, seed, zc) for (N, nf, q, ex, seed), zc in zip(JOBS, (16, 8, 24, 16, 32, 16))]
    jobs += [(28, 3, 50.0, True, 17, 28), (36, 3, 10.0, False, 18, 12)]  # three-field TMA group
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _TMA_GROUP_SCRIPT, json.dumps(jobs), str(tmp_path / "tune.txt")],
                         cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-3000:]
    res = json.loads(out.stdout.strip().splitlines()[-1][len("RESULT "):])
    assert res["f64"] < 1e-12, res


def test_batch_membership_rules_and_a_batch_of_one():
    """A lattice belongs to at most one batch at a time (a second batch is refused until the first
    is destroyed), lattices of different precisions cannot share a batch, and a batch of one lattice
    steps bitwise like that lattice alone on its batch shape."""
    N, nf, q, ex, seed = JOBS[1]
    a = make(N, nf, q, ex, "f32")
    fill(a, N, nf, seed, "f32")
    other = make(32, 1, 0.0, True, "f64")
    fill(other, 32, 1, 5, "f64")
    with pytest.raises(T.TLError) as e:
        T.Batch([a, other])
    assert e.value.code == T.EINVAL
    b1 = T.Batch([a])
    with pytest.raises(T.TLError) as e:
        T.Batch([a])
    assert e.value.code == T.EINVAL and "already in a batch" in str(e.value)
    b1.step(8, 0.01, "verlet")
    b1.close()
    T.Batch([a]).close()  # allowed again once the first batch is gone
    twin = make(N, nf, q, ex, "f32")
    fill(twin, N, nf, seed, "f32")
    twin.step(8, 0.01, "verlet")
    assert np.array_equal(a.get_all()[0], twin.get_all()[0]) and np.array_equal(a.get_all()[1], twin.get_all()[1])
    Ea, Et = a.energies(), twin.energies()
    assert np.array_equal(Ea.vector(), Et.vector()) and Ea.a == Et.a and Ea.b == Et.b
    for lat in (a, other, twin):
        lat.close()
