"""Writes tests/golden/oracle_cases.json: small seeded cases evaluated by the
oracle alone (regression values: a later change to the oracle's arithmetic
shows up as a mismatch in tests/test_golden.py and has to name the passage
that justifies it).  Run from the repository root:
    python tests/golden/make_oracle_cases.py"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as o  # noqa: E402
from oracle import su2 as osu2  # noqa: E402
from paper_2607_24908_gb300.workloads import plane_wave, random_su2_links, white_noise_state  # noqa: E402


def checksum(a):
    a = np.asarray(a, dtype=np.float64)
    return [float(a.sum()), float((a * a).sum())]


def cases():
    out = {}
    # free plane wave, static, 100 Verlet steps
    p = o.Params(N=16, nf=1, kIR=0.5, lam=0.0, q=0.0, m2=(1.0, 0.0, 0.0))
    phi = plane_wave(16, (1, 2, 3))[None]
    f, g, a, b = o.run(p, phi, np.zeros_like(phi), 1.0, 0.0, 0.05, 100, o.VERLET)
    out["plane_wave_16_verlet_100"] = {"phi": checksum(f), "pi": checksum(g), "E": o.energies(p, f, g, 1.0).tolist()}
    # two coupled fields, expanding (alpha = 1), 20 Yoshida steps
    p = o.Params(N=8, nf=2, kIR=0.5, expanding=True, alpha=1.0, lam=1.0, q=10.0, m2=(0.0, 0.2, 0.0))
    phi, pi = white_noise_state(8, 2, seed=3, phi0=(1.0, 0.0), sigma_phi=1e-2, sigma_pi=1e-2)
    b0 = float(np.sqrt(np.sum(o.energies(p, phi, pi, 1.0)) / 3.0))
    f, g, a, b = o.run(p, phi, pi, 1.0, b0, 0.01, 20, o.YOSHIDA4)
    out["two_field_expanding_8_yoshida_20"] = {"phi": checksum(f), "pi": checksum(g), "a": a, "b": b,
                                               "E": o.energies(p, f, g, a).tolist()}
    # initial Gaussian field and its binned spectrum
    p = o.Params(N=16, nf=1, kIR=0.5, lam=1.0)
    f, g, a, b = o.init_fluctuations(p, 11, o.InitSpec(A=1e-4, meff2=(3.0, 0.0, 0.0), phi0=(1.0, 0.0, 0.0)))
    k, P, cnt = o.spectrum(p, f[0])
    out["init_16_seed11"] = {"phi": checksum(f), "P_bins_0_4": [float(x) for x in P[:5]],
                             "count_bins_0_4": [int(x) for x in cnt[:5]]}
    # Langevin phi^4, 10 steps
    phi = np.full((8, 8, 8), 0.5)
    f = o.langevin_run(8, 0.5, phi, 0.01, 10, 1.0, 0.5, 0.3, seed=7)
    out["langevin_8_10"] = {"phi": checksum(f)}
    # SU(2) Yang-Mills, 5 leapfrog steps on 4^3
    U = random_su2_links(4, seed=5, amp=0.5)
    E = np.zeros((3, 3, 4, 4, 4))
    U1, E1 = osu2.step(U, E, 0.02, 5)
    out["su2_4_5"] = {"U": checksum(U1), "E": checksum(E1), "plaquette_energy": osu2.plaquette_energy(U1),
                      "electric_energy": osu2.electric_energy(E1)}
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_cases.json")
    with open(path, "w") as fh:
        json.dump(cases(), fh, indent=1)
        fh.write("\n")
    print("wrote", path)
