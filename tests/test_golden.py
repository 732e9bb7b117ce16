"""Stored expected values (tests/golden/).

- minimal_example_sec2_1.json: the one number the paper prints for a worked
  example (Sec. 2.1: the average of 2 plus a configuration-space Gaussian
  field on 128^3).  Its exact digits depend on the paper's own seeding of its
  generator, which the paper does not define, so what is checked is our
  reading of `average` (mean over the N^3 sites) and of the field (unit
  variance per site): under it the printed value lies within 4 standard
  errors of 2, and an average of 2 plus unit white noise on 128^3 does too.
- oracle_cases.json: small seeded cases written by make_oracle_cases.py,
  which calls only oracle/; the oracle must keep reproducing them."""
import json
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    with open(os.path.join(HERE, "golden", name)) as fh:
        return json.load(fh)


def test_paper_minimal_example_average():
    g = load("minimal_example_sec2_1.json")
    N = g["lattice_N"]
    se = 1.0 / math.sqrt(N ** 3)  # standard error of the mean of N^3 unit-variance sites
    assert abs(g["printed_average"] - 2.0) < 4 * se
    rng = np.random.default_rng(0)
    assert abs(np.mean(2.0 + rng.standard_normal((N, N, N))) - 2.0) < 4 * se


def _close(x, ref, rtol=1e-11):
    x, ref = np.asarray(x, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return bool(np.all(np.abs(x - ref) <= rtol * np.maximum(1.0, np.abs(ref))))


def test_oracle_reproduces_stored_cases():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_oracle_cases", os.path.join(HERE, "golden", "make_oracle_cases.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    now = mod.cases()
    ref = load("oracle_cases.json")
    assert set(now) == set(ref)
    for case, vals in ref.items():
        for key, v in vals.items():
            assert _close(now[case][key], v), (case, key, now[case][key], v)
