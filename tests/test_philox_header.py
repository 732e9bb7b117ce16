"""The library's Philox-2x64-10 (csrc/tl_philox.cuh, the generator of the
initial fields, the Langevin noise and the random SU(2) links) compiled for
the host and checked against the generator's published known answers
(tests/golden/philox2x64_10_kat.json): the rounds, constants and word order
that the device shares; its host 128-bit product against Python's integers.
CPU only (the device's product, __umul64hi and a 64-bit multiply, is checked
bitwise through the GPU parity tests of the initial fields and the noise)."""
import json
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2607_24908_gb300", "csrc")

MAIN = r"""
#include <stdio.h>
#include <stdlib.h>
#include "tl_philox.cuh"
int main(int argc, char **argv)
{
    // "p c0 c1 key" -> Philox words; "m a b" -> (hi, lo) of a * b; hex in, hex out
    char op[4];
    unsigned long long x, y, z;
    while (scanf("%3s", op) == 1) {
        if (op[0] == 'p' && scanf("%llx %llx %llx", &x, &y, &z) == 3) {
            uint64_t o0, o1;
            tl::philox2x64_10(x, y, z, o0, o1);
            printf("%016llx %016llx\n", (unsigned long long)o0, (unsigned long long)o1);
        } else if (op[0] == 'm' && scanf("%llx %llx", &x, &y) == 2) {
            uint64_t hi, lo;
            tl::mul_64x64_128(x, y, hi, lo);
            printf("%016llx %016llx\n", (unsigned long long)hi, (unsigned long long)lo);
        } else {
            return 1;
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("philox")
    src, exe = d / "main.cpp", d / "philox"
    src.write_text(MAIN)
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])
    return str(exe)


def run(prog, lines):
    out = subprocess.run([prog], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return [tuple(int(w, 16) for w in ln.split()) for ln in out.stdout.splitlines()]


def test_known_answers(prog):
    with open(os.path.join(ROOT, "tests", "golden", "philox2x64_10_kat.json")) as f:
        rows = json.load(f)["rows"]
    got = run(prog, [f"p {r['ctr'][0]} {r['ctr'][1]} {r['key']}" for r in rows])
    assert got == [(int(r["out"][0], 16), int(r["out"][1], 16)) for r in rows]


def test_wide_product_against_python_integers(prog):
    rng = random.Random(7)
    M = 0xD2B74407B1CE6E93
    edge = [0, 1, 2 ** 32 - 1, 2 ** 32, 2 ** 63, 2 ** 64 - 1]
    pairs = [(a, b) for a in edge for b in edge] + [(M, rng.getrandbits(64)) for _ in range(200)]
    pairs += [(rng.getrandbits(64), rng.getrandbits(64)) for _ in range(200)]
    got = run(prog, [f"m {a:x} {b:x}" for a, b in pairs])
    assert got == [((a * b) >> 64, (a * b) & (2 ** 64 - 1)) for a, b in pairs]
