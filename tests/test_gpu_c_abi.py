"""The C ABI from a plain C program (tests/c_abi_parity.c, compiled with gcc as
C11 against include/tl.h and linked with libtl.so and the oracle's C library):
an expanding two-field FP64 lattice stepped with Yoshida-4 on the GPU agrees
with the oracle to 1e-12, without Python in between."""
import os
import subprocess

import pytest

import oracle
from paper_2607_24908_gb300 import tl as T

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_steps_on_the_gpu_like_the_oracle(tmp_path):
    T.lib()  # libtl.so is built
    oracle.lib()  # and the oracle's library
    libtl_dir = os.path.dirname(T.LIB_PATH)
    libo = oracle.lib()._name
    exe = str(tmp_path / "c_abi_parity")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_parity.c"), "-o", exe,
           "-L", libtl_dir, "-ltl", libo, "-lm", f"-Wl,-rpath,{libtl_dir}",
           f"-Wl,-rpath,{os.path.dirname(libo)}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, (out.stdout, out.stderr)
    assert "c-abi parity" in out.stdout
