"""CPU checks of the boundary: libtl.so builds, loads without a GPU and
exports every function include/tl.h declares; the binding covers them all."""
import os
import pathlib
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = pathlib.Path(ROOT, "include", "tl.h").read_text()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tl_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    from paper_2607_24908_gb300 import build, tl
    lib = build.build()
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib], text=True)
    exported = set(re.findall(r" T (tl_[a-z0-9_]+)$", out, flags=re.M))
    declared = header_functions()
    assert declared, "no functions parsed from include/tl.h"
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    L = tl.lib()  # dlopen works without a GPU
    for f in declared:
        assert hasattr(L, f)
    assert sorted(tl.declared_symbols()) == declared


def test_spectrum_bins_and_state_bytes_without_gpu():
    from paper_2607_24908_gb300 import tl
    import math
    for N in (8, 32, 48, 1024):
        assert tl.tl_spectrum_bins(N) == math.ceil(math.sqrt(3) * N / 2) + 1
    # padded device layout: W = 16/sizeof ghost elements per row side, one ghost row per plane side
    for N, dt, esz in ((1024, tl.F32, 4), (32, tl.F64, 8), (40, tl.F32, 4)):
        W = 16 // esz
        elems, pitch, plane, origin = tl.tl_array_layout(N, dt)
        lpad = 128 // esz
        assert pitch >= lpad + N + W and (pitch * esz) % 128 == 0
        assert plane == (N + 2) * pitch and elems == N * plane and origin == pitch + lpad
        assert (origin * esz) % 128 == 0
    assert tl.tl_state_bytes(1024, 2, tl.F32) == 4 * 2 * tl.tl_array_layout(1024, tl.F32)[0] * 4
    assert tl.tl_state_bytes(32, 1, tl.F64) == 4 * tl.tl_array_layout(32, tl.F64)[0] * 8


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2607_24908_gb300 import tl
    with pytest.raises(tl.TLError) as e:
        tl.Lattice(32, 0.5, 1, "f64")
    assert e.value.code in (tl.ECUDA, tl.ENOMEM)
    with pytest.raises(tl.TLError) as e:
        tl.Lattice(30, 0.5, 1, "f64")
    assert e.value.code == tl.EINVAL


def test_host_alloc_argument_errors_and_no_gpu():
    """tl_host_alloc / tl_host_free: argument errors on any machine; without a
    GPU the registration fails with TL_ECUDA and nothing stays allocated."""
    import ctypes
    import torch
    from paper_2607_24908_gb300 import tl
    with pytest.raises(tl.TLError) as e:
        tl.tl_host_alloc(0)
    assert e.value.code == tl.EINVAL
    tl.tl_host_free(0)  # NULL is a no-op
    junk = ctypes.create_string_buffer(64)
    with pytest.raises(tl.TLError) as e:
        tl.tl_host_free(ctypes.addressof(junk))
    assert e.value.code == tl.EINVAL
    assert tl.host_empty((0, 4), np.float32).shape == (0, 4)
    if not torch.cuda.is_available():
        with pytest.raises(tl.TLError) as e:
            tl.host_empty((1 << 20,), np.float32)
        assert e.value.code == tl.ECUDA


def test_serving_job_generator_and_budget_arithmetic():
    """Host-side pieces of the server that need no GPU."""
    from paper_2607_24908_gb300 import serve as S
    jobs = S.poisson_jobs(50, seed=12345, rate=10.0)
    assert len(jobs) == 50
    arr = [j.arrival for j in jobs]
    assert arr == sorted(arr) and arr[0] > 0
    for j in jobs:
        assert j.N in (64, 128, 256, 384) and 1 <= j.n_fields <= 3 and j.q in (1.0, 100.0)
        assert 500 <= j.steps <= 5000 and j.steps % 100 == 0 and j.dtype in ("f32", "f64")
        esz = 4 if j.dtype == "f32" else 8
        line = 128 // esz
        pitch = -(-(line + j.N + 16 // esz) // line) * line
        assert j.state_bytes() == 4 * j.n_fields * j.N * (j.N + 2) * pitch * esz
        assert j.budget_bytes() > j.state_bytes()
    # mean inter-arrival ~ 1/rate
    gaps = np.diff([0.0] + arr)
    assert 0.05 < gaps.mean() < 0.2
    srv = S.Server(budget_bytes=jobs[0].budget_bytes())
    assert srv.fits(jobs[0])
    srv.used = 1
    assert not srv.fits(jobs[0])


def test_product_path_never_imports_or_links_the_oracle():
    """The package (binding, serving loop, build script) imports nothing from oracle/,
    and no kernel or header source includes a file from it."""
    import ast
    import glob
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2607_24908_gb300")
    for path in glob.glob(os.path.join(pkg, "*.py")):
        tree = ast.parse(pathlib.Path(path).read_text(), path)
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
            elif isinstance(node, ast.ImportFrom):
                assert node.level > 0 or (node.module or "").split(".")[0] != "oracle", path
    for path in glob.glob(os.path.join(pkg, "csrc", "*")) + glob.glob(os.path.join(root, "include", "*")):
        for line in pathlib.Path(path).read_text(errors="replace").splitlines():
            if line.lstrip().startswith("#include"):
                assert "oracle" not in line and "tlo" not in line, (path, line)
    build = pathlib.Path(pkg, "build.py").read_text()
    assert "oracle" not in build and "tlo.c" not in build


def test_header_is_plain_c11():
    """include/tl.h compiles as C11 (no C++ in the boundary's declarations)."""
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = '#include "tl.h"\nint main(void) { tl_energies_t e; (void)e; return TL_OK; }\n'
    out = subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-pedantic", "-fsyntax-only", "-x", "c",
                          "-I", os.path.join(root, "include"), "-"], input=src, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
