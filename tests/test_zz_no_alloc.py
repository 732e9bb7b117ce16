"""tl_energies_noalloc: energies of a caller-owned device state computed
without any device allocation.

It exists for callers that cannot call cudaMalloc: a host framework that
owns all device memory and hands out only its own buffers, or code that must
not allocate because an allocation can synchronise the device.  The entry
point keeps its reduction scratch in a fixed static device array shared by
every call, so these tests call it twice in a row (the second call finds the
first call's leftovers) and compare each result with tl_energies on the same
state, within the parity tolerances used elsewhere (FP64 1e-12, FP32 1e-5,
relative to the total energy density).
"""
import numpy as np
import pytest

from paper_2607_24908_gb300 import tl as T
from paper_2607_24908_gb300.workloads import white_noise_state

pytestmark = pytest.mark.gpu

M2 = (0.1, 0.2, 0.3)


@pytest.mark.parametrize("dtype,N,nf,expanding", [("f64", 40, 2, True), ("f32", 72, 3, False),
                                                   ("f32", 128, 2, True)])
def test_noalloc_energies_match_lattice_energies(dtype, N, nf, expanding):
    npd = np.float32 if dtype == "f32" else np.float64
    phi, pi = white_noise_state(N, nf, seed=N + nf, phi0=(1.0, 0.2, 0.1), sigma_phi=1e-2, sigma_pi=1e-2)
    a = 1.3 if expanding else 1.0
    import torch
    with T.Lattice(N, 0.5, nf, dtype, expanding, 1.0, 1.0, 1.0) as lat:
        lat.set_potential(1.0, 20.0, M2)
        lat.set_state(phi.astype(npd), pi.astype(npd), a, 0.1, False)
        ref = lat.energies().vector()
        # the entry point takes dense caller-owned device arrays [z][y][x]
        dev = [torch.from_numpy(np.ascontiguousarray(x[f].astype(npd))).cuda() for x in (phi, pi) for f in range(nf)]
        torch.cuda.synchronize()
        phip = [t.data_ptr() for t in dev[:nf]]
        pip = [t.data_ptr() for t in dev[nf:]]
        ex = T.tl_expansion(int(expanding), 1.0, 1.0, 1.0)
        tol = 1e-12 if dtype == "f64" else 1e-5
        for _ in range(2):
            got = T.tl_energies_noalloc(N, 0.5, nf, T.DTYPES[dtype], 1.0, 20.0, M2, ex, a, phip, pip, 0)
            assert np.max(np.abs(got - ref)) / np.sum(np.abs(ref)) <= tol, (got, ref)


def test_noalloc_rejects_lattices_beyond_the_scratch_limit():
    with T.Lattice(16, 0.5, 1, "f64") as lat:
        ptr = [lat.device_ptr(0, 0)]
        with pytest.raises(T.TLError) as e:  # 2048^3 FP64 needs 131072 CTA slots > 16384
            T.tl_energies_noalloc(2048, 0.5, 1, T.F64, 1.0, 0.0, (0, 0, 0), None, 1.0, ptr, ptr, 0)
        assert e.value.code == T.EINVAL
        assert "scratch" in str(e.value)
