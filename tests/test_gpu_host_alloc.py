"""tl_host_alloc / tl_host_free on the GPU: page-locked memory that the state
copies and plain CUDA copies use; freed when the last view goes."""
import numpy as np
import pytest

from paper_2607_24908_gb300 import tl as T

pytestmark = pytest.mark.gpu


def huge_page_bytes():
    try:
        with open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size") as f:
            return int(f.read())
    except (OSError, ValueError):
        return 2 << 20


@pytest.mark.parametrize("nbytes", [1000, "huge"])
def test_host_alloc_is_pinned_zeroed_and_copies_round_trip(nbytes):
    import torch
    if nbytes == "huge":  # at least one huge page: the aligned, huge-page path
        nbytes = huge_page_bytes() + 12345
    n = nbytes // 8
    a = T.host_empty((n,), np.float64)
    assert a.ctypes.data % 64 == 0
    assert not a.any()  # zero-filled
    t = torch.from_numpy(a)
    assert t.is_pinned()
    a[:] = np.arange(n, dtype=np.float64) * 0.5 - 3.0
    d = t.to("cuda", non_blocking=True)
    b = T.host_empty((n,), np.float64)
    torch.from_numpy(b).copy_(d * 2.0, non_blocking=True)
    torch.cuda.synchronize()
    assert np.array_equal(b, 2.0 * a)


def test_state_copies_through_host_alloc_memory_are_bitwise():
    N, nf = 48, 2
    rng = np.random.default_rng(3)
    src = [rng.standard_normal((N, N, N)).astype(np.float32) for _ in range(2 * nf)]
    host = [T.host_empty((N, N, N), np.float32) for _ in range(2 * nf)]
    with T.Lattice(N, 0.5, nf, "f32") as lat:
        lat.set_potential(1.0, 0.0, (0.0, 0.0, 0.0))
        for i, x in enumerate(src):
            host[i][...] = x
            T.tl_set_state(lat.h, i // 2, i % 2, host[i])
        for h in host:
            h[...] = 0.0
        for i in range(2 * nf):
            T.tl_get_state(lat.h, i // 2, i % 2, host[i])
            assert np.array_equal(host[i], src[i])
            assert np.array_equal(lat.get(i // 2, i % 2), src[i])


def test_host_free_rules():
    p = T.tl_host_alloc(4096)
    T.tl_host_free(p)
    with pytest.raises(T.TLError) as e:  # already freed
        T.tl_host_free(p)
    assert e.value.code == T.EINVAL
    # views keep the memory: dropping the array but keeping a slice is safe
    a = T.host_empty((1 << 16,), np.int32)
    a[:] = np.arange(1 << 16, dtype=np.int32)
    tail = a[-4:]
    del a
    assert list(tail) == [65532, 65533, 65534, 65535]
