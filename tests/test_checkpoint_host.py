"""The checkpoint file format on the CPU: save_checkpoint / load_checkpoint
round-trip every field exactly (arrays bitwise, the FP64 scalars and the
clock unchanged), with and without a potential, and the file holds no
pickled objects."""
import numpy as np

from paper_2607_24908_gb300 import tl as T


def _ck(dtype, with_potential):
    rng = np.random.default_rng(5)
    npd = np.float32 if dtype == "f32" else np.float64
    ck = {"N": 8, "n_fields": 2, "dtype": dtype, "kIR": 0.1 + 1e-17, "phi": rng.standard_normal((2, 8, 8, 8)).astype(npd),
          "pi": rng.standard_normal((2, 8, 8, 8)).astype(npd), "a": 1.0 + 2.0 ** -50, "b": float(np.nextafter(0.3, 1.0)),
          "pass_config": {"kind": "tma", "warps": 7, "stages": 6, "z_chunk": 16, "tile_x": 0, "threads": 0},
          "step": 123456789012, "time": 1234.5678901234567, "langevin_steps": 7}
    if with_potential:
        ck["potential"] = (1.0, 100.0, (0.0, 0.1 + 2.0 ** -40, 0.0))
    return ck


def test_checkpoint_file_round_trip(tmp_path):
    for dtype in ("f32", "f64"):
        for pot in (False, True):
            ck = _ck(dtype, pot)
            path = tmp_path / f"ck_{dtype}_{pot}.npz"
            T.save_checkpoint(path, ck)
            back = T.load_checkpoint(path)
            assert set(back) == set(ck)
            for k, v in ck.items():
                if isinstance(v, np.ndarray):
                    assert back[k].dtype == v.dtype and np.array_equal(back[k], v)
                else:
                    assert back[k] == v and type(back[k]) is type(v), k
            with np.load(path, allow_pickle=False) as z:  # readable without pickle
                assert all(z[k].dtype != object for k in z.files)
