"""ctypes binding of include/tl.h (argument marshalling only).

Functions keep the C names (``tl_lattice_create`` ...) and raise ``TLError``
on a negative return code.  ``Lattice`` wraps one lattice handle.  Every step
of the computation runs in libtl.so, loaded on the first call; if the library
is missing that call raises ImportError -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtl.so")

MAX_FIELDS = 3
F32, F64 = 0, 1
LEAPFROG, VERLET, YOSHIDA4 = 0, 1, 2
INTEGRATORS = {"leapfrog": LEAPFROG, "verlet": VERLET, "yoshida4": YOSHIDA4}
DTYPES = {"f32": F32, "f64": F64}
OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6
_NAMES = {EINVAL: "TL_EINVAL", ENOMEM: "TL_ENOMEM", ECUDA: "TL_ECUDA", EUNSTABLE: "TL_EUNSTABLE",
          ETIMEOUT: "TL_ETIMEOUT", ESTATE: "TL_ESTATE"}


class TLError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class tl_expansion(ctypes.Structure):
    _fields_ = [("expanding", ctypes.c_int), ("alpha", ctypes.c_double),
                ("fstar_over_mp", ctypes.c_double), ("a0", ctypes.c_double)]


class tl_potential(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("q", ctypes.c_double), ("m2", ctypes.c_double * MAX_FIELDS)]


class tl_init_spec(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double), ("meff2", ctypes.c_double * MAX_FIELDS),
                ("phi0", ctypes.c_double * MAX_FIELDS), ("pi0", ctypes.c_double * MAX_FIELDS),
                ("fluct_pi", ctypes.c_int), ("fixed_modulus", ctypes.c_int)]


class tl_langevin_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("m2", ctypes.c_double), ("noise", ctypes.c_double)]


class tl_energies_t(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("time", ctypes.c_double), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("K", ctypes.c_double * MAX_FIELDS),
                ("G", ctypes.c_double * MAX_FIELDS), ("V", ctypes.c_double),
                ("hubble_resid", ctypes.c_double)]


class tl_clock(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("time", ctypes.c_double), ("langevin_steps", ctypes.c_int64)]


PASS_STREAM, PASS_TMA = 0, 1
PASS_KINDS = {"stream": PASS_STREAM, "tma": PASS_TMA}


class tl_pass_config(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("warps", ctypes.c_int), ("stages", ctypes.c_int),
                ("z_chunk", ctypes.c_int), ("tile_x", ctypes.c_int), ("threads", ctypes.c_int)]


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "tl_lattice_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, ctypes.POINTER(tl_expansion), ctypes.c_void_p]),
    "tl_lattice_create_with_buffers": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_double,
                                                      ctypes.c_int, ctypes.c_int, ctypes.POINTER(tl_expansion),
                                                      ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]),
    "tl_state_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "tl_array_layout": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(ctypes.c_size_t)]),
    "tl_lattice_destroy": (None, [ctypes.c_void_p]),
    "tl_set_potential": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tl_potential)]),
    "tl_init_fluctuations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(tl_init_spec)]),
    "tl_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int]),
    "tl_energies": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tl_energies_t)]),
    "tl_spectrum_bins": (ctypes.c_int, [ctypes.c_int]),
    "tl_spectrum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int64)]),
    "tl_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]),
    "tl_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]),
    "tl_set_background": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int]),
    "tl_get_clock": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tl_clock)]),
    "tl_set_clock": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tl_clock)]),
    "tl_state_device_ptr": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "tl_energies_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(tl_potential), ctypes.POINTER(tl_expansion),
                                           ctypes.c_double, ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_double)]),
    "tl_host_alloc": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "tl_host_free": (ctypes.c_int, [ctypes.c_void_p]),
    "tl_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                       ctypes.c_void_p]),
    "tl_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int]),
    "tl_batch_destroy": (None, [ctypes.c_void_p]),
    "tl_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "tl_batch_get_options": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "tl_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "tl_set_pass_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tl_pass_config)]),
    "tl_commit_state": (ctypes.c_int, [ctypes.c_void_p]),
    "tl_batch_pass_config": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(tl_pass_config)]),
    "tl_probe_fma_rates": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_void_p]),
    "tl_get_pass_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tl_pass_config)]),
    "tl_langevin_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                        ctypes.POINTER(tl_langevin_params), ctypes.c_uint64]),
    "tl_su2_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "tl_su2_destroy": (None, [ctypes.c_void_p]),
    "tl_su2_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tl_su2_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tl_su2_init_random": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double]),
    "tl_su2_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    "tl_su2_measure": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "tl_last_error": (ctypes.c_char_p, []),
}


def lib() -> ctypes.CDLL:
    """Load libtl.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2607_24908_gb300.build` "
                              "(no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def _check(rc: int):
    if rc != OK:
        raise TLError(rc, lib().tl_last_error().decode(errors="replace"))


def _f3(vals, fill=0.0):
    v = list(vals) + [fill] * MAX_FIELDS
    return (ctypes.c_double * MAX_FIELDS)(*v[:MAX_FIELDS])


# --- the C functions, same names ------------------------------------------------

def tl_lattice_create(N: int, kIR: float, n_fields: int, dtype: int, expansion: Optional[tl_expansion] = None,
                      cuda_stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().tl_lattice_create(ctypes.byref(h), N, kIR, n_fields, dtype,
                                   ctypes.byref(expansion) if expansion is not None else None,
                                   ctypes.c_void_p(cuda_stream)))
    return h


def tl_lattice_create_with_buffers(N: int, kIR: float, n_fields: int, dtype: int, expansion: Optional[tl_expansion],
                                   cuda_stream: int, dev_ptrs: Sequence[int]) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * len(dev_ptrs))(*dev_ptrs)
    _check(lib().tl_lattice_create_with_buffers(ctypes.byref(h), N, kIR, n_fields, dtype,
                                                ctypes.byref(expansion) if expansion is not None else None,
                                                ctypes.c_void_p(cuda_stream), arr, len(dev_ptrs)))
    return h


def tl_state_bytes(N: int, n_fields: int, dtype: int) -> int:
    return lib().tl_state_bytes(N, n_fields, dtype)


def tl_array_layout(N: int, dtype: int):
    """(elems, row_pitch, plane_pitch, origin) of one device field array."""
    v = [ctypes.c_size_t() for _ in range(4)]
    _check(lib().tl_array_layout(N, dtype, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def tl_lattice_destroy(h):
    lib().tl_lattice_destroy(h)


def tl_set_potential(h, lam: float, q: float, m2: Sequence[float]):
    p = tl_potential(lam, q, _f3(m2))
    _check(lib().tl_set_potential(h, ctypes.byref(p)))


def tl_init_fluctuations(h, seed: int, A: float, meff2, phi0, pi0=(0, 0, 0), fluct_pi: bool = False,
                         fixed_modulus: bool = False):
    s = tl_init_spec(A, _f3(meff2), _f3(phi0), _f3(pi0), int(bool(fluct_pi)), int(bool(fixed_modulus)))
    _check(lib().tl_init_fluctuations(h, ctypes.c_uint64(seed), ctypes.byref(s)))


def tl_step(h, n: int, dt: float, integrator: int):
    _check(lib().tl_step(h, n, dt, integrator))


def tl_energies(h) -> tl_energies_t:
    e = tl_energies_t()
    _check(lib().tl_energies(h, ctypes.byref(e)))
    return e


def tl_spectrum_bins(N: int) -> int:
    return lib().tl_spectrum_bins(N)


def tl_spectrum(h, N: int, field: int, which: int):
    nb = tl_spectrum_bins(N)
    k = np.zeros(nb)
    P = np.zeros(nb)
    c = np.zeros(nb, dtype=np.int64)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().tl_spectrum(h, field, which, nb, k.ctypes.data_as(dp), P.ctypes.data_as(dp),
                             c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return k, P, c


def tl_get_state(h, field: int, which: int, out: np.ndarray):
    _check(lib().tl_get_state(h, field, which, ctypes.c_void_p(out.ctypes.data), out.nbytes))


def tl_set_state(h, field: int, which: int, arr: np.ndarray):
    a = np.ascontiguousarray(arr)
    _check(lib().tl_set_state(h, field, which, ctypes.c_void_p(a.ctypes.data), a.nbytes))


def tl_set_background(h, a: float, b: float, from_constraint: bool):
    _check(lib().tl_set_background(h, a, b, int(bool(from_constraint))))


def tl_get_clock(h) -> tl_clock:
    c = tl_clock()
    _check(lib().tl_get_clock(h, ctypes.byref(c)))
    return c


def tl_set_clock(h, step: int, time: float, langevin_steps: int = 0):
    c = tl_clock(step, time, langevin_steps)
    _check(lib().tl_set_clock(h, ctypes.byref(c)))


def tl_state_device_ptr(h, field: int, which: int) -> int:
    p = ctypes.c_void_p()
    _check(lib().tl_state_device_ptr(h, field, which, ctypes.byref(p)))
    return p.value or 0


def tl_energies_noalloc(N: int, kIR: float, n_fields: int, dtype: int, lam: float, q: float, m2,
                        expansion: Optional[tl_expansion], a: float, phi_ptrs: Sequence[int],
                        pi_ptrs: Sequence[int], cuda_stream: int = 0) -> np.ndarray:
    """Energies [K_0.., G_0.., V] of caller-owned device arrays; allocates nothing on the device."""
    pot = tl_potential(lam, q, _f3(m2))
    ph = (ctypes.c_void_p * n_fields)(*phi_ptrs)
    pp = (ctypes.c_void_p * n_fields)(*pi_ptrs)
    out = np.zeros(2 * n_fields + 1)
    _check(lib().tl_energies_noalloc(N, kIR, n_fields, dtype, ctypes.byref(pot),
                                     ctypes.byref(expansion) if expansion is not None else None, a, ph, pp,
                                     ctypes.c_void_p(cuda_stream), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def tl_host_alloc(nbytes: int) -> int:
    p = ctypes.c_void_p()
    _check(lib().tl_host_alloc(nbytes, ctypes.byref(p)))
    return int(p.value)


def tl_host_free(ptr: int):
    _check(lib().tl_host_free(ctypes.c_void_p(ptr)))


class _HostBuffer:
    """Bytes from tl_host_alloc, freed when the last numpy view of them goes."""

    def __init__(self, nbytes: int):
        self.nbytes = nbytes
        self.ptr = tl_host_alloc(nbytes)
        self.__array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (self.ptr, False),
                                    "version": 3}

    def __del__(self):
        ptr, self.ptr = getattr(self, "ptr", None), None
        if ptr:
            try:
                tl_host_free(ptr)
            except Exception:  # at interpreter exit the CUDA context may be gone first
                pass


def host_empty(shape, dtype) -> np.ndarray:
    """A numpy array in page-locked host memory from tl_host_alloc (huge pages
    where the kernel grants them), for state copies to and from the device;
    zero-filled.  The memory lives as long as the array or any view of it."""
    dtype = np.dtype(dtype)
    shape = tuple(int(x) for x in np.atleast_1d(shape))
    nbytes = int(np.prod(shape, dtype=np.int64)) * dtype.itemsize
    if nbytes == 0:
        return np.zeros(shape, dtype)
    return np.asarray(_HostBuffer(nbytes)).view(dtype).reshape(shape)


def tl_langevin_step(h, n: int, dt: float, lam: float, m2: float, noise: float, seed: int):
    p = tl_langevin_params(lam, m2, noise)
    _check(lib().tl_langevin_step(h, n, dt, ctypes.byref(p), ctypes.c_uint64(seed)))


class SU2:
    """SU(2) Yang-Mills lattice in temporal gauge (see tl_su2_* in tl.h);
    states as numpy arrays U[3, 4, N, N, N], E[3, 3, N, N, N]."""

    def __init__(self, N: int, dtype: str = "f64", stream: int = 0):
        self.N, self.dtype = N, dtype
        self.np_dtype = np.float32 if dtype == "f32" else np.float64
        self.h = ctypes.c_void_p()
        _check(lib().tl_su2_create(ctypes.byref(self.h), N, DTYPES[dtype], ctypes.c_void_p(stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().tl_su2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, U: np.ndarray, E: np.ndarray):
        U = np.ascontiguousarray(U, dtype=self.np_dtype)
        E = np.ascontiguousarray(E, dtype=self.np_dtype)
        assert U.shape == (3, 4) + (self.N,) * 3 and E.shape == (3, 3) + (self.N,) * 3
        _check(lib().tl_su2_set_state(self.h, ctypes.c_void_p(U.ctypes.data), ctypes.c_void_p(E.ctypes.data)))

    def get_state(self):
        U = np.empty((3, 4) + (self.N,) * 3, self.np_dtype)
        E = np.empty((3, 3) + (self.N,) * 3, self.np_dtype)
        _check(lib().tl_su2_get_state(self.h, ctypes.c_void_p(U.ctypes.data), ctypes.c_void_p(E.ctypes.data)))
        return U, E

    def init_random(self, seed: int, amp: float):
        _check(lib().tl_su2_init_random(self.h, ctypes.c_uint64(seed), amp))

    def step(self, n: int, dt: float):
        _check(lib().tl_su2_step(self.h, n, dt))

    def measure(self) -> np.ndarray:
        """[electric, magnetic (plaquette) energy per site, max |Gauss|, rms |Gauss|]."""
        out = np.zeros(4)
        _check(lib().tl_su2_measure(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out


def tl_batch_create(handles: Sequence, cuda_stream: int = 0) -> ctypes.c_void_p:
    b = ctypes.c_void_p()
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    _check(lib().tl_batch_create(ctypes.byref(b), arr, len(handles), ctypes.c_void_p(cuda_stream)))
    return b


def tl_batch_step(b, n: int, dt: float, integrator: int):
    _check(lib().tl_batch_step(b, n, dt, integrator))


def tl_batch_destroy(b):
    lib().tl_batch_destroy(b)


def tl_batch_autotune(b) -> float:
    ms = ctypes.c_double()
    _check(lib().tl_batch_autotune(b, ctypes.byref(ms)))
    return ms.value


def tl_batch_get_options(b) -> dict:
    v = [ctypes.c_int() for _ in range(3)]
    _check(lib().tl_batch_get_options(b, *[ctypes.byref(x) for x in v]))
    return {"prefetch": v[0].value, "split": v[1].value, "share": v[2].value}


def tl_autotune(h) -> float:
    ms = ctypes.c_double()
    _check(lib().tl_autotune(h, ctypes.byref(ms)))
    return ms.value


def tl_commit_state(h):
    _check(lib().tl_commit_state(h))


def tl_probe_fma_rates(cuda_stream: int = 0):
    """(FP64, FP32) FMA operations per second measured on the current device."""
    f64, f32 = ctypes.c_double(), ctypes.c_double()
    _check(lib().tl_probe_fma_rates(ctypes.byref(f64), ctypes.byref(f32), ctypes.c_void_p(cuda_stream)))
    return f64.value, f32.value


def tl_set_pass_config(h, kind: int, warps: int = 0, stages: int = 0, z_chunk: int = 0, tile_x: int = 0,
                       threads: int = 0):
    cfg = tl_pass_config(kind, warps, stages, z_chunk, tile_x, threads)
    _check(lib().tl_set_pass_config(h, ctypes.byref(cfg)))


def _cfg_dict(cfg: tl_pass_config) -> dict:
    kind = {v: k for k, v in PASS_KINDS.items()}[cfg.kind]
    return {"kind": kind, "warps": cfg.warps, "stages": cfg.stages, "z_chunk": cfg.z_chunk,
            "tile_x": cfg.tile_x, "threads": cfg.threads}


def tl_get_pass_config(h) -> dict:
    cfg = tl_pass_config()
    _check(lib().tl_get_pass_config(h, ctypes.byref(cfg)))
    return _cfg_dict(cfg)


def batch_pass_config(N: int, n_fields: int, dtype: str) -> dict:
    """The launch shape tl_batch_create gives a lattice of this size (keyword
    arguments for Lattice.set_pass_config)."""
    cfg = tl_pass_config()
    _check(lib().tl_batch_pass_config(N, n_fields, DTYPES[dtype], ctypes.byref(cfg)))
    return _cfg_dict(cfg)


class Batch:
    """Several lattices advanced together (see tl_batch_step)."""

    def __init__(self, lattices: Sequence["Lattice"], stream: int = 0):
        self.lattices = list(lattices)
        self.b = tl_batch_create([l.h for l in self.lattices], stream)

    def step(self, n: int, dt: float, integrator="verlet"):
        tl_batch_step(self.b, n, dt, INTEGRATORS[integrator] if isinstance(integrator, str) else integrator)

    def autotune(self) -> float:
        """Choose the members' batch shapes and the batch options by
        measurement (see tl_batch_autotune); returns ms per grouped pass."""
        return tl_batch_autotune(self.b)

    def options(self) -> dict:
        return tl_batch_get_options(self.b)

    def close(self):
        if getattr(self, "b", None):
            tl_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# --- convenience wrapper --------------------------------------------------------

@dataclass
class Energies:
    step: int
    time: float
    a: float
    b: float
    K: np.ndarray
    G: np.ndarray
    V: float
    hubble_resid: float

    def vector(self) -> np.ndarray:
        """[K_0.., G_0.., V] like the oracle's energies()."""
        return np.concatenate([self.K, self.G, [self.V]])


class Lattice:
    """One lattice on the current CUDA device (state resident in HBM)."""

    def __init__(self, N: int, kIR: float, n_fields: int = 1, dtype: str = "f64", expanding: bool = False,
                 alpha: float = 0.0, fstar_over_mp: float = 1.0, a0: float = 1.0, stream: int = 0):
        self.N, self.nf, self.kIR = N, n_fields, kIR
        self.dtype = dtype
        self.expanding, self.alpha = bool(expanding), alpha
        self.np_dtype = np.float32 if dtype == "f32" else np.float64
        ex = tl_expansion(int(bool(expanding)), alpha, fstar_over_mp, a0)
        self.h = tl_lattice_create(N, kIR, n_fields, DTYPES[dtype], ex, stream)
        self.potential = None  # (lambda, q, m2) once set

    def close(self):
        if getattr(self, "h", None):
            tl_lattice_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_potential(self, lam: float = 1.0, q: float = 0.0, m2=(0.0, 0.0, 0.0)):
        tl_set_potential(self.h, lam, q, m2)
        self.potential = (float(lam), float(q), tuple(float(v) for v in _f3(m2)))

    def init_fluctuations(self, seed: int, A: float = 1e-10, meff2=(3.0, 0, 0), phi0=(1.0, 0, 0), pi0=(0, 0, 0),
                          fluct_pi: bool = False, fixed_modulus: bool = False):
        tl_init_fluctuations(self.h, seed, A, meff2, phi0, pi0, fluct_pi, fixed_modulus)

    def step(self, n: int, dt: float, integrator="verlet"):
        tl_step(self.h, n, dt, INTEGRATORS[integrator] if isinstance(integrator, str) else integrator)

    def energies(self) -> Energies:
        e = tl_energies(self.h)
        nf = self.nf
        return Energies(e.step, e.time, e.a, e.b, np.array(e.K[:nf]), np.array(e.G[:nf]), e.V, e.hubble_resid)

    def spectrum(self, field: int = 0, which: int = 0):
        return tl_spectrum(self.h, self.N, field, which)

    def get(self, field: int, which: int) -> np.ndarray:
        out = np.empty((self.N, self.N, self.N), dtype=self.np_dtype)
        tl_get_state(self.h, field, which, out)
        return out

    def get_all(self):
        phi = np.stack([self.get(f, 0) for f in range(self.nf)])
        pi = np.stack([self.get(f, 1) for f in range(self.nf)])
        return phi, pi

    def set_state(self, phi: np.ndarray, pi: np.ndarray, a: float = 1.0, b: float = 0.0,
                  b_from_constraint: bool = False):
        for f in range(self.nf):
            tl_set_state(self.h, f, 0, np.ascontiguousarray(phi[f], dtype=self.np_dtype))
            tl_set_state(self.h, f, 1, np.ascontiguousarray(pi[f], dtype=self.np_dtype))
        tl_set_background(self.h, a, b, b_from_constraint)

    def clock(self) -> dict:
        """Completed steps and program time since the state was set, and Langevin steps."""
        c = tl_get_clock(self.h)
        return {"step": c.step, "time": c.time, "langevin_steps": c.langevin_steps}

    def set_clock(self, step: int, time: float = 0.0, langevin_steps: int = 0):
        tl_set_clock(self.h, step, time, langevin_steps)

    def checkpoint(self) -> dict:
        """What a resumed run needs: the lattice's size, fields, precision and
        kIR (checked on restore), the potential, the pass shape, the state at
        the current integer time, a, a' and the clock (see tl_set_clock)."""
        E = self.energies()
        phi, pi = self.get_all()
        ck = {"N": self.N, "n_fields": self.nf, "dtype": self.dtype, "kIR": self.kIR, "phi": phi, "pi": pi,
              "a": E.a, "b": E.b, "pass_config": self.pass_config(), **self.clock()}
        if self.potential is not None:
            ck["potential"] = self.potential
        return ck

    def restore(self, ck: dict):
        """Continue from ``checkpoint()`` of a lattice created with the same
        arguments: the same tl_step calls then give bitwise its results."""
        for key, mine in (("N", self.N), ("n_fields", self.nf), ("dtype", self.dtype), ("kIR", self.kIR)):
            if ck[key] != mine:
                raise ValueError(f"checkpoint {key} {ck[key]!r} does not match the lattice's {mine!r}")
        if ck.get("potential") is not None:
            lam, q, m2 = ck["potential"]
            self.set_potential(lam, q, m2)
        if ck["pass_config"] != self.pass_config():
            self.set_pass_config(**ck["pass_config"])
        self.set_state(ck["phi"], ck["pi"], ck["a"], ck["b"], b_from_constraint=False)
        self.set_clock(int(ck["step"]), float(ck["time"]), int(ck["langevin_steps"]))

    def device_ptr(self, field: int, which: int) -> int:
        return tl_state_device_ptr(self.h, field, which)

    def langevin(self, n: int, dt: float, lam: float, m2: float = 0.0, noise: float = 1.0, seed: int = 0):
        """n Euler-Maruyama Langevin steps of phi_0 (see tl_langevin_step)."""
        tl_langevin_step(self.h, n, dt, lam, m2, noise, seed)

    def autotune(self) -> float:
        """Pick the fastest launch geometry for this lattice shape; returns ms per pass."""
        return tl_autotune(self.h)

    def set_pass_config(self, kind: str = "tma", warps: int = 0, stages: int = 0, z_chunk: int = 0,
                        tile_x: int = 0, threads: int = 0):
        """Launch shape of the fused pass (see tl_set_pass_config); kind "stream" or "tma"."""
        tl_set_pass_config(self.h, PASS_KINDS[kind], warps, stages, z_chunk, tile_x, threads)

    def pass_config(self) -> dict:
        """The launch shape in use, automatic values resolved."""
        return tl_get_pass_config(self.h)


def save_checkpoint(path, ck: dict):
    """Write a ``Lattice.checkpoint()`` to an .npz file (no pickled objects)."""
    flat = {k: v for k, v in ck.items() if k not in ("potential", "pass_config")}
    if ck.get("potential") is not None:
        lam, q, m2 = ck["potential"]
        flat["potential"] = np.array([lam, q, *m2])
    pc = ck["pass_config"]
    flat["pass_config_kind"] = pc["kind"]
    flat["pass_config"] = np.array([pc[k] for k in _PASS_INTS], dtype=np.int64)
    np.savez(path, **flat)


def load_checkpoint(path) -> dict:
    """Read a checkpoint written by ``save_checkpoint``."""
    with np.load(path, allow_pickle=False) as z:
        ck = {k: z[k] for k in z.files}
    out = {"N": int(ck["N"]), "n_fields": int(ck["n_fields"]), "dtype": str(ck["dtype"]), "kIR": float(ck["kIR"]),
           "phi": ck["phi"], "pi": ck["pi"], "a": float(ck["a"]), "b": float(ck["b"]), "step": int(ck["step"]),
           "time": float(ck["time"]), "langevin_steps": int(ck["langevin_steps"])}
    pc = {k: int(v) for k, v in zip(_PASS_INTS, ck["pass_config"])}
    pc["kind"] = str(ck["pass_config_kind"])
    out["pass_config"] = pc
    if "potential" in ck:
        p = ck["potential"]
        out["potential"] = (float(p[0]), float(p[1]), tuple(float(v) for v in p[2:]))
    return out


_PASS_INTS = ("warps", "stages", "z_chunk", "tile_x", "threads")
