"""Continuous-batching server for lattice simulation jobs.

Jobs (lattice size, fields, couplings, steps, precision, seed) arrive over
time.  The server admits a waiting job as soon as its device memory fits in
the budget beside the jobs already resident, draws its initial state on the
device, and from then on advances it together with every other resident job:
each scheduler tick runs ``chunk`` velocity-Verlet steps of all resident jobs
of one precision as one batched call (``tl_batch_step``: one grouped launch per
pass, replayed as a CUDA graph), FP32 and FP64 jobs on two streams so their
work overlaps.  A job that has run all its steps is reaped (final energies and
spectrum read back, lattice destroyed, memory returned) and the freed budget
admits the next arrivals at the following tick.

Every job advances in the same ``chunk``-step calls whatever else is resident,
and keeps the launch geometry it has alone, so its results are bitwise those
of running it alone (``run_alone``).  Step counts must be multiples of
``chunk``.  All device work goes through the C ABI (paper_2607_24908_gb300.tl).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np

from . import tl as T


@dataclass
class JobSpec:
    """One simulation request: phi^4 plus (q/2) phi^2 chi^2 couplings to
    n_fields-1 further fields, expanding background (alpha = 1), velocity
    Verlet with step dt, vacuum fluctuations A/(2 omega_k)."""
    job_id: int
    N: int
    n_fields: int
    q: float
    steps: int
    dtype: str
    seed: int
    kIR: float = 0.1
    dt: float = 0.01
    A: float = 1e-10
    arrival: float = 0.0  # seconds after the server starts

    def state_bytes(self) -> int:
        return T.tl_state_bytes(self.N, self.n_fields, T.DTYPES[self.dtype])

    def init_scratch_bytes(self) -> int:
        # FP64 half spectrum + FP64 real array while the initial field is drawn
        return 16 * self.N * self.N * (self.N // 2 + 1) + 8 * self.N ** 3

    def budget_bytes(self) -> int:
        return self.state_bytes() + self.init_scratch_bytes()


@dataclass
class JobResult:
    job_id: int
    arrival: float
    admitted: float
    finished: float
    energies: np.ndarray          # [K_0.., G_0.., V] at the last step
    a: float
    b: float
    hubble_resid: float
    spectrum: np.ndarray          # binned P_b of field 0 at the last step

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def _new_lattice(spec: JobSpec, stream: int) -> T.Lattice:
    lat = T.Lattice(spec.N, spec.kIR, spec.n_fields, spec.dtype, True, 1.0, 1.0, 1.0, stream=stream)
    lat.set_potential(1.0, spec.q, (0.0, 0.0, 0.0))
    meff2 = (3.0,) + (spec.q,) * (spec.n_fields - 1)
    lat.init_fluctuations(spec.seed, A=spec.A, meff2=meff2, phi0=(1.0, 0.0, 0.0))
    return lat


def _result(spec: JobSpec, lat: T.Lattice, admitted: float, t0: float) -> JobResult:
    E = lat.energies()
    _, P, _ = lat.spectrum(0, 0)
    return JobResult(spec.job_id, spec.arrival, admitted, time.perf_counter() - t0, E.vector(), E.a, E.b,
                     E.hubble_resid, P)


@dataclass
class _Active:
    spec: JobSpec
    lat: T.Lattice
    done_steps: int
    admitted: float


class Server:
    """Continuous batching over resident lattices (see the module docstring)."""

    def __init__(self, budget_bytes: int, chunk: int = 100, streams: Optional[Dict[str, int]] = None):
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.streams = streams or {"f32": 0, "f64": 0}
        self.active: List[_Active] = []
        self.used = 0
        self._batches: Dict[str, T.Batch] = {}
        self._members: Dict[str, tuple] = {}
        self.rejected: List[int] = []

    def fits(self, spec: JobSpec) -> bool:
        return self.used + spec.budget_bytes() <= self.budget

    def admit(self, spec: JobSpec, now: float) -> None:
        if spec.steps % self.chunk != 0:
            raise ValueError(f"job {spec.job_id}: steps must be a multiple of {self.chunk}")
        lat = _new_lattice(spec, self.streams[spec.dtype])
        self.active.append(_Active(spec, lat, 0, now))
        self.used += spec.budget_bytes()

    def _batch(self, dtype: str) -> Optional[T.Batch]:
        members = tuple(id(a.lat) for a in self.active if a.spec.dtype == dtype)
        if not members:
            self._drop(dtype)
            return None
        if self._members.get(dtype) != members:
            self._drop(dtype)
            lats = [a.lat for a in self.active if a.spec.dtype == dtype]
            self._batches[dtype] = T.Batch(lats, self.streams[dtype])
            self._members[dtype] = members
        return self._batches[dtype]

    def _drop(self, dtype: str) -> None:
        b = self._batches.pop(dtype, None)
        self._members.pop(dtype, None)
        if b is not None:
            b.close()

    def tick(self) -> None:
        """Advance every resident job by one chunk (both precisions, two streams)."""
        for dtype in ("f32", "f64"):
            b = self._batch(dtype)
            if b is not None:
                b.step(self.chunk, 0.01, "verlet")
        for a in self.active:
            a.done_steps += self.chunk

    def reap(self, t0: float) -> List[JobResult]:
        out, keep = [], []
        for a in self.active:
            if a.done_steps >= a.spec.steps:
                out.append((a, None))
            else:
                keep.append(a)
        if not out:
            return []
        # results are read on the lattices' own streams after the batch work
        for dtype in ("f32", "f64"):
            if any(a.spec.dtype == dtype for a, _ in out):
                self._drop(dtype)
        results = []
        for a, _ in out:
            results.append(_result(a.spec, a.lat, a.admitted, t0))
            a.lat.close()
            self.used -= a.spec.budget_bytes()
        self.active = keep
        return results

    def close(self):
        for d in list(self._batches):
            self._drop(d)
        for a in self.active:
            a.lat.close()
        self.active = []
        self.used = 0


def serve(jobs: List[JobSpec], budget_bytes: int, chunk: int = 100,
          clock: Callable[[], float] = time.perf_counter, streams: Optional[Dict[str, int]] = None):
    """Run ``jobs`` (sorted by arrival) through a continuous-batching server in
    real time.  Returns (results in completion order, makespan seconds)."""
    srv = Server(budget_bytes, chunk, streams)
    pending = sorted(jobs, key=lambda j: j.arrival)
    for j in pending:
        if j.budget_bytes() > budget_bytes:
            raise ValueError(f"job {j.job_id} alone exceeds the budget")
    t0 = clock()
    results: List[JobResult] = []
    i = 0
    try:
        while len(results) < len(jobs):
            now = clock() - t0
            # admit arrivals in order while they fit
            while i < len(pending) and pending[i].arrival <= now and srv.fits(pending[i]):
                srv.admit(pending[i], now)
                i += 1
            if not srv.active:
                if i < len(pending):  # idle until the next arrival
                    wait = pending[i].arrival - (clock() - t0)
                    if wait > 0:
                        time.sleep(wait)
                continue
            srv.tick()
            results.extend(srv.reap(t0))
    finally:
        srv.close()
    return results, clock() - t0


def run_alone(jobs: List[JobSpec], chunk: int = 100, clock: Callable[[], float] = time.perf_counter,
              stream: int = 0):
    """The plain loop: jobs one at a time in arrival order, each stepped on its
    own in the same chunks.  Returns (results, makespan seconds)."""
    t0 = clock()
    results = []
    for spec in sorted(jobs, key=lambda j: j.arrival):
        now = clock() - t0
        if spec.arrival > now:
            time.sleep(spec.arrival - now)
        admitted = clock() - t0
        lat = _new_lattice(spec, stream)
        for _ in range(spec.steps // chunk):
            lat.step(chunk, spec.dt, "verlet")
        results.append(_result(spec, lat, admitted, t0))
        lat.close()
    return results, clock() - t0


def poisson_jobs(n: int, seed: int, rate: float, sizes=(64, 128, 256, 384), steps=(500, 5000),
                 chunk: int = 100) -> List[JobSpec]:
    """n jobs with exponential inter-arrival times (rate per second); N from
    ``sizes``, 1-3 fields, q from {1, 100}, steps a multiple of ``chunk`` in
    ``steps``, FP32 or FP64, per-job seeds."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n):
        t += float(rng.exponential(1.0 / rate)) if rate > 0 else 0.0
        s = int(rng.integers(steps[0] // chunk, steps[1] // chunk + 1)) * chunk
        out.append(JobSpec(job_id=k, N=int(rng.choice(sizes)), n_fields=int(rng.integers(1, 4)),
                           q=float(rng.choice([1.0, 100.0])), steps=s, dtype=str(rng.choice(["f32", "f64"])),
                           seed=int(rng.integers(1, 2 ** 31)), arrival=t))
    return out
