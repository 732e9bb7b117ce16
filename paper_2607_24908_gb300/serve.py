"""Continuous-batching server for lattice simulation jobs.

Jobs (lattice size, fields, couplings, steps, precision, seed) arrive over
time.  The server admits a waiting job as soon as its device memory fits in
the budget beside the jobs already resident, draws its initial state on the
device, and from then on advances it together with the other resident jobs
of its lane.  A lane is one precision and one size class with its own CUDA
stream; whenever a lane is idle the host reaps its finished jobs and starts
its next ``chunk`` velocity-Verlet steps for all its jobs as one batched call
(``tl_batch_step``: one grouped launch per pass, replayed as a CUDA graph).
Lanes run concurrently on the device, so small jobs are not held to the pace
of large ones.  A reaped job's final energies and spectrum are read back, its
lattice destroyed and its memory returned, and the freed budget admits the
next arrivals.

Every job advances in the same ``chunk``-step calls whatever else is resident,
and keeps the launch geometry it has alone, so its results are bitwise those
of running it alone (``run_alone``).  Step counts must be multiples of
``chunk``.  All device work goes through the C ABI (paper_2607_24908_gb300.tl).
"""
from __future__ import annotations

import time
from dataclasses import dataclass
from typing import Callable, List, Optional

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
    # served jobs advance in batches; every job starts on the batch launch
    # shape, so its energy sums (and thus its expansion) are the same served
    # and alone
    lat.set_pass_config(**T.batch_pass_config(spec.N, spec.n_fields, spec.dtype))
    lat.set_potential(1.0, spec.q, (0.0, 0.0, 0.0))
    meff2 = (3.0,) + (spec.q,) * (spec.n_fields - 1)
    lat.init_fluctuations(spec.seed, A=spec.A, meff2=meff2, phi0=(1.0, 0.0, 0.0))
    return lat


def _result(spec: JobSpec, lat: T.Lattice, admitted: float, t0: float,
            clock: Callable[[], float] = time.perf_counter) -> JobResult:
    E = lat.energies()
    _, P, _ = lat.spectrum(0, 0)
    return JobResult(spec.job_id, spec.arrival, admitted, clock() - t0, E.vector(), E.a, E.b, E.hubble_resid, P)


@dataclass
class _Active:
    spec: JobSpec
    lat: T.Lattice
    done_steps: int
    admitted: float


def job_cost(spec: JobSpec) -> float:
    """Relative device time per step (FP64 runs ALU-bound, ~8x an FP32 site)."""
    return spec.N ** 3 * spec.n_fields * (8.0 if spec.dtype == "f64" else 1.0)


SMALL_COST = 128 ** 3 * 3  # jobs up to this per-step cost share the "small" lanes


class _Lane:
    """Jobs of one precision and size class, advanced together on their own
    stream; the host starts the lane's next chunk as soon as the last one is
    done, independently of the other lanes."""

    def __init__(self, dtype: str, stream):
        self.dtype = dtype
        self.stream = stream
        self.jobs: List[_Active] = []
        self.batch: Optional[T.Batch] = None
        self.members: tuple = ()
        self.event = None
        self.inflight: List[_Active] = []

    def busy(self) -> bool:
        return self.event is not None and not self.event.query()


class Server:
    """Continuous batching over resident lattices (see the module docstring)."""

    def __init__(self, budget_bytes: int, chunk: int = 100, clock: Callable[[], float] = time.perf_counter):
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.clock = clock
        self.lanes = {}  # (dtype, size class) -> _Lane, created with its stream on first use
        self.used = 0

    @property
    def active(self) -> List[_Active]:
        return [a for lane in self.lanes.values() for a in lane.jobs]

    def fits(self, spec: JobSpec) -> bool:
        return self.used + spec.budget_bytes() <= self.budget

    def lane_of(self, spec: JobSpec) -> _Lane:
        key = (spec.dtype, "small" if job_cost(spec) <= SMALL_COST else "big")
        if key not in self.lanes:
            import torch
            self.lanes[key] = _Lane(spec.dtype, torch.cuda.Stream())
        return self.lanes[key]

    def admit(self, spec: JobSpec, now: float) -> None:
        if spec.steps % self.chunk != 0:
            raise ValueError(f"job {spec.job_id}: steps must be a multiple of {self.chunk}")
        lane = self.lane_of(spec)
        lat = _new_lattice(spec, lane.stream.cuda_stream)
        lane.jobs.append(_Active(spec, lat, 0, now))
        self.used += spec.budget_bytes()

    def service(self, t0: float) -> List[JobResult]:
        """Reap finished jobs of idle lanes and start their next chunk.  Returns
        the jobs completed now."""
        done: List[JobResult] = []
        for lane in self.lanes.values():
            if lane.busy():
                continue
            lane.event = None
            for a in lane.inflight:
                a.done_steps += self.chunk
            lane.inflight = []
            finished = [a for a in lane.jobs if a.done_steps >= a.spec.steps]
            if finished:
                lane.jobs = [a for a in lane.jobs if a.done_steps < a.spec.steps]
                if lane.batch is not None:
                    lane.batch.close()
                    lane.batch, lane.members = None, ()
                for a in finished:
                    done.append(_result(a.spec, a.lat, a.admitted, t0, self.clock))
                    a.lat.close()
                    self.used -= a.spec.budget_bytes()
            if not lane.jobs:
                continue
            members = tuple(id(a.lat) for a in lane.jobs)
            if members != lane.members:
                if lane.batch is not None:
                    lane.batch.close()
                lane.batch = T.Batch([a.lat for a in lane.jobs], lane.stream.cuda_stream)
                lane.members = members
            lane.batch.step(self.chunk, 0.01, "verlet")
            lane.inflight = list(lane.jobs)
            import torch
            lane.event = torch.cuda.Event()
            lane.event.record(lane.stream)
        return done

    def close(self):
        for lane in self.lanes.values():
            if lane.batch is not None:
                lane.batch.close()
            for a in lane.jobs:
                a.lat.close()
            lane.jobs, lane.batch, lane.members, lane.inflight = [], None, (), []
        self.used = 0


def serve(jobs: List[JobSpec], budget_bytes: int, chunk: int = 100,
          clock: Callable[[], float] = time.perf_counter):
    """Run ``jobs`` (sorted by arrival) through a continuous-batching server in
    real time.  Returns (results in completion order, makespan seconds)."""
    srv = Server(budget_bytes, chunk, clock)
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
            while i < len(pending) and pending[i].arrival <= now and srv.fits(pending[i]):
                srv.admit(pending[i], now)
                i += 1
            got = srv.service(t0)
            results.extend(got)
            if not got:
                if not srv.active and i < len(pending):
                    wait = pending[i].arrival - (clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
                else:
                    time.sleep(0.0005)
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
        results.append(_result(spec, lat, admitted, t0, clock))
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
