"""Continuous-batching server for lattice simulation jobs.

Jobs (lattice size, fields, couplings, steps, step size, integrator,
precision, seed) arrive over time.  The server admits a waiting job as soon as
its device memory fits in the budget beside the jobs already resident, draws
its initial state on the device, and from then on advances it in
``chunk``-step calls on a lane of its own kind:

* small jobs (per-step cost up to ``SMALL_COST``) share a batched lane per
  (precision, dt, integrator): whenever the lane is idle the host reaps its
  finished jobs and starts the next ``chunk`` steps of all its jobs as one
  batched call (``tl_batch_step``: one grouped launch per pass, replayed as a
  CUDA graph), so many small lattices fill the GPU together;
* a big job fills the GPU by itself, so batching it buys nothing: it gets a
  solo lane (its own stream) and runs ``tl_step`` on the launch shape the
  library gives it alone.

Lanes run concurrently on the device on their own CUDA streams, so small jobs
are not held to the pace of large ones.  A reaped job's final energies and
spectrum (and, on request, its final fields) are read back, its lattice
destroyed and its memory returned, and the freed budget admits the next
arrivals.

A job's launch shape depends only on the job (the batch shape for small jobs,
the library default for big ones), every job advances in the same
``chunk``-step calls whatever else is resident, and lanes never mix step
sizes or integrators, so its results are bitwise those of running it alone on
that shape (``run_alone(..., shape="served")``).  The plain one-job-at-a-time
loop a user would write (``run_alone(..., shape="default")``) runs every job
on the library's default launch shape; its results agree with the served ones
to rounding (the energy sums of small jobs are reduced in another order).
Step counts must be multiples of ``chunk``.  All device work goes through the
C ABI (paper_2607_24908_gb300.tl).
"""
from __future__ import annotations

import time
from dataclasses import dataclass
from typing import Callable, List, Optional, Tuple

import numpy as np

from . import tl as T


@dataclass
class JobSpec:
    """One simulation request: phi^4 plus (q/2) phi^2 chi^2 couplings to
    n_fields-1 further fields, expanding background (alpha = 1), ``integrator``
    with step dt, vacuum fluctuations A/(2 omega_k)."""
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
    integrator: str = "verlet"

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
    state: Optional[Tuple[np.ndarray, np.ndarray]] = None  # (phi, pi) [field, z, y, x] if kept
    status: str = "done"          # "done", "failed" (its lattice could not be set up) or "cancelled"
    error: str = ""               # the library's message for a failed job

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def _no_result(spec: JobSpec, admitted: float, finished: float, status: str, error: str = "") -> JobResult:
    """The result of a job that did not run to its end."""
    nan = float("nan")
    return JobResult(spec.job_id, spec.arrival, admitted, finished, np.zeros(0), nan, nan, nan, np.zeros(0), None,
                     status, error)


def job_cost(spec: JobSpec) -> float:
    """Relative device time per step (FP64 runs ALU-bound, ~8x an FP32 site)."""
    return spec.N ** 3 * spec.n_fields * (8.0 if spec.dtype == "f64" else 1.0)


SMALL_COST = 128 ** 3 * 3  # jobs up to this per-step cost share batched lanes


def is_batched(spec: JobSpec) -> bool:
    """Small jobs are served in batched lanes, big ones each on a solo lane."""
    return job_cost(spec) <= SMALL_COST


def _new_lattice(spec: JobSpec, stream: int, shape: str = "served") -> T.Lattice:
    """The job's lattice with its initial state.  shape "served": the shape the
    server steps it on (the batch shape for batched jobs, the library default
    otherwise); "default": the library default for every job."""
    if shape not in ("served", "default"):
        raise ValueError(f"unknown shape {shape!r}")
    lat = T.Lattice(spec.N, spec.kIR, spec.n_fields, spec.dtype, True, 1.0, 1.0, 1.0, stream=stream)
    try:
        if shape == "served" and is_batched(spec):
            lat.set_pass_config(**T.batch_pass_config(spec.N, spec.n_fields, spec.dtype))
        lat.set_potential(1.0, spec.q, (0.0, 0.0, 0.0))
        meff2 = (3.0,) + (spec.q,) * (spec.n_fields - 1)
        lat.init_fluctuations(spec.seed, A=spec.A, meff2=meff2, phi0=(1.0, 0.0, 0.0))
    except BaseException:
        lat.close()
        raise
    return lat


def _result(spec: JobSpec, lat: T.Lattice, admitted: float, t0: float,
            clock: Callable[[], float] = time.perf_counter, keep_state: bool = False) -> JobResult:
    E = lat.energies()
    _, P, _ = lat.spectrum(0, 0)
    state = lat.get_all() if keep_state else None
    return JobResult(spec.job_id, spec.arrival, admitted, clock() - t0, E.vector(), E.a, E.b, E.hubble_resid, P,
                     state)


@dataclass
class _Active:
    spec: JobSpec
    lat: T.Lattice
    done_steps: int
    admitted: float


class _Lane:
    """Jobs advanced together on one stream: a batched lane (small jobs of one
    precision, dt and integrator) or a solo lane (one big job).  The host
    starts the lane's next chunk as soon as the last one is done,
    independently of the other lanes."""

    def __init__(self, key, stream, batched: bool, dt: float, integrator: str):
        self.key = key
        self.stream = stream
        self.batched = batched
        self.dt = dt
        self.integrator = integrator
        self.jobs: List[_Active] = []
        self.batch: Optional[T.Batch] = None
        self.members: tuple = ()
        self.event = None
        self.started = 0.0  # host time the chunk in flight was started
        self.inflight: List[_Active] = []

    def busy(self) -> bool:
        return self.event is not None and not self.event.query()


class Server:
    """Continuous batching over resident lattices (see the module docstring).
    ``lane_log`` records (lane key, chunk start, time the host saw it done)
    for every chunk, in the server clock's seconds since ``t0``."""

    def __init__(self, budget_bytes: int, chunk: int = 100, clock: Callable[[], float] = time.perf_counter,
                 keep_state: bool = False):
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.clock = clock
        self.keep_state = keep_state
        self.lanes = {}  # key -> _Lane, created with a stream on first use
        self._streams: list = []  # streams of closed solo lanes, reused
        self.used = 0
        self.lane_log: List[tuple] = []
        self.cancelled: set = set()  # resident jobs to drop when their lane is next idle

    @property
    def active(self) -> List[_Active]:
        return [a for lane in self.lanes.values() for a in lane.jobs]

    def fits(self, spec: JobSpec) -> bool:
        return self.used + spec.budget_bytes() <= self.budget

    @staticmethod
    def lane_key(spec: JobSpec):
        if is_batched(spec):
            return ("batch", spec.dtype, float(spec.dt), spec.integrator)
        return ("solo", spec.job_id)

    def lane_of(self, spec: JobSpec) -> _Lane:
        key = self.lane_key(spec)
        if key not in self.lanes:
            import torch
            stream = self._streams.pop() if self._streams else torch.cuda.Stream()
            self.lanes[key] = _Lane(key, stream, is_batched(spec), float(spec.dt), spec.integrator)
        return self.lanes[key]

    def admit(self, spec: JobSpec, now: float) -> Optional[JobResult]:
        """Make the job resident.  If the library cannot set up its lattice (a
        device allocation that fails, say) the job is not admitted and its
        "failed" result is returned; otherwise None."""
        if spec.steps % self.chunk != 0:
            raise ValueError(f"job {spec.job_id}: steps must be a multiple of {self.chunk}")
        if spec.integrator not in T.INTEGRATORS:
            raise ValueError(f"job {spec.job_id}: unknown integrator {spec.integrator!r}")
        if not (np.isfinite(spec.dt) and spec.dt > 0):
            raise ValueError(f"job {spec.job_id}: dt must be positive")
        if not is_batched(spec) and self.lane_key(spec) in self.lanes:
            raise ValueError(f"job id {spec.job_id} is already resident")
        lane = self.lane_of(spec)
        try:
            lat = _new_lattice(spec, lane.stream.cuda_stream, "served")
        except T.TLError as e:
            if not lane.jobs and not lane.batched:  # the solo lane opened for this job
                self._streams.append(lane.stream)
                del self.lanes[self.lane_key(spec)]
            return _no_result(spec, now, now, "failed", str(e))
        lane.jobs.append(_Active(spec, lat, 0, now))
        self.used += spec.budget_bytes()
        return None

    def cancel(self, job_id: int) -> None:
        """Drop a resident job: at the next service of its lane, once any chunk
        in flight is done, its lattice is destroyed, its memory returned and a
        "cancelled" result reported (a "done" one if that chunk was its last)."""
        self.cancelled.add(job_id)

    def service(self, t0: float) -> List[JobResult]:
        """Reap finished jobs of idle lanes and start their next chunk.  Returns
        the jobs completed now."""
        done: List[JobResult] = []
        for key in list(self.lanes):
            lane = self.lanes[key]
            if lane.busy():
                continue
            if lane.event is not None:
                self.lane_log.append((key, lane.started, self.clock() - t0))
            lane.event = None
            for a in lane.inflight:
                a.done_steps += self.chunk
            lane.inflight = []
            finished = [a for a in lane.jobs if a.done_steps >= a.spec.steps or a.spec.job_id in self.cancelled]
            if finished:
                lane.jobs = [a for a in lane.jobs if a not in finished]
                if lane.batch is not None:
                    lane.batch.close()
                    lane.batch, lane.members = None, ()
                for a in finished:
                    self.cancelled.discard(a.spec.job_id)
                    if a.done_steps >= a.spec.steps:  # a job that completed before its cancel is done
                        done.append(_result(a.spec, a.lat, a.admitted, t0, self.clock, self.keep_state))
                    else:
                        done.append(_no_result(a.spec, a.admitted, self.clock() - t0, "cancelled"))
                    a.lat.close()
                    self.used -= a.spec.budget_bytes()
            if not lane.jobs:
                if not lane.batched:  # a solo lane ends with its job; its stream is reused
                    self._streams.append(lane.stream)
                    del self.lanes[key]
                continue
            if lane.batched:
                members = tuple(id(a.lat) for a in lane.jobs)
                if members != lane.members:
                    if lane.batch is not None:
                        lane.batch.close()
                    lane.batch = T.Batch([a.lat for a in lane.jobs], lane.stream.cuda_stream)
                    lane.members = members
                lane.batch.step(self.chunk, lane.dt, lane.integrator)
            else:
                lane.jobs[0].lat.step(self.chunk, lane.dt, lane.integrator)
            lane.inflight = list(lane.jobs)
            import torch
            lane.started = self.clock() - t0
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
        self.lanes = {}
        self.used = 0


def serve(jobs: List[JobSpec], budget_bytes: int, chunk: int = 100,
          clock: Callable[[], float] = time.perf_counter, keep_state: bool = False, log: Optional[list] = None,
          cancel: Optional[List[Tuple[float, int]]] = None):
    """Run ``jobs`` (sorted by arrival) through a continuous-batching server in
    real time.  Returns (results in completion order, makespan seconds); every
    job gives one result, "done", "failed" or "cancelled".  ``cancel``: (time,
    job id) requests, applied when their time has come (a job not yet admitted
    is dropped at once, a resident one at its lane's next idle point).  With
    ``log`` a list, the server's lane_log is appended to it."""
    srv = Server(budget_bytes, chunk, clock, keep_state)
    pending = sorted(jobs, key=lambda j: j.arrival)
    for j in pending:
        if j.budget_bytes() > budget_bytes:
            raise ValueError(f"job {j.job_id} alone exceeds the budget")
    requests = sorted(cancel or [])
    dropped: set = set()
    t0 = clock()
    results: List[JobResult] = []
    i = 0
    try:
        while len(results) < len(jobs):
            now = clock() - t0
            while requests and requests[0][0] <= now:
                _, jid = requests.pop(0)
                if any(j.job_id == jid for j in pending[i:]):
                    dropped.add(jid)
                elif any(a.spec.job_id == jid for a in srv.active):
                    srv.cancel(jid)
            while i < len(pending) and (pending[i].job_id in dropped or
                                        (pending[i].arrival <= now and srv.fits(pending[i]))):
                if pending[i].job_id in dropped:
                    results.append(_no_result(pending[i], now, now, "cancelled"))
                else:
                    failed = srv.admit(pending[i], now)
                    if failed is not None:
                        results.append(failed)
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
        if log is not None:
            log.extend(srv.lane_log)
        srv.close()
    return results, clock() - t0


def run_alone(jobs: List[JobSpec], chunk: int = 100, clock: Callable[[], float] = time.perf_counter,
              stream: int = 0, shape: str = "default", keep_state: bool = False):
    """The plain loop: jobs one at a time in arrival order, each stepped on its
    own in the same chunks with its own dt and integrator.  shape "default"
    runs every job on the library's default launch shape (the loop a user
    would write); "served" on the shape the server gives it (bitwise the served
    results).  Returns (results, makespan seconds)."""
    t0 = clock()
    results = []
    for spec in sorted(jobs, key=lambda j: j.arrival):
        now = clock() - t0
        if spec.arrival > now:
            time.sleep(spec.arrival - now)
        admitted = clock() - t0
        lat = _new_lattice(spec, stream, shape)
        for _ in range(spec.steps // chunk):
            lat.step(chunk, spec.dt, spec.integrator)
        results.append(_result(spec, lat, admitted, t0, clock, keep_state))
        lat.close()
    return results, clock() - t0


def lane_overlap(log: List[tuple], makespan: float) -> dict:
    """Busy fractions from a lane log: the share of the makespan in which at
    least one / at least two lanes had a chunk in flight, and each lane kind's
    summed busy time (seconds)."""
    ev = []
    per_kind = {}
    for key, t_start, t_end in log:
        ev.append((t_start, 1))
        ev.append((t_end, -1))
        kind = key[0] if key[0] == "solo" else f"batch-{key[1]}"
        per_kind[kind] = per_kind.get(kind, 0.0) + (t_end - t_start)
    ev.sort()
    busy1 = busy2 = 0.0
    depth, last = 0, 0.0
    for t, d in ev:
        if depth >= 1:
            busy1 += t - last
        if depth >= 2:
            busy2 += t - last
        depth += d
        last = t
    span = max(makespan, 1e-12)
    return {"any_lane_busy": busy1 / span, "two_or_more_lanes_busy": busy2 / span,
            "busy_s_by_lane_kind": per_kind}


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
