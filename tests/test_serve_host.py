"""The serving loop's host logic on the CPU: admission by budget in arrival
order, batched lanes per (precision, dt, integrator) and solo lanes for big
jobs, the step size and integrator each job is advanced with, reaping, batch
rebuilds and clean-up, failed and cancelled jobs, with the device calls (lattices, batches, streams,
events) replaced by fakes that record what the server asks of them."""
import types

import numpy as np
import pytest

from paper_2607_24908_gb300 import serve as S
from paper_2607_24908_gb300 import tl as realT


class FakeLattice:
    created = []

    def __init__(self, N, kIR, nf, dtype, expanding, alpha, a0, fstar, stream=0):
        self.N, self.nf, self.dtype, self.stream = N, nf, dtype, stream
        self.steps, self.closed, self.in_batch, self.shape = 0, False, None, None
        self.calls = []  # (n, dt, integrator) of every step this lattice took
        FakeLattice.created.append(self)

    def set_pass_config(self, **shape):
        assert self.in_batch is None
        self.shape = shape

    def set_potential(self, lam, q, m2):
        pass

    def init_fluctuations(self, seed, A, meff2, phi0):
        self.seed = seed

    def step(self, n, dt, integ):  # a solo lane or the one-at-a-time loop
        assert not self.closed and self.in_batch is None
        self.steps += n
        self.calls.append((n, dt, integ))

    def energies(self):
        assert not self.closed
        return types.SimpleNamespace(vector=lambda: np.array([float(self.steps)]), a=1.0, b=0.0,
                                     hubble_resid=0.0)

    def spectrum(self, f, which):
        return np.zeros(2), np.zeros(2), np.zeros(2)

    def close(self):
        assert self.in_batch is None, "a lattice closed while still in an open batch"
        self.closed = True


class FakeBatch:
    def __init__(self, lats, stream):
        for lat in lats:
            assert lat.in_batch is None, "a lattice in two open batches"
            assert lat.stream == stream
            lat.in_batch = self
        self.lats, self.open = list(lats), True

    def step(self, n, dt, integ):
        assert self.open
        for lat in self.lats:
            assert not lat.closed
            lat.steps += n
            lat.calls.append((n, dt, integ))

    def close(self):
        for lat in self.lats:
            lat.in_batch = None
        self.open = False


class FakeStream:
    count = 0

    def __init__(self):
        FakeStream.count += 1
        self.cuda_stream = 1000 + FakeStream.count


class FakeEvent:
    """Completes on its third query, so chunks are in flight for a while."""

    def __init__(self):
        self.queries = 0

    def record(self, stream):
        pass

    def query(self):
        self.queries += 1
        return self.queries >= 3


@pytest.fixture
def fakes(monkeypatch):
    import torch
    FakeLattice.created = []
    fake_T = types.SimpleNamespace(Lattice=FakeLattice, Batch=FakeBatch, DTYPES=realT.DTYPES,
                                   INTEGRATORS=realT.INTEGRATORS,
                                   tl_state_bytes=realT.tl_state_bytes,
                                   batch_pass_config=lambda N, nf, dtype: {"kind": "stream", "z_chunk": min(N, 32)})
    monkeypatch.setattr(S, "T", fake_T)
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    return fake_T


def _jobs():
    jobs = S.poisson_jobs(24, seed=7, rate=2000.0, sizes=(32, 64, 160), steps=(100, 600))
    return jobs


def test_serve_loop_completes_every_job_within_budget(fakes, monkeypatch):
    jobs = _jobs()
    budget = max(j.budget_bytes() for j in jobs) * 2
    used_after_admit, admitted_ids = [], []
    orig_admit = S.Server.admit

    def admit(self, spec, now):
        assert orig_admit(self, spec, now) is None
        used_after_admit.append(self.used)
        admitted_ids.append(spec.job_id)
        for key, lane in self.lanes.items():  # batched lanes: one precision, dt, integrator; solo: one job
            for a in lane.jobs:
                if S.is_batched(a.spec):
                    assert key == ("batch", a.spec.dtype, a.spec.dt, a.spec.integrator)
                else:
                    assert key == ("solo", a.spec.job_id) and len(lane.jobs) == 1

    monkeypatch.setattr(S.Server, "admit", admit)
    results, _ = S.serve(jobs, budget, chunk=100)
    assert sorted(r.job_id for r in results) == [j.job_id for j in jobs]
    assert max(used_after_admit) <= budget
    assert admitted_ids == sorted(admitted_ids)  # first come, first admitted
    by_id = {j.job_id: j for j in jobs}
    for r in results:  # each job saw exactly its own step count
        assert r.energies[0] == by_id[r.job_id].steps
        assert r.admitted >= by_id[r.job_id].arrival - 1e-9 and r.latency >= 0
    assert len(FakeLattice.created) == len(jobs)
    assert all(lat.closed for lat in FakeLattice.created)
    # batched jobs start on the batch shape, big ones keep the library default
    for lat in FakeLattice.created:
        small = S.job_cost(types.SimpleNamespace(N=lat.N, n_fields=lat.nf, dtype=lat.dtype)) <= S.SMALL_COST
        assert (lat.shape is not None and lat.shape["kind"] == "stream") if small else lat.shape is None
    assert any(lat.shape is None for lat in FakeLattice.created)  # the mix has big jobs


def test_tight_budget_serialises_and_still_finishes(fakes):
    jobs = _jobs()[:8]
    budget = max(j.budget_bytes() for j in jobs)  # room for the largest job alone
    results, _ = S.serve(jobs, budget, chunk=100)
    assert len(results) == len(jobs)
    assert all(lat.closed for lat in FakeLattice.created)


def test_server_refuses_bad_jobs(fakes):
    jobs = _jobs()[:3]
    with pytest.raises(ValueError):
        S.serve(jobs, min(j.budget_bytes() for j in jobs) - 1)
    srv = S.Server(budget_bytes=10 ** 12, chunk=100)
    bad = S.JobSpec(job_id=99, N=32, n_fields=1, q=1.0, steps=150, dtype="f32", seed=1)
    with pytest.raises(ValueError):
        srv.admit(bad, 0.0)
    srv.close()


def test_results_are_stamped_with_the_callers_clock(fakes):
    """Arrival, admission and finish times all come from the clock given to serve()."""
    ticks = iter(range(10 ** 9))
    clock = lambda: 1000.0 + next(ticks) * 1e-3  # noqa: E731  (a synthetic clock far from perf_counter)
    jobs = _jobs()[:6]
    results, makespan = S.serve(jobs, max(j.budget_bytes() for j in jobs) * 3, chunk=100, clock=clock)
    for r in results:
        assert 0.0 <= r.admitted <= r.finished <= makespan < 1000.0


def test_run_alone_steps_each_job_in_chunks(fakes):
    jobs = _jobs()[:5]
    results, _ = S.run_alone(jobs, chunk=100)
    assert [r.job_id for r in results] == [j.job_id for j in sorted(jobs, key=lambda j: j.arrival)]
    for r, j in zip(results, sorted(jobs, key=lambda j: j.arrival)):
        assert r.energies[0] == j.steps
    assert all(lat.closed for lat in FakeLattice.created)


def test_each_job_is_stepped_with_its_own_dt_and_integrator(fakes):
    """Jobs with a non-default step size or integrator are never advanced with
    another job's: lanes are keyed by them, and solo lanes use the job's own."""
    base = _jobs()[:10]
    jobs = []
    for k, j in enumerate(base):
        j.dt = (0.01, 0.004, 0.02)[k % 3]
        j.integrator = ("verlet", "yoshida4", "leapfrog")[k % 3]
        jobs.append(j)
    results, _ = S.serve(jobs, max(j.budget_bytes() for j in jobs) * 4, chunk=100)
    assert len(results) == len(jobs)
    by_seed = {j.seed: j for j in jobs}
    for lat in FakeLattice.created:
        j = by_seed[lat.seed]
        assert lat.calls and all(c == (100, j.dt, j.integrator) for c in lat.calls), (j.job_id, lat.calls)
        assert lat.steps == j.steps
    FakeLattice.created = []
    alone, _ = S.run_alone(jobs, chunk=100)
    for lat in FakeLattice.created:
        j = by_seed[lat.seed]
        assert all(c == (100, j.dt, j.integrator) for c in lat.calls)


def test_run_alone_shapes(fakes):
    """The plain loop runs every job on the library default ("default"); the
    "served" form reproduces the server's shapes (batch shape for batched jobs)."""
    jobs = _jobs()[:8]
    S.run_alone(jobs, chunk=100)
    assert all(lat.shape is None for lat in FakeLattice.created)
    FakeLattice.created = []
    S.run_alone(jobs, chunk=100, shape="served")
    for lat, j in zip(FakeLattice.created, sorted(jobs, key=lambda j: j.arrival)):
        assert (lat.shape is not None) == S.is_batched(j)
    with pytest.raises(ValueError):
        S.run_alone(jobs[:1], chunk=100, shape="tuned")


def test_server_refuses_unknown_integrator_and_bad_dt(fakes):
    srv = S.Server(budget_bytes=10 ** 12, chunk=100)
    for kw in ({"integrator": "rk4"}, {"dt": 0.0}, {"dt": float("nan")}):
        bad = S.JobSpec(job_id=7, N=32, n_fields=1, q=1.0, steps=100, dtype="f32", seed=1, **kw)
        with pytest.raises(ValueError):
            srv.admit(bad, 0.0)
    srv.close()


def test_lane_overlap_accounting():
    log = [(("solo", 1), 0.0, 4.0), (("batch", "f32", 0.01, "verlet"), 1.0, 2.0),
           (("batch", "f32", 0.01, "verlet"), 2.0, 3.0), (("solo", 2), 5.0, 6.0)]
    o = S.lane_overlap(log, 8.0)
    assert abs(o["any_lane_busy"] - 5.0 / 8.0) < 1e-12
    assert abs(o["two_or_more_lanes_busy"] - 2.0 / 8.0) < 1e-12
    assert o["busy_s_by_lane_kind"] == {"solo": 5.0, "batch-f32": 2.0}


def test_a_job_whose_lattice_cannot_be_set_up_fails_alone(fakes, monkeypatch):
    """A lattice creation that the library refuses (a failed device
    allocation, say) gives that job a "failed" result with the library's
    message; its budget is never taken, the lane it opened is dropped and every
    other job still runs to its end."""
    jobs = _jobs()[:10]
    doomed = {jobs[2].job_id, jobs[5].job_id}
    seeds = {j.seed: j.job_id for j in jobs}

    class Refusing(FakeLattice):
        def init_fluctuations(self, seed, A, meff2, phi0):
            if seeds[seed] in doomed:
                raise realT.TLError(-3, "cudaMalloc: out of memory")
            super().init_fluctuations(seed, A, meff2, phi0)

    fakes.TLError = realT.TLError
    fakes.Lattice = Refusing
    budget = max(j.budget_bytes() for j in jobs) * 3
    log = []
    results, _ = S.serve(jobs, budget, chunk=100, log=log)
    assert sorted(r.job_id for r in results) == [j.job_id for j in jobs]
    by_id = {r.job_id: r for r in results}
    steps = {j.job_id: j.steps for j in jobs}
    for jid, r in by_id.items():
        if jid in doomed:
            assert r.status == "failed" and "out of memory" in r.error and r.energies.size == 0
        else:
            assert r.status == "done" and r.energies[0] == steps[jid]
    assert all(lat.closed for lat in FakeLattice.created)  # the refused lattices too
    assert not any(key == ("solo", jid) for key, _, _ in log for jid in doomed)


def test_cancelled_jobs_release_their_memory(fakes, monkeypatch):
    """A cancel request drops a waiting job at once and a resident one at its
    lane's next idle point: the lattice is closed, its budget returned, the
    batch rebuilt without it, and the job reported "cancelled"; the others are
    unaffected."""
    jobs = S.poisson_jobs(12, seed=3, rate=1e6, sizes=(32, 64), steps=(600, 1000))
    budget = max(j.budget_bytes() for j in jobs) * 2  # the first jobs are resident, the rest wait
    ticks = iter(range(10 ** 9))
    clock = lambda: next(ticks) * 1e-3  # noqa: E731
    resident, waiting = jobs[1].job_id, jobs[-1].job_id
    used = []
    orig = S.Server.service

    def service(self, t0):
        out = orig(self, t0)
        used.append(self.used)
        assert 0 <= self.used <= budget
        return out

    monkeypatch.setattr(S.Server, "service", service)
    results, _ = S.serve(jobs, budget, chunk=100, clock=clock, cancel=[(0.004, resident), (0.004, waiting)])
    by_id = {r.job_id: r for r in results}
    assert sorted(by_id) == sorted(j.job_id for j in jobs)
    assert by_id[resident].status == "cancelled" and by_id[waiting].status == "cancelled"
    lat_of = {lat.seed: lat for lat in FakeLattice.created}
    seed = {j.job_id: j.seed for j in jobs}
    assert seed[waiting] not in lat_of  # never admitted
    assert lat_of[seed[resident]].closed and lat_of[seed[resident]].steps < jobs[1].steps
    for j in jobs:
        if j.job_id not in (resident, waiting):
            assert by_id[j.job_id].status == "done" and by_id[j.job_id].energies[0] == j.steps
    assert used[-1] == 0 and all(lat.closed for lat in FakeLattice.created)
