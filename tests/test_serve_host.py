"""The serving loop's host logic on the CPU: admission by budget in arrival
order, lanes per precision and size class, reaping, batch rebuilds and
clean-up, with the device calls (lattices, batches, streams, events) replaced
by fakes that record what the server asks of them."""
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
        FakeLattice.created.append(self)

    def set_pass_config(self, **shape):
        assert self.in_batch is None
        self.shape = shape

    def set_potential(self, lam, q, m2):
        pass

    def init_fluctuations(self, seed, A, meff2, phi0):
        self.seed = seed

    def step(self, n, dt, integ):  # the one-at-a-time loop
        assert not self.closed and self.in_batch is None
        self.steps += n

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
        orig_admit(self, spec, now)
        used_after_admit.append(self.used)
        admitted_ids.append(spec.job_id)
        for key, lane in self.lanes.items():  # each lane holds one precision and one size class
            for a in lane.jobs:
                assert key == (a.spec.dtype, "small" if S.job_cost(a.spec) <= S.SMALL_COST else "big")

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
    assert all(lat.shape["kind"] == "stream" for lat in FakeLattice.created)


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
