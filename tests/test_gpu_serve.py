"""Continuous-batching server on the GPU.

- Jobs arriving while others run are admitted as memory frees up, their work
  overlaps, and each job's state, energies and scale factor are bitwise those
  of the job run alone on the shape the server gives it (batch shape for the
  batched small jobs, the library default for solo big jobs); the binned
  spectrum to 1e-12, since the shell sums use FP64 atomics.  The mix has
  batched and solo lanes, FP32 and FP64, and several step sizes and
  integrators.
- Served jobs against the FP64 oracle: each job's initial state is drawn on
  both sides from its seed (Philox from its published definition on each
  side), and the final fields, energies, a and a' of the served job meet the
  parity tolerances (FP64 1e-12, FP32 1e-5, FP32 momenta ``f32_pi_tol``;
  Hubble residual as ``check_hubble``).
- The plain loop on the library's default shapes agrees with the served
  results within the same tolerances.
- Cancelling resident jobs (one in a batched lane, one solo) mid-run leaves
  every other job bitwise equal to the job run alone, and every cancelled
  lattice's memory returned."""
import numpy as np
import pytest

import oracle as o
from paper_2607_24908_gb300 import serve as S
from _tol import TOL, check_hubble, f32_pi_tol, normwise

pytestmark = pytest.mark.gpu

OINT = {"leapfrog": o.LEAPFROG, "verlet": o.VERLET, "yoshida4": o.YOSHIDA4}


def mixed_jobs():
    jobs = S.poisson_jobs(12, seed=7, rate=200.0, sizes=(16, 24, 32), steps=(100, 400), chunk=100)
    for k, j in enumerate(jobs):
        j.kIR = 0.5
        j.dt = (0.01, 0.005)[k % 2]
        j.integrator = ("verlet", "yoshida4", "verlet", "leapfrog")[k % 4]
    # two jobs big enough for solo lanes
    jobs.append(S.JobSpec(job_id=12, N=96, n_fields=2, q=100.0, steps=200, dtype="f64", seed=901, kIR=0.5,
                          arrival=jobs[3].arrival))
    jobs.append(S.JobSpec(job_id=13, N=192, n_fields=1, q=1.0, steps=100, dtype="f32", seed=902, kIR=0.5,
                          dt=0.005, integrator="yoshida4", arrival=jobs[5].arrival))
    assert sum(not S.is_batched(j) for j in jobs) == 2
    return jobs


def test_served_results_equal_alone_and_budget_respected():
    jobs = mixed_jobs()
    budget = 3 * max(j.budget_bytes() for j in jobs)  # a few jobs resident at a time: forces queueing
    peak = {"used": 0}
    orig_admit = S.Server.admit

    def admit(self, spec, now):
        assert orig_admit(self, spec, now) is None
        peak["used"] = max(peak["used"], self.used)
        assert self.used <= self.budget
    S.Server.admit = admit
    log = []
    try:
        served, t_served = S.serve(jobs, budget, chunk=100, log=log)
    finally:
        S.Server.admit = orig_admit
    alone, _ = S.run_alone(jobs, chunk=100, shape="served")
    assert len(served) == len(jobs) and peak["used"] <= budget
    by_id = {r.job_id: r for r in alone}
    for r in served:
        a = by_id[r.job_id]
        assert np.array_equal(r.energies, a.energies), r.job_id
        assert r.a == a.a and r.b == a.b
        # the state is bitwise equal; spectrum shell sums use FP64 atomics (order-dependent rounding)
        assert np.allclose(r.spectrum, a.spectrum, rtol=1e-12, atol=0.0)
        assert r.finished >= r.admitted >= r.arrival - 1e-9
    # several jobs were resident together at some point (continuous batching, not a queue)
    assert peak["used"] > max(j.budget_bytes() for j in jobs)
    assert S.lane_overlap(log, t_served)["two_or_more_lanes_busy"] > 0.0
    # the plain loop on default shapes: the same physics to rounding
    plain, _ = S.run_alone(jobs, chunk=100, shape="default")
    spec = {j.job_id: j for j in jobs}
    for r in plain:
        s = by_id[r.job_id]
        tol = TOL[spec[r.job_id].dtype]
        assert np.max(np.abs(r.energies - s.energies)) / np.sum(np.abs(s.energies)) < tol, r.job_id
        assert abs(r.a - s.a) / s.a < tol and abs(r.b - s.b) / abs(s.b) < tol, r.job_id


def test_served_jobs_match_the_oracle():
    jobs = [
        S.JobSpec(job_id=0, N=16, n_fields=2, q=100.0, steps=200, dtype="f64", seed=11, kIR=0.5),
        S.JobSpec(job_id=1, N=24, n_fields=1, q=1.0, steps=200, dtype="f32", seed=12, kIR=0.5),
        S.JobSpec(job_id=2, N=20, n_fields=3, q=100.0, steps=100, dtype="f64", seed=13, kIR=0.5, dt=0.005,
                  integrator="yoshida4"),
        S.JobSpec(job_id=3, N=32, n_fields=2, q=1.0, steps=100, dtype="f32", seed=15, kIR=0.5, dt=0.005,
                  integrator="leapfrog"),
        S.JobSpec(job_id=4, N=96, n_fields=2, q=100.0, steps=100, dtype="f64", seed=14, kIR=0.5),  # solo lane
    ]
    assert not S.is_batched(jobs[-1])
    served, _ = S.serve(jobs, 4 * sum(j.budget_bytes() for j in jobs), chunk=100, keep_state=True)
    assert len(served) == len(jobs)
    for r in served:
        j = jobs[r.job_id]
        p = o.Params(N=j.N, nf=j.n_fields, kIR=j.kIR, expanding=True, alpha=1.0, lam=1.0, q=j.q)
        spec = o.InitSpec(A=j.A, meff2=(3.0,) + (j.q,) * (j.n_fields - 1), phi0=(1.0, 0.0, 0.0))
        phi0, pi0, a0, b0 = o.init_fluctuations(p, j.seed, spec)
        ophi, opi, oa, ob = o.run(p, phi0, pi0, a0, b0, j.dt, j.steps, OINT[j.integrator])
        oE = o.energies(p, ophi, opi, oa)
        phi, pi = r.state
        tol = TOL[j.dtype]
        passes = j.steps * (3 if j.integrator == "yoshida4" else 1) + j.steps // 100
        tol_pi = tol if j.dtype == "f64" else f32_pi_tol(p, passes, np.max(np.abs(ophi)), np.max(np.abs(opi)))
        assert normwise(phi, ophi) < tol, (j.job_id, normwise(phi, ophi))
        assert normwise(pi, opi) < tol_pi, (j.job_id, normwise(pi, opi), tol_pi)
        assert np.max(np.abs(r.energies - oE)) / float(np.sum(oE)) < tol, (j.job_id, r.energies, oE)
        assert abs(r.a - oa) / oa < tol and abs(r.b - ob) / abs(ob) < tol, (j.job_id, r.a, oa, r.b, ob)
        check_hubble(p, r.hubble_resid, r.energies, r.a, r.b, oE, oa, ob)


def test_cancelled_jobs_leave_the_others_bitwise_unchanged():
    """All jobs resident at once; after the first chunk is started, one job of a
    batched lane and one solo job are cancelled.  Their lanes go on without them
    (the batch rebuilt), and every other job is bitwise the job run alone."""
    import time
    import torch
    jobs = mixed_jobs()
    small = [j for j in jobs if S.is_batched(j) and j.steps >= 200][0]
    solo = [j for j in jobs if not S.is_batched(j) and j.steps >= 200][0]
    lane_mates = [j for j in jobs if S.is_batched(j) and j.job_id != small.job_id
                  and S.Server.lane_key(j) == S.Server.lane_key(small)]
    assert lane_mates, "the cancelled batched job must share its lane"
    srv = S.Server(sum(j.budget_bytes() for j in jobs), chunk=100)
    results = []
    try:
        for j in jobs:
            assert srv.admit(j, 0.0) is None
        t0 = time.perf_counter()
        results += srv.service(t0)  # every lane's first chunk is in flight
        srv.cancel(small.job_id)
        srv.cancel(solo.job_id)
        while len(results) < len(jobs):
            results += srv.service(t0)
        assert srv.used == 0
    finally:
        srv.close()
    torch.cuda.synchronize()
    status = {r.job_id: r.status for r in results}
    assert status.pop(small.job_id) == "cancelled" and status.pop(solo.job_id) == "cancelled"
    assert set(status.values()) == {"done"}
    alone = {r.job_id: r for r in S.run_alone([j for j in jobs if j.job_id in status], chunk=100,
                                              shape="served")[0]}
    for r in results:
        if r.job_id in status:
            a = alone[r.job_id]
            assert np.array_equal(r.energies, a.energies), r.job_id
            assert r.a == a.a and r.b == a.b
