"""Throughput of the fused lattice step on one GB300 (per rank).

Workload: phi^4 + (q/2) phi^2 chi^2, q = 100, two fields, 1024^3 sites,
kIR = 0.05, expanding (alpha = 1, fstar/m_p = 1), 4th-order Yoshida,
dt = 0.005, FP32 fields and momenta with FP64 energy reductions, initial
state phi = 1, chi = 0 plus Gaussian fluctuations with power A/(2 omega_k),
A = 1e-10 (drawn on the device).  One bench step = one Yoshida step =
three fused passes.  The state (32 GiB) is far larger than L2, so no flush
is needed between timed iterations.

Metric: site-updates/s per field = N^3 * n_fields * passes / s (a pass is
one force evaluation: 1 per leapfrog/Verlet step, 3 per Yoshida step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With torchrun (N > 1) every rank runs its own replica (the path has no
exchange step on one lattice per GPU), so value = sum over ranks (weak).
``--impl reference`` times the FP64 CPU oracle on the host cores instead, on
a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2607_24908_gb300.workloads import TWO_FIELD_1024 as WL  # noqa: E402

METRIC = "site-updates/s per field"
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal (context beside the measured copy peak)
PASSES = {"leapfrog": 1, "verlet": 1, "yoshida4": 3}[WL.integrator]
BYTES_PER_SITE_FIELD_PASS = 4 * (4 if WL.dtype == "f32" else 8)  # read phi, pi; write phi, pi
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fused_pass_1024cubed_2f_f32.md")
KERNEL_SRCS = [os.path.join(ROOT, "paper_2607_24908_gb300", "csrc", n)
               for n in ("tl_pass_impl.cuh", "tl_pass.cu", "tl_pass_f32.cu", "tl_tma_maps.cu", "tl_lattice.cuh")]


def kernel_hash() -> str:
    """sha256 of what fixes the fused pass's DRAM traffic: the kernel, its
    geometry and FP32 instantiation, the tensor-map encoding and the padded
    array layout."""
    h = hashlib.sha256()
    for p in KERNEL_SRCS:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def kernel_name(shape) -> str:
    """The fused-pass kernel a launch shape runs (FP32, two fields)."""
    if shape is None:
        return "fused_pass<float,2>"
    if shape["kind"] == "tma":
        return f"fused_pass_tma<float,2> ({shape['warps']}+1 warps, {shape['stages']} stages)"
    return f"fused_pass_ldg<float,2> ({shape['threads']} threads)"


def shape_tag(shape) -> str:
    """The launch shape as written in the profile summary."""
    if not shape:
        return ""
    if shape["kind"] == "tma":
        return f"tma warps={shape['warps']} stages={shape['stages']} z_chunk={shape['z_chunk']}"
    return f"stream threads={shape['threads']} tile_x={shape['tile_x']} z_chunk={shape['z_chunk']}"


def measured_traffic(shape=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source and launch shape (else None)."""
    try:
        with open(TRAFFIC_FILE) as f:
            txt = f.read()
    except OSError:
        return None
    h = re.search(r"kernel source sha256\[:16\]:\s*([0-9a-f]+)", txt)
    b = re.search(r"dram bytes per full launch:\s*([0-9.eE+]+)", txt)
    sh = re.search(r"launch shape of the capture:\s*(.+)", txt)
    if not h or not b or h.group(1) != kernel_hash():
        return None
    if shape is not None and (not sh or sh.group(1).strip() != shape_tag(shape)):
        return None
    return float(b.group(1))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(rank: int) -> int:
    """Seed of a replica's initial state: every rank evolves its own lattice."""
    return WL.seed + 1000 * rank


def max_over_ranks(x: float, ws: int, device) -> float:
    """Max of x over all ranks (all_reduce MAX of one FP64 value on `device`:
    the GPU under NCCL, the CPU under gloo)."""
    if ws <= 1:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(work_per_rank: float, ws: int, t_max_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return work_per_rank * ws / (t_max_ms / 1e3)


# ---------------------------------------------------------------------------------
# CPU oracle leg (reported baseline / --impl reference)
# ---------------------------------------------------------------------------------

def oracle_sample(seconds_target: float = 15.0, max_steps: int = 1000):
    """Time the FP64 oracle on host cores on a bounded sample of the workload:
    same model, dt and integrator on a 96^3 two-field lattice."""
    import oracle as o
    n = 96
    p = o.Params(N=n, nf=WL.nf, kIR=WL.kIR * WL.N / n, expanding=WL.expanding, alpha=WL.alpha,
                 fstar_over_mp=WL.fstar_over_mp, lam=WL.lam, q=WL.q, m2=WL.m2)
    spec = o.InitSpec(A=WL.A, meff2=WL.meff2, phi0=WL.phi0)
    phi, pi, a, b = o.init_fluctuations(p, WL.seed, spec)
    integ = {"leapfrog": o.LEAPFROG, "verlet": o.VERLET, "yoshida4": o.YOSHIDA4}[WL.integrator]
    t0 = time.perf_counter()
    phi, pi, a, b = o.run(p, phi, pi, a, b, WL.dt, 1, integ)
    one = time.perf_counter() - t0
    steps = max(1, min(max_steps, int(seconds_target / max(one, 1e-6))))
    t0 = time.perf_counter()
    phi, pi, a, b = o.run(p, phi, pi, a, b, WL.dt, steps, integ)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = n ** 3 * WL.nf * PASSES * steps / el
    final = {"N": n, "kIR": p.kIR, "steps": 1 + steps, "E": o.energies(p, phi, pi, a), "a": a, "b": b,
             "R": o.hubble_residual(p, o.energies(p, phi, pi, a), a, b)}
    return {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{n}^3 x {WL.nf} fields, same model/dt/{WL.integrator}, FP64, {steps} steps in {el:.1f} s "
                      f"(OpenMP {cores} threads)"}, final


def gpu_vs_oracle(final):
    """The oracle sample's run (same seed, model, dx, dt, integrator and step
    count) on the GPU in each precision, one tl_step call: the largest error of
    K_f, G_f, V relative to K+G+V and of a, a' relative to themselves, against
    the FP64 oracle (the error statement of the reported FP32 result)."""
    from paper_2607_24908_gb300 import tl as T
    oE = np.asarray(final["E"])
    rho = float(np.sum(oE))
    out = {"sample": f"{final['N']}^3 x {WL.nf} fields, {final['steps']} {WL.integrator} steps "
                     f"(dt {WL.dt}, same dx as {WL.N}^3), initial state drawn from the same seed on each side"}
    for dtype in ("f32", "f64"):
        lat = T.Lattice(final["N"], final["kIR"], WL.nf, dtype, WL.expanding, WL.alpha, WL.fstar_over_mp, 1.0)
        lat.set_potential(WL.lam, WL.q, WL.m2)
        lat.init_fluctuations(WL.seed, A=WL.A, meff2=WL.meff2, phi0=WL.phi0)
        lat.step(final["steps"], WL.dt, WL.integrator)
        E = lat.energies()
        lat.close()
        out[dtype] = {"energies_rel_to_rho": float(np.max(np.abs(E.vector() - oE)) / rho),
                      "a_rel": abs(E.a - final["a"]) / final["a"], "b_rel": abs(E.b - final["b"]) / abs(final["b"]),
                      "hubble_resid": E.hubble_resid, "hubble_resid_oracle": final["R"]}
        out[dtype]["max"] = max(out[dtype]["energies_rel_to_rho"], out[dtype]["a_rel"], out[dtype]["b_rel"])
    return out


# FP64 operations a fused pass must do per site of one field, as the pass is
# written: drift 1; phi^2 1; the weighted dV/dphi in factored form 2 (the force's
# weight a^(3+alpha) folded into the coefficients); Laplacian (neighbour sum
# minus 6 phi) 6; force 1; momentum at the evaluation time and the kicked
# momentum 2; kinetic and gradient sums (summation by parts: -phi Lap phi) 2;
# V(phi) in factored form accumulated straight into its sum 2.  The FP64 pass
# is bound by the FP64 pipe; each thread also redoes the drift of its four
# in-plane neighbours (3 more per site), which is not counted here.
FP64_OPS_PER_SITE_1F = 17


def fp64_pass():
    """The paper's own precision: the 256^3 one-field expanding phi^4 workload
    in FP64 (velocity Verlet, one fused pass per step), ms per pass and its
    FP64-pipe roofline against the device's measured FP64 FMA issue rate."""
    import torch
    from paper_2607_24908_gb300 import tl as T
    from paper_2607_24908_gb300.workloads import PHI4_EXPANDING_256 as W2
    stream = torch.cuda.Stream()
    lat = T.Lattice(W2.N, W2.kIR, 1, "f64", True, W2.alpha, W2.fstar_over_mp, 1.0, stream=stream.cuda_stream)
    lat.set_potential(W2.lam, 0.0, W2.m2)
    lat.init_fluctuations(W2.seed, A=W2.A, meff2=W2.meff2, phi0=W2.phi0)
    for _ in range(3):
        lat.step(1, W2.dt, "verlet")
    lat.energies()
    steps = 40
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lat.step(steps, W2.dt, "verlet")
    e1.record(stream)
    torch.cuda.synchronize()
    ms_pass = e0.elapsed_time(e1) / (steps + 1)
    shape = lat.pass_config()
    lat.close()
    rate64, _ = T.tl_probe_fma_rates(stream.cuda_stream)
    sites = W2.N ** 3
    achieved = FP64_OPS_PER_SITE_1F * sites / (ms_pass / 1e3)
    hbm, _ = peaks()
    return {"workload": W2.name, "ms_per_pass": ms_pass, "site_updates_per_s": sites / (ms_pass / 1e3),
            "pass_shape": shape,
            "roofline": {"bound": "alu", "unit": "G FP64 operations/s", "ops_per_site": FP64_OPS_PER_SITE_1F,
                         "achieved": achieved / 1e9, "peak": rate64 / 1e9,
                         "peak_source": "tl_probe_fma_rates (measured FP64 FMA issue rate)",
                         "frac": achieved / rate64},
            "hbm_frac": 32 * sites / (ms_pass / 1e3) / 1e9 / hbm}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as o
    n = 96
    p = o.Params(N=n, nf=WL.nf, kIR=WL.kIR * WL.N / n, expanding=WL.expanding, alpha=WL.alpha,
                 fstar_over_mp=WL.fstar_over_mp, lam=WL.lam, q=WL.q, m2=WL.m2)
    phi, pi, a, b = o.init_fluctuations(p, WL.seed, o.InitSpec(A=WL.A, meff2=WL.meff2, phi0=WL.phi0))
    integ = {"leapfrog": o.LEAPFROG, "verlet": o.VERLET, "yoshida4": o.YOSHIDA4}[WL.integrator]
    for _ in range(args.warmup):
        phi, pi, a, b = o.run(p, phi, pi, a, b, WL.dt, 1, integ)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        phi, pi, a, b = o.run(p, phi, pi, a, b, WL.dt, 1, integ)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = n ** 3 * WL.nf * PASSES * args.steps / el
    sample = f"{n}^3 x {WL.nf} fields per step (bounded sample of {WL.N}^3), FP64, OpenMP {cores} threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WL.name, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------------

def run_ours(args):
    import torch
    from paper_2607_24908_gb300 import tl as T

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    sptr = stream.cuda_stream

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    integ = T.INTEGRATORS[WL.integrator]
    N = args.N or WL.N
    kIR = WL.kIR * WL.N / N  # same lattice spacing dx when N is reduced for profiling
    lat = T.Lattice(N, kIR, WL.nf, WL.dtype, WL.expanding, WL.alpha, WL.fstar_over_mp, 1.0, stream=sptr)
    lat.set_potential(WL.lam, WL.q, WL.m2)
    lat.init_fluctuations(replica_seed(rank), A=WL.A, meff2=WL.meff2, phi0=WL.phi0)
    args.pass_shape = lat.pass_config()
    # the end-to-end leg's page-locked host buffers (tl_host_alloc: huge pages,
    # registered), allocated and touched now: pinning tens of GB makes the host
    # rearrange memory for a while, which would slow the transfers if it
    # happened inside that leg's timed region
    host = []
    if not args.no_e2e:
        host = [T.host_empty((N,) * 3, np.float32 if WL.dtype == "f32" else np.float64) for _ in range(2 * WL.nf)]
        for f in range(WL.nf):
            for w in range(2):
                T.tl_get_state(lat.h, f, w, host[2 * f + w])

    # warm-up: W steps (one call each)
    for _ in range(args.warmup):
        lat.step(1, WL.dt, integ)
    lat.energies()
    barrier()

    # device-timed region: exactly K steps in one call (3K+1 fused passes)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    barrier()
    ev0.record(stream)
    lat.step(args.steps, WL.dt, integ)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    E = lat.energies()
    launches = PASSES * args.steps + 1
    ms_pass = ms / launches

    t_max = max_over_ranks(ms, ws, "cuda")
    sites = N ** 3
    work_per_rank = sites * WL.nf * PASSES * args.steps
    value = job_value(work_per_rank, ws, t_max)

    # end-to-end through the C ABI with host buffers: H2D of the state from
    # page-locked memory (tl_host_alloc), K steps, energies and D2H of the state, every call inside
    # the timed region; three such jobs, the median reported (the host link's
    # speed varies between jobs on a busy host; all three are in the phases).
    npd = np.float32 if WL.dtype == "f32" else np.float64
    if args.no_e2e:
        lat.close()
        t_e2e, E2 = float("nan"), E
        state_bytes = 2 * WL.nf * sites * np.dtype(npd).itemsize
        return _report(args, ws, rank, N, ms, t_max, ms_pass, launches, value, work_per_rank, t_e2e, state_bytes,
                       E, E2, clk)
    runs = []
    for f in range(WL.nf):  # the state the first job starts from
        for w in range(2):
            T.tl_get_state(lat.h, f, w, host[2 * f + w])
    a_in, b_in = E.a, E.b
    for rep in range(3):  # each job continues from the previous job's returned state
        barrier()
        t0 = time.perf_counter()
        for f in range(WL.nf):
            for w in range(2):
                T.tl_set_state(lat.h, f, w, host[2 * f + w])
        T.tl_set_background(lat.h, a_in, b_in, False)
        t1 = time.perf_counter()
        lat.step(args.steps, WL.dt, integ)
        E2 = lat.energies()
        t2 = time.perf_counter()
        for f in range(WL.nf):
            for w in range(2):
                T.tl_get_state(lat.h, f, w, host[2 * f + w])
        t3 = time.perf_counter()
        runs.append({"total_s": t3 - t0, "set_state_s": t1 - t0, "steps_and_energies_s": t2 - t1,
                     "get_state_s": t3 - t2})
        a_in, b_in = E2.a, E2.b
    mid = sorted(runs, key=lambda r: r["total_s"])[1]
    t_e2e = mid["total_s"]
    args.e2e_phases = {"median_job": mid, "jobs": runs}
    t_e2e = max_over_ranks(t_e2e, ws, "cuda")
    state_bytes = 2 * WL.nf * sites * np.dtype(npd).itemsize
    lat.close()
    return _report(args, ws, rank, N, ms, t_max, ms_pass, launches, value, work_per_rank, t_e2e, state_bytes,
                   E, E2, clk)


def _report(args, ws, rank, N, ms, t_max, ms_pass, launches, value, work_per_rank, t_e2e, state_bytes, E, E2, clk):
    import torch
    sites = N ** 3
    e2e_value = work_per_rank * ws / t_e2e if t_e2e == t_e2e else None
    if rank == 0:
        peak, peak_kind = peaks()
        alg_bytes = sites * WL.nf * BYTES_PER_SITE_FIELD_PASS
        achieved = alg_bytes / (ms_pass / 1e3) / 1e9
        cpu, extras = None, {}
        if ws == 1 and not args.no_cpu_baseline:
            cpu, final = oracle_sample()
            extras["oracle_error"] = gpu_vs_oracle(final)
        if ws == 1 and not args.no_extras and N == WL.N:
            extras["fp64"] = fp64_pass()
            extras["ensemble"] = ensemble_measure(96, 1000)
        line = {
            "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": WL.dtype, "data": "synthetic",
            "config": {"workload": WL.name if N == WL.N else f"{WL.name} reduced to {N}^3 (same dx)", "N": N, "n_fields": WL.nf, "integrator": WL.integrator,
                       "passes_per_step": PASSES, "dt": WL.dt, "storage": "fp32 fields/momenta, fp64 reductions",
                       "pass_shape": getattr(args, "pass_shape", None),
                       "l2": f"inputs ({4 * WL.nf * sites * (4 if WL.dtype == 'f32' else 8) / 2**30:.1f} GiB "
                             "state) larger than L2; no flush", "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind,
                         "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                         "traffic": measured_traffic(getattr(args, "pass_shape", None)) if N == WL.N else None,
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "kernel": kernel_name(getattr(args, "pass_shape", None)), "ms_per_launch": ms_pass},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "site-updates/s", "h2d_bytes_per_step": state_bytes / args.steps,
                    "d2h_bytes_per_step": (state_bytes + 136) / args.steps,
                    "note": "state H2D once from tl_host_alloc memory, K steps, energies + state D2H, per K-step job; "
                            "median of 3 jobs",
                    "phases": getattr(args, "e2e_phases", None)},
            "gpu_launches": launches,
            "clocks": clk,
            "physics": {"a": E.a, "hubble_resid": E.hubble_resid, "a_after_e2e": E2.a},
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------------
# Batched ensemble: many small uneven lattices, batched vs one job at a time
# ---------------------------------------------------------------------------------

def ensemble_jobs(n_jobs=96, seed=4242):
    """Per job: N from {32, 48, 64, 96, 128}, 1-2 fields, q from {0, 10, 100},
    its own seed; expanding (alpha = 1, kIR = 0.5), FP32 storage."""
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n_jobs):
        jobs.append(dict(N=int(rng.choice([32, 48, 64, 96, 128])), nf=int(rng.choice([1, 2])),
                         q=float(rng.choice([0.0, 10.0, 100.0])), seed=int(rng.integers(1, 2 ** 31))))
    return jobs


def ensemble_measure(n_jobs: int = 96, steps: int = 1000, dt: float = 0.01, tune_batch: bool = True) -> dict:
    """The batched ensemble (every job resident, one grouped launch per pass
    and field count, graph replay; member shapes and batch options from
    tl_batch_autotune) against one job at a time with tl_step on its
    autotuned shape; wall times include each job's init."""
    import torch
    from paper_2607_24908_gb300 import tl as T
    jobs = ensemble_jobs(n_jobs)

    def new(j, tune=True):
        lat = T.Lattice(j["N"], 0.5, j["nf"], "f32", True, 1.0, 1.0, 1.0)
        lat.set_potential(1.0, j["q"], (0.0, 0.0, 0.0))
        lat.init_fluctuations(j["seed"], A=1e-10, meff2=(3.0, j["q"], 0.0), phi0=(1.0, 0.0, 0.0))
        if tune:
            lat.autotune()
        return lat

    # warm the per-shape caches (FFT plans, autotuners) and the kernels once:
    # each shape tuned alone for the one-at-a-time arm, and a batch of the
    # same composition tuned for the batched arm (tl_batch_autotune caches its
    # member shapes and options for the batch created below)
    shapes = {(j["N"], j["nf"]) for j in jobs}
    for N, nf in shapes:
        lat = new(dict(N=N, nf=nf, q=0.0, seed=1))
        lat.step(2, dt, "verlet")
        lat.energies()
        lat.close()
    warm = [new(dict(j, seed=j["seed"] + 1), tune=False) for j in jobs]
    with T.Batch(warm) as b:
        b.step(2, dt, "verlet")
        tuned_ms_per_pass = b.autotune() if tune_batch else None
    for lat in warm:
        lat.close()
    torch.cuda.synchronize()

    # one job at a time
    t0 = time.perf_counter()
    seq = []
    t_seq_init = 0.0
    for j in jobs:
        ti = time.perf_counter()
        lat = new(j)
        torch.cuda.synchronize()
        t_seq_init += time.perf_counter() - ti
        lat.step(steps, dt, "verlet")
        seq.append(lat.energies())
        lat.close()
    t_seq = time.perf_counter() - t0

    # batched: all jobs resident, one grouped launch per pass, graph replay
    t0 = time.perf_counter()
    lats = [new(j, tune=False) for j in jobs]
    torch.cuda.synchronize()
    t_bat_init = time.perf_counter() - t0
    with T.Batch(lats) as b:
        b.step(steps, dt, "verlet")
        opts = b.options()
    bat = [lat.energies() for lat in lats]
    shapes_used = sorted({(lat.N, lat.nf, json.dumps(lat.pass_config(), sort_keys=True)) for lat in lats})
    for lat in lats:
        lat.close()
    t_bat = time.perf_counter() - t0

    diff = max(float(np.max(np.abs(x.vector() - y.vector()))) / float(np.sum(np.abs(y.vector()))) for x, y in
               zip(bat, seq))
    # the batched FP32 results against the FP64 oracle, on the cheapest jobs
    err = oracle_job_errors([(j["N"], j["nf"], j["q"], j["seed"], 0.5, dt, steps, "verlet", E.vector(), E.a, E.b)
                             for j, E in zip(jobs, bat)])
    site_updates = sum(j["N"] ** 3 * j["nf"] for j in jobs) * steps
    alg_bytes = sum(j["N"] ** 3 * j["nf"] for j in jobs) * 16 * (steps + 1)
    hbm, _ = peaks()
    return {"workload": f"{len(jobs)} jobs, N in {{32,48,64,96,128}}, 1-2 fields, q in {{0,10,100}}, "
                        f"{steps} Verlet steps dt={dt}, FP32 storage, expanding alpha=1, kIR=0.5",
            "jobs": len(jobs), "steps": steps,
            "batched_jobs_per_s": len(jobs) / t_bat, "sequential_jobs_per_s": len(jobs) / t_seq,
            "batched_s": t_bat, "sequential_s": t_seq,
            "init_s": {"batched": t_bat_init, "sequential": t_seq_init},
            "stepping_s": {"batched": t_bat - t_bat_init, "sequential": t_seq - t_seq_init},
            "speedup": t_seq / t_bat, "site_updates_per_s_batched": site_updates / t_bat,
            "batched_stepping_hbm_frac": alg_bytes / (t_bat - t_bat_init) / 1e9 / hbm,
            "batch_shapes": [{"N": n, "fields": f, "shape": json.loads(c)} for n, f, c in shapes_used],
            "batch_options": opts, "batch_tuned_ms_per_pass": tuned_ms_per_pass,
            "max_rel_energy_diff_batched_vs_sequential": diff,
            "oracle_error_fp32_batched": err}


def oracle_job_errors(cases, max_cases: int = 4):
    """Error of GPU results against the FP64 oracle on a bounded sample of
    jobs: each case (N, fields, q, seed, kIR, dt, steps, integrator, GPU
    energies [K.., G.., V], a, a') is rerun by the oracle from the same seed
    (Philox drawn from its definition on the CPU side), cheapest first.
    Returns the largest errors (energies relative to K+G+V; a, a' relative)."""
    import oracle as o
    integ = {"leapfrog": o.LEAPFROG, "verlet": o.VERLET, "yoshida4": o.YOSHIDA4}
    cases = sorted(cases, key=lambda c: c[0] ** 3 * c[1] * c[6])[:max_cases]
    worst = {"energies_rel_to_rho": 0.0, "a_rel": 0.0, "b_rel": 0.0}
    sample = []
    for N, nf, q, seed, kIR, dt, steps, integrator, E, a, b in cases:
        p = o.Params(N=N, nf=nf, kIR=kIR, expanding=True, alpha=1.0, lam=1.0, q=q)
        spec = o.InitSpec(A=1e-10, meff2=(3.0,) + (q,) * (nf - 1), phi0=(1.0, 0.0, 0.0))
        phi, pi, a0, b0 = o.init_fluctuations(p, seed, spec)
        ophi, opi, oa, ob = o.run(p, phi, pi, a0, b0, dt, steps, integ[integrator])
        oE = o.energies(p, ophi, opi, oa)
        worst["energies_rel_to_rho"] = max(worst["energies_rel_to_rho"],
                                           float(np.max(np.abs(np.asarray(E) - oE)) / np.sum(oE)))
        worst["a_rel"] = max(worst["a_rel"], abs(a - oa) / oa)
        worst["b_rel"] = max(worst["b_rel"], abs(b - ob) / abs(ob))
        sample.append(f"{N}^3x{nf} {steps} {integrator}")
    worst["max"] = max(worst["energies_rel_to_rho"], worst["a_rel"], worst["b_rel"])
    worst["sample"] = ", ".join(sample)
    return worst


def run_ensemble(args):
    import torch
    torch.cuda.set_device(0)
    r = ensemble_measure(args.jobs, args.ens_steps, tune_batch=not args.no_batch_tune)
    line = {"metric": "jobs/s", "value": r["batched_jobs_per_s"], "unit": "jobs/s", "higher_is_better": True,
            "mode": "ensemble", "n_gpus": 1, "config": {"workload": r["workload"], "jobs": r["jobs"],
                                                        "steps": r["steps"]}}
    line.update(r)
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------
# Serving: continuous batching vs a plain sequential loop
# ---------------------------------------------------------------------------------

def run_serve(args):
    import torch
    from paper_2607_24908_gb300 import serve as S
    torch.cuda.set_device(0)
    budget = int(150e9)
    n = args.jobs
    repeats = max(1, args.repeats)
    base = S.poisson_jobs(n, seed=12345, rate=0.0)
    # warm-up: one small and one big job of each precision on both shapes (kernels, FFT plans)
    warm = [S.JobSpec(-1, 64, 2, 100.0, 100, "f32", 1), S.JobSpec(-2, 64, 2, 100.0, 100, "f64", 2),
            S.JobSpec(-3, 256, 2, 100.0, 100, "f32", 3), S.JobSpec(-4, 256, 1, 100.0, 100, "f64", 4)]
    for shape in ("served", "default"):
        S.run_alone(warm, shape=shape)
    # mean service time of the plain loop from the first jobs, arrivals at t = 0
    probe = [S.JobSpec(**{**j.__dict__, "arrival": 0.0}) for j in base[:4]]
    _, t_probe = S.run_alone(probe, shape="default")
    mean_service = t_probe / len(probe)
    rate = 0.8 / mean_service
    jobs = S.poisson_jobs(n, seed=12345, rate=rate)
    sat = [S.JobSpec(**{**j.__dict__, "arrival": 0.0}) for j in jobs]

    def stats(res, span):
        lat = np.array([r.latency for r in res])
        return {"jobs_per_s": len(res) / span, "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "makespan_s": span}

    def agreement(a, b):
        """max relative difference of the final energies (to K+G+V), a and a'
        between two runs of the same jobs, per precision"""
        out = {}
        bb = {r.job_id: r for r in b}
        spec = {j.job_id: j for j in jobs}
        for r in a:
            s_ = bb[r.job_id]
            d = max(float(np.max(np.abs(r.energies - s_.energies)) / np.sum(np.abs(s_.energies))),
                    abs(r.a - s_.a) / s_.a, abs(r.b - s_.b) / abs(s_.b))
            k = spec[r.job_id].dtype
            out[k] = max(out.get(k, 0.0), d)
        return out

    runs = {"poisson_load_0.8": [], "saturation": []}
    agree = {}
    served_last = None
    for rep in range(repeats):
        for name, js in (("poisson_load_0.8", jobs), ("saturation", sat)):
            log = []
            served, span_s = S.serve(js, budget, log=log)
            served_last = served
            plain, span_p = S.run_alone(js, shape="default")
            for k, v in agreement(served, plain).items():
                agree[k] = max(agree.get(k, 0.0), v)
            runs[name].append({"served": stats(served, span_s), "plain_loop": stats(plain, span_p),
                               "speedup_jobs_per_s": span_p / span_s,
                               "served_lanes": S.lane_overlap(log, span_s)})

    def spread(name, arm, key):
        v = [r[arm][key] for r in runs[name]]
        return {"mean": float(np.mean(v)), "min": float(np.min(v)), "max": float(np.max(v))}

    summary = {name: {f"{arm}_{key}": spread(name, arm, key) for arm in ("served", "plain_loop")
                      for key in ("jobs_per_s", "p50_s", "p99_s")} for name in runs}
    sat_served = summary["saturation"]["served_jobs_per_s"]["mean"]
    spec = {j.job_id: j for j in jobs}
    oerr = {}
    for dt_ in ("f32", "f64"):
        cases = [(spec[r.job_id].N, spec[r.job_id].n_fields, spec[r.job_id].q, spec[r.job_id].seed,
                  spec[r.job_id].kIR, spec[r.job_id].dt, spec[r.job_id].steps, spec[r.job_id].integrator,
                  r.energies, r.a, r.b) for r in served_last if spec[r.job_id].dtype == dt_]
        if cases:
            oerr[dt_] = oracle_job_errors(cases, max_cases=1)
    line = {"metric": "served jobs/s", "value": sat_served, "unit": "jobs/s", "higher_is_better": True,
            "mode": "serve", "n_gpus": 1,
            "config": {"workload": f"{n} Poisson jobs: N in {{64,128,256,384}}, 1-3 fields, q in {{1,100}}, "
                                   "500-5000 Verlet steps (dt 0.01), FP32 or FP64, expanding alpha=1, kIR=0.1",
                       "budget_bytes": budget, "chunk_steps": 100, "arrival_rate_per_s": rate,
                       "mean_plain_service_s": mean_service, "repeats": repeats,
                       "plain_loop": "one job at a time, tl_step on the library's default launch shape",
                       "served": "batched lanes (small jobs, batch shape) + solo lanes (big jobs, default shape)"},
            "summary": summary, "runs": runs,
            "max_rel_diff_served_vs_plain": agree,
            "oracle_error_served": oerr,
            "accuracy_note": "served and plain results agree within the parity tolerances of each precision "
                             "(FP64 1e-12, FP32 1e-5); served results are bitwise those of each job alone on "
                             "its served shape (tests/test_gpu_serve.py)"}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------
# phi^4 through parametric resonance in an expanding box (256^3, VV, FP64 and FP32)
# ---------------------------------------------------------------------------------

def run_expanding256(args):
    import torch
    from paper_2607_24908_gb300 import tl as T
    from paper_2607_24908_gb300.workloads import PHI4_EXPANDING_256 as W2
    torch.cuda.set_device(0)
    steps = args.ens_steps if args.ens_steps != 1000 else W2.steps
    every = 100
    out = {}
    for dtype in ("f64", "f32"):
        stream = torch.cuda.Stream()
        lat = T.Lattice(W2.N, W2.kIR, 1, dtype, True, W2.alpha, W2.fstar_over_mp, 1.0, stream=stream.cuda_stream)
        lat.set_potential(W2.lam, 0.0, (0.0, 0.0, 0.0))
        lat.init_fluctuations(W2.seed, A=W2.A, meff2=W2.meff2, phi0=W2.phi0)
        series = []
        t_step = 0.0
        for s0 in range(0, steps, every):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(every, W2.dt, "verlet")
            e1.record(stream)
            E = lat.energies()
            t_step += e0.elapsed_time(e1)
            k, P, c = lat.spectrum(0, 0)
            series.append({"step": E.step, "a": E.a, "H_resid": E.hubble_resid, "K": float(E.K[0]),
                           "G": float(E.G[0]), "V": E.V, "P": P})
        lat.close()
        out[dtype] = (series, t_step / (steps + steps // every) )
    s64, ms64 = out["f64"]
    s32, ms32 = out["f32"]
    rows = []
    for a, b in zip(s64, s32):
        sel = a["P"] > 1e-6 * a["P"].max()
        rows.append({"step": a["step"], "a": a["a"], "hubble_resid_f64": a["H_resid"], "hubble_resid_f32": b["H_resid"],
                     "rho_f64": a["K"] + a["G"] + a["V"],
                     "f32_vs_f64_energy_rel": max(abs(b[q] - a[q]) / (a["K"] + a["G"] + a["V"]) for q in ("K", "G", "V")),
                     "f32_vs_f64_spectrum_rel_max": float(np.max(np.abs(b["P"][sel] - a["P"][sel]) / a["P"][sel])),
                     "P_bins_1_4_16_f64": [float(a["P"][i]) for i in (1, 4, 16)]})
    sites = W2.N ** 3
    fp64_rate, fp32_rate = T.tl_probe_fma_rates()
    line = {"mode": "expanding256", "workload": W2.name, "steps": steps,
            "ms_per_pass": {"f64": ms64, "f32": ms32},
            "fp64_fma_per_s_measured": fp64_rate, "fp32_fma_per_s_measured": fp32_rate,
            "site_updates_per_s": {"f64": sites / (ms64 / 1e3), "f32": sites / (ms32 / 1e3)},
            "every_100_steps": rows}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------
# The 32^3 FP64 static phi^4 workload: launch-bound, time per step direct vs graph replay
# ---------------------------------------------------------------------------------

def run_static32(args):
    import torch
    from paper_2607_24908_gb300 import tl as T
    from paper_2607_24908_gb300.workloads import PHI4_STATIC_32 as W1
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    lat = T.Lattice(W1.N, W1.kIR, 1, W1.dtype, False, 0.0, 1.0, 1.0, stream=stream.cuda_stream)
    lat.set_potential(W1.lam, 0.0, W1.m2)
    lat.init_fluctuations(W1.seed, A=W1.A, meff2=W1.meff2, phi0=W1.phi0)
    E0 = lat.energies()
    times = []
    for _ in range(4):  # call 1 launches directly, call 2 captures, calls 3-4 replay the graph
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.step(W1.steps, W1.dt, W1.integrator)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / W1.steps)
    E = lat.energies()
    lat.close()
    e0t, et = float(np.sum(E0.vector())), float(np.sum(E.vector()))
    fp64_rate, _ = T.tl_probe_fma_rates()
    print(json.dumps({"mode": "static32", "workload": W1.name, "steps_per_call": W1.steps,
                      "fp64_fma_per_s_measured": fp64_rate,
                      "ms_per_step_direct": times[0], "ms_per_step_graph": min(times[2:]),
                      "site_updates_per_s_graph": W1.N ** 3 / (min(times[2:]) / 1e3),
                      "energy_rel_change_after_1600_steps": abs(et - e0t) / e0t}), flush=True)
    return 0


# ---------------------------------------------------------------------------------
# Langevin phi^4 (the paper's interface example) throughput
# ---------------------------------------------------------------------------------

def run_langevin(args):
    import torch
    from paper_2607_24908_gb300 import tl as T
    torch.cuda.set_device(0)
    N = args.N or 512
    peak, peak_kind = peaks()
    out = {}
    for dtype in ("f32", "f64"):
        stream = torch.cuda.Stream()
        lat = T.Lattice(N, 0.5, 1, dtype, stream=stream.cuda_stream)
        npd = np.float32 if dtype == "f32" else np.float64
        lat.set_state(np.full((1, N, N, N), 0.5, npd), np.zeros((1, N, N, N), npd))
        lat.langevin(args.warmup, 0.01, 1.0, 0.5, 1.0, 7)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.langevin(args.steps, 0.01, 1.0, 0.5, 1.0, 7)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        esz = 4 if dtype == "f32" else 8
        out[dtype] = {"ms_per_step": ms, "site_updates_per_s": N ** 3 / (ms / 1e3),
                      "hbm_gbs": 2 * esz * N ** 3 / (ms / 1e3) / 1e9,
                      "frac_of_hbm": 2 * esz * N ** 3 / (ms / 1e3) / 1e9 / peak}
        lat.close()
    print(json.dumps({"mode": "langevin", "N": N, "steps": args.steps, "peak_gbs": peak, "peak_source": peak_kind,
                      "results": out}), flush=True)
    return 0


# ---------------------------------------------------------------------------------
# SU(2) Yang-Mills leapfrog (the paper's benchmark workload), ns per site per step
# ---------------------------------------------------------------------------------

def run_su2(args):
    import torch
    from paper_2607_24908_gb300 import tl as T
    torch.cuda.set_device(0)
    N = args.N or 576
    peak, peak_kind = peaks()
    out = {}
    for dtype in ("f64", "f32"):
        stream = torch.cuda.Stream()
        lat = T.SU2(N, dtype, stream=stream.cuda_stream)
        lat.init_random(7, 0.8)
        lat.step(args.warmup, 0.02)
        m0 = lat.measure()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(args.steps, 0.02)
        e1.record(stream)
        m1 = lat.measure()
        ms = e0.elapsed_time(e1) / args.steps
        esz = 4 if dtype == "f32" else 8
        alg = 42 * esz * N ** 3  # read 12 link + 9 field values, write 9 + 12, per site
        out[dtype] = {"ms_per_step": ms, "ns_per_site_step": ms * 1e6 / N ** 3,
                      "achieved_gbs": alg / (ms / 1e3) / 1e9, "frac_of_hbm": alg / (ms / 1e3) / 1e9 / peak,
                      "energy_drift_rel": abs(m1[0] + m1[1] - m0[0] - m0[1]) / (m0[0] + m0[1]),
                      "gauss_max": m1[2]}
        lat.close()
    print(json.dumps({"mode": "su2", "N": N, "steps": args.steps, "dt": 0.02, "peak_gbs": peak,
                      "peak_source": peak_kind, "results": out}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--N", type=int, default=0, help="lattice size (default: the workload's 1024; for profiling)")
    ap.add_argument("--mode", default="step",
                    choices=["step", "ensemble", "serve", "expanding256", "static32", "langevin", "su2"],
                    help="step: the 1024^3 fused step (default); ensemble: batched small lattices vs a plain loop; "
                         "serve: continuous batching of Poisson-arriving jobs vs a sequential loop")
    ap.add_argument("--jobs", type=int, default=0, help="jobs for --mode ensemble (96) / serve (16)")
    ap.add_argument("--repeats", type=int, default=2, help="--mode serve: repeats of each arm")
    ap.add_argument("--no-batch-tune", action="store_true",
                    help="--mode ensemble: batch on the untuned batch shapes (for comparison)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line without the fp64 and ensemble keys (profiling runs)")
    ap.add_argument("--ens-steps", type=int, default=1000)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: warm-up raised to the minimum of 3 steps", file=sys.stderr)
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "ensemble":
        args.jobs = args.jobs or 96
        return run_ensemble(args)
    if args.mode == "su2":
        return run_su2(args)
    if args.mode == "langevin":
        return run_langevin(args)
    if args.mode == "expanding256":
        return run_expanding256(args)
    if args.mode == "static32":
        return run_static32(args)
    if args.mode == "serve":
        args.jobs = args.jobs or 16
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
