#!/usr/bin/env python
"""Throughput of the convex-limited graph-dG stage sweep on GB300 (DoF-stage updates per second).

Workload (default): 2D Euler, gamma = 1.4, dG Q2 on 1024 x 1024 uniform quads of [0,1]^2 (9,437,184
nodes), four-quadrant Riemann data drawn from default_rng(0), slip walls, full limited scheme (two limiter
passes), CFL 0.5.  One step = one SSP-RK3 step = one gdg_ssprk3_step call (the time step is reduced
on the device from the first stage's sweep, no host round trip), i.e. 3 DoF-stage updates per node.  Inputs are synthetic and resident in HBM; the working set (several GB) is larger than
L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank runs its own instance (replicas: the path has no
exchange step); value = all ranks' DoF-stage updates / max over ranks of the timed region.
At N = 1 the line also carries the batched workload (its 512 seeded Q1 instances: batched solves/s
against one at a time) and a sample of the served workload (48 Poisson-arrival Q1/Q2
requests with meshes up to 256^2 and end times capped at 0.01: solves/s and p50/p99 time-to-solution
against one at a time); --workload batched_q1_riemann / served_stream run either at any size.
--impl reference times the FP64 CPU oracle on all host cores (rank 0 only) on a bounded sample of the
same workload (the same four-quadrant data on a 128 x 128 Q2 mesh).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DoF-stage updates/s"
WORKLOADS = {
    "q2_1024_four_quadrant": dict(N=1024, k=2, seed=0),
    "q2_512_four_quadrant": dict(N=512, k=2, seed=0),
    "q1_512_vortex_periodic": dict(N=512, k=1, vortex=True),
}
SAMPLE_N = 128  # oracle sample: same data on a 128 x 128 mesh
SOLVE_STEPS = 50  # a batched solve: 50 SSP-RK3 steps of one instance
# samples of the batched and served workloads that the default run reports beside the main line
COMBINED_BATCH_INSTANCES = 512
COMBINED_SERVED = dict(requests=48, rate=20.0, n_max=256, t_cap=0.01)


def make_problem(spec):
    from paper_2402_04514_gb300 import assembly, workloads

    N, k = spec["N"], spec["k"]
    if spec.get("vortex"):
        P = assembly.assemble_2d(N, N, k, box=(-5.0, 5.0, -5.0, 5.0), periodic=(True, True))
        U = workloads.vortex(P.x[0], P.x[1], 0.0, gamma=1.4)
    else:
        P = assembly.assemble_2d(N, N, k)
        U = workloads.four_quadrant(P.x[0], P.x[1], gamma=1.4, seed=spec.get("seed", 0))
    return P, U


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(", ") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({nm for r in rows for nm, v in zip(names, r[5:9]) if v.strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (all ranks get it): the job is done when its last rank is."""
    import torch

    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms_max):
    """Units processed by all ranks (replicas: each rank the same work) per second of the slowest rank."""
    return world * units_per_rank / (ms_max / 1e3)


def oracle_sample_rate(steps, warmup=0, openmp=False):
    """DoF-stage updates/s of the CPU oracle on the 128^2 sample: the pinned single-thread build, or with
    openmp=True the same code with its row loops shared among all host cores (bit-identical results).
    Returns (value, seconds, nodes, threads)."""
    from oracle import oracle as om

    spec = dict(WORKLOADS["q2_1024_four_quadrant"], N=SAMPLE_N)
    P, U = make_problem(spec)
    O = om.Oracle(P, openmp=openmp)
    for _ in range(warmup):
        tau = O.max_dt(U, 0.5)
        U, _ = O.ssprk3_step(U, tau)
    t0 = time.perf_counter()
    for _ in range(steps):
        tau = O.max_dt(U, 0.5)
        U, _ = O.ssprk3_step(U, tau)
    dt = time.perf_counter() - t0
    return P.n * 3 * steps / dt, dt, P.n, om.threads(openmp)


def oracle_full_size_rate(P, U, steps):
    """The all-core oracle on the full bench mesh itself for a few SSP-RK3 steps (the time step from the
    oracle's own max_dt): its DoF-stage rate, which extrapolates per stage to any number of steps.
    Returns (value, seconds, threads)."""
    from oracle import oracle as om

    O = om.Oracle(P, openmp=True)
    t0 = time.perf_counter()
    for _ in range(steps):
        U, _ = O.ssprk3_step(U, O.max_dt(U, 0.5))
    dt = time.perf_counter() - t0
    return P.n * 3 * steps / dt, dt, om.threads(True)


def measure_developed(N=256, t_dev=0.05, steps=20):
    """How representative steps from the initial data are: the same four-quadrant Q2 problem on N^2 quads,
    stepped to t_dev (the waves then cross a good part of the domain), against its first steps.  Returns
    ms per SSP-RK3 step at the start and at t_dev (autotuned once at the start, as the main line)."""
    import torch

    from paper_2402_04514_gb300.gdg import Solver

    P, U0 = make_problem(dict(N=N, k=2, seed=0))
    S = Solver(P)
    S.set_clock(0.0, float("inf"), 0.5)
    U = torch.from_numpy(U0).cuda()
    work = (torch.empty_like(U), torch.empty_like(U))
    stream = torch.cuda.current_stream()
    for _ in range(3):
        S.step(U, work)
    S.autotune(U, work, trials=1)

    def timed():
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            S.step(U, work)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    early = timed()
    taken = 3 + steps
    while S.clock()[0] < t_dev:
        for _ in range(50):
            S.step(U, work)
        taken += 50
    late = timed()
    return {"workload": f"Q2 {N}x{N} four-quadrant (seed 0), the same sweep and schedule", "ms_per_step_initial": early,
            "ms_per_step_developed": late, "t_developed": S.clock()[0], "steps_taken": taken + steps,
            "ratio": late / early, "status_flags": S.status()}


def run_vortex_sweep(args):
    """The isentropic-vortex throughput sweep (Q1 on periodic [-5,5]^2 meshes of 64^2 .. 512^2 quads, gamma
    = 1.4): per N, the GPU's DoF-stage updates/s over fused SSP-RK3 steps (after warm-up and autotuning)
    and the FP64 oracle's on the same mesh and data, single-threaded and on all host cores, over a bounded
    number of steps.  Prints one JSON line."""
    import torch

    from oracle import oracle as om
    from paper_2402_04514_gb300.gdg import Solver

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rows = []
    for N in (64, 128, 256, 512):
        P, U0 = make_problem(dict(N=N, k=1, vortex=True))
        S = Solver(P)
        S.set_clock(0.0, float("inf"), 0.5)
        U = torch.from_numpy(U0).cuda()
        work = (torch.empty_like(U), torch.empty_like(U))
        for _ in range(args.warmup):
            S.step(U, work)
        S.autotune(U, work, trials=1)
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            S.step(U, work)
        e1.record(stream)
        torch.cuda.synchronize()
        gpu = P.n * 3 * args.steps / (e0.elapsed_time(e1) / 1e3)
        row = {"N": N, "dofs": int(P.n), "gpu": gpu, "gpu_ms_per_step": e0.elapsed_time(e1) / args.steps,
               "status_flags": S.status()}
        S.close()
        for openmp in (False, True):
            O = om.Oracle(P, openmp=openmp)
            steps = max(1, int(2e6 / P.n)) if not openmp else max(2, int(5e6 / P.n))
            V = U0.copy()
            t0 = time.perf_counter()
            for _ in range(steps):
                V, _ = O.ssprk3_step(V, O.max_dt(V, 0.5))
            dt = time.perf_counter() - t0
            row["oracle_all_cores" if openmp else "oracle_1_thread"] = P.n * 3 * steps / dt
            row["oracle_steps_all_cores" if openmp else "oracle_steps_1_thread"] = steps
        row["oracle_threads"] = om.threads(True)
        rows.append(row)
    print(json.dumps({"metric": METRIC, "unit": METRIC, "workload": "q1_vortex_periodic_sweep", "gamma": 1.4,
                      "cfl": 0.5, "steps": args.steps, "warmup": args.warmup, "rows": rows}), flush=True)
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    value, secs, n_s, threads = oracle_sample_rate(args.steps, args.warmup, openmp=True)
    sample = (f"Q2 {SAMPLE_N}x{SAMPLE_N} four-quadrant (seed 0, {n_s} DoFs), {args.steps} SSP-RK3 steps after "
              f"{args.warmup} warm-up steps, {threads} threads (the oracle's row loops shared by OpenMP), "
              f"{secs:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(args, None),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def c4_instances(count, seed=1):
    """The batched workload: `count` instances of 2D Q1 on [0,1]^2 with N = round(32 * 16^u) quads per side
    (u ~ U[0,1], so N is log-uniform in [32, 512]), slip walls, two-state Riemann data split by a line
    through the centre at a random angle (rho, p log-uniform in [0.1, 10], |u| <= 2), all from
    default_rng(seed).  Yields (N, problem, U0)."""
    import numpy as np

    from paper_2402_04514_gb300 import assembly, workloads

    rng = np.random.default_rng(seed)
    Ns = [int(round(32 * 16 ** u)) for u in rng.uniform(0.0, 1.0, count)]
    for N in Ns:
        P = assembly.assemble_2d(N, N, 1)
        yield N, P, workloads.two_state_riemann(P.x[0], P.x[1], rng)


def measure_batched(instances, steps, warmup, autotune=True):
    """Batched solves: one gdg_batch_step advances every instance by one SSP-RK3 step in shared launches;
    against the same instances stepped one at a time (gdg_ssprk3_step per instance, in turn, on one
    stream).  A solve is SOLVE_STEPS steps of one instance; solves/s = instances x timed steps /
    SOLVE_STEPS / time.  `instances` takes the first instances of the seeded 512-instance stream."""
    import torch

    from paper_2402_04514_gb300.gdg import Batch, Solver

    solvers, states, works, sizes = [], [], [], []
    t0 = time.perf_counter()
    stream_ = c4_instances(512)
    for _ in range(instances):
        N, P, U = next(stream_)
        S = Solver(P)
        S.set_clock(0.0, float("inf"), 0.5)
        Ud = torch.from_numpy(U).cuda()
        solvers.append(S)
        states.append(Ud)
        works.append((torch.empty_like(Ud), torch.empty_like(Ud)))
        sizes.append(P.n)
    setup_s = time.perf_counter() - t0
    B = Batch(solvers, states, works)
    stream = torch.cuda.current_stream()
    dofs = sum(sizes)

    def timed(fn, k):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def one_at_a_time():
        for S, U, w in zip(solvers, states, works):
            S.step(U, w)

    for _ in range(warmup):
        B.step()
        one_at_a_time()
    schedule = B.autotune(trials=1) if autotune else B.schedule()  # states restored
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    t_batch = timed(B.step, steps)
    t_single = timed(one_at_a_time, steps)
    # the same batch as one cooperative launch per stage (gdg_batch_set_persistent)
    B.set_persistent(True)
    B.step()
    t_persist = timed(B.step, steps)
    B.set_persistent(False)
    clocks = sampler.stop()
    flags = max(S.status() for S in solvers)
    B.close()
    for S in solvers:
        S.close()
    inst = len(solvers)
    return {"value": inst * steps / SOLVE_STEPS / t_batch, "unit": "solves/s", "steps": steps, "warmup": warmup,
            "ms_per_step": 1e3 * t_batch / steps,
            "config": {"workload": "batched_q1_riemann", "instances": inst,
                       "sample": ("all 512 instances" if inst == 512 else
                                  f"the first {inst} of the 512 instances of the seeded stream"),
                       "mesh": "N x N Q1 quads, N log-uniform in [32, 512]", "dofs_total": dofs,
                       "solve": f"{SOLVE_STEPS} SSP-RK3 steps", "scheme": "convex-limited, 2 limiter passes",
                       "cfl": 0.5, "seed": 1, "setup_s": round(setup_s, 1), "schedule": schedule},
            "dof_stage_per_s": dofs * 3 * steps / t_batch,
            "one_at_a_time": {"value": inst * steps / SOLVE_STEPS / t_single, "unit": "solves/s",
                              "ms_per_step": 1e3 * t_single / steps,
                              "dof_stage_per_s": dofs * 3 * steps / t_single},
            "persistent": {"value": inst * steps / SOLVE_STEPS / t_persist, "unit": "solves/s",
                           "ms_per_step": 1e3 * t_persist / steps, "gpu_launches": 3 * steps,
                           "launch": "one cooperative launch per SSP-RK3 stage over all instances"},
            "speedup_vs_one_at_a_time": t_single / t_batch, "gpu_launches": 26 * steps,
            "clocks": clocks, "status_flags": flags}


def run_batched(args):
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    r = measure_batched(args.instances, args.steps, args.warmup, autotune=not args.no_autotune)
    line = {"metric": "batched solves/s", "value": r["value"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": r["config"],
            **{k: r[k] for k in ("dof_stage_per_s", "one_at_a_time", "persistent", "speedup_vs_one_at_a_time",
                                 "gpu_launches", "clocks", "status_flags")}}
    print(json.dumps(line), flush=True)
    return 0


def served_requests(count, rate, seed=2, n_max=64, t_cap=None):
    """The served stream: `count` requests with Poisson arrivals at `rate` per second, all from
    default_rng(seed): Q1 or Q2 (even odds), N x N quads of [0,1]^2 with N log-uniform in [16, n_max], slip
    walls, two-state Riemann data (as the batched workload) or the isentropic vortex of Sec. 6.2 scaled to the
    unit square (even odds), end time uniform in [0.1, 1] (capped at t_cap when given, so that a stream with
    large meshes ends in minutes).  Yields (arrival_s, problem, U0, t_end)."""
    import numpy as np

    from paper_2402_04514_gb300 import assembly, workloads

    rng = np.random.default_rng(seed)
    t = 0.0
    for _ in range(count):
        t += rng.exponential(1.0 / rate)
        k = 1 + int(rng.integers(0, 2))
        N = int(round(16 * (n_max / 16.0) ** rng.uniform(0.0, 1.0)))
        P = assembly.assemble_2d(N, N, k)
        if rng.uniform() < 0.5:
            U = workloads.two_state_riemann(P.x[0], P.x[1], rng)
        else:
            U = workloads.vortex(10.0 * P.x[0] - 5.0, 10.0 * P.x[1] - 5.0, 0.0, gamma=1.4)
        t_end = float(rng.uniform(0.1, 1.0))
        yield t, P, np.ascontiguousarray(U), (t_end if t_cap is None else min(t_end, t_cap))


def measure_served(requests, rate, n_max, t_cap=None, skip_one_at_a_time=False):
    """Served stream: requests submitted at their arrival times to the continuous-batching server
    (gdg_server), against the same stream solved one request at a time (each with gdg_ssprk3_step to its
    end time, in arrival order).  Reports solves/s over the makespan and p50/p99 time-to-solution."""
    import threading

    import numpy as np
    import torch

    from paper_2402_04514_gb300.gdg import Server, Solver

    reqs = list(served_requests(requests, rate, n_max=n_max, t_cap=t_cap))
    dofs = sum(P.n for _, P, _, _ in reqs)

    def pct(v, q):
        return float(np.percentile(np.asarray(v), q))

    # continuous batching
    srv = Server()
    ids = [None] * len(reqs)
    t0 = time.perf_counter()

    def client():
        for i, (ta, P, U, te) in enumerate(reqs):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids[i] = srv.submit(P, U, te)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    th = threading.Thread(target=client)
    th.start()
    th.join()
    infos = [srv.wait(r)[1] for r in ids]
    srv.close()
    tts = [i["t_done"] - i["t_submit"] for i in infos]
    span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
    steps = sum(i["steps"] for i in infos)
    flags = max(i["flags"] for i in infos)
    status = max(i["status"] for i in infos)

    # one at a time, in arrival order, each request as soon as it has arrived and the previous one is done
    t1 = time.perf_counter()
    tts1 = []
    for ta, P, U, te in ([] if skip_one_at_a_time else reqs):
        now = time.perf_counter() - t1
        if now < ta:
            time.sleep(ta - now)
        S = Solver(P)
        S.set_clock(0.0, te, 0.5)
        Ud = torch.from_numpy(U).cuda()
        work = (torch.empty_like(Ud), torch.empty_like(Ud))
        while True:
            for _ in range(8):  # finished steps are no-ops: check the clock every 8 steps
                S.step(Ud, work)
            if S.clock()[0] >= te:
                break
        Ud.cpu()
        tts1.append(time.perf_counter() - t1 - ta)
        S.close()
    span1 = time.perf_counter() - t1 - reqs[0][0]
    clocks = sampler.stop()
    one = None if skip_one_at_a_time else {
        "value": len(reqs) / span1, "unit": "solves/s", "tts_p50_s": pct(tts1, 50), "tts_p99_s": pct(tts1, 99),
        "makespan_s": span1}
    return {"value": len(reqs) / span, "unit": "solves/s", "steps": steps,
            "config": {"workload": "served_stream", "requests": len(reqs), "rate_per_s": rate,
                       "mesh": f"N x N Q1/Q2 quads, N log-uniform in [16, {n_max}]",
                       "t_end": "uniform in [0.1, 1]" + ("" if t_cap is None else f", capped at {t_cap}"),
                       "data": "Riemann or scaled vortex", "seed": 2, "dofs_total": dofs,
                       "budget": "80% of free HBM"},
            "tts_p50_s": pct(tts, 50), "tts_p99_s": pct(tts, 99), "makespan_s": span,
            "one_at_a_time": one, "speedup_vs_one_at_a_time": None if one is None else span1 / span,
            "clocks": clocks, "status_flags": flags, "status": status}


def run_served(args):
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    r = measure_served(args.requests, args.rate, args.n_max, args.t_cap, args.skip_one_at_a_time)
    line = {"metric": "served solves/s", "value": r["value"], "unit": "solves/s", "n_gpus": 1, "steps": r["steps"],
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": r["config"],
            **{k: r[k] for k in ("tts_p50_s", "tts_p99_s", "makespan_s", "one_at_a_time", "speedup_vs_one_at_a_time",
                                 "clocks", "status_flags", "status")}}
    print(json.dumps(line), flush=True)
    return 0


def config_block(args, n):
    spec = WORKLOADS[args.workload]
    return {"workload": args.workload, "mesh": f"{spec['N']}x{spec['N']} quads", "degree": spec["k"],
            "dofs_per_gpu": n, "gamma": 1.4, "cfl": 0.5, "scheme": "convex-limited, 2 limiter passes",
            "step": "SSP-RK3 step (gdg_ssprk3_step: tau chosen on the device + 3 stages)", "parallelism": f"replicas x{args.gpus}",
            "l2": "no flush: working set larger than L2 (129 MB)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="q2_1024_four_quadrant",
                    choices=sorted(WORKLOADS) + ["batched_q1_riemann", "served_stream", "q1_vortex_periodic_sweep"])
    ap.add_argument("--requests", type=int, default=32, help="served workload: number of requests")
    ap.add_argument("--rate", type=float, default=20.0, help="served workload: arrivals per second")
    ap.add_argument("--n-max", type=int, default=48, help="served workload: largest N")
    ap.add_argument("--t-cap", type=float, default=None, help="served workload: cap on the end times")
    ap.add_argument("--skip-one-at-a-time", action="store_true", help="served workload: no one-at-a-time run")
    ap.add_argument("--no-batched", action="store_true", help="main line: skip the batched sample")
    ap.add_argument("--no-developed", action="store_true",
                    help="main line: skip the step cost of a developed flow (Q2 256^2 at t = 0.05)")
    ap.add_argument("--no-served", action="store_true", help="main line: skip the served sample")
    ap.add_argument("--cpu-c3-steps", type=int, default=3,
                    help="main line: SSP-RK3 steps of the all-core oracle on the full mesh (0: none)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch schedule")
    ap.add_argument("--instances", type=int, default=512, help="batched workload: number of instances")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-steps", type=int, default=8)
    ap.add_argument("--fp64-rates", action="store_true", help="print the measured arithmetic rates and exit")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="arithmetic of the sweep (mixed: GDG_PRECISION_MIXED, reported separately)")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the separately reported mixed-precision measurement of the fp64 run")
    args = ap.parse_args()
    if args.fp64_rates:
        import torch

        from paper_2402_04514_gb300.gdg import fp64_throughput

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps({"fp64_rates_ops_per_s": fp64_throughput()}))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched_q1_riemann":
        return run_batched(args)
    if args.workload == "served_stream":
        return run_served(args)
    if args.workload == "q1_vortex_periodic_sweep":
        return run_vortex_sweep(args)

    import numpy as np
    import torch

    from paper_2402_04514_gb300 import costmodel
    from paper_2402_04514_gb300.gdg import Solver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    spec = WORKLOADS[args.workload]
    P, U0 = make_problem(spec)
    counts = costmodel.Counts.of(P)
    n = P.n
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    def measure(mixed, with_e2e):
        """Times args.steps fused SSP-RK3 steps of one instance (after warm-up and autotuning) and, with
        with_e2e, the same through host buffers; returns the pieces of the JSON line."""
        solver = Solver(P, params=dict(precision=1 if mixed else 0))
        solver.set_clock(0.0, float("inf"), 0.5)
        stream = torch.cuda.current_stream()
        U = torch.from_numpy(U0).cuda()
        work = (torch.empty_like(U), torch.empty_like(U))

        def step():
            solver.step(U, work)  # gdg_ssprk3_step: tau chosen on the device, U updated in place

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        assert solver.status() == 0, "inadmissible state or CFL violation during warm-up"
        schedule = solver.schedule() if args.no_autotune else solver.autotune(U, work, trials=2)  # state restored

        sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
            time.sleep(0.3)
        solver.profile(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop() if sampler else None
        ms = ev0.elapsed_time(ev1)
        prof = solver.profile_read()
        solver.profile(False)
        flags = solver.status()
        ms_max = max_over_ranks(ms, dist, "cuda")
        value = whole_job_rate(world, n * 3 * args.steps, ms_max)
        launches = sum(c for _, c in prof.values())

        # roofline of the dominant kernel (its own launches' CUDA-event times inside the timed region)
        top = max(prof, key=lambda k: prof[k][0])
        top_ms, top_cnt = prof[top]
        avg_s = top_ms / top_cnt / 1e3
        fl = costmodel.flops_per_launch(counts)[top]
        by = costmodel.bytes_per_launch(counts)[top]
        # DRAM bytes per launch of the top kernel from the committed ncu table, scaled to this mesh by its
        # node count; None when the table was taken from other library sources than the ones built here
        traffic = costmodel.measured_traffic(
            os.path.join(ROOT, "profiles", "dram_traffic_q2_512_four_quadrant.txt"), top, n,
            "mixed" if mixed else "fp64")
        alu = {"bound": "alu", "kernel": f"k_{top}", "achieved": fl / avg_s / 1e12,
               "peak": costmodel.ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": fl / avg_s / 1e12 / costmodel.ALU_PEAK_TFLOPS, "traffic": traffic,
               "peak_source": "unit counts and clock (2.07 GHz, 152 SMs): FP64 pipe 2 DFMA/clk/SM x 2 flop "
                              f"({costmodel.FP64_PEAK_TFLOPS:.3f}) + integer-pipe binary64 products, 64 ALU lanes/clk/SM / "
                              f"{costmodel.INT_MUL_ALU_INST} ALU instructions per product ({costmodel.INT_MUL_PEAK_TFLOPS:.3f})",
               "fp64_pipe_peak": costmodel.FP64_PEAK_TFLOPS, "alg_flops_per_launch": fl}
        hbm = {"bound": "hbm", "kernel": f"k_{top}", "achieved": by / avg_s / 1e9, "peak": hbm_peak,
               "unit": "GB/s", "frac": by / avg_s / 1e9 / hbm_peak, "alg_bytes_per_launch": by,
               "traffic": traffic, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
        kernels = {k: {"ms_total": v[0], "launches": v[1],
                       "share": v[0] / max(1e-9, sum(x[0] for x in prof.values()))}
                   for k, v in prof.items() if v[1]}

        # end to end through the public API with host buffers (gdg_ssprk3_step_host): every step reads its
        # input from page-locked host memory and writes its result back there, and the host waits for it
        e2e = None
        if with_e2e:
            hin = torch.empty(U.shape, dtype=torch.float64, pin_memory=True)
            hin.copy_(U)
            hout = torch.empty_like(hin, pin_memory=True)
            for _ in range(2):  # untimed: the first transfers through freshly pinned buffers run slower
                solver.step_host(hin, hout, U, work)
                stream.synchronize()
                hin, hout = hout, hin
            torch.cuda.synchronize()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                solver.step_host(hin, hout, U, work)
                stream.synchronize()
                hin, hout = hout, hin
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            ems = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
            e2e = {"value": whole_job_rate(world, n * 3 * args.steps, ems), "unit": METRIC,
                   "h2d_bytes_per_step": int(U.numel() * 8), "d2h_bytes_per_step": int(U.numel() * 8),
                   "api": "gdg_ssprk3_step_host", "ms_per_step": ems / args.steps}
        solver.close()
        # the mixed path is not bound by the FP64 pipe: its roofline is the HBM one
        roofline, other = (hbm, alu) if mixed else (alu, hbm)
        return {"value": value, "ms_per_step": ms_max / args.steps, "schedule": schedule, "roofline": roofline,
                "other": other, "kernels": kernels, "e2e": e2e, "launches": launches, "clocks": clocks,
                "flags": flags}

    main_mixed = args.precision == "mixed"
    res = measure(main_mixed, not args.no_e2e)
    mixed_res = None
    if not main_mixed and not args.no_mixed:
        mixed_res = measure(True, False)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    # the batched and served workloads, measured on samples sized to end in about a minute each (their own
    # --workload runs take any size)
    batched = served = developed = None
    if world == 1 and not args.no_developed:
        developed = measure_developed()
    if world == 1 and not args.no_batched:
        batched = measure_batched(COMBINED_BATCH_INSTANCES, steps=3, warmup=1)
    if world == 1 and not args.no_served:
        served = measure_served(**COMBINED_SERVED)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v1, secs1, n_s, _ = oracle_sample_rate(args.cpu_baseline_steps)
        v, secs, _, threads = oracle_sample_rate(args.cpu_baseline_steps, openmp=True)
        sample = f"Q2 {SAMPLE_N}x{SAMPLE_N} four-quadrant (seed 0, {n_s} DoFs), {args.cpu_baseline_steps} SSP-RK3 steps"
        cpu = {"value": v, "unit": METRIC, "cores": threads, "kind": "oracle",
               "sample": f"{sample}, {threads} threads (the oracle's row loops shared by OpenMP), {secs:.1f} s",
               "single_thread": {"value": v1, "unit": METRIC, "cores": 1,
                                 "sample": f"{sample}, single thread, {secs1:.1f} s"}}
        if args.cpu_c3_steps > 0:
            v3, secs3, threads3 = oracle_full_size_rate(P, np.ascontiguousarray(U0), args.cpu_c3_steps)
            cpu["full_size_extrapolated"] = {
                "value": v3, "unit": METRIC, "cores": threads3,
                "sample": (f"the full {args.workload} mesh ({n} DoFs), {args.cpu_c3_steps} SSP-RK3 steps "
                           f"({3 * args.cpu_c3_steps} stages) from the initial data, {threads3} threads, "
                           f"{secs3:.1f} s; the per-stage rate extrapolates to the workload's 200 steps")}
    line = {"metric": METRIC, "value": res["value"], "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64 mixed" if main_mixed else "f64",
            "data": "synthetic",
            "config": {**config_block(args, n), "precision": args.precision, "schedule": res["schedule"]},
            "roofline": res["roofline"], "roofline_hbm" if not main_mixed else "roofline_alu": res["other"],
            "cpu_baseline": cpu, "e2e": res["e2e"], "gpu_launches": res["launches"] * world,
            "clocks": res["clocks"], "kernels": res["kernels"], "status_flags": res["flags"]}
    if developed is not None:
        line["developed_flow"] = developed
    if batched is not None:
        line["batched"] = batched
    if served is not None:
        line["served"] = served
    if mixed_res is not None:
        # the mixed-precision path (GDG_PRECISION_MIXED) on the same workload, reported on its own: its
        # results differ from the FP64 path's by up to ~1e-5 of max |U| per stage
        line["mixed_precision"] = {
            "value": mixed_res["value"], "unit": METRIC, "ms_per_step": mixed_res["ms_per_step"],
            "dtype": "f32/f64 mixed", "schedule": mixed_res["schedule"], "roofline": mixed_res["roofline"],
            "kernels": mixed_res["kernels"], "gpu_launches": mixed_res["launches"] * world,
            "clocks": mixed_res["clocks"], "status_flags": mixed_res["flags"]}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
