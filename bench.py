"""Benchmark of the HDD likelihood path on GB300 (one JSON line on stdout).

Default workload: 513 x 513 grid (261,121 unknowns), 256 samples per step,
40 KL terms (correlation length 0.1, variance 2), 16 x 16 observations, leaves of
4 x 4 cells.  One step = assemble + upsweep + pruned point solve + log-likelihood
for the whole batch, inputs resident in HBM.  The step's working set (tens of GB
of fronts and factors) is far larger than the 129 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Under torchrun (N > 1) every rank evaluates its own batch on its own GPU
(replicas: the samples are independent; no data-path collective); value is the
total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workload as w  # noqa: E402

METRIC = "log-likelihood evals/s at 513^2 grid"
# FP64 FMA throughput of GB300: 2 FP64 FMA per clock per SM (1.25 TFLOP/s nominal
# at 2070 MHz over 152 SMs), i.e. 152 * 2 * 2 * 2.07e9 flop/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 SIMT: 128 FMA per clock per SM.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


MEASURED = _measured_peaks()

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of a stage's kernels, summed over
# the launches of one evaluation of a 16-sample run of the same workload and divided by 16
# (taken on the kernel versions of this tree; a stage whose kernels change gets null).
MEASURED_TRAFFIC = {
    "large_fronts": {"workload": "grid513", "leaf": 4, "precision": "mixed", "bytes_per_sample": 4.3483e9 / 16,
                     "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_front_fill, k_potrf*, "
                               "k_trsm*, k_chol_trsm, k_syrk_tc, k_syrk_rhs over one 16-sample evaluation"},
}


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._thr = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._thr = threading.Thread(target=self._run, daemon=True)
        self._thr.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._thr:
            self._thr.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for n, v in zip(names, s[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "n_samples": len(self.samples)}


def cpu_baseline(cfg, prob, n_samples, processes):
    """The oracle (FP64 P1 FEM + banded Cholesky) on host cores, spawn pool, 1 BLAS thread each."""
    from oracle import fem
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        t0 = time.perf_counter()
        fem.evaluate_batch(cfg.N, prob.phi, prob.Z[:n_samples], prob.obs, prob.y, cfg.sigma, cfg.f,
                           processes=processes)
        dt = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return n_samples / dt, dt


def aggregate(total_ms: float, batch: int, steps: int, dist=None, device="cpu"):
    """Replica timing: the slowest rank's time and the whole-job rate (all ranks'
    samples / that time).  The samples of different ranks are independent, so the
    only collective is this reduction of the elapsed time."""
    world = dist.get_world_size() if dist is not None else 1
    if dist is not None:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * batch * steps / (total_ms / 1e3)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, cfg):
    """--impl reference: the FP64 CPU oracle timed on the host cores."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    P = host_cores()
    per_step = P
    prob = w.make_problem(cfg, batch=max(per_step, cfg.batch))
    for _ in range(args.warmup):
        cpu_baseline(cfg, prob, per_step, P)
    times = []
    for _ in range(args.steps):
        _, dt = cpu_baseline(cfg, prob, per_step, P)
        times.append(dt)
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{cfg.name}: {cfg.N}x{cfg.N} grid, {per_step} samples per step (of {cfg.batch}),"
                               f" n_z {cfg.n_z}, {cfg.obs_side ** 2} observations", "batch": per_step},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": P, "kind": "oracle",
                         "sample": f"{per_step} samples per step, one per process"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# Uneven batch (many grids in one batch): samples over four grids, 40/30/20/10 %
# by count, n_Z uniform in {10, 20, 40}, per plan an m x m observation lattice with m
# uniform in 4..32 (16 to 1024 points); KL field with correlation length 0.2, variance 1.
UNEVEN_MIX = ((129, 0.4), (257, 0.3), (513, 0.2), (1025, 0.1))


def uneven_groups(total: int):
    """The plans of the uneven batch: one per (grid, n_Z) with its sample count and lattice."""
    rng = np.random.default_rng(np.random.SeedSequence(w.ROOT_SEED).spawn(4)[3])
    counts = [int(round(total * f)) for _, f in UNEVEN_MIX]
    counts[-1] = total - sum(counts[:-1])
    groups = []
    for (N, _), cnt in zip(UNEVEN_MIX, counts):
        nz = rng.choice([10, 20, 40], size=cnt)
        for z in (10, 20, 40):
            k = int((nz == z).sum())
            if k:
                groups.append({"N": N, "n_z": z, "count": k, "m": int(rng.integers(4, 33))})
    return groups, rng


def run_uneven(args, hdd, torch, dev, stream, local):
    """The uneven batch through hdd_multi_* (one launch per tree height and front class over
    all plans) against the same samples evaluated plan by plan, leaves and refinement steps
    from the autotuner's table."""
    from paper_1708_02207_gb300 import autotune
    prec_name = args.precision
    prec = hdd.HDD_MIXED_FP32 if prec_name == "mixed" else hdd.HDD_FP64
    groups, rng = uneven_groups(args.uneven_samples)
    grids = sorted({g["N"] for g in groups})
    tuned = {N: autotune.choose(N, prec_name) for N in grids}
    phis = {N: w.kl_basis(N, 40, 0.2, 1.0) for N in grids}
    plans = []
    for g in groups:
        t = tuned[g["N"]]
        phi = np.ascontiguousarray(phis[g["N"]][:, :g["n_z"]])
        plans.append(hdd.Plan(g["N"], t["leaf"], phi, w.obs_vertices(g["N"], g["m"]), 0.01, precision=prec,
                              ir_max_iter=t["ir_max_iter"], ir_tol=args.ir_tol, device=local))
    free = torch.cuda.mem_get_info(dev)[0]
    chunks = 1
    while sum(p.workspace_size(-(-g["count"] // chunks)) for p, g in zip(plans, groups)) > 0.6 * free:
        chunks += 1
    batches = [-(-g["count"] // chunks) for g in groups]
    mp = hdd.MultiPlan(plans, batches)
    Zs = [[torch.from_numpy(rng.standard_normal((b, g["n_z"]))).to(dev) for b, g in zip(batches, groups)]
          for _ in range(chunks)]
    ys = [torch.from_numpy(0.01 * rng.standard_normal(p.n_obs)).to(dev) for p in plans]
    failed = 0

    def multi():
        nonlocal failed
        for c in range(chunks):
            outs = mp.evaluate(Zs[c], ys, stream)
        failed = sum(int((o[2] != 0).sum().item()) for o in outs)

    def alone():
        for c in range(chunks):
            for q, p in enumerate(plans):
                p.evaluate(Zs[c][q], ys[q], ws=mp.ws[q], stream=stream)

    def timed(fn, steps):
        with torch.cuda.stream(stream):
            fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / steps

    t_multi = timed(multi, args.uneven_steps)
    t_alone = timed(alone, args.uneven_steps)
    # the same chunks as captured CUDA graphs (hdd_multi_capture), one replay per chunk
    graphs = [mp.capture(Zs[c], ys) for c in range(chunks)]

    def replay():
        for g in graphs:
            g.launch(stream)

    t_graph = timed(replay, args.uneven_steps)
    for g in graphs:
        g.close()
    evaluated = sum(batches) * chunks
    info = mp.info()
    out = {"samples": args.uneven_samples, "evaluated_per_step": evaluated, "plans": len(plans), "chunks": chunks,
           "grids": {str(N): sum(g["count"] for g in groups if g["N"] == N) for N in grids},
           "precision": prec_name, "tuned": {str(N): tuned[N] for N in grids},
           "ms_per_step": t_multi, "evals_per_s": args.uneven_samples / (t_multi / 1e3),
           "ms_per_step_plans_alone": t_alone, "evals_per_s_plans_alone": args.uneven_samples / (t_alone / 1e3),
           "ms_per_step_graph": t_graph, "evals_per_s_graph": args.uneven_samples / (t_graph / 1e3),
           "launches_per_chunk": info["launches_evaluate"],
           "launches_per_chunk_plans_alone": sum(p.info()["launches_evaluate"] for p in plans),
           "failed_samples": failed,
           "note": "one step = every sample once (chunks of per-plan batches that fit 60% of free HBM; "
                   "padded samples of the last chunk count as work, not as evaluations)"}
    del mp, Zs
    torch.cuda.empty_cache()
    return out


def run_policy(args, cfg, hdd, torch, dev, stream, local, prob, Z, y):
    """The precision split with FP64 Cholesky of the top two tree levels beside the
    benched all-FP32 factorisation: per setting the fewest refinement steps with no sample
    flagged HDD_ENOCONV at the tolerance, and its speed."""
    B = Z.shape[0]
    res = {}
    for top in (0, 2):
        for K in (1, 2, 3):
            plan = hdd.Plan(cfg.N, args.leaf or cfg.leaf, prob.phi, prob.obs, cfg.sigma, f=cfg.f,
                            precision=hdd.HDD_MIXED_FP32, ir_max_iter=K, ir_tol=args.ir_tol, fp64_top_levels=top,
                            device=local)
            ws = plan.workspace(B)
            with torch.cuda.stream(stream):
                ll, u, st = plan.evaluate(Z, y, ws=ws, stream=stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(2):
                    plan.evaluate(Z, y, ws=ws, stream=stream)
                e1.record(stream)
            stream.synchronize()
            bad = int((st != 0).sum().item())
            ms = e0.elapsed_time(e1) / 2
            del ws
            torch.cuda.empty_cache()
            if bad == 0 or K == 3:
                res[f"fp64_top_levels_{top}"] = {"ir_steps": K, "failed_samples": bad, "ms_per_step": ms,
                                                 "evals_per_s": B / (ms / 1e3)}
                break
    return res


def run_means_leg(args, cfg, hdd, torch, dev, stream, local, prob, Z):
    """Subdomain means as the observation operator (Sec. 5.1-5.2): the 256 cells of depth 8
    (32 x 32 cells each) of the same grid and samples."""
    B = Z.shape[0]
    probe = hdd.Plan(cfg.N, args.leaf or cfg.leaf, None, np.array([0], dtype=np.int32), cfg.sigma,
                     device=-1, obs_kind=hdd.HDD_OBS_MEANS)
    ids = probe.nodes_at_depth(8)
    plan = hdd.Plan(cfg.N, args.leaf or cfg.leaf, prob.phi, ids, cfg.sigma, f=cfg.f, precision=hdd.HDD_MIXED_FP32,
                    ir_max_iter=args.ir_iters, ir_tol=args.ir_tol, device=local, obs_kind=hdd.HDD_OBS_MEANS)
    ws = plan.workspace(B)
    yv = torch.zeros(ids.size, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        ll, m, st = plan.evaluate(Z, yv, ws=ws, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            plan.evaluate(Z, yv, ws=ws, stream=stream)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / 2
    out = {"observed_nodes": int(ids.size), "depth": 8, "ms_per_step": ms, "evals_per_s": B / (ms / 1e3),
           "failed_samples": int((st != 0).sum().item()), "visited_nodes": plan.info()["n_visited"],
           "launches_per_evaluation": plan.info()["launches_evaluate"]}
    del ws
    torch.cuda.empty_cache()
    return out


def run_serving(args, hdd, torch, dev, local):
    """The serving workload: 64 random-walk Metropolis chains (step 0.1, n_Z 40) spread over the
    grids, each with one request in flight, Poisson arrivals at offered loads that are
    fractions of the measured saturation rate; continuous batching admitted by workspace
    bytes (paper_1708_02207_gb300.serving).  Per load point: offered rate, throughput and
    per-request p50/p99 latency."""
    from paper_1708_02207_gb300 import autotune, serving
    rng = np.random.default_rng(np.random.SeedSequence(w.ROOT_SEED).spawn(5)[4])
    grids = args.serve_grids
    out = {"chains": 64, "grids": grids, "step": 0.1, "n_z": 40, "points": {}}
    for prec_name in args.serve_precisions:
        prec = hdd.HDD_MIXED_FP32 if prec_name == "mixed" else hdd.HDD_FP64
        plans, ydata = {}, {}
        for N in grids:
            t = autotune.choose(N, prec_name)
            obs = w.obs_vertices(N, 16)
            # the chains wander into fields of higher contrast than the prior samples the
            # tuner saw, where the tuned minimum of refinement steps leaves requests above the
            # tolerance (flagged HDD_ENOCONV): serving plans take one step more
            K = t["ir_max_iter"] + (1 if prec_name == "mixed" else 0)
            phi = w.kl_basis(N, 40, 0.1, 2.0)
            plans[str(N)] = hdd.Plan(N, t["leaf"], phi, obs, 0.01, precision=prec,
                                     ir_max_iter=K, ir_tol=args.ir_tol, device=local)
            ydata[str(N)] = 0.05 + 0.01 * rng.standard_normal(obs.size)
            if prec_name == "mixed":
                # a request that still does not converge is answered by an FP64 plan
                t64 = autotune.choose(N, "fp64")
                plans[f"{N}-fp64"] = hdd.Plan(N, t64["leaf"], phi, obs, 0.01, precision=hdd.HDD_FP64,
                                              ir_max_iter=0, device=local)
        fallback = {str(N): f"{N}-fp64" for N in grids} if prec_name == "mixed" else None
        budget = int(min(80e9, 0.5 * torch.cuda.mem_get_info(dev)[0]))
        backend = serving.CudaBackend(plans, n_slots=4, device=local)
        server = serving.Server(backend, budget_bytes=budget, max_batch=64, n_slots=4, fallback=fallback)
        chains = [serving.MetropolisChain(str(grids[k % len(grids)]), rng.standard_normal(40),
                                          ydata[str(grids[k % len(grids)])], 0.1, rng) for k in range(64)]
        n_req = args.serve_requests if prec_name == "mixed" else max(1, args.serve_requests // 5)
        serving.run_offered_load(server, chains, float("inf"), min(n_req, 256), rng)   # warm-up
        sat = serving.run_offered_load(server, chains, float("inf"), n_req, rng)
        pts = [{"load": "saturation", "offered_per_s": None, "evals_per_s": sat["evals_per_s"],
                "p50_ms": 1e3 * sat["p50_s"], "p99_ms": 1e3 * sat["p99_s"], "requests": sat["requests"]}]
        for f in args.serve_loads:
            r = serving.run_offered_load(server, chains, f * sat["evals_per_s"], n_req, rng)
            pts.append({"load": f, "offered_per_s": f * sat["evals_per_s"], "evals_per_s": r["evals_per_s"],
                        "p50_ms": 1e3 * r["p50_s"], "p99_ms": 1e3 * r["p99_s"], "requests": r["requests"]})
        fails = {}
        for r in server.done:
            if r.status != 0 or r.rejected:
                key = f"{r.plan}:" + ("rejected" if r.rejected else str(-(r.status & 0xFF)))
                fails[key] = fails.get(key, 0) + 1
        out["points"][prec_name] = {"budget_bytes": budget, "peak_admitted_bytes": server.peak_bytes,
                                    "batches": server.batches, "requests_per_point": n_req, "sweep": pts,
                                    "requests": len(server.done),
                                    "escalated_to_fp64": server.escalated,
                                    "failed": sum(fails.values()), "failed_by_grid_and_status": fails}
        del server, backend, plans
        torch.cuda.empty_cache()
    return out


def run_hdd(args, cfg):
    import torch
    from paper_1708_02207_gb300 import build as hdd_build, hdd

    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        hdd_build.build()
    if dist:
        dist.barrier()

    B = args.batch or cfg.batch
    prob = w.make_problem(cfg, batch=B)
    precision = hdd.HDD_MIXED_FP32 if args.precision == "mixed" else hdd.HDD_FP64
    plan = hdd.Plan(cfg.N, args.leaf or cfg.leaf, prob.phi, prob.obs, cfg.sigma, f=cfg.f, precision=precision,
                    ir_max_iter=args.ir_iters, ir_tol=args.ir_tol, device=local)
    if args.sweep_fusion is not None:
        plan.set_sweep_fusion(args.sweep_fusion)
    info = plan.info()
    ws = plan.workspace(B)
    Z = torch.from_numpy(prob.Z).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    u_obs = torch.empty(B, plan.n_obs, dtype=torch.float64, device=dev)
    ll = torch.empty(B, dtype=torch.float64, device=dev)
    st_t = torch.empty(B, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    stages = ("assemble", "upsweep", "point_solve", "loglik")

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        plan.assemble(Z, ws, stream)
        if evs is not None:
            evs[1].record(stream)
        plan.upsweep(B, ws, stream)
        if evs is not None:
            evs[2].record(stream)
        plan.point_solve(B, ws, u_obs, stream)
        if evs is not None:
            evs[3].record(stream)
        plan.loglik(B, ws, u_obs, y, ll, st_t, stream)
        if evs is not None:
            evs[4].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    bad = int((st_t != 0).sum().item())

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # the headline: K steps with no per-kernel events (only one event per stage boundary)
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            t_start.record(stream)
            for k in range(args.steps):
                step(evs[k])
            t_end.record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms, value = aggregate(t_start.elapsed_time(t_end), B, args.steps, dist, dev)
    # a second pass of the same K steps with a CUDA event pair around every launch
    # (hdd_profile_begin), for the per-kernel-family times and rooflines
    plan.profile_begin()
    with torch.cuda.stream(stream):
        p_start = torch.cuda.Event(enable_timing=True)
        p_end = torch.cuda.Event(enable_timing=True)
        p_start.record(stream)
        for k in range(args.steps):
            step()
        p_end.record(stream)
    stream.synchronize()
    kstats = plan.profile_end()
    profiled_ms = p_start.elapsed_time(p_end) / args.steps
    stage_ms = {s: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i, s in enumerate(stages)}
    step_ms = sorted(e[0].elapsed_time(e[4]) for e in evs)

    def pct(q):
        return step_ms[min(len(step_ms) - 1, int(round(q * (len(step_ms) - 1))))]


    # end to end through the C ABI with host buffers (pinned), copies inside
    Zh = torch.from_numpy(prob.Z).pin_memory()
    yh = torch.from_numpy(prob.y).pin_memory()
    llh = torch.empty(B, dtype=torch.float64).pin_memory()
    uh = torch.empty(B, plan.n_obs, dtype=torch.float64).pin_memory()
    sh = torch.empty(B, dtype=torch.int32).pin_memory()

    def e2e_call():
        plan.evaluate_host_ptrs(B, ws, Zh.data_ptr(), yh.data_ptr(), 0, llh.data_ptr(), uh.data_ptr(),
                                sh.data_ptr(), stream)

    for _ in range(max(1, min(args.warmup, 2))):
        e2e_call()
    e2e_steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_call()
    e2e_s = time.perf_counter() - t0
    e2e_value = world * B * e2e_steps / e2e_s
    h2d = B * plan.n_z * 8 + plan.n_obs * 8
    d2h = B * 8 + B * plan.n_obs * 8 + B * 4

    # per-kernel-family times and algorithmic flops over the timed region
    kernels = {}
    for name, st_ in kstats.items():
        ms = st_["ms"] / args.steps
        kernels[name] = {"ms_per_step": ms, "launches_per_step": st_["launches"] / args.steps,
                         "share": st_["ms"] / max(1e-9, sum(v["ms"] for v in kstats.values())),
                         "tflops": (st_["flops"] / args.steps) / (ms / 1e3) / 1e12 if st_["flops"] > 0 and ms > 0 else None}
    # Rooflines per kernel family and stage: t_roof = max(flops / compute peak, algorithmic
    # bytes / HBM bandwidth) and frac = t_roof / measured time.  Algorithmic bytes come from the
    # plan (each input read once, each output written once); flops from the profiler.
    hbm = MEASURED.get("hbm_gbs", 6756.5)
    tf32_peak = MEASURED.get("bf16_tflops", 1899.9) * 1.1 / 2.25
    if precision == hdd.HDD_FP64:
        simt_peak, simt_src = FP64_PEAK_TFLOPS, "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz"
    else:
        simt_peak, simt_src = FP32_PEAK_TFLOPS, "derived: 128 FP32 FMA/clk/SM x 152 SMs x 2070 MHz"
    K = args.ir_iters if precision != hdd.HDD_FP64 else 0
    n_desc_all, n_desc_vis, n_fwd, n_res = (K, 1, K, K) if K > 0 else (0, 1, 0, 0)
    stage_bytes = {   # per step
        "kappa": info["bytes_assemble"] * B + info["bytes_kl_basis"],
        "leaf_front": info["bytes_upsweep_leaf"] * B,
        "front_warp": info["bytes_upsweep_tiny"] * B,
        "front_small": info["bytes_upsweep_small"] * B,
        "large_fronts": info["bytes_upsweep_large"] * B,
        "subtree": info["bytes_upsweep_fused"] * B,
        "forward": n_fwd * info["bytes_forward"] * B,
        "descent": (n_desc_all * info["bytes_descent_all"] + n_desc_vis * info["bytes_descent_visited"]) * B,
        "residual": n_res * info["bytes_residual"] * B,
    }
    groups = {"large_fronts": ("front_fill", "potrf", "chol_trsm", "trsm", "syrk_simt", "syrk_tc", "syrk_rhs")}

    def fam_roof(name, members):
        ms = sum(kernels[m]["ms_per_step"] for m in members if m in kernels)
        if ms <= 0:
            return None
        t_alu = 0.0
        for m in members:
            fl = kstats.get(m, {}).get("flops", 0.0) / args.steps
            pk = tf32_peak / 3.0 if m == "syrk_tc" else simt_peak   # 3xTF32: 3 tensor products per FMA
            t_alu += fl / (pk * 1e12) * 1e3
        by = stage_bytes.get(name, 0.0)
        t_hbm = by / (hbm * 1e9) * 1e3
        bound = "hbm" if t_hbm >= t_alu else "alu"
        return {"ms_per_step": ms, "bytes_per_step": by, "gbs": by / (ms / 1e3) / 1e9,
                "t_roof_ms": max(t_hbm, t_alu), "bound": bound, "frac": max(t_hbm, t_alu) / ms}

    stages_roof = {}
    for name in ("kappa", "leaf_front", "front_warp", "front_small", "large_fronts", "subtree", "forward", "descent",
                 "residual"):
        r = fam_roof(name, groups.get(name, (name,)))
        if r:
            stages_roof[name] = r
    # the stage with the largest device time (a kernel family, or the group of kernels
    # that runs the large fronts) carries the headline roofline
    roof = None
    if stages_roof:
        dom = max(stages_roof, key=lambda k: stages_roof[k]["ms_per_step"])
        r = stages_roof[dom]
        if r["bound"] == "hbm":
            # DRAM bytes per step from ncu (profiles/), per sample; only for the family and
            # kernel version the counters were taken on
            tr = MEASURED_TRAFFIC.get(dom)
            same = tr and cfg.name == tr["workload"] and (args.leaf or cfg.leaf) == tr["leaf"] \
                and args.precision == tr["precision"]
            traffic = tr["bytes_per_sample"] * B if same else None
            roof = {"bound": "hbm", "achieved": r["gbs"], "peak": hbm, "unit": "GB/s", "frac": r["gbs"] / hbm,
                    "traffic": traffic, "traffic_unit": "bytes per step (all launches of the stage's kernels)",
                    "traffic_source": tr["source"] if traffic else None, "kernel": dom,
                    "kernels": list(groups.get(dom, (dom,))), "ms_per_step": r["ms_per_step"],
                    "peak_source": "of measured: MEASURED_PEAKS hbm_gbs (copy bandwidth)",
                    "algorithmic_bytes_per_step": r["bytes_per_step"],
                    "bytes_note": "per front and sample: sons' lower Schur triangles (leaves: kappa) read once; "
                                  "factor columns, y_g and the lower Schur triangle written once"}
        else:
            ach = sum(kstats.get(m_, {}).get("flops", 0.0) for m_ in groups.get(dom, (dom,))) / args.steps \
                / (r["ms_per_step"] / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": simt_peak, "unit": "TFLOP/s", "frac": r["frac"],
                    "traffic": None, "kernel": dom, "kernels": list(groups.get(dom, (dom,))),
                    "ms_per_step": r["ms_per_step"], "peak_source": simt_src}
    tc = kernels.get("syrk_tc")
    if tc and tc["tflops"]:
        # 3xTF32: three tensor-core products per FP32 multiply-add; TF32 peak = measured BF16
        # burst x the nominal TF32/BF16 ratio (1.1 / 2.25)
        ach_tc = 3.0 * tc["tflops"]
        kernels["syrk_tc"]["roofline"] = {"bound": "tensor", "achieved": ach_tc, "peak": tf32_peak,
                                          "unit": "TFLOP/s (TF32 tensor ops, 3 per FP32 FMA)",
                                          "frac": ach_tc / tf32_peak,
                                          "peak_source": "of measured: MEASURED_PEAKS bf16_tflops x 1.1/2.25"}
    up_flops = info["flops_upsweep"] * B
    upsweep_roof = {"achieved": up_flops / (stage_ms["upsweep"] / 1e3) / 1e12, "unit": "TFLOP/s",
                    "note": "whole hdd_upsweep call"}

    # many loads at a fixed coefficient field (hdd_solve_loads on the factors of one upsweep)
    # and the subdomain means of the result; timed after the headline step, not part of it
    loads = None
    if args.loads > 0:
        NN = cfg.N * cfg.N
        gen = torch.Generator(device=dev)
        gen.manual_seed(1708_02207)
        c_l = torch.rand(B, args.loads, NN, dtype=torch.float64, device=dev, generator=gen) / (cfg.N - 1) ** 2
        u_l = torch.empty_like(c_l)
        s_l = torch.empty(B, dtype=torch.int32, device=dev)
        means = torch.empty(B, info["n_nodes"], dtype=torch.float64, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ws_l = ws
        with torch.cuda.stream(stream):
            plan.assemble(Z, ws, stream)
            plan.upsweep(B, ws, stream)
            for _ in range(args.warmup):
                plan.solve_loads(B, ws, c_l, u_l, s_l, stream)
                plan.subdomain_means(u_l[:, 0, :], means, stream)
            ev[0].record(stream)
            for _ in range(args.steps):
                plan.solve_loads(B, ws, c_l, u_l, s_l, stream)
            ev[1].record(stream)
            for _ in range(args.steps):
                plan.subdomain_means(u_l[:, 0, :], means, stream)
            ev[2].record(stream)
        stream.synchronize()
        # slowest rank (replicas: the same reduction as the headline)
        t_l = aggregate(ev[0].elapsed_time(ev[1]), 1, 1, dist, dev)[0] / args.steps
        t_m = aggregate(ev[1].elapsed_time(ev[2]), 1, 1, dist, dev)[0] / args.steps
        v8 = 8.0 * NN   # one FP64 vertex vector
        # per load and sample: zero u; (1 + K) sweeps and full descents; K residuals (kappa, u
        # and c in, r out), updates (u, du in, u out) and correction maxima (du in; u at the last)
        by_load = v8 + (1 + K) * (info["bytes_forward"] + info["bytes_descent_all"]) \
            + K * (info["bytes_residual"] + v8) + K * 3 * v8 + (K * v8 + v8 if K else 0.0)
        by_l = by_load * B * args.loads
        by_m = (v8 + 8.0 * info["n_nodes"]) * B
        # four loads per sample: hdd_solve_loads (one load per sweep) against hdd_solve_data
        # (four right-hand sides per factor read), with Dirichlet data, and with coarse-grid loads
        data = None
        if args.data:
            c4 = torch.rand(B, 4, NN, dtype=torch.float64, device=dev, generator=gen) / (cfg.N - 1) ** 2
            g4 = torch.rand(B, 4, NN, dtype=torch.float64, device=dev, generator=gen)
            NH = (cfg.N + 1) // 2
            f4 = torch.rand(B, 4, NH * NH, dtype=torch.float64, device=dev, generator=gen)
            u4 = torch.empty_like(c4)
            scratch = torch.empty(plan.data_scratch_size(B), dtype=torch.uint8, device=dev)
            runs = {"solve_loads": lambda: plan.solve_loads(B, ws_l, c4, u4, s_l, stream),
                    "solve_data": lambda: plan.solve_data(B, ws_l, u4, c=c4, g=g4, status=s_l, scratch=scratch,
                                                          stream=stream),
                    "solve_data_coarse": lambda: plan.solve_data(B, ws_l, u4, f_coarse=f4, g=g4, status=s_l,
                                                                 scratch=scratch, stream=stream)}
            data = {"loads_per_sample": 4}
            for name, fn in runs.items():
                with torch.cuda.stream(stream):
                    fn()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(args.steps):
                        fn()
                    e1.record(stream)
                stream.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                # samples flagged by this call alone: a fresh upsweep clears the status words
                with torch.cuda.stream(stream):
                    plan.assemble(Z, ws_l, stream)
                    plan.upsweep(B, ws_l, stream)
                    fn()
                stream.synchronize()
                data[name] = {"ms_per_call": ms, "load_solves_per_s": 4 * B / (ms / 1e3),
                              "flagged_samples": int((s_l != 0).sum().item())}
            data["speedup_of_grouped_sweeps"] = data["solve_loads"]["ms_per_call"] / data["solve_data"]["ms_per_call"]
            del c4, g4, f4, u4, scratch
        loads = {"loads_per_sample": args.loads, "ms_per_call": t_l, "four_loads_with_data": data,
                 "load_solves_per_s": world * B * args.loads / (t_l / 1e3),
                 "failed_samples": int((s_l != 0).sum().item()),
                 "roofline": {"bound": "hbm", "achieved": by_l / (t_l / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                              "frac": by_l / (t_l / 1e3) / 1e9 / hbm, "algorithmic_bytes_per_call": by_l},
                 "subdomain_means": {"ms_per_call": t_m, "nodes": info["n_nodes"],
                                     "achieved_gbs": by_m / (t_m / 1e3) / 1e9,
                                     "frac": by_m / (t_m / 1e3) / 1e9 / hbm}}
        del c_l, u_l
        torch.cuda.empty_cache()

    # legs beside the headline (each after the headline's workspace is released)
    del ws
    torch.cuda.empty_cache()
    policy = means_leg = uneven = serve = None
    if precision != hdd.HDD_FP64 and args.policy:
        policy = run_policy(args, cfg, hdd, torch, dev, stream, local, prob, Z, y)
    if precision != hdd.HDD_FP64 and args.means and cfg.N >= 257:
        means_leg = run_means_leg(args, cfg, hdd, torch, dev, stream, local, prob, Z)
    if args.uneven_samples > 0:
        uneven = run_uneven(args, hdd, torch, dev, stream, local)
    if args.serve_requests > 0:
        serve = run_serving(args, hdd, torch, dev, local)

    # the plain FP64 path on the same inputs (the speedup of the mixed path is over it)
    fp64 = None
    if precision != hdd.HDD_FP64 and args.fp64_steps > 0:
        plan64 = hdd.Plan(cfg.N, args.leaf or cfg.leaf, prob.phi, prob.obs, cfg.sigma, f=cfg.f,
                          precision=hdd.HDD_FP64, device=local)
        ws64 = plan64.workspace(B)
        u64 = torch.empty(B, plan.n_obs, dtype=torch.float64, device=dev)
        ll64 = torch.empty(B, dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            plan64.assemble(Z, ws64, stream)
            plan64.upsweep(B, ws64, stream)
            plan64.point_solve(B, ws64, u64, stream)
            plan64.loglik(B, ws64, u64, y, ll64, None, stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.fp64_steps):
                plan64.assemble(Z, ws64, stream)
                plan64.upsweep(B, ws64, stream)
                plan64.point_solve(B, ws64, u64, stream)
                plan64.loglik(B, ws64, u64, y, ll64, None, stream)
            e1.record(stream)
        stream.synchronize()
        t64 = e0.elapsed_time(e1) / args.fp64_steps
        rel = ((u_obs - u64).abs().max(dim=1).values / u64.abs().max(dim=1).values).max().item()
        fp64 = {"value": world * B / (t64 / 1e3), "unit": "evals/s", "ms_per_step": t64,
                "speedup_of_mixed": (world * B / (t64 / 1e3)) and value / (world * B / (t64 / 1e3)),
                "max_rel_diff_u_obs_mixed_vs_fp64": rel, "steps": args.fp64_steps}
        del ws64
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        P = min(host_cores(), B)
        v, dt = cpu_baseline(cfg, prob, P, P)
        cpu = {"value": v, "unit": "evals/s", "cores": P, "kind": "oracle",
               "sample": f"{P} of the {B} samples, one per process ({dt:.1f} s)"}

    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if precision == hdd.HDD_FP64 else "f32+f64",
        "data": "synthetic",
        "config": {"workload": f"{cfg.name}: {cfg.N}x{cfg.N} grid ({(cfg.N - 2) ** 2} unknowns), {B} samples/step,"
                               f" n_z {cfg.n_z}, corr {cfg.corr_len}, var {cfg.variance},"
                               f" {cfg.obs_side ** 2} observations, leaf {args.leaf or cfg.leaf}",
                   "batch": B, "precision": args.precision, "parallelism": f"replicas x{world}",
                   "l2": "working set >> 129 MB L2 (no flush needed)"},
        "stage_ms": stage_ms, "failed_samples": bad,
        "batch_latency_ms": {"p50": pct(0.5), "p99": pct(0.99),
                             "note": "device time of one whole batch step; per-request latency is in 'serving'"},
        "profiled_ms_per_step": profiled_ms,
        "fp64_path": fp64,
        "precision_policy": policy,
        "subdomain_means": means_leg,
        "uneven": uneven,
        "serving": serve,
        "solve_loads": loads,
        "roofline": roof,
        "upsweep": upsweep_roof,
        "stages": stages_roof,
        "kernels": kernels,
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": info["launches_evaluate"] * args.steps,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "plan": {"flops_upsweep_per_sample": info["flops_upsweep"], "nodes": info["n_nodes"],
                 "visited": info["n_visited"], "workspace_gb": plan.workspace_size(B) / 1e9,
                 "sweep_fuse_height": info["sweep_fuse_height"]},
    }
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hdd", choices=["hdd", "reference"])
    ap.add_argument("--config", default="grid513", choices=sorted(w.CONFIGS))
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the plain FP64 path reported beside the mixed one (0: skip)")
    ap.add_argument("--leaf", type=int, default=0)
    ap.add_argument("--batch", type=int, default=0, help="samples per step (default: the workload's)")
    ap.add_argument("--ir-iters", type=int, default=2)
    ap.add_argument("--sweep-fusion", type=int, default=None,
                    help="largest height of the fused bottom subtrees of the full sweeps (0: level by level; "
                         "default: the plan's own choice)")
    ap.add_argument("--ir-tol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--policy", type=int, default=1, help="precision-policy leg (FP64 top levels; 0: skip)")
    ap.add_argument("--means", type=int, default=1, help="subdomain-means leg (0: skip)")
    ap.add_argument("--data", type=int, default=1, help="loads-with-data leg inside the loads leg (0: skip)")
    ap.add_argument("--uneven-samples", type=int, default=4096, help="samples of the uneven batch (0: skip)")
    ap.add_argument("--uneven-steps", type=int, default=2)
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="requests per load point of the serving leg (0: skip; FP64 takes a fifth)")
    ap.add_argument("--serve-grids", type=int, nargs="+", default=[513])
    ap.add_argument("--serve-precisions", nargs="+", default=["mixed"], choices=["mixed", "fp64"])
    ap.add_argument("--serve-loads", type=float, nargs="+", default=[0.25, 0.75, 1.25])
    ap.add_argument("--loads", type=int, default=1,
                    help="load vectors per sample of the hdd_solve_loads measurement (0: skip)")
    args = ap.parse_args(argv)
    cfg = w.CONFIGS[args.config]
    if args.impl == "reference":
        return run_reference(args, cfg)
    return run_hdd(args, cfg)


if __name__ == "__main__":
    sys.exit(main())
