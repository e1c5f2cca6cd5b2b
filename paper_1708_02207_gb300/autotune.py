"""Autotuner of the plan parameters that trade speed against nothing but speed: for each
grid size N and precision it picks the leaf size (the cells per side of the subdomains
eliminated directly, the paper's leaves generalised from single triangles) and, for mixed
plans, the number of refinement steps.

For every candidate leaf in {4, 8, 16} the tuner times one batch evaluation through the C
ABI (CUDA events, after warm-up).  Mixed plans take, per leaf, the fewest refinement steps
K in {1, 2, 3} for which no sample of the batch is flagged HDD_ENOCONV at the tolerance
(wider leaves factorise larger blocks in FP32 and may need a step more), so a choice never
buys speed with accuracy.  The fastest candidate wins.  The table is JSON keyed by
"<N>/<precision>" with the winner and every measured candidate; `choose` reads it and falls
back to leaf 4 with two refinement steps for grids it does not hold.

The front-kernel thresholds inside the library (fronts of up to 32 rows one per warp, up
to 128 FP32 / 160 FP64 rows in shared memory, larger ones on the global-memory and
tensor-core path) are fixed: they follow from register and shared-memory capacity and were
chosen by measurement.

  python -m paper_1708_02207_gb300.autotune --grids 129 257 513 1025 --out tuning.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
LEAVES = (4, 8, 16)
IR_STEPS = (1, 2, 3)
# samples per timed batch: enough to fill the GPU, small enough for any leaf's workspace
DEFAULT_BATCH = {129: 1024, 257: 512, 513: 256, 1025: 64}


def _key(N: int, precision: str) -> str:
    return f"{N}/{precision}"


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def choose(N: int, precision: str, table: dict | None = None) -> dict:
    """{"leaf", "ir_max_iter"} for a grid and precision ("mixed" or "fp64")."""
    t = load_table() if table is None else table
    e = t.get(_key(N, precision))
    if e:
        return {"leaf": int(e["leaf"]), "ir_max_iter": int(e["ir_max_iter"])}
    return {"leaf": 4, "ir_max_iter": 2 if precision == "mixed" else 0}


def _time_eval(plan, Z, y, ws, reps: int):
    import torch
    stream = torch.cuda.current_stream()
    ll, u, st = plan.evaluate(Z, y, ws=ws)   # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ll, u, st = plan.evaluate(Z, y, ws=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, st


def tune(N: int, precision: str, batch: int | None = None, n_z: int = 40, corr_len: float = 0.1,
         variance: float = 2.0, obs_side: int = 16, leaves=LEAVES, ir_steps=IR_STEPS, ir_tol: float = 1e-8,
         reps: int = 2, phi: np.ndarray | None = None, device: int = 0) -> dict:
    """Time every candidate on synthetic inputs of the workload recipe; returns the table entry."""
    import torch

    import workload as w
    from . import hdd

    B = batch or DEFAULT_BATCH.get(N, 64)
    phi = w.kl_basis(N, n_z, corr_len, variance) if phi is None else phi
    obs = w.obs_vertices(N, obs_side)
    rng = np.random.default_rng(N)
    dev = torch.device("cuda", device)
    Z = torch.from_numpy(rng.standard_normal((B, phi.shape[1]))).to(dev)
    y = torch.from_numpy(0.01 * rng.standard_normal(obs.size)).to(dev)
    prec = hdd.HDD_MIXED_FP32 if precision == "mixed" else hdd.HDD_FP64
    cands = []
    for leaf in leaves:
        if leaf >= N - 1:
            continue
        for K in (ir_steps if precision == "mixed" else (0,)):
            plan = hdd.Plan(N, leaf, phi, obs, 0.01, precision=prec, ir_max_iter=K, ir_tol=ir_tol, device=device)
            free, _ = torch.cuda.mem_get_info(dev)
            need = plan.workspace_size(B)
            if need > 0.8 * free:
                cands.append({"leaf": leaf, "ir_max_iter": K, "skipped": "workspace larger than free memory"})
                break
            ws = plan.workspace(B)
            ms, st = _time_eval(plan, Z, y, ws, reps)
            failed = int((st != 0).sum().item())
            cands.append({"leaf": leaf, "ir_max_iter": K, "ms_per_batch": ms, "ms_per_sample": ms / B,
                          "failed_samples": failed, "workspace_gb": need / 1e9})
            del ws, plan
            torch.cuda.empty_cache()
            if failed == 0:
                break   # the fewest refinement steps that meet the tolerance for this leaf
    ok = [c for c in cands if c.get("failed_samples") == 0]
    if not ok:
        raise RuntimeError(f"no candidate for N={N} {precision} met the tolerance: {cands}")
    best = min(ok, key=lambda c: c["ms_per_sample"])
    return {"leaf": best["leaf"], "ir_max_iter": best["ir_max_iter"], "ms_per_sample": best["ms_per_sample"],
            "batch": B, "n_z": int(phi.shape[1]), "obs": int(obs.size), "ir_tol": ir_tol, "candidates": cands}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--grids", type=int, nargs="+", default=[129, 257, 513, 1025])
    ap.add_argument("--precisions", nargs="+", default=["mixed", "fp64"], choices=["mixed", "fp64"])
    ap.add_argument("--out", default=TABLE)
    args = ap.parse_args(argv)
    import workload as w
    table = load_table(args.out)
    for N in args.grids:
        phi = w.kl_basis(N, 40, 0.1, 2.0)
        for prec in args.precisions:
            entry = tune(N, prec, phi=phi)
            table[_key(N, prec)] = entry
            print(json.dumps({"grid": N, "precision": prec, "leaf": entry["leaf"], "ir_max_iter": entry["ir_max_iter"],
                              "ms_per_sample": entry["ms_per_sample"]}), flush=True)
            with open(args.out, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
    return 0


if __name__ == "__main__":
    ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    sys.exit(main())
