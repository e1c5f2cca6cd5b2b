"""Continuous-batching request loop for likelihood evaluations.

Plans (one per grid, KL basis and observation set) stay resident on the device.  Each
request carries one parameter vector Z and its data y and names its plan.  Requests wait in
arrival order; a scheduling pass first collects the batches whose completion event has
fired, then admits new batches: it takes the plan of the oldest waiting request and gathers
up to `max_batch` waiting requests of that plan, shrinking the batch until the device memory
of its workspace (hdd_workspace_size: the Schur stacks, factors and vectors of that many
samples) fits into what the batches in flight leave of the budget.  An admitted batch runs
on a free stream, so batches of different plans overlap on the device, and requests that
arrive while others run are admitted as soon as memory and a stream are free.  Latency is
measured per request from submission to collection.

Every sample of a batch is computed independently of the others (the library's kernels
never combine samples), so a result does not depend on what it was batched with.

A plan may name a fallback plan (`fallback={"513": "513-fp64"}`): a request whose result comes
back with one of the `escalate` codes (by default HDD_ENOCONV, a mixed-precision sample
whose refinement did not reach the tolerance) goes back to the head of the queue under the
fallback plan, keeping its submission time, and is reported once, with the fallback's result
and `escalated_from` set.  An FP64 plan as the fallback of a mixed one turns the rare sample
of high contrast that the FP32 factors cannot refine into a slower, exact answer instead of a
failure.

The loop itself is host logic over a small backend interface: `CudaBackend` runs batches
through the C ABI (paper_1708_02207_gb300.hdd); tests drive the same loop with a fake.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass

import numpy as np


@dataclass
class Request:
    rid: int
    plan: str
    Z: np.ndarray
    y: np.ndarray
    t_submit: float
    t_done: float = float("nan")
    loglik: float = float("nan")
    u_obs: np.ndarray | None = None
    status: int = 0
    rejected: str = ""
    escalated_from: str = ""

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


@dataclass
class _Batch:
    handle: object
    plan: str
    requests: list
    bytes: int
    slot: int


class Server:
    """The request loop.  `backend` provides workspace_bytes(plan, batch),
    launch(plan, Z[B, n_z], y[B, n_obs], slot) -> handle, done(handle) -> bool,
    collect(handle) -> (loglik[B], u_obs[B, n_obs], status[B]) and release(handle)."""

    def __init__(self, backend, budget_bytes: int, max_batch: int = 64, n_slots: int = 4, clock=time.perf_counter,
                 fallback: dict | None = None, escalate=(-5,)):
        if budget_bytes <= 0 or max_batch < 1 or n_slots < 1:
            raise ValueError("budget_bytes, max_batch and n_slots must be positive")
        self.fallback = dict(fallback or {})
        for a, b in self.fallback.items():
            backend.workspace_bytes(a, 1)   # unknown plans raise here
            backend.workspace_bytes(b, 1)
            if self.fallback.get(b) is not None:
                raise ValueError(f"fallback plan {b!r} has a fallback of its own")
        self.escalate = frozenset(int(e) for e in escalate)
        self.escalated = 0
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.clock = clock
        self.waiting: deque = deque()
        self.in_flight: list = []
        self.free_slots = list(range(n_slots))
        self.done: list = []
        self.bytes_in_flight = 0
        self.peak_bytes = 0
        self.batches = 0
        self._next = 0

    # ---- requests ------------------------------------------------------
    def submit(self, plan: str, Z, y, t: float | None = None) -> Request:
        self.backend.workspace_bytes(plan, 1)   # an unknown plan raises here, not in the loop
        r = Request(self._next, plan, np.asarray(Z, dtype=np.float64), np.asarray(y, dtype=np.float64),
                    self.clock() if t is None else t)
        self._next += 1
        self.waiting.append(r)
        return r

    # ---- scheduling ----------------------------------------------------
    def _collect(self):
        still = []
        for b in self.in_flight:
            if not self.backend.done(b.handle):
                still.append(b)
                continue
            ll, u, st = self.backend.collect(b.handle)
            t = self.clock()
            again = []
            for k, r in enumerate(b.requests):
                code = -(int(st[k]) & 0xFF)   # a sample's status is (-code) | (node << 8)
                if code in self.escalate and b.plan in self.fallback:
                    r.escalated_from, r.plan = b.plan, self.fallback[b.plan]
                    again.append(r)
                    continue
                r.loglik, r.u_obs, r.status, r.t_done = float(ll[k]), np.array(u[k]), int(st[k]), t
                self.done.append(r)
            self.waiting.extendleft(reversed(again))   # ahead of every later arrival, in order
            self.escalated += len(again)
            self.backend.release(b.handle)
            self.bytes_in_flight -= b.bytes
            self.free_slots.append(b.slot)
        self.in_flight = still

    def _admit(self):
        while self.waiting and self.free_slots:
            plan = self.waiting[0].plan
            group = [r for r in self.waiting if r.plan == plan][: self.max_batch]
            n = len(group)
            left = self.budget - self.bytes_in_flight
            while n > 0 and self.backend.workspace_bytes(plan, n) > left:
                n -= 1
            if n == 0:
                if not self.in_flight and self.backend.workspace_bytes(plan, 1) > self.budget:
                    r = self.waiting.popleft()   # can never fit: refuse it rather than wait forever
                    r.rejected = "workspace of one sample exceeds the budget"
                    r.t_done = self.clock()
                    self.done.append(r)
                    continue
                return   # wait for memory to free up
            group = group[:n]
            ids = {r.rid for r in group}
            self.waiting = deque(r for r in self.waiting if r.rid not in ids)
            nbytes = self.backend.workspace_bytes(plan, n)
            slot = self.free_slots.pop()
            Z = np.stack([r.Z for r in group])
            y = np.stack([r.y for r in group])
            handle = self.backend.launch(plan, Z, y, slot)
            self.in_flight.append(_Batch(handle, plan, group, nbytes, slot))
            self.bytes_in_flight += nbytes
            self.peak_bytes = max(self.peak_bytes, self.bytes_in_flight)
            self.batches += 1

    def step(self):
        """One scheduling pass: collect finished batches, then admit what fits."""
        self._collect()
        self._admit()

    def idle(self) -> bool:
        return not self.waiting and not self.in_flight

    def run_until_idle(self, poll_s: float = 0.0):
        while not self.idle():
            self.step()
            if poll_s:
                time.sleep(poll_s)

    def latency_percentiles(self, qs=(0.5, 0.99)) -> dict:
        lat = sorted(r.latency for r in self.done if not r.rejected)
        if not lat:
            return {q: float("nan") for q in qs}
        return {q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))] for q in qs}


class CudaBackend:
    """Batches through the C ABI on one device: per plan a resident hdd.Plan, per in-flight
    batch its own workspace (from PyTorch's caching allocator, returned when the batch is
    collected), one CUDA stream per slot, inputs copied from pinned host memory and results
    copied back on that stream, and a CUDA event that marks completion."""

    def __init__(self, plans: dict, n_slots: int = 4, device: int = 0):
        import torch
        self.torch = torch
        self.plans = plans
        self.dev = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(n_slots)]

    def workspace_bytes(self, plan: str, batch: int) -> int:
        return self.plans[plan].workspace_size(batch)

    def launch(self, plan: str, Z: np.ndarray, y: np.ndarray, slot: int):
        torch = self.torch
        p = self.plans[plan]
        B = Z.shape[0]
        st = self.streams[slot]
        with torch.cuda.stream(st):
            ws = p.workspace(B)
        Zh = torch.from_numpy(np.ascontiguousarray(Z)).pin_memory()
        yh = torch.from_numpy(np.ascontiguousarray(y)).pin_memory()
        out = {"ll": torch.empty(B, dtype=torch.float64).pin_memory(),
               "u": torch.empty(B, p.n_obs, dtype=torch.float64).pin_memory(),
               "st": torch.empty(B, dtype=torch.int32).pin_memory()}
        with torch.cuda.stream(st):
            Zd = Zh.to(self.dev, non_blocking=True)
            yd = yh.to(self.dev, non_blocking=True)
            u = torch.empty(B, p.n_obs, dtype=torch.float64, device=self.dev)
            ll = torch.empty(B, dtype=torch.float64, device=self.dev)
            sd = torch.empty(B, dtype=torch.int32, device=self.dev)
            p.assemble(Zd, ws, st)
            p.upsweep(B, ws, st)
            p.point_solve(B, ws, u, st)
            p.loglik(B, ws, u, yd, ll, sd, st)
            out["ll"].copy_(ll, non_blocking=True)
            out["u"].copy_(u, non_blocking=True)
            out["st"].copy_(sd, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        # the device tensors of this batch stay alive until it is released
        return {"ev": ev, "out": out, "keep": (ws, Zh, yh, Zd, yd, u, ll, sd)}

    def done(self, h) -> bool:
        return h["ev"].query()

    def collect(self, h):
        h["ev"].synchronize()
        o = h["out"]
        return o["ll"].numpy(), o["u"].numpy(), o["st"].numpy()

    def release(self, h):
        h["keep"] = None   # collected, so the stream is past every use of these buffers


class MetropolisChain:
    """Random-walk Metropolis on Z with prior N(0, I) and the served log-likelihood:
    propose Z' = Z + step * xi (xi ~ N(0, I)); once l(Z') is back, accept with probability
    min(1, exp(l(Z') - |Z'|^2 / 2 - l(Z) + |Z|^2 / 2)).  A chain has at most one request in
    flight; its first request evaluates its starting point, which is always taken."""

    def __init__(self, plan: str, Z0, y, step: float, rng: np.random.Generator):
        self.plan, self.y, self.step, self.rng = plan, np.asarray(y, dtype=np.float64), float(step), rng
        self.Z = np.asarray(Z0, dtype=np.float64)
        self.logpost = None          # log-likelihood + log-prior at Z, once known
        self.pending = None          # (request, proposal) in flight
        self.accepted = 0
        self.steps = 0

    def propose(self) -> np.ndarray:
        if self.logpost is None:
            return self.Z.copy()
        return self.Z + self.step * self.rng.standard_normal(self.Z.shape)

    def update(self, Zp: np.ndarray, loglik: float, status: int):
        lp = loglik - 0.5 * float(Zp @ Zp) if status == 0 else -np.inf
        if self.logpost is None:
            self.logpost = lp
            return
        self.steps += 1
        if np.log(self.rng.random()) < lp - self.logpost:
            self.Z, self.logpost = Zp, lp
            self.accepted += 1


def run_offered_load(server: Server, chains: list, rate: float, n_requests: int, rng: np.random.Generator,
                     tick=None) -> dict:
    """Requests arrive as a Poisson process of `rate` per second over all chains; at an arrival
    the longest-idle chain without a request in flight proposes and submits (if every chain
    is waiting for a result, the arrival waits for the first one to come back).  Runs until
    `n_requests` results are back and returns their throughput, p50/p99 latency and the
    acceptance rate.  `rate` = inf submits whenever a chain is free (saturation).
    `tick()` is called when a pass did nothing (default: sleep 50 us)."""
    clock = server.clock
    tick = tick or (lambda: time.sleep(5e-5))
    idle = deque(chains)
    t0 = clock()
    next_arrival = t0 if np.isinf(rate) else t0 + rng.exponential(1.0 / rate)
    submitted, seen, results = 0, len(server.done), []
    while len(results) < n_requests:
        busy = False
        while submitted < n_requests and idle and clock() >= next_arrival:
            c = idle.popleft()
            Zp = c.propose()
            c.pending = (server.submit(c.plan, Zp, c.y), Zp)
            submitted += 1
            busy = True
            if not np.isinf(rate):
                next_arrival += rng.exponential(1.0 / rate)
        server.step()
        while seen < len(server.done):
            r = server.done[seen]
            seen += 1
            for c in chains:
                if c.pending is not None and c.pending[0] is r:
                    c.update(c.pending[1], r.loglik, r.status if not r.rejected else -1)
                    c.pending = None
                    idle.append(c)
                    results.append(r)
                    busy = True
        if not busy:
            tick()
    t1 = clock()
    lat = sorted(r.latency for r in results)
    pick = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    steps = sum(c.steps for c in chains)
    return {"offered_per_s": rate, "evals_per_s": len(results) / (t1 - t0) if t1 > t0 else float("inf"),
            "p50_s": pick(0.5), "p99_s": pick(0.99), "requests": len(results),
            "accept_rate": sum(c.accepted for c in chains) / steps if steps else float("nan")}
