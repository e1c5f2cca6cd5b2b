"""Host logic of the continuous-batching request loop (paper_1708_02207_gb300.serving),
driven by a fake backend on a manual clock: every request gets its own result whatever it
was batched with, the memory budget holds at every instant, requests that arrive while
batches run are admitted as soon as a batch completes, and a request that can never fit is
refused instead of blocking the queue."""
import numpy as np
import pytest

from paper_1708_02207_gb300.serving import Server


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """workspace = fixed + per-sample bytes; a batch of n samples of a plan finishes
    `dur[plan] * (1 + n / 8)` after launch; loglik is a fixed function of each row."""

    def __init__(self, clock, per_sample, fixed=100, dur=None):
        self.clock, self.per_sample, self.fixed = clock, per_sample, fixed
        self.dur = dur or {k: 1.0 for k in per_sample}
        self.launches = []
        self.budget_seen = []

    def workspace_bytes(self, plan, n):
        return self.fixed + self.per_sample[plan] * n

    def launch(self, plan, Z, y, slot):
        h = {"t_end": self.clock() + self.dur[plan] * (1 + Z.shape[0] / 8), "Z": Z, "y": y}
        self.launches.append((plan, Z.shape[0], slot, self.clock()))
        return h

    def done(self, h):
        return self.clock() >= h["t_end"]

    def collect(self, h):
        ll = -(h["Z"] ** 2).sum(axis=1) + h["y"].sum(axis=1)
        return ll, h["Z"][:, :2] * 3.0, np.zeros(len(ll), dtype=np.int32)

    def release(self, h):
        pass


def drive(server, clock, dt=0.25, limit=10000):
    for _ in range(limit):
        if server.idle():
            return
        server.step()
        assert server.bytes_in_flight <= server.budget
        clock.t += dt
    raise AssertionError("the loop did not drain")


def test_results_belong_to_their_requests():
    clock = Clock()
    be = FakeBackend(clock, {"a": 10, "b": 30})
    srv = Server(be, budget_bytes=1000, max_batch=5, n_slots=3, clock=clock)
    rng = np.random.default_rng(0)
    reqs = []
    for k in range(37):
        plan = "a" if rng.random() < 0.6 else "b"
        Z, y = rng.standard_normal(4), rng.standard_normal(3)
        reqs.append((srv.submit(plan, Z, y), Z, y))
        if k % 5 == 0:
            srv.step()
            clock.t += 0.1
    drive(srv, clock)
    assert len(srv.done) == 37
    for r, Z, y in reqs:
        assert r.rejected == ""
        assert r.loglik == pytest.approx(-(Z ** 2).sum() + y.sum(), abs=1e-12)
        assert np.allclose(r.u_obs, Z[:2] * 3.0)
        assert r.t_done >= r.t_submit
    assert max(n for _, n, _, _ in be.launches) <= 5


def test_batches_shrink_to_the_memory_budget():
    clock = Clock()
    be = FakeBackend(clock, {"a": 100}, fixed=50)
    srv = Server(be, budget_bytes=400, max_batch=16, n_slots=4, clock=clock)   # room for 3 samples
    for _ in range(10):
        srv.submit("a", np.zeros(2), np.zeros(1))
    drive(srv, clock)
    assert all(n <= 3 for _, n, _, _ in be.launches)
    assert srv.peak_bytes <= 400
    assert len(srv.done) == 10


def test_arrivals_are_admitted_while_other_batches_run():
    clock = Clock()
    be = FakeBackend(clock, {"slow": 10, "fast": 10}, dur={"slow": 50.0, "fast": 1.0})
    srv = Server(be, budget_bytes=10_000, max_batch=4, n_slots=2, clock=clock)
    srv.submit("slow", np.zeros(2), np.zeros(1))
    srv.submit("fast", np.zeros(2), np.zeros(1))
    srv.step()                                  # both slots busy
    assert len(srv.in_flight) == 2
    clock.t = 5.0
    late = srv.submit("fast", np.ones(2), np.zeros(1))
    srv.step()                                  # the fast batch is done: its slot takes the new request
    assert late not in srv.waiting and any(late in b.requests for b in srv.in_flight)
    assert any(b.plan == "slow" for b in srv.in_flight)   # still running beside it
    drive(srv, clock)
    assert late.t_done < 50.0


def test_oversized_request_is_refused_not_blocking():
    clock = Clock()
    be = FakeBackend(clock, {"small": 10, "huge": 10_000})
    srv = Server(be, budget_bytes=1000, max_batch=4, n_slots=2, clock=clock)
    big = srv.submit("huge", np.zeros(2), np.zeros(1))
    ok = [srv.submit("small", np.zeros(2), np.zeros(1)) for _ in range(3)]
    drive(srv, clock)
    assert big.rejected and np.isnan(big.loglik)
    assert all(r.rejected == "" and np.isfinite(r.loglik) for r in ok)
    assert srv.latency_percentiles()[0.5] >= 0.0


def test_oldest_request_chooses_the_plan():
    clock = Clock()
    be = FakeBackend(clock, {"a": 10, "b": 10})
    srv = Server(be, budget_bytes=10_000, max_batch=8, n_slots=1, clock=clock)
    for plan in ("b", "a", "b", "a", "a"):
        srv.submit(plan, np.zeros(2), np.zeros(1))
    drive(srv, clock)
    assert [(p, n) for p, n, _, _ in be.launches] == [("b", 2), ("a", 3)]


def test_unknown_plan_and_bad_settings_raise():
    clock = Clock()
    be = FakeBackend(clock, {"a": 10})
    srv = Server(be, budget_bytes=100, clock=clock)
    with pytest.raises(KeyError):
        srv.submit("nope", np.zeros(2), np.zeros(1))
    with pytest.raises(ValueError):
        Server(be, budget_bytes=0)


def test_offered_load_run_with_metropolis_chains():
    from paper_1708_02207_gb300.serving import MetropolisChain, run_offered_load

    class GaussBackend(FakeBackend):
        # log-likelihood of a Gaussian centred at 1 in every coordinate
        def collect(self, h):
            ll = -0.5 * ((h["Z"] - 1.0) ** 2).sum(axis=1)
            return ll, h["Z"][:, :2], np.zeros(len(ll), dtype=np.int32)

    clock = Clock()
    be = GaussBackend(clock, {"a": 10, "b": 10}, dur={"a": 0.01, "b": 0.02})
    srv = Server(be, budget_bytes=10_000, max_batch=8, n_slots=2, clock=clock)
    rng = np.random.default_rng(3)
    chains = [MetropolisChain("a" if k % 2 else "b", np.zeros(3), np.zeros(1), 0.5, np.random.default_rng(k))
              for k in range(6)]

    def tick():
        clock.t += 0.001

    out = run_offered_load(srv, chains, rate=200.0, n_requests=600, rng=rng, tick=tick)
    assert out["requests"] == 600 and len(srv.done) == 600
    assert 0.05 < out["accept_rate"] < 0.95
    assert 0.0 <= out["p50_s"] <= out["p99_s"]
    # offered 200/s for 600 requests: about 3 s of arrivals on the fake clock
    assert 120.0 < out["evals_per_s"] < 260.0
    # the chains drift to the likelihood's centre (posterior mean 0.5 per coordinate)
    assert np.mean([c.Z.mean() for c in chains]) > 0.1
    sat = run_offered_load(srv, chains, rate=float("inf"), n_requests=120, rng=rng, tick=tick)
    assert sat["evals_per_s"] > out["evals_per_s"]


class FlakyBackend(FakeBackend):
    """Plan "mixed" reports HDD_ENOCONV at tree node 7 ((5) | (7 << 8)) for rows whose first
    entry is negative; plan "fp64" always succeeds and shifts loglik by +1000 so that the
    test can tell which plan produced a result."""

    def collect(self, h):
        ll, u, st = super().collect(h)
        if h["plan"] == "mixed":
            st = np.where(h["Z"][:, 0] < 0, 5 | (7 << 8), 0).astype(np.int32)
        else:
            ll = ll + 1000.0
        return ll, u, st

    def launch(self, plan, Z, y, slot):
        h = super().launch(plan, Z, y, slot)
        h["plan"] = plan
        return h


def test_non_converged_requests_escalate_to_the_fallback_plan():
    clock = Clock()
    be = FlakyBackend(clock, {"mixed": 10, "fp64": 40}, dur={"mixed": 1.0, "fp64": 4.0})
    srv = Server(be, budget_bytes=10_000, max_batch=8, clock=clock, fallback={"mixed": "fp64"})
    rng = np.random.default_rng(3)
    reqs = [srv.submit("mixed", rng.standard_normal(4), np.ones(2)) for _ in range(20)]
    drive(srv, clock)
    assert len(srv.done) == 20 and {r.rid for r in srv.done} == {r.rid for r in reqs}
    bad = [r for r in reqs if r.Z[0] < 0]
    assert bad and srv.escalated == len(bad)
    for r in reqs:
        ref = -(r.Z ** 2).sum() + 2.0
        assert r.status == 0
        if r.Z[0] < 0:
            assert r.escalated_from == "mixed" and r.plan == "fp64" and r.loglik == pytest.approx(ref + 1000.0)
        else:
            assert r.escalated_from == "" and r.plan == "mixed" and r.loglik == pytest.approx(ref)
        assert r.t_done > r.t_submit
    # the re-run of a request never precedes its first attempt, and fp64 batches hold only escalated rows
    assert all(p == "mixed" for p, _, _, t in be.launches if t == 0.0)
    assert sum(n for p, n, _, _ in be.launches if p == "fp64") == len(bad)


def test_escalation_only_for_the_named_codes_and_plans():
    clock = Clock()
    be = FlakyBackend(clock, {"mixed": 10, "fp64": 40})
    # HDD_ENOTSPD (-4) is escalated, HDD_ENOCONV is not: the failures come back as they are
    srv = Server(be, budget_bytes=10_000, max_batch=8, clock=clock, fallback={"mixed": "fp64"}, escalate=(-4,))
    rng = np.random.default_rng(4)
    reqs = [srv.submit("mixed", rng.standard_normal(4), np.ones(2)) for _ in range(12)]
    drive(srv, clock)
    assert srv.escalated == 0
    assert all((r.status == (5 | (7 << 8))) == (r.Z[0] < 0) for r in reqs)
    with pytest.raises(ValueError):
        Server(be, budget_bytes=10_000, fallback={"mixed": "fp64", "fp64": "mixed"})
    with pytest.raises(KeyError):
        Server(be, budget_bytes=10_000, fallback={"mixed": "nope"})
