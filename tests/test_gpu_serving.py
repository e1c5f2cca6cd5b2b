"""The request loop on the GPU: batches of two resident plans (33² FP64 and 65² mixed)
admitted by workspace memory and overlapped on three streams; every request's result equals
the same request evaluated alone."""
import numpy as np
import pytest

import workload as w
from tests.gpu_common import small_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_served_results_equal_alone():
    from paper_1708_02207_gb300 import build, hdd, serving
    build.build()
    phi33, _ = small_problem(33, batch=1, seed=1)
    phi65, _ = small_problem(65, n_z=20, corr_len=0.2, variance=2.0, batch=1, seed=2)
    obs33, obs65 = w.obs_vertices(33, 3), w.obs_vertices(65, 4)
    plans = {"g33": hdd.Plan(33, 8, phi33, obs33, 0.01),
             "g65": hdd.Plan(65, 4, phi65, obs65, 0.01, precision=hdd.HDD_MIXED_FP32, ir_max_iter=2)}
    budget = plans["g65"].workspace_size(4) + 2 * plans["g33"].workspace_size(4)
    srv = serving.Server(serving.CudaBackend(plans, n_slots=3), budget, max_batch=4, n_slots=3)
    rng = np.random.default_rng(7)
    reqs = []
    for k in range(30):
        name = "g33" if k % 3 else "g65"
        p = plans[name]
        Z = rng.standard_normal(p.n_z)
        y = 0.01 * rng.standard_normal(p.n_obs)
        reqs.append(srv.submit(name, Z, y))
        if k % 4 == 0:
            srv.step()
    srv.run_until_idle()
    assert len(srv.done) == 30 and srv.peak_bytes <= budget
    for r in reqs:
        assert r.rejected == "" and r.status == 0
        ll, u, st = plans[r.plan].evaluate(torch.from_numpy(r.Z[None]).cuda(), torch.from_numpy(r.y[None]).cuda())
        torch.cuda.synchronize()
        u = u.cpu().numpy()[0]
        assert st.item() == 0
        assert abs(r.loglik - ll.item()) <= 1e-13 * abs(ll.item())
        assert np.max(np.abs(r.u_obs - u)) <= 1e-13 * np.max(np.abs(u))
    p50, p99 = srv.latency_percentiles().values()
    assert 0.0 <= p50 <= p99


def test_non_converged_requests_are_answered_by_the_fp64_fallback():
    # a mixed plan whose tolerance no refinement reaches flags every sample HDD_ENOCONV;
    # the loop re-runs each on the FP64 plan of the same problem and reports that result
    from paper_1708_02207_gb300 import build, hdd, serving
    build.build()
    phi, _ = small_problem(65, n_z=20, corr_len=0.2, variance=2.0, batch=1, seed=5)
    obs = w.obs_vertices(65, 4)
    plans = {"mixed": hdd.Plan(65, 4, phi, obs, 0.01, precision=hdd.HDD_MIXED_FP32, ir_max_iter=1, ir_tol=1e-300),
             "fp64": hdd.Plan(65, 8, phi, obs, 0.01)}
    budget = 2 * plans["mixed"].workspace_size(4) + 2 * plans["fp64"].workspace_size(4)
    srv = serving.Server(serving.CudaBackend(plans, n_slots=2), budget, max_batch=4, n_slots=2,
                         fallback={"mixed": "fp64"})
    rng = np.random.default_rng(8)
    reqs = [srv.submit("mixed", rng.standard_normal(20), 0.01 * rng.standard_normal(obs.size)) for _ in range(10)]
    srv.run_until_idle()
    assert len(srv.done) == 10 and srv.escalated == 10
    for r in reqs:
        assert r.status == 0 and r.plan == "fp64" and r.escalated_from == "mixed"
        ll, u, st = plans["fp64"].evaluate(torch.from_numpy(r.Z[None]).cuda(), torch.from_numpy(r.y[None]).cuda())
        torch.cuda.synchronize()
        assert st.item() == 0 and abs(r.loglik - ll.item()) <= 1e-13 * abs(ll.item())
        assert np.max(np.abs(r.u_obs - u.cpu().numpy()[0])) <= 1e-13 * np.max(np.abs(u.cpu().numpy()))
