"""hdd_evaluate_static: the evaluation for callers that cannot allocate device memory.

Such callers (a host application whose device memory is all reserved up front by
another framework's pool, a plug-in without an allocator, a sampling loop that
must not call cudaMalloc/cudaFree) get the workspace from one static device array
inside the library.  This test calls that entry point through the C ABI twice in
a row and checks both results against the workspace-based entry points with the
parity tolerance of the FP64 path (1e-11 relative).  It is collected last.
"""
import numpy as np
import pytest

import workload as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


def test_static_workspace_entry_matches_workspace_entry():
    from paper_1708_02207_gb300 import build, hdd
    build.build()
    cfg = w.CONFIGS["grid33"]
    prob = w.make_problem(cfg, batch=4)
    plan = hdd.Plan(cfg.N, cfg.leaf, prob.phi, prob.obs, cfg.sigma)
    assert plan.workspace_size(4) <= hdd.STATIC_WORKSPACE_BYTES
    y = torch.from_numpy(prob.y).cuda()
    Z1 = torch.from_numpy(prob.Z).cuda()
    Z2 = torch.from_numpy(prob.Z[::-1].copy() * 0.5).cuda()
    ref = [plan.evaluate(Z, y) for Z in (Z1, Z2)]          # caller-provided torch workspace
    for Z, (ll_ref, u_ref, st_ref) in zip((Z1, Z2), ref):  # two static-workspace calls in a row
        ll = torch.empty(4, dtype=torch.float64, device="cuda")
        u = torch.empty(4, plan.n_obs, dtype=torch.float64, device="cuda")
        st = torch.full((4,), 7, dtype=torch.int32, device="cuda")
        plan.evaluate_static(Z, y, ll, u, st)
        torch.cuda.synchronize()
        assert torch.equal(st, st_ref) and int(st.abs().sum()) == 0
        err_u = ((u - u_ref).abs().max(dim=1).values / u_ref.abs().max(dim=1).values).max().item()
        err_ll = ((ll - ll_ref).abs() / ll_ref.abs()).max().item()
        assert err_u <= TOL and err_ll <= TOL
    # a batch whose workspace exceeds the static array is refused
    big = 1
    while plan.workspace_size(big) <= hdd.STATIC_WORKSPACE_BYTES:
        big *= 2
    Zb = torch.zeros(big, cfg.n_z, dtype=torch.float64, device="cuda")
    llb = torch.empty(big, dtype=torch.float64, device="cuda")
    with pytest.raises(hdd.HDDError) as e:
        plan.evaluate_static(Zb, y, llb)
    assert e.value.status == hdd.HDD_EINVAL
