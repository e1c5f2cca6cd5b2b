"""GPU: the fused bottom-subtree sweeps (hdd_set_sweep_fusion) against the level-by-level
sweeps and the oracle.  The same elimination in another order of operations: full
fields of hdd_solve_loads and refined u_obs agree to 1e-13 relative (FP32 factors: the
refinement removes the rounding differences to its tolerance and beyond), and the
fused path meets the oracle's tolerances on its own."""
import numpy as np
import pytest

import workload as w
from oracle import fem
from tests.gpu_common import rel_err_field, small_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hdd():
    from paper_1708_02207_gb300 import build, hdd as binding
    build.build()
    return binding


def run(hdd, plan, Z, c):
    B = Z.shape[0]
    ws = plan.workspace(B)
    Zd = torch.from_numpy(Z).cuda()
    plan.assemble(Zd, ws)
    plan.upsweep(B, ws)
    u = torch.empty(B, c.shape[1], plan.N * plan.N, dtype=torch.float64, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    plan.solve_loads(B, ws, torch.from_numpy(c).cuda(), u, status=st)
    ll, uo, st2 = plan.evaluate(Zd, torch.zeros(plan.n_obs, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    return u.cpu().numpy(), uo.cpu().numpy(), st.cpu().numpy(), st2.cpu().numpy()


@pytest.mark.parametrize("N,leaf,prec,heights", [(65, 4, 1, (1, 2, 3)), (129, 4, 1, (2, 3)), (50, 5, 1, (1, 2, 6)),
                                                 (33, 4, 0, (1, 2)), (65, 3, 0, (1, 3, 6))])
def test_fused_equals_level_by_level(hdd, N, leaf, prec, heights):
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=11, seed=N + 7 * leaf)
    plan = hdd.Plan(N, leaf, phi, w.obs_vertices(N, 4), 0.01, precision=prec, ir_max_iter=2 if prec else 0,
                    ir_tol=1e-9)
    c = np.random.default_rng(N).standard_normal((Z.shape[0], 2, N * N)) / (N - 1) ** 2
    plan.set_sweep_fusion(0)
    assert plan.info()["sweep_fuse_height"] == 0
    ref = run(hdd, plan, Z, c)
    used = set()
    for h in heights:
        plan.set_sweep_fusion(h)
        hu = plan.info()["sweep_fuse_height"]
        assert 1 <= hu <= h   # the largest height <= h whose subtrees fit
        if hu in used:
            continue
        used.add(hu)
        got = run(hdd, plan, Z, c)
        assert (got[2] == 0).all() and (got[3] == 0).all()
        assert rel_err_field(got[0].reshape(-1, N * N), ref[0].reshape(-1, N * N)).max() <= 1e-13
        assert np.abs(got[1] - ref[1]).max() <= 1e-13 * np.abs(ref[1]).max()


def test_fused_loads_match_the_oracle(hdd):
    N = 129
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=3, seed=5)
    plan = hdd.Plan(N, 4, phi, w.obs_vertices(N, 4), 0.01)
    plan.set_sweep_fusion(6)
    assert plan.info()["sweep_fuse_height"] >= 2   # FP64 subtrees: height 2 fits the shared-memory budget
    c = np.random.default_rng(2).standard_normal((3, 1, N * N)) / (N - 1) ** 2
    u, _, st, _ = run(hdd, plan, Z, c)
    assert (st == 0).all()
    for s in range(3):
        ref = fem.solve_load(N, fem.kappa_from_kl(phi, Z[s]), c[s, 0], refine=True)
        assert rel_err_field(u[s, 0][None], ref.reshape(1, -1)).max() <= 1e-11
