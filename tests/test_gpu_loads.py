"""GPU parity of the calls that reuse the factors of one upsweep: many load vectors
at a fixed coefficient field (hdd_solve_loads, Sec. 2) and the mean of u over every
subdomain of the tree (hdd_subdomain_means, Sec. 5, Eq. mean; Sec. 5.1).

Tolerances as for the point solve: 1e-11 relative (FP64 plans) and 1e-8 relative
after refinement (mixed plans), max_k |u_k - u_k^oracle| / max_k |u_k^oracle| over
every vertex; subdomain means of a given field agree to FP64 rounding (1e-13
relative to the largest |u|).
"""
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
    assert torch.cuda.is_available()
    return binding


def make_loads(N, batch, seed):
    """[batch, 3, N*N]: the f = 1 load h^2, a random nonnegative load, a point load;
    boundary entries hold noise, which the solve must ignore."""
    h2 = 1.0 / (N - 1) ** 2
    rng = np.random.default_rng(seed)
    c = np.empty((batch, 3, N * N))
    c[:, 0] = h2
    c[:, 1] = h2 * rng.random((batch, N * N))
    c[:, 2] = 0.0
    c[:, 2, (N // 3) * N + N // 2] = 1.0
    c[:, 2, 2 * N + 3] = -0.5
    bnd = np.setdiff1d(np.arange(N * N), fem.interior_ids(N))
    c[:, :, bnd] = rng.standard_normal((batch, 3, bnd.size))
    return c


def gpu_solve_loads(hdd, N, leaf, phi, Z, c, **kw):
    obs = np.array([(N // 2) * N + N // 2], dtype=np.int32)
    plan = hdd.Plan(N, leaf, phi, obs, 0.1, **kw)
    batch = Z.shape[0]
    ws = plan.workspace(batch)
    Zd = torch.from_numpy(np.ascontiguousarray(Z)).cuda()
    cd = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    u = torch.full_like(cd, float("nan"))
    st = torch.full((batch,), -99, dtype=torch.int32, device="cuda")
    plan.assemble(Zd, ws)
    plan.upsweep(batch, ws)
    plan.solve_loads(batch, ws, cd, u, st)
    torch.cuda.synchronize()
    return plan, u.cpu().numpy(), st.cpu().numpy()


def oracle_loads(N, phi, Z, c):
    out = np.empty_like(c)
    for s, z in enumerate(Z):
        kap = fem.kappa_from_kl(phi, z)
        for k in range(c.shape[1]):
            out[s, k] = fem.solve_load(N, kap, c[s, k], refine=True)
    return out


@pytest.mark.parametrize("N,leaf", [(33, 8), (65, 4), (129, 8), (50, 5)])
def test_solve_loads_fp64(hdd, N, leaf):
    phi, Z = small_problem(N, batch=2, seed=100 + N)
    c = make_loads(N, 2, N)
    _, u, st = gpu_solve_loads(hdd, N, leaf, phi, Z, c)
    ref = oracle_loads(N, phi, Z, c)
    assert (st == 0).all()
    assert np.isfinite(u).all()
    assert rel_err_field(u, ref).max() <= 1e-11


@pytest.mark.parametrize("N,leaf,top", [(33, 8, 0), (65, 4, 0), (129, 8, 2), (257, 16, 0)])
def test_solve_loads_mixed(hdd, N, leaf, top):
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=2, seed=200 + N)
    c = make_loads(N, 2, N + 1)
    _, u, st = gpu_solve_loads(hdd, N, leaf, phi, Z, c, precision=hdd.HDD_MIXED_FP32, ir_max_iter=2,
                               fp64_top_levels=top)
    ref = oracle_loads(N, phi, Z, c)
    assert (st == 0).all()
    assert np.isfinite(u).all()
    assert rel_err_field(u, ref).max() <= 1e-8


def test_solve_loads_matches_the_point_solve(hdd):
    # the f = 1 load through hdd_solve_loads gives the u_obs of hdd_point_solve (FP64 plan:
    # the same factors; y_gamma comes from the sweep kernels instead of the bordered fronts,
    # so only the rounding differs)
    cfg = w.CONFIGS["grid33"]
    prob = w.make_problem(cfg, batch=3)
    N = cfg.N
    plan = hdd.Plan(N, cfg.leaf, prob.phi, prob.obs, cfg.sigma)
    ws = plan.workspace(3)
    Zd = torch.from_numpy(prob.Z).cuda()
    u_obs = torch.empty(3, prob.obs.size, dtype=torch.float64, device="cuda")
    plan.assemble(Zd, ws)
    plan.upsweep(3, ws)
    plan.point_solve(3, ws, u_obs)
    c = torch.full((3, 1, N * N), 1.0 / (N - 1) ** 2, dtype=torch.float64, device="cuda")
    u = torch.empty_like(c)
    plan.solve_loads(3, ws, c, u)
    torch.cuda.synchronize()
    got = u[:, 0, torch.from_numpy(prob.obs).long().cuda()].cpu().numpy()
    assert rel_err_field(got, u_obs.cpu().numpy()).max() <= 1e-13


def test_solve_loads_no_convergence_is_flagged(hdd):
    N, leaf = 65, 4
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=2, seed=7)
    c = make_loads(N, 2, 8)
    _, u, st = gpu_solve_loads(hdd, N, leaf, phi, Z, c, precision=hdd.HDD_MIXED_FP32, ir_max_iter=1,
                               ir_tol=1e-30)
    assert ((st & 0xFF) == -hdd.HDD_ENOCONV).all()
    assert np.isfinite(u).all()


@pytest.mark.parametrize("N,leaf", [(33, 8), (65, 4), (50, 5)])
def test_subdomain_means_of_a_field(hdd, N, leaf):
    # a random field (boundary values included), rows strided in memory
    batch = 3
    obs = np.array([(N // 2) * N + N // 2], dtype=np.int32)
    phi, _ = small_problem(N, batch=1, seed=N)
    plan = hdd.Plan(N, leaf, phi, obs, 0.1)
    n_nodes = plan.info()["n_nodes"]
    u = np.random.default_rng(N).standard_normal((batch, N * N + 5))
    ud = torch.from_numpy(u).cuda()[:, : N * N]
    means = torch.full((batch, n_nodes), float("nan"), dtype=torch.float64, device="cuda")
    plan.subdomain_means(ud, means)
    torch.cuda.synchronize()
    got = means.cpu().numpy()
    for k in range(n_nodes):
        nd = plan.node(k)
        for s in range(batch):
            ref = fem.subdomain_mean(N, u[s, : N * N], nd["x0"], nd["x1"], nd["y0"], nd["y1"])
            assert abs(got[s, k] - ref) <= 1e-13, (k, s)


def test_subdomain_means_of_the_solution(hdd):
    # chained: loads solved on the GPU, means over every subdomain of the solution
    N, leaf = 65, 4
    phi, Z = small_problem(N, batch=2, seed=9)
    c = make_loads(N, 2, 10)
    plan, _, _ = gpu_solve_loads(hdd, N, leaf, phi, Z, c)
    # solve again into a device tensor kept for the means call
    ws = plan.workspace(2)
    plan.assemble(torch.from_numpy(Z).cuda(), ws)
    plan.upsweep(2, ws)
    cd = torch.from_numpy(c).cuda()
    u = torch.empty_like(cd)
    plan.solve_loads(2, ws, cd, u)
    n_nodes = plan.info()["n_nodes"]
    means = torch.empty((2, n_nodes), dtype=torch.float64, device="cuda")
    plan.subdomain_means(u[:, 1, :], means)   # the random load; row stride 3 N^2
    torch.cuda.synchronize()
    got = means.cpu().numpy()
    ref_u = oracle_loads(N, phi, Z, c[:, 1:2])[:, 0]
    ref = np.array([[fem.subdomain_mean(N, ref_u[s], **{q: plan.node(k)[q] for q in ("x0", "x1", "y0", "y1")})
                     for k in range(n_nodes)] for s in range(2)])
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
