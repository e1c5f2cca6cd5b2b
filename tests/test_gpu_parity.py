"""GPU parity of the FP64 HDD path against the FP64 oracle, through the C ABI.

Tolerance (stated by the target of this path): 1e-11 relative per result, i.e.
max_k |u_k - u_k^oracle| / max_k |u_k^oracle| <= 1e-11 for the solution at the
observation vertices and |loglik - loglik^oracle| / |loglik^oracle| <= 1e-11.
The oracle reference is refined once with a long-double residual, so the error
measured is the GPU path's.
"""
import numpy as np
import pytest

import workload as w
from oracle import fem
from tests.gpu_common import interior, oracle_eval, oracle_full, rel_err_field, rel_err_scalar, small_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def hdd():
    from paper_1708_02207_gb300 import build, hdd as binding
    build.build()
    assert torch.cuda.is_available()
    return binding


def gpu_eval(hdd, N, leaf, phi, obs, Z, y, sigma, **kw):
    plan = hdd.Plan(N, leaf, phi, obs, sigma, **kw)
    Zd = torch.from_numpy(np.ascontiguousarray(Z)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    ll, u_obs, st = plan.evaluate(Zd, yd)
    torch.cuda.synchronize()
    return ll.cpu().numpy(), u_obs.cpu().numpy(), st.cpu().numpy()


def test_grid33_workload(hdd):
    # 33 x 33, 8 x 8-cell leaves (depth 4), 10 KL terms, 3 x 3 observations
    cfg = w.CONFIGS["grid33"]
    prob = w.make_problem(cfg)
    ll, u, st = gpu_eval(hdd, cfg.N, cfg.leaf, prob.phi, prob.obs, prob.Z, prob.y, cfg.sigma)
    u_ref, ll_ref = oracle_eval(cfg.N, prob.phi, prob.Z, prob.obs, prob.y, cfg.sigma)
    assert (st == 0).all()
    assert rel_err_field(u, u_ref).max() <= TOL
    assert rel_err_scalar(ll, ll_ref).max() <= TOL


@pytest.mark.parametrize("N,leaf", [(33, 8), (65, 4), (129, 8), (50, 5), (9, 1), (17, 2)])
def test_full_field_every_vertex(hdd, N, leaf):
    # observations at every unknown: the pruned descent becomes the full descent and
    # the whole FE solution is compared element by element (129: fronts above the
    # shared-memory limit take the POTRF/TRSM/SYRK path; 50: unbalanced tree)
    phi, Z = small_problem(N, batch=3, seed=N)
    obs = interior(N)
    y = np.zeros(obs.size)
    _, u, st = gpu_eval(hdd, N, leaf, phi, obs, Z, y, 0.1)
    ref = oracle_full(N, phi, Z)[:, obs]
    assert (st == 0).all()
    assert rel_err_field(u, ref).max() <= TOL


@pytest.mark.parametrize("N,leaf,fuse", [(65, 4, 4), (129, 4, 5), (129, 8, 2)])
def test_fused_subtrees_full_field(hdd, N, leaf, fuse):
    # bottom subtrees eliminated by one CTA each (Schur complements on chip)
    phi, Z = small_problem(N, batch=2, seed=N + fuse)
    obs = interior(N)
    _, u, st = gpu_eval(hdd, N, leaf, phi, obs, Z, np.zeros(obs.size), 0.1, fuse_height=fuse)
    ref = oracle_full(N, phi, Z)[:, obs]
    assert (st == 0).all()
    assert rel_err_field(u, ref).max() <= TOL


def test_leaf_size_invariance(hdd):
    # the Schur complement onto a separator does not depend on the elimination order
    N = 65
    phi, Z = small_problem(N, batch=2, seed=3)
    obs = w.obs_vertices(N, 7)
    y = np.zeros(obs.size)
    res = [gpu_eval(hdd, N, leaf, phi, obs, Z, y, 0.1)[1] for leaf in (1, 2, 4, 8, 16, 32, 64)]
    for u in res[1:]:
        assert rel_err_field(u, res[0]).max() <= 1e-12


def test_alone_equals_in_batch_and_deterministic(hdd):
    N = 65
    phi, Z = small_problem(N, batch=6, seed=4)
    obs = w.obs_vertices(N, 5)
    y = np.zeros(obs.size)
    ll_b, u_b, _ = gpu_eval(hdd, N, 4, phi, obs, Z, y, 0.1)
    ll_b2, u_b2, _ = gpu_eval(hdd, N, 4, phi, obs, Z, y, 0.1)
    assert np.array_equal(u_b, u_b2) and np.array_equal(ll_b, ll_b2)
    for s in (0, 3, 5):
        ll_1, u_1, _ = gpu_eval(hdd, N, 4, phi, obs, Z[s:s + 1], y, 0.1)
        assert np.array_equal(u_1[0], u_b[s]) and ll_1[0] == ll_b[s]


def test_evaluate_host_matches_device(hdd):
    cfg = w.CONFIGS["grid33"]
    prob = w.make_problem(cfg, batch=4)
    plan = hdd.Plan(cfg.N, cfg.leaf, prob.phi, prob.obs, cfg.sigma)
    ws = plan.workspace(4)
    ll_h, u_h, st_h = plan.evaluate_host(prob.Z, prob.y, ws)
    ll_d, u_d, st_d = plan.evaluate(torch.from_numpy(prob.Z).cuda(), torch.from_numpy(prob.y).cuda(), ws)
    assert np.array_equal(ll_h, ll_d.cpu().numpy()) and np.array_equal(u_h, u_d.cpu().numpy())
    # per-sample data y
    Y = np.stack([prob.y, prob.y + 0.01, prob.y, prob.y - 0.02])
    ll_y, _, _ = plan.evaluate_host(prob.Z, Y, ws)
    assert ll_y[0] == ll_h[0] and ll_y[2] == ll_h[2] and ll_y[1] != ll_h[1]


def test_non_spd_sample_is_flagged_not_trapped(hdd):
    # kappa = exp(q) overflows for |q| ~ 800: the sample is marked HDD_ENOTSPD with
    # loglik = -inf; the other samples and the context are unaffected
    N = 33
    phi, Z = small_problem(N, batch=3, seed=5)
    Z = Z.copy()
    Z[1] *= 800.0 / np.abs(phi @ Z[1]).max()
    obs = w.obs_vertices(N, 3)
    y = np.zeros(obs.size)
    ll, u, st = gpu_eval(hdd, N, 8, phi, obs, Z, y, 0.1)
    assert st[0] == 0 and st[2] == 0
    assert (st[1] & 0xFF) == -hdd.HDD_ENOTSPD
    assert ll[1] == -np.inf and np.isfinite(ll[[0, 2]]).all()
    u_ref, _ = oracle_eval(N, phi, Z[[0, 2]], obs, y, 0.1)
    assert rel_err_field(u[[0, 2]], u_ref).max() <= TOL


def _full_size(hdd, name, samples):
    cfg = w.CONFIGS[name]
    prob = w.make_problem(cfg)
    plan = hdd.Plan(cfg.N, cfg.leaf, prob.phi, prob.obs, cfg.sigma)
    need = plan.workspace_size(cfg.batch)
    free, _ = torch.cuda.mem_get_info()
    assert need < 0.9 * free, f"workspace {need / 1e9:.1f} GB does not fit"
    ws = plan.workspace(cfg.batch)
    ll, u, st = plan.evaluate(torch.from_numpy(prob.Z).cuda(), torch.from_numpy(prob.y).cuda(), ws)
    ll, u, st = ll.cpu().numpy(), u.cpu().numpy(), st.cpu().numpy()
    del ws
    torch.cuda.empty_cache()
    assert (st == 0).all() and np.isfinite(ll).all()
    u_ref, ll_ref = oracle_eval(cfg.N, prob.phi, prob.Z[samples], prob.obs, prob.y, cfg.sigma)
    return rel_err_field(u[samples], u_ref), rel_err_scalar(ll[samples], ll_ref)


def test_grid257_full_batch_sampled(hdd):
    # 257 x 257, 16 x 16-cell leaves, 1024 samples, 8 x 8 observations; the oracle
    # checks three samples of the full launch
    eu, el = _full_size(hdd, "grid257", [0, 511, 1023])
    assert eu.max() <= TOL and el.max() <= TOL


def test_grid513_full_batch_sampled(hdd):
    # 513 x 513, 4 x 4-cell leaves, 256 samples, 16 x 16 observations
    eu, el = _full_size(hdd, "grid513", [0, 255])
    assert eu.max() <= TOL and el.max() <= TOL
