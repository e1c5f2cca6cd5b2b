"""GPU parity of the mixed-precision path (FP32 Schur factorisation, FP64 residual,
iterative refinement) against the FP64 oracle.

Tolerance after refinement (stated by the target of this path): 1e-8 relative
per result, max_k |u_k - u_k^oracle| / max_k |u_k^oracle| and
|loglik - loglik^oracle| / |loglik^oracle|.
"""
import numpy as np
import pytest

import workload as w
from tests.gpu_common import interior, oracle_eval, oracle_full, rel_err_field, rel_err_scalar, small_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module")
def hdd():
    from paper_1708_02207_gb300 import build, hdd as binding
    build.build()
    return binding


def gpu_eval(hdd, N, leaf, phi, obs, Z, y, sigma, **kw):
    kw.setdefault("precision", hdd.HDD_MIXED_FP32)
    plan = hdd.Plan(N, leaf, phi, obs, sigma, **kw)
    ll, u_obs, st = plan.evaluate(torch.from_numpy(np.ascontiguousarray(Z)).cuda(),
                                  torch.from_numpy(np.ascontiguousarray(y)).cuda())
    torch.cuda.synchronize()
    return ll.cpu().numpy(), u_obs.cpu().numpy(), st.cpu().numpy()


def test_grid33_mixed(hdd):
    cfg = w.CONFIGS["grid33"]
    prob = w.make_problem(cfg, batch=4)
    ll, u, st = gpu_eval(hdd, cfg.N, cfg.leaf, prob.phi, prob.obs, prob.Z, prob.y, cfg.sigma, ir_max_iter=2)
    u_ref, ll_ref = oracle_eval(cfg.N, prob.phi, prob.Z, prob.obs, prob.y, cfg.sigma)
    assert (st == 0).all()
    assert rel_err_field(u, u_ref).max() <= TOL
    assert rel_err_scalar(ll, ll_ref).max() <= TOL


@pytest.mark.parametrize("N,leaf,top", [(65, 4, 0), (129, 8, 0), (129, 8, 2), (50, 5, 1), (257, 16, 0)])
def test_full_field_mixed(hdd, N, leaf, top):
    # 257 with 16 x 16-cell leaves: fronts above the shared-memory limit (tensor-core SYRK)
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=3 if N < 200 else 2, seed=N + top)
    obs = interior(N)
    _, u, st = gpu_eval(hdd, N, leaf, phi, obs, Z, np.zeros(obs.size), 0.1, ir_max_iter=3, fp64_top_levels=top)
    ref = oracle_full(N, phi, Z)[:, obs]
    assert (st == 0).all()
    assert rel_err_field(u, ref).max() <= TOL


@pytest.mark.parametrize("fuse", [4, 5])
def test_fused_subtrees_mixed(hdd, fuse):
    N = 129
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=2, seed=77)
    obs = interior(N)
    _, u, st = gpu_eval(hdd, N, 4, phi, obs, Z, np.zeros(obs.size), 0.1, ir_max_iter=2, fuse_height=fuse)
    ref = oracle_full(N, phi, Z)[:, obs]
    assert (st == 0).all()
    assert rel_err_field(u, ref).max() <= TOL


def test_refinement_contracts(hdd):
    # each refinement step multiplies the error by the contraction factor of the
    # FP32 factorisation; no refinement leaves an FP32-sized error
    N = 129
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=2, seed=7)
    obs = w.obs_vertices(N, 8)
    ref, _ = oracle_eval(N, phi, Z, obs, np.zeros(obs.size), 0.1)
    errs = []
    for K in (0, 1, 2, 3):
        _, u, _ = gpu_eval(hdd, N, 8, phi, obs, Z, np.zeros(obs.size), 0.1, ir_max_iter=K, ir_tol=1.0)
        errs.append(rel_err_field(u, ref).max())
    assert 1e-9 < errs[0] < 1e-3
    assert errs[1] < 0.1 * errs[0] and errs[2] < 0.1 * errs[1]
    assert errs[3] <= TOL


def test_no_convergence_is_flagged(hdd):
    N = 33
    phi, Z = small_problem(N, batch=2, seed=9)
    obs = w.obs_vertices(N, 3)
    ll, _, st = gpu_eval(hdd, N, 8, phi, obs, Z, np.zeros(obs.size), 0.1, ir_max_iter=1, ir_tol=0.0)
    assert ((st & 0xFF) == -hdd.HDD_ENOCONV).all() and np.isneginf(ll).all()


def test_grid513_full_batch_mixed_sampled(hdd):
    cfg = w.CONFIGS["grid513"]
    prob = w.make_problem(cfg)
    plan = hdd.Plan(cfg.N, cfg.leaf, prob.phi, prob.obs, cfg.sigma, precision=hdd.HDD_MIXED_FP32, ir_max_iter=2)
    ll, u, st = plan.evaluate(torch.from_numpy(prob.Z).cuda(), torch.from_numpy(prob.y).cuda())
    ll, u, st = ll.cpu().numpy(), u.cpu().numpy(), st.cpu().numpy()
    torch.cuda.empty_cache()
    assert (st == 0).all()
    samples = [0, 128, 255]
    u_ref, ll_ref = oracle_eval(cfg.N, prob.phi, prob.Z[samples], prob.obs, prob.y, cfg.sigma)
    assert rel_err_field(u[samples], u_ref).max() <= TOL
    assert rel_err_scalar(ll[samples], ll_ref).max() <= TOL


def test_double_float_assembly_matches_fp64_exp(hdd):
    # mixed plans form kappa = exp(Phi Z) in double-float arithmetic; compare with
    # the FP64 plan's kappa (CUDA's FP64 exp) entry by entry, and check overflow
    N = 65
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=3, seed=21)
    Z = Z.copy()
    Z[2] *= 900.0 / np.abs(phi @ Z[2]).max()        # |q| up to 900: kappa overflows / underflows
    obs = w.obs_vertices(N, 4)
    Zd = torch.from_numpy(Z).cuda()
    ks = []
    for prec in (hdd.HDD_FP64, hdd.HDD_MIXED_FP32):
        plan = hdd.Plan(N, 4, phi, obs, 0.1, precision=prec)
        ws = plan.workspace(3)
        plan.assemble(Zd, ws)
        k = torch.empty(3, 2 * (N - 1) ** 2, dtype=torch.float64, device="cuda")
        plan.kappa(3, ws, k)
        ks.append(k.cpu().numpy())
    k64, kdf = ks
    # double-float arithmetic carries ~48 bits (unit 2^-48 = 3.6e-15).  The error of
    # q is bounded by ~2 n_z 2^-48 sum_k |Phi_tk Z_k|, which is also the relative error
    # it causes in exp(q); the table-driven exp (2^(j/16) pairs, a degree-6 series, the
    # product of the two) adds a few units more.
    u = 2.0 ** -48
    for s in range(3):
        q = phi @ Z[s]
        fin = np.abs(q) < 700.0
        bound = 2 * phi.shape[1] * u * (np.abs(phi) @ np.abs(Z[s])) + 16 * u
        rel = np.abs(kdf[s][fin] - k64[s][fin]) / k64[s][fin]
        assert (rel <= bound[fin]).all()
        if s < 2:
            assert rel.max() <= 1e-12 and np.median(rel) <= 2e-14
    q2 = phi @ Z[2]
    assert np.isinf(kdf[2][q2 > 710.0]).all() and np.isinf(k64[2][q2 > 710.0]).all()
    assert (kdf[2][q2 < -750.0] == 0.0).all()


def test_bounded_wait_runs_out_and_flags_only_its_sample(hdd):
    # The tensor-core Schur update waits on shared-memory barriers for its operand
    # copies.  The plan's test hook withholds the copies of one operand chunk of one
    # (node, sample), so that wait is certain to run out after the given number of polls
    # (every other wait of the launch has the same bound and completes well within it):
    # the sample must read HDD_ETIMEOUT at that node with loglik = -inf, and every other
    # sample must still match the oracle.  Nothing faults or hangs: the kernel drains
    # what it issued and returns.
    N, leaf = 129, 8
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=3, seed=21)
    obs = w.obs_vertices(N, 8)
    y = np.zeros(obs.size)
    plan = hdd.Plan(N, leaf, phi, obs, 0.1, precision=hdd.HDD_MIXED_FP32, ir_max_iter=3)
    n_nodes = plan.info()["n_nodes"]
    # a front on the tensor-core path (more than 128 rows, boundary rows) with at least
    # two 8-column operand chunks
    node = next(k for k in range(n_nodes)
                if plan.node(k)["m"] + plan.node(k)["b"] + 1 > 128 and plan.node(k)["b"] > 0
                and plan.node(k)["m"] > 8)
    Zt = torch.from_numpy(Z).cuda()
    yt = torch.from_numpy(y).cuda()
    plan.set_wait_bound(1 << 16, node, 1)
    ll, u, st = (t.cpu().numpy() for t in plan.evaluate(Zt, yt))
    assert st[1] & 0xFF == -hdd.HDD_ETIMEOUT and st[1] >> 8 == node
    assert np.isneginf(ll[1])
    u_ref, ll_ref = oracle_eval(N, phi, Z, obs, y, 0.1)
    ok = [0, 2]
    assert (st[ok] == 0).all()
    assert rel_err_field(u[ok], u_ref[ok]).max() <= TOL
    assert rel_err_scalar(ll[ok], ll_ref[ok]).max() <= TOL
    # back to the default bound: the same plan evaluates every sample again
    plan.set_wait_bound()
    ll, u, st = (t.cpu().numpy() for t in plan.evaluate(Zt, yt))
    assert (st == 0).all()
    assert rel_err_field(u, u_ref).max() <= TOL
