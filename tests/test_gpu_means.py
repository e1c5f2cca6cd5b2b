"""GPU parity of subdomain-mean observations through the mean functionals of Sec. 5.1-5.2.

A plan with obs_kind = HDD_OBS_MEANS observes the mean of u over tree nodes (Eq. mean).  The
library descends only to the observed nodes' ancestors and builds, leaves to root through the
stored factors, the vectors of the Lemma of Sec. 5.1: lambda^g over each node's boundary
unknowns and mu^f = (lambda^f, c) for the load c.  Checked against the oracle:
  * lambda^g of every node and (lambda^f, c) against oracle/functionals.py (the recursion of
    the Lemma, itself pinned against the definition on each node's own triangles);
  * the means against Eq. mean of the oracle's global solution (oracle/fem.py), and the
    log-likelihood of those means.
Tolerances: 1e-11 relative on FP64 plans, 1e-8 after refinement on mixed plans (per result,
relative to the largest value of the quantity).
"""
import numpy as np
import pytest

from oracle import fem
from oracle import functionals as fn
from tests.gpu_common import small_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hdd():
    from paper_1708_02207_gb300 import build, hdd as binding
    build.build()
    return binding


def oracle_means(N, phi, Z, nodes_xy):
    """Eq. mean of the oracle's (refined) global solution over each rectangle, per sample."""
    out = []
    for z in np.atleast_2d(Z):
        u = fem.solve_full(N, fem.kappa_from_kl(phi, z), refine=True)
        out.append([fem.subdomain_mean(N, u, *r) for r in nodes_xy])
    return np.array(out)


def rects(plan, ids):
    return [(plan.node(int(k))["x0"], plan.node(int(k))["x1"], plan.node(int(k))["y0"], plan.node(int(k))["y1"])
            for k in ids]


def run(hdd, N, leaf, phi, Z, ids, y, sigma, **kw):
    plan = hdd.Plan(N, leaf, phi, ids, sigma, obs_kind=hdd.HDD_OBS_MEANS, **kw)
    B = Z.shape[0]
    ws = plan.workspace(B)
    ll, m, st = plan.evaluate(torch.from_numpy(np.ascontiguousarray(Z)).cuda(),
                              torch.from_numpy(np.ascontiguousarray(y)).cuda(), ws=ws)
    lam, mu = plan.mean_functionals(B, ws)
    torch.cuda.synchronize()
    return plan, ll.cpu().numpy(), m.cpu().numpy(), st.cpu().numpy(), lam.cpu().numpy(), mu.cpu().numpy()


@pytest.mark.parametrize("N,leaf", [(17, 4), (33, 8), (30, 5)])
def test_fp64_functionals_of_every_node(hdd, N, leaf):
    # every node observed: lambda^g, mu^f and the mean of each node against the oracle
    phi, Z = small_problem(N, n_z=10, corr_len=0.3, variance=1.5, batch=2, seed=N)
    n_nodes = hdd.Plan(N, leaf, None, np.array([1], dtype=np.int32), 0.1, device=-1,
                       obs_kind=hdd.HDD_OBS_MEANS).info()["n_nodes"]
    ids = np.arange(n_nodes, dtype=np.int32)
    y = np.zeros(n_nodes)
    plan, ll, m, st, lam, mu = run(hdd, N, leaf, phi, Z, ids, y, 0.05)
    assert (st == 0).all()
    h2 = 1.0 / (N - 1) ** 2
    for s, z in enumerate(Z):
        kap = fem.kappa_from_kl(phi, z)
        onodes, olam = fn.mean_functionals_by_recursion(N, kap, leaf)
        assert len(onodes) == n_nodes
        off = 0
        for k, nd in enumerate(onodes):
            info = plan.node(k)
            assert (info["x0"], info["x1"], info["y0"], info["y1"]) == (nd.x0, nd.x1, nd.y0, nd.y1)
            g_ref, f_ref = olam[k]
            b = len(nd.bnd)
            scale = max(np.abs(g_ref).max(initial=0.0), np.abs(f_ref).max(initial=0.0))
            assert np.abs(lam[s, off:off + b] - g_ref).max(initial=0.0) <= 1e-11 * scale, k
            mu_ref = f_ref.sum() * h2   # (lambda^f, c) with c = h^2 f, f = 1, at the unknowns inside
            assert abs(mu[s, k] - mu_ref) <= 1e-11 * max(abs(mu_ref), 1e-300) + 1e-14 * np.abs(mu[s]).max(), k
            off += b
    ref = oracle_means(N, phi, Z, rects(plan, ids))
    assert np.abs(m - ref).max() <= 1e-11 * np.abs(ref).max()
    ll_ref = np.array([fem.loglik(r, y, 0.05) for r in ref])
    assert np.abs(ll - ll_ref).max() <= 1e-11 * np.abs(ll_ref).max()


def test_sixteen_cells_and_the_domain(hdd):
    # Sec. 5, Example (16 subdomains, "cells"): the means of the 16 nodes at depth 4 of the
    # 33 x 33 tree, plus the mean over Omega itself (its functional has no boundary part)
    N, leaf = 33, 4
    phi, Z = small_problem(N, n_z=10, corr_len=0.3, variance=1.0, batch=3, seed=5)
    probe = hdd.Plan(N, leaf, None, np.array([0], dtype=np.int32), 0.1, device=-1, obs_kind=hdd.HDD_OBS_MEANS)
    cells = probe.nodes_at_depth(4)
    assert cells.size == 16
    ids = np.concatenate([cells, [0]]).astype(np.int32)
    rng = np.random.default_rng(1)
    y = rng.random(ids.size) * 0.01
    plan, ll, m, st, _, _ = run(hdd, N, leaf, phi, Z, ids, y, 0.01)
    assert (st == 0).all()
    ref = oracle_means(N, phi, Z, rects(plan, ids))
    assert np.abs(m - ref).max() <= 1e-11 * np.abs(ref).max()
    ll_ref = np.array([fem.loglik(r, y, 0.01) for r in ref])
    assert np.abs(ll - ll_ref).max() <= 1e-11 * np.abs(ll_ref).max()
    # the descent visits only the ancestors of the 16 cells (depths 0..3) and the root
    info = plan.info()
    visited = [k for k in range(info["n_nodes"]) if plan.node(k)["visited"]]
    assert visited and max(plan.node(k)["depth"] for k in visited) <= 3


def test_root_only(hdd):
    N, leaf = 33, 8
    phi, Z = small_problem(N, n_z=10, batch=2, seed=3)
    ids = np.array([0], dtype=np.int32)
    plan, _, m, st, _, mu = run(hdd, N, leaf, phi, Z, ids, np.zeros(1), 0.1)
    ref = oracle_means(N, phi, Z, rects(plan, ids))
    assert (st == 0).all()
    assert np.abs(m - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.allclose(m[:, 0], mu[:, 0], rtol=1e-15, atol=0)   # g = 0 on d Omega


@pytest.mark.parametrize("N,leaf,K,top", [(65, 4, 2, 0), (129, 8, 3, 0), (129, 8, 2, 2), (257, 16, 3, 0)])
def test_mixed_refined_means(hdd, N, leaf, K, top):
    # mixed plans: Eq. mean of the refined iterate + the functional of the last correction;
    # 257 with 16 x 16-cell leaves has tensor-core fronts
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=2, seed=N + K)
    probe = hdd.Plan(N, leaf, None, np.array([0], dtype=np.int32), 0.1, device=-1, obs_kind=hdd.HDD_OBS_MEANS)
    d = min(6, probe.info()["depth"] - 1)
    ids = np.concatenate([probe.nodes_at_depth(d), probe.nodes_at_depth(2)]).astype(np.int32)
    y = np.zeros(ids.size)
    plan, ll, m, st, _, _ = run(hdd, N, leaf, phi, Z, ids, y, 0.1, precision=hdd.HDD_MIXED_FP32, ir_max_iter=K,
                                fp64_top_levels=top)
    assert (st == 0).all()
    ref = oracle_means(N, phi, Z, rects(plan, ids))
    assert np.abs(m - ref).max() <= 1e-8 * np.abs(ref).max()


def test_mixed_without_refinement_is_fp32_accurate(hdd):
    N, leaf = 65, 4
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=2, seed=8)
    probe = hdd.Plan(N, leaf, None, np.array([0], dtype=np.int32), 0.1, device=-1, obs_kind=hdd.HDD_OBS_MEANS)
    ids = probe.nodes_at_depth(4)
    plan, _, m, st, _, _ = run(hdd, N, leaf, phi, Z, ids, np.zeros(ids.size), 0.1,
                               precision=hdd.HDD_MIXED_FP32, ir_max_iter=0)
    ref = oracle_means(N, phi, Z, rects(plan, ids))
    err = np.abs(m - ref).max() / np.abs(ref).max()
    assert (st == 0).all() and 1e-12 < err < 1e-4
