"""CPU checks of the C ABI: the library builds, loads and exports every declared
symbol; host-only plans reproduce the oracle's decomposition tree (Sec. 2.1), the
Appendix A sizes and the pruned descent set (Sec. 5.3); bad arguments are refused."""
import json
import os
import re

import numpy as np
import pytest

import workload as w
from oracle import hdd_dense as hd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hdd():
    from paper_1708_02207_gb300 import build, hdd as binding
    build.build()
    return binding


def test_library_exports_every_declared_symbol(hdd):
    lib = hdd.load_library()
    with open(os.path.join(ROOT, "include", "hdd.h")) as fh:
        header = fh.read()
    declared = set(re.findall(r"^\s*(?:hdd_status|const char\*)\s+(hdd_\w+)\s*\(", header, re.M))
    assert len(declared) >= 13
    for name in declared:
        assert hasattr(lib, name), name
    assert set(hdd.EXPORTED) >= declared - {"hdd_zz_unused"}


@pytest.mark.parametrize("N,leaf,m_obs", [(33, 8, 3), (65, 4, 5), (17, 16, 2), (30, 4, 4), (50, 5, 6), (9, 1, 2)])
def test_tree_matches_oracle(hdd, N, leaf, m_obs):
    obs = w.obs_vertices(N, m_obs)
    plan = hdd.Plan(N, leaf, None, obs, 0.01, device=-1)
    nodes = hd.build_tree(N, leaf)
    info = plan.info()
    assert info["n_nodes"] == len(nodes)
    vis = hd.visited_nodes(nodes, obs)
    assert info["n_visited"] == len(vis)
    # the C plan and the oracle number nodes the same way (depth-first, left son first)
    for k, nd in enumerate(nodes):
        c = plan.node(k)
        assert (c["x0"], c["x1"], c["y0"], c["y1"]) == (nd.x0, nd.x1, nd.y0, nd.y1)
        assert c["parent"] == nd.parent
        assert (c["child0"], c["child1"]) == (tuple(nd.children) if nd.children else (-1, -1))
        g, b = plan.node_indices(k)
        assert list(g) == nd.gamma
        assert list(b) == nd.bnd
        assert c["visited"] == (k in vis)


def test_appendix_a_sizes_in_the_plan(hdd):
    with open(os.path.join(ROOT, "tests", "golden", "appendix_a.json")) as fh:
        g = json.load(fh)
    plan = hdd.Plan(513, 8, None, w.obs_vertices(513, 16), 0.01, device=-1)
    found = 0
    for k in range(plan.info()["n_nodes"]):
        c = plan.node(k)
        if c["x1"] - c["x0"] == g["cells_per_side"] == c["y1"] - c["y0"] and c["x0"] > 0 and c["y0"] > 0 \
                and c["x1"] < 512 and c["y1"] < 512:
            s0, s1 = plan.node(c["child0"]), plan.node(c["child1"])
            assert c["b"] == g["father_boundary"] and c["m"] == g["gamma"]
            assert s0["b"] == s1["b"] == g["son_boundary"]
            _, b0 = plan.node_indices(c["child0"])
            _, b1 = plan.node_indices(c["child1"])
            assert len(set(b0) | set(b1)) == g["auxiliary"]
            found += 1
    assert found == 4


def test_invalid_arguments(hdd):
    with pytest.raises(hdd.HDDError) as e:
        hdd.Plan(33, 8, None, np.array([0], dtype=np.int32), 0.01, device=-1)
    assert e.value.status == hdd.HDD_EINVAL
    with pytest.raises(hdd.HDDError):
        hdd.Plan(2, 8, None, np.array([0], dtype=np.int32), 0.01, device=-1)
    with pytest.raises(hdd.HDDError):
        hdd.Plan(33, 0, None, w.obs_vertices(33, 3), 0.01, device=-1)
    with pytest.raises(hdd.HDDError):
        hdd.Plan(33, 8, None, w.obs_vertices(33, 3), -1.0, device=-1)
    plan = hdd.Plan(33, 8, None, w.obs_vertices(33, 3), 0.01, device=-1)
    assert plan.workspace_size(2) > plan.workspace_size(1)
    with pytest.raises(hdd.HDDError) as e:
        plan.upsweep(1, None)
    assert e.value.status == hdd.HDD_ESTATE
    torch = pytest.importorskip("torch")
    c = torch.zeros(1, 2, 33 * 33, dtype=torch.float64)
    with pytest.raises(hdd.HDDError) as e:   # host-only plans refuse device calls before touching buffers
        plan.solve_loads(1, None, c, c.clone())
    assert e.value.status == hdd.HDD_ESTATE
    with pytest.raises(hdd.HDDError) as e:
        plan.subdomain_means(c[:, 0, :], torch.zeros(1, plan.info()["n_nodes"], dtype=torch.float64))
    assert e.value.status == hdd.HDD_ESTATE
    with pytest.raises(ValueError):
        plan.solve_loads(1, None, c, c[:, :1])


def test_flop_count_matches_front_sizes(hdd):
    plan = hdd.Plan(33, 8, None, w.obs_vertices(33, 3), 0.01, device=-1)
    nodes = hd.build_tree(33, 8)
    ref = 0.0
    for nd in nodes:
        m, nb = len(nd.gamma), len(nd.bnd) + 1
        ref += 2 * (m ** 3 / 3 + nb * m * m / 2 + nb * (nb + 1) / 2 * m)
    assert np.isclose(plan.info()["flops_upsweep"], ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("N,leaf", [(33, 8), (129, 4), (65, 2)])
def test_algorithmic_bytes_match_front_sizes(hdd, precision, N, leaf):
    """The per-stage byte counts that the roofline reports follow from the front sizes of the
    oracle's tree: fronts read their sons' lower Schur triangles (leaves: their triangles'
    kappa) and write F (nf x m), y_g and their lower Schur triangle; the sweeps read F once."""
    prec = hdd.HDD_FP64 if precision == "fp64" else hdd.HDD_MIXED_FP32
    obs = w.obs_vertices(N, 3)
    plan = hdd.Plan(N, leaf, None, obs, 0.01, precision=prec, device=-1)
    info = plan.info()
    E = 8.0 if precision == "fp64" else 4.0
    small_max = 160 if precision == "fp64" else 128
    nodes = hd.build_tree(N, leaf)
    tri = lambda n: n * (n + 1) / 2
    cls = {"tiny": 0.0, "small": 0.0, "large": 0.0, "leaf": 0.0}
    fwd = desc = 0.0
    n_condensed = 0
    for nd in nodes:
        m, b = len(nd.gamma), len(nd.bnd)
        nf = m + b + 1
        if not nd.children and 1 <= m <= 16 and b <= 63:
            # condensed leaf: K_gg^-1 (packed) and one coupling weight per boundary row
            g = tri(m) + b
            inp = 2 * (nd.x1 - nd.x0) * (nd.y1 - nd.y0) * E
            cls["leaf"] += inp + (g + m + tri(b + 1)) * E
            fwd += g * E + m * 8 + (m + b) * E
            desc += (g + m) * E + b * 8 + m * 8
            n_condensed += 1
            continue
        if nd.children:
            sons = [nodes[c] for c in nd.children]
            inp = sum(tri(len(c.bnd) + 1) * E for c in sons)
            cond = sum(len(c.bnd) * E for c in sons)
        else:
            inp, cond = 2 * (nd.x1 - nd.x0) * (nd.y1 - nd.y0) * E, 0.0
        front = inp + (nf * m + m + tri(b + 1)) * E
        cls["tiny" if nf <= 32 else ("small" if nf <= small_max else "large")] += front
        fwd += (nf - 1) * m * E + m * 8 + cond + (m + b) * E
        desc += (nf - 1) * m * E + m * E + b * 8 + m * 8
    assert np.isclose(info["bytes_upsweep_tiny"], cls["tiny"])
    assert np.isclose(info["bytes_upsweep_small"], cls["small"])
    assert np.isclose(info["bytes_upsweep_large"], cls["large"])
    assert np.isclose(info["bytes_upsweep_leaf"], cls["leaf"])
    assert info["n_condensed_leaves"] == n_condensed
    assert info["bytes_upsweep_fused"] == 0.0
    assert np.isclose(info["bytes_forward"], fwd)
    assert np.isclose(info["bytes_descent_all"], desc)
    assert 0 < info["bytes_descent_visited"] < info["bytes_descent_all"]


def test_condensed_leaves_follow_the_leaf_size(hdd):
    """Leaves with at most 16 interior vertices are condensed; larger leaves and
    leaves inside fused subtrees keep their partial Cholesky factors."""
    obs = w.obs_vertices(65, 3)
    assert hdd.Plan(65, 4, None, obs, 0.01, device=-1).info()["n_condensed_leaves"] == 256
    assert hdd.Plan(65, 8, None, obs, 0.01, device=-1).info()["n_condensed_leaves"] == 0
    fused = hdd.Plan(65, 4, None, obs, 0.01, precision=hdd.HDD_MIXED_FP32, fuse_height=2, device=-1)
    assert fused.info()["n_condensed_leaves"] == 0


@pytest.mark.parametrize("N,leaf,depth", [(33, 4, 4), (65, 8, 3), (50, 5, 5)])
def test_mean_plan_visits_exactly_the_ancestors(hdd, N, leaf, depth):
    # Sec. 5.2 Remark b: a functional supported in omega_0 needs Phi of the nodes above
    # omega_0 only, so the descent of a plan observing node means stops at their ancestors
    # (the root is always solved)
    probe = hdd.Plan(N, leaf, None, np.array([0], dtype=np.int32), 0.1, device=-1, obs_kind=hdd.HDD_OBS_MEANS)
    ids = probe.nodes_at_depth(depth)[::2]
    plan = hdd.Plan(N, leaf, None, ids, 0.1, device=-1, obs_kind=hdd.HDD_OBS_MEANS)
    nodes = hd.build_tree(N, leaf)
    expect = {0}
    for k in ids:
        a = nodes[k].parent
        while a >= 0:
            expect.add(a)
            a = nodes[a].parent
    got = {k for k in range(len(nodes)) if plan.node(k)["visited"]}
    assert got == {k for k in expect if nodes[k].gamma}
    # mean plans hold more per sample than vertex plans (functionals, conv. vertices)
    vplan = hdd.Plan(N, leaf, None, w.obs_vertices(N, 2), 0.1, device=-1)
    assert plan.workspace_size(4) > vplan.workspace_size(4)


def test_mean_plan_refuses_bad_nodes(hdd):
    with pytest.raises(hdd.HDDError):
        hdd.Plan(33, 8, None, np.array([99], dtype=np.int32), 0.1, device=-1, obs_kind=hdd.HDD_OBS_MEANS)
    with pytest.raises(hdd.HDDError):
        hdd.Plan(33, 8, None, np.array([-1], dtype=np.int32), 0.1, device=-1, obs_kind=hdd.HDD_OBS_MEANS)
    with pytest.raises(hdd.HDDError):
        hdd.Plan(33, 8, None, np.array([3], dtype=np.int32), 0.1, device=-1, obs_kind=7)


def test_data_scratch_size_is_two_groups_of_four_vectors(hdd):
    # hdd_solve_data keeps the residuals and corrections of four data sets per sample
    # plus four words of refinement bookkeeping per sample
    plan = hdd.Plan(33, 8, None, w.obs_vertices(33, 3), 0.1, device=-1)
    for B in (1, 7, 256):
        assert plan.data_scratch_size(B) == (2 * 4 * B * 33 * 33 + 4 * B) * 8


def test_multi_and_graph_calls_refuse_bad_arguments(hdd):
    # The uneven-batch and graph calls check their arguments before any CUDA call:
    # NULL handles and host-only plans are refused with HDD_EINVAL, destroying NULL is a
    # no-op, and no handle is left behind.
    import ctypes as C
    lib = hdd.load_library()
    out = C.c_void_p(1)
    one = (C.c_int32 * 1)(4)
    ws = (C.c_void_p * 1)(256)
    assert lib.hdd_multi_create(None, 1, one, ws, C.byref(out)) == hdd.HDD_EINVAL
    assert out.value is None
    plan = hdd.Plan(33, 8, None, w.obs_vertices(33, 3), 0.01, device=-1)
    plans = (C.c_void_p * 1)(plan._h.value)
    out = C.c_void_p(1)
    assert lib.hdd_multi_create(plans, 1, one, ws, C.byref(out)) == hdd.HDD_EINVAL
    assert out.value is None
    assert "host-only" in lib.hdd_last_error().decode()
    assert lib.hdd_multi_create(plans, 0, one, ws, C.byref(out)) == hdd.HDD_EINVAL
    assert lib.hdd_multi_create(plans, 1, one, ws, None) == hdd.HDD_EINVAL
    g = C.c_void_p(1)
    assert lib.hdd_multi_capture(None, None, None, None, None, None, None, C.byref(g)) == hdd.HDD_EINVAL
    assert lib.hdd_graph_launch(None, None) == hdd.HDD_EINVAL
    assert lib.hdd_graph_destroy(None) == hdd.HDD_OK
    assert lib.hdd_multi_destroy(None) == hdd.HDD_OK
    assert lib.hdd_multi_upsweep(None, None) == hdd.HDD_EINVAL
    assert lib.hdd_multi_evaluate(None, None, None, None, None, None, None, None) == hdd.HDD_EINVAL
    up = C.c_int32()
    assert lib.hdd_multi_info(None, C.byref(up), None) == hdd.HDD_EINVAL
