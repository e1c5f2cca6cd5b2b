"""Pins of the dense HDD restatement (oracle/hdd_dense.py).

HDD is exact up to rounding (abstract; end of Sec. 3.4), so its interface values
must equal the global FE solve; the Schur complements must have the properties
of Sec. 2.4 / Sec. 3.2; the tree must reproduce the sizes of Appendix A.
"""
import json
import os

import numpy as np
import pytest

import workload as w
from oracle import fem, hdd_dense as hd


def _kappa(N, seed, amp=1.0):
    rng = np.random.default_rng(seed)
    return np.exp(amp * rng.standard_normal(2 * (N - 1) ** 2))


@pytest.mark.parametrize("N,leaf", [(17, 4), (33, 8), (33, 4), (65, 16)])
def test_hdd_equals_global_solve(N, leaf):
    # T8: values on all gamma (all unknowns) equal the banded Cholesky solution
    kap = _kappa(N, N + leaf, amp=1.5)
    u, nodes, _, _ = hd.solve(N, kap, leaf)
    ref = fem.solve_full(N, kap)
    assert np.max(np.abs(u - ref)) < 1e-12 * np.max(np.abs(ref))
    # every unknown is eliminated exactly once (I(Omega) = union of I(gamma))
    own = [v for nd in nodes for v in nd.gamma]
    assert len(own) == len(set(own)) == (N - 2) ** 2


def test_pruned_descent_equals_full_at_points():
    # Sec. 5.3: "Root to Leaves" restricted to the root-to-point paths
    N, leaf = 33, 4
    kap = _kappa(N, 3)
    obs = w.obs_vertices(N, 3)
    u_full, nodes, _, phi = hd.solve(N, kap, leaf)
    vis = hd.visited_nodes(nodes, obs)
    assert len(vis) < len(nodes)
    u_p = hd.root_to_leaves(N, nodes, phi, vis)
    assert np.array_equal(u_p[obs], u_full[obs])
    assert np.isnan(u_p).sum() > 0


def test_schur_recursion_matches_definition_and_is_spd():
    # Eq. SchurC1 two ways: recursive (Sec. 3.3) vs directly from the node's triangles;
    # T6: symmetric, PSD; S 1 = 0 for a floating node (constants solve the Neumann
    # problem); SPD for nodes touching the Dirichlet boundary; gamma block SPD (Remark on M)
    N, leaf = 33, 4
    kap = _kappa(N, 4, amp=1.0)
    h = 1.0 / (N - 1)
    load = np.full(N * N, h * h)
    nodes = hd.build_tree(N, leaf)
    psi, _ = hd.leaves_to_root(N, kap, load, nodes)
    n_float = 0
    for k, nd in enumerate(nodes):
        S_rec, g_rec = psi[k]
        S_def, g_def = hd.schur_by_definition(N, kap, load, nd)
        if S_def.size == 0:          # the root: no boundary unknowns
            assert S_rec.size == 0
            continue
        assert np.allclose(S_rec, S_def, atol=1e-12 * max(1.0, np.abs(S_def).max()))
        assert np.allclose(g_rec, g_def, atol=1e-12 * max(1e-3, np.abs(g_def).max()))
        assert np.allclose(S_def, S_def.T, atol=1e-13)
        ev = np.linalg.eigvalsh(S_def)
        floating = nd.x0 > 0 and nd.y0 > 0 and nd.x1 < N - 1 and nd.y1 < N - 1
        if floating:
            n_float += 1
            assert np.allclose(S_def @ np.ones(len(nd.bnd)), 0.0, atol=1e-12)
            assert abs(ev[0]) < 1e-12 and ev[1] > 1e-8
        else:
            assert ev[0] > 1e-10
    assert n_float > 0


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def test_appendix_a_sizes():
    # Appendix A: Psi^g of a 512-boundary node built from two 384 x 384 sons
    # through a 639 x 639 auxiliary matrix; |gamma| = 127 (floating 128 x 128 cells)
    g = _golden("appendix_a.json")
    c = g["cells_per_side"]
    nodes = hd.build_tree(513, 8)
    found = 0
    for nd in nodes:
        if nd.x1 - nd.x0 == c and nd.y1 - nd.y0 == c and nd.x0 > 0 and nd.y0 > 0 \
                and nd.x1 < 512 and nd.y1 < 512:
            c1, c2 = (nodes[k] for k in nd.children)
            assert len(nd.bnd) == g["father_boundary"]
            assert len(c1.bnd) == len(c2.bnd) == g["son_boundary"]
            assert len(set(c1.bnd) | set(c2.bnd)) == g["auxiliary"]
            assert len(nd.gamma) == g["gamma"]
            found += 1
    assert found == 4


def test_figure_ex_points_sizes():
    # Fig. ex_points: a floating subdomain with 12 nodes has 10 boundary nodes and 2 interior
    # ones.  The oracle's own tree builds such a subdomain: on the 11 x 11 grid with leaves of
    # at most 3 cells the bisection (Sec. 2.1) leaves floating 2 x 3-cell leaves, whose index
    # sets I(d omega) and I(omega) \ I(d omega) must have the figure's sizes.
    g = _golden("fig_ex_points.json")
    N = 11
    nodes = hd.build_tree(N, 3)
    found = 0
    for nd in nodes:
        floating = nd.x0 > 0 and nd.y0 > 0 and nd.x1 < N - 1 and nd.y1 < N - 1
        if nd.leaf and floating and {nd.x1 - nd.x0, nd.y1 - nd.y0} == {2, 3}:
            assert len(nd.bnd) == g["boundary"] and len(nd.gamma) == g["interior"]
            assert len(set(nd.bnd) | set(nd.gamma)) == g["nodes"]
            # the two interior vertices are the ones off the rectangle's edges
            for v in nd.gamma:
                i, j = v % N, v // N
                assert nd.x0 < i < nd.x1 and nd.y0 < j < nd.y1
            found += 1
    assert found >= 1


def test_tree_shape_rules():
    # 33 x 33 with 8 x 8-cell leaves: 16 leaves, depth 4 (the 33^2 workload)
    nodes = hd.build_tree(33, 8)
    leaves = [nd for nd in nodes if nd.leaf]
    assert len(leaves) == 16 and {nd.depth for nd in leaves} == {4}
    assert nodes[0].split == "x" and nodes[0].cut == 16
    # leaf-size invariance of the answer (T9 on the CPU side)
    kap = _kappa(33, 8)
    u8, *_ = hd.solve(33, kap, 8)
    u4, *_ = hd.solve(33, kap, 4)
    assert np.max(np.abs(u8 - u4)) < 1e-13 * np.max(np.abs(u8))


@pytest.mark.parametrize("N,leaf", [(17, 4), (21, 3), (33, 8), (30, 5)])
def test_leaf_boundary_rows_couple_to_one_interior_vertex(N, leaf):
    # The condensed leaves store K_gg^-1 and one weight per boundary row: on this mesh (each
    # cell cut by its "/" diagonal, hypotenuse couplings zero) a boundary vertex of a leaf
    # rectangle couples to at most one interior vertex, and that weight is the only nonzero
    # of its row of K_Bg.  Corner vertices couple to none.
    rng = np.random.default_rng(N + leaf)
    kap = np.exp(rng.standard_normal(2 * (N - 1) ** 2))
    for nd in hd.build_tree(N, leaf):
        if not nd.leaf:
            continue
        A, ids = hd.local_neumann(N, kap, nd)
        pos = {v: a for a, v in enumerate(ids)}
        bset = set(nd.bnd)
        I = [pos[v] for v in ids if v not in bset]
        for v in nd.bnd:
            row = A[pos[v], I]
            nz = np.flatnonzero(np.abs(row) > 1e-14 * np.abs(A).max())
            assert nz.size <= 1, (nd.x0, nd.y0, v)
            i, j = v % N, v // N
            corner = i in (nd.x0, nd.x1) and j in (nd.y0, nd.y1)
            if corner:
                assert nz.size == 0
