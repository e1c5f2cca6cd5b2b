"""Pins of the tree functionals of the oracle (oracle/functionals.py; Sec. 5.1 Lemma, Sec. 5.2).

The recursion is checked against the functional's definition on each node's own triangles,
the functional applied to the data of a solution against the mean of that solution
(Eq. mean, itself pinned in test_oracle_fem), one cell against the paper's initialisation
of a triangle leaf, and the root against the self-adjoint identity lambda^f = u(f=1) / |Omega|.
"""
import numpy as np
import pytest

from oracle import fem
from oracle import functionals as fn
from oracle.hdd_dense import build_tree


def _kappa(N, seed, amp=1.0):
    return np.exp(amp * np.random.default_rng(seed).standard_normal(2 * (N - 1) ** 2))


@pytest.mark.parametrize("N,leaf", [(17, 4), (21, 3), (13, 2)])
def test_recursion_equals_definition(N, leaf):
    kap = _kappa(N, N + leaf, 1.5)
    nodes, lam = fn.mean_functionals_by_recursion(N, kap, leaf)
    for k, nd in enumerate(nodes):
        g_def, f_def = fn.mean_functional_by_definition(N, kap, nd)
        g_rec, f_rec = lam[k]
        scale = max(1e-300, np.abs(np.concatenate([g_def, f_def])).max())
        assert np.abs(g_rec - g_def).max(initial=0.0) <= 1e-12 * scale, k
        assert np.abs(f_rec - f_def).max(initial=0.0) <= 1e-12 * scale, k


def test_functional_of_a_solution_is_its_mean():
    # Eq. prop1 applied to the data of the FE solution of a random load gives Eq. mean
    N, leaf = 17, 4
    kap = _kappa(N, 3, 1.0)
    c = np.random.default_rng(4).random(N * N) / (N - 1) ** 2
    u = fem.solve_load(N, kap, c)
    nodes, lam = fn.mean_functionals_by_recursion(N, kap, leaf)
    for k, nd in enumerate(nodes):
        got = fn.apply_functional(N, nd, lam[k][0], lam[k][1], u, c)
        ref = fem.subdomain_mean(N, u, nd.x0, nd.x1, nd.y0, nd.y1)
        assert abs(got - ref) <= 1e-12 * np.abs(u).max(), k


def test_one_cell_is_the_average_of_its_triangles_initial_vectors():
    # Sec. 5.2 starts a triangle leaf from lambda^g = (1/3, 1/3, 1/3), lambda^f = 0; a cell is two
    # triangles of equal area, so its vector is their average: 1/3 at the two corners on the
    # diagonal, 1/6 at the other two (here the corners that are unknowns)
    N = 6
    nodes = build_tree(N, 1)
    kap = _kappa(N, 5)
    for nd in nodes:
        if not nd.leaf:
            continue
        i, j = nd.x0, nd.y0
        lam_g, lam_f = fn.mean_functional_by_definition(N, kap, nd)
        assert lam_f.size == 0
        expect = {j * N + i: 1 / 3, (j + 1) * N + i + 1: 1 / 3, j * N + i + 1: 1 / 6, (j + 1) * N + i: 1 / 6}
        for a, v in enumerate(nd.bnd):
            assert abs(lam_g[a] - expect[v]) < 1e-15


def test_root_functional_is_the_unit_load_solution():
    # the mean over Omega is (w, u) / |Omega| with w the f = 1 vertex-quadrature load, so by
    # symmetry of A its load vector is A^-1 w / |Omega| = u(f = 1) (|Omega| = 1)
    N = 17
    kap = _kappa(N, 6, 1.0)
    nodes, lam = fn.mean_functionals_by_recursion(N, kap, 4)
    lam_g, lam_f = lam[0]
    assert lam_g.size == 0
    u1 = fem.solve_full(N, kap, 1.0)
    ref = u1[fn.interior_unknowns(N, nodes[0])]
    assert np.abs(lam_f - ref).max() <= 1e-12 * np.abs(ref).max()
