"""Linear functionals of the solution built up the decomposition tree (test infrastructure only).

Sec. 5.1 represents a linear functional of the solution in a subdomain omega by two vectors,
    lambda_omega(d_omega) = (lambda^g_omega, g_omega) + (lambda^f_omega, f_omega)     (Eq. prop1)
with g_omega the values of u on the boundary unknowns of omega and f_omega the load at the
unknowns inside omega, and builds them for a father from its sons (Eq. prop2 and the Lemma of
Sec. 5.1; the two algorithms of Sec. 5.2):
    z            = c_1 lambda^g_1 |gamma + c_2 lambda^g_2 |gamma
    lambda^g     = c_1 lambda^g_1 |^Gamma + c_2 lambda^g_2 |^Gamma + (Phi^g_omega)^T z
    lambda^f     = c_1 lambda^f_1 |^omega + c_2 lambda^f_2 |^omega + (Phi^f_omega)^T z
where u_gamma = Phi^g_omega g_omega + Phi^f_omega f_omega is the interface solution of omega.
The functional here is the mean value over omega (Sec. 5, Eq. mean), with c_i = |omega_i| / |omega|.

Two routes, small grids only (dense matrices):
  * by definition: the local problem of omega over its own triangles,
    K_II u_I = f_I - K_IB g_B, and Eq. mean, sum_v w_v u_v / |omega| with w_v = sum over the
    triangles t of omega at v of |t|/3, give
        lambda^f = K_II^-1 w_I / |omega|,   lambda^g = (w_B - K_BI K_II^-1 w_I) / |omega|;
  * by recursion, following the steps above, with Phi^g, Phi^f of every father from its own
    local problem (u_gamma is the gamma part of u_I) and the leaves' vectors by definition.

Readings: the paper's leaves are single triangles, initialised with lambda^g = (1/3, 1/3, 1/3)
and lambda^f = 0; the leaves here are rectangles of cells, started from the definition (a test
checks that one cell gives the average of its two triangles' initial vectors).  Boundary
vertices of the domain carry Dirichlet data g = 0 and have no entries.
"""
from __future__ import annotations

import numpy as np

from . import fem
from .hdd_dense import build_tree, heights, local_neumann


def interior_unknowns(N: int, nd) -> list:
    """Unknowns strictly inside the node's rectangle (the index set of f_omega), ascending."""
    return [j * N + i for j in range(nd.y0 + 1, nd.y1) for i in range(nd.x0 + 1, nd.x1)]


def mean_weights(N: int, nd):
    """Eq. mean for the node's rectangle: {vertex: sum over its triangles t in omega of |t|/3}
    and |omega| (the summed area of those triangles)."""
    coords, tris = fem.mesh(N)
    _, area = fem.element_matrices(coords, tris, np.ones(tris.shape[0]))
    w, total = {}, 0.0
    for j in range(nd.y0, nd.y1):
        for i in range(nd.x0, nd.x1):
            for t in (2 * (j * (N - 1) + i), 2 * (j * (N - 1) + i) + 1):
                total += area[t]
                for v in tris[t]:
                    w[int(v)] = w.get(int(v), 0.0) + area[t] / 3.0
    return w, total


def _local(N, kappa, nd):
    """The node's local stiffness split into interior (I) and boundary (B) unknowns."""
    A, ids = local_neumann(N, kappa, nd)
    pos = {v: a for a, v in enumerate(ids)}
    I_ids = interior_unknowns(N, nd)
    I = [pos[v] for v in I_ids]
    B = [pos[v] for v in nd.bnd]
    return A[np.ix_(I, I)], A[np.ix_(I, B)], I_ids


def mean_functional_by_definition(N: int, kappa: np.ndarray, nd):
    """(lambda^g over nd.bnd, lambda^f over interior_unknowns) of the mean over nd."""
    K_II, K_IB, I_ids = _local(N, kappa, nd)
    w, total = mean_weights(N, nd)
    w_I = np.array([w.get(v, 0.0) for v in I_ids])
    w_B = np.array([w.get(v, 0.0) for v in nd.bnd])
    if not I_ids:
        return w_B / total, np.zeros(0)
    x = np.linalg.solve(K_II, w_I)          # K_II^-1 w_I (K_II symmetric)
    return (w_B - K_IB.T @ x) / total, x / total


def interface_maps(N: int, kappa: np.ndarray, nd):
    """Phi^g (gamma x bnd) and Phi^f (gamma x interior unknowns) of a father: the gamma rows
    of u_I = K_II^-1 (f_I - K_IB g_B) on its own triangles."""
    K_II, K_IB, I_ids = _local(N, kappa, nd)
    rows = [I_ids.index(v) for v in nd.gamma]
    Kinv = np.linalg.inv(K_II)
    return -(Kinv @ K_IB)[rows], Kinv[rows]


def mean_functionals_by_recursion(N: int, kappa: np.ndarray, leaf: int):
    """The vectors of every node of the tree by the recursion of Sec. 5.1-5.2.

    Returns (nodes, lam) with lam[k] = (lambda^g over nodes[k].bnd, lambda^f over
    interior_unknowns(N, nodes[k]))."""
    nodes = build_tree(N, leaf)
    h = heights(nodes)
    area = lambda nd: float((nd.x1 - nd.x0) * (nd.y1 - nd.y0))
    lam = {}
    for k in sorted(range(len(nodes)), key=lambda q: h[q]):
        nd = nodes[k]
        if nd.leaf:
            lam[k] = mean_functional_by_definition(N, kappa, nd)
            continue
        s1, s2 = nd.children
        c = {s1: area(nodes[s1]) / area(nd), s2: area(nodes[s2]) / area(nd)}
        # boundary part: the sons' entries on d omega (the parts Gamma_{omega,1}, Gamma_{omega,2})
        bpos = {v: a for a, v in enumerate(nd.bnd)}
        lg = np.zeros(len(nd.bnd))
        z = np.zeros(len(nd.gamma))
        gpos = {v: a for a, v in enumerate(nd.gamma)}
        for s in (s1, s2):
            lg_s, _ = lam[s]
            for a, v in enumerate(nodes[s].bnd):
                if v in bpos:
                    lg[bpos[v]] += c[s] * lg_s[a]
                if v in gpos:
                    z[gpos[v]] += c[s] * lg_s[a]
        # interior part: the sons' interiors, extended by zero to omega
        I_ids = interior_unknowns(N, nd)
        ipos = {v: a for a, v in enumerate(I_ids)}
        lf = np.zeros(len(I_ids))
        for s in (s1, s2):
            _, lf_s = lam[s]
            for a, v in enumerate(interior_unknowns(N, nodes[s])):
                lf[ipos[v]] += c[s] * lf_s[a]
        # the interface values enter through Phi: (Phi^g)^T z and (Phi^f)^T z
        if nd.gamma:
            Pg, Pf = interface_maps(N, kappa, nd)
            lg += Pg.T @ z
            lf += Pf.T @ z
        lam[k] = (lg, lf)
    return nodes, lam


def apply_functional(N: int, nd, lam_g: np.ndarray, lam_f: np.ndarray, u: np.ndarray, c: np.ndarray) -> float:
    """lambda_omega(d_omega) = (lambda^g, u on the boundary unknowns) + (lambda^f, load inside)."""
    u = np.asarray(u, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    return float(lam_g @ u[nd.bnd] + lam_f @ c[interior_unknowns(N, nd)])
