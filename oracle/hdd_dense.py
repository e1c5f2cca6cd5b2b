"""The HDD method written out densely in NumPy (test infrastructure only).

Small grids only (every map is a dense matrix).  Used by the tests to pin:
  * the decomposition tree and its index sets (Sec. 2.1, Eq. gamma_def; the sizes
    of the Appendix A example, 384 + 384 -> 639 -> 512);
  * the Schur-complement maps of Sec. 2.4 (Eq. SchurMinus1, Eq. SchurC1):
      Psi^g = A11 - A12 A22^{-1} A21,  Psi^f c = F1 c - A12 A22^{-1} F2 c,
      Phi^g = -A22^{-1} A21,           Phi^f c = A22^{-1} F2 c,
    with block 1 = the node's boundary unknowns and block 2 = its interface gamma;
  * the father system of Sec. 3.3 (Eq. block_equation4): the sons' Psi embedded in
    the union of their boundaries and added, the shared gamma block summed;
  * "Leaves to Root" / "Root to Leaves" (Sec. 3.4) and the pruned descent to a
    point (Sec. 5.3): the values on all interfaces equal the global FE solution.

Readings taken where the paper is open:
  * leaves are rectangles of leaf x leaf cells whose interior vertices play the
    role of gamma (the paper's leaves are single triangles; the Schur complement
    onto a separator set does not depend on the elimination order);
  * the load of a vertex enters once, at the node that eliminates it (its gamma or
    leaf interior); a son's condensed right-hand side therefore carries no load of
    its own boundary vertices.  The sum over all nodes is the global load vector,
    so the global system is unchanged;
  * the tree splits the longer side of a node at the cell-aligned midpoint
    (x first on ties) and stops when both sides are at most `leaf` cells;
  * Dirichlet data g = 0: vertices on the boundary of Omega are not unknowns and
    belong to no index set.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import fem


@dataclass
class Node:
    x0: int
    x1: int
    y0: int
    y1: int
    depth: int
    parent: int = -1
    children: tuple = ()
    split: str = ""                      # "x" (vertical line) or "y" (horizontal line)
    cut: int = -1                        # vertex index of the split line
    gamma: list = field(default_factory=list)   # eliminated vertices (interface, or leaf interior)
    bnd: list = field(default_factory=list)     # boundary unknowns I(d omega) minus Dirichlet vertices

    @property
    def leaf(self):
        return not self.children


def _unknown(N, i, j):
    return 1 <= i <= N - 2 and 1 <= j <= N - 2


def build_tree(N: int, leaf: int):
    """Binary decomposition tree of the (N-1)^2-cell square (Sec. 2.1).  Node 0 is Omega."""
    nodes = [Node(0, N - 1, 0, N - 1, 0)]
    stack = [0]
    while stack:
        k = stack.pop()
        nd = nodes[k]
        w, hgt = nd.x1 - nd.x0, nd.y1 - nd.y0
        if w <= leaf and hgt <= leaf:
            continue
        if w >= hgt:
            xm = nd.x0 + w // 2
            kids = [Node(nd.x0, xm, nd.y0, nd.y1, nd.depth + 1, k), Node(xm, nd.x1, nd.y0, nd.y1, nd.depth + 1, k)]
            nd.split, nd.cut = "x", xm
        else:
            ym = nd.y0 + hgt // 2
            kids = [Node(nd.x0, nd.x1, nd.y0, ym, nd.depth + 1, k), Node(nd.x0, nd.x1, ym, nd.y1, nd.depth + 1, k)]
            nd.split, nd.cut = "y", ym
        base = len(nodes)
        nodes.extend(kids)
        nd.children = (base, base + 1)
        stack.extend([base + 1, base])
    for nd in nodes:
        bnd = []
        for j in range(nd.y0, nd.y1 + 1):
            for i in range(nd.x0, nd.x1 + 1):
                on_edge = i in (nd.x0, nd.x1) or j in (nd.y0, nd.y1)
                if on_edge and _unknown(N, i, j):
                    bnd.append(j * N + i)
        nd.bnd = bnd
        if nd.leaf:
            nd.gamma = [j * N + i for j in range(nd.y0 + 1, nd.y1) for i in range(nd.x0 + 1, nd.x1)]
        elif nd.split == "x":
            nd.gamma = [j * N + nd.cut for j in range(nd.y0 + 1, nd.y1)]
        else:
            nd.gamma = [nd.cut * N + i for i in range(nd.x0 + 1, nd.x1)]
    return nodes


def heights(nodes):
    h = [0] * len(nodes)
    for k in sorted(range(len(nodes)), key=lambda k: -nodes[k].depth):
        if nodes[k].children:
            h[k] = 1 + max(h[c] for c in nodes[k].children)
    return h


def local_neumann(N: int, kappa: np.ndarray, nd: Node):
    """Stiffness of the triangles inside the closed rectangle of nd, over its unknowns.

    Returns (A_loc dense, ids) with ids the node's unknown vertices, sorted.
    """
    coords, tris = fem.mesh(N)
    cells = [(i, j) for j in range(nd.y0, nd.y1) for i in range(nd.x0, nd.x1)]
    t_idx = np.array([2 * (j * (N - 1) + i) + s for (i, j) in cells for s in (0, 1)])
    Ke, _ = fem.element_matrices(coords, tris[t_idx], kappa[t_idx])
    ids = sorted({int(v) for v in tris[t_idx].ravel() if _unknown(N, v % N, v // N)})
    pos = {v: a for a, v in enumerate(ids)}
    A = np.zeros((len(ids), len(ids)))
    for e, t in enumerate(tris[t_idx]):
        for a in range(3):
            for b in range(3):
                if t[a] in pos and t[b] in pos:
                    A[pos[t[a]], pos[t[b]]] += Ke[e, a, b]
    return A, ids


def schur_by_definition(N, kappa, load, nd: Node):
    """Psi^g and the condensed load of nd computed directly from its own triangles.

    Eliminates every unknown strictly inside the rectangle (Eq. SchurC1) with the
    load of those vertices; the boundary unknowns carry no load of their own.
    """
    A, ids = local_neumann(N, kappa, nd)
    pos = {v: a for a, v in enumerate(ids)}
    bset = set(nd.bnd)
    I = [pos[v] for v in ids if v not in bset]
    B = [pos[v] for v in nd.bnd]
    rhs_I = np.array([load[v] for v in ids if v not in bset])
    if not I:
        return A[np.ix_(B, B)], np.zeros(len(B))
    X = np.linalg.solve(A[np.ix_(I, I)], np.column_stack([A[np.ix_(I, B)], rhs_I]))
    S = A[np.ix_(B, B)] - A[np.ix_(B, I)] @ X[:, :-1]
    g = -A[np.ix_(B, I)] @ X[:, -1]
    return S, g


def leaves_to_root(N: int, kappa: np.ndarray, load: np.ndarray, nodes):
    """"Leaves to Root" (Sec. 3.4): Psi for every node, Phi stored for every node.

    Returns dicts psi[k] = (Psi^g, Psi^f c) over nodes[k].bnd and
    phi[k] = (Phi^g, Phi^f c) mapping nodes[k].bnd data to nodes[k].gamma.
    """
    psi, phi = {}, {}
    order = sorted(range(len(nodes)), key=lambda k: heights(nodes)[k])
    for k in order:
        nd = nodes[k]
        if nd.leaf:
            A, ids = local_neumann(N, kappa, nd)
            pos = {v: a for a, v in enumerate(ids)}
            J = nd.bnd + nd.gamma                                  # block 1 = boundary, block 2 = gamma
            Aj = A[np.ix_([pos[v] for v in J], [pos[v] for v in J])]
            Fc = np.array([0.0] * len(nd.bnd) + [load[v] for v in nd.gamma])
        else:
            c1, c2 = nd.children
            J = nd.bnd + nd.gamma
            pos = {v: a for a, v in enumerate(J)}
            Aj = np.zeros((len(J), len(J)))
            Fc = np.zeros(len(J))
            for c in (c1, c2):                                     # Eq. block_equation4
                P = [pos[v] for v in nodes[c].bnd]
                Aj[np.ix_(P, P)] += psi[c][0]
                Fc[P] += psi[c][1]
            for v in nd.gamma:
                Fc[pos[v]] += load[v]
        nb = len(nd.bnd)
        A11, A12 = Aj[:nb, :nb], Aj[:nb, nb:]
        A21, A22 = Aj[nb:, :nb], Aj[nb:, nb:]
        F1, F2 = Fc[:nb], Fc[nb:]
        if A22.shape[0]:
            X = np.linalg.solve(A22, np.column_stack([A21, F2]))
            phi_g, phi_f = -X[:, :-1], X[:, -1]                    # Phi^g, Phi^f c
            psi_g = A11 - A12 @ X[:, :-1]                          # Psi^g
            psi_f = F1 - A12 @ X[:, -1]                            # Psi^f c
        else:
            phi_g, phi_f = np.zeros((0, nb)), np.zeros(0)
            psi_g, psi_f = A11, F1
        psi[k] = (psi_g, psi_f)
        phi[k] = (phi_g, phi_f)
    return psi, phi


def owner_map(nodes):
    """Vertex id -> index of the node that eliminates it (its gamma or leaf interior)."""
    own = {}
    for k, nd in enumerate(nodes):
        for v in nd.gamma:
            own[v] = k
    return own


def visited_nodes(nodes, obs):
    """Nodes on the root-to-owner paths of the observation vertices (Sec. 5.3)."""
    own = owner_map(nodes)
    vis = set()
    for v in obs:
        k = own[int(v)]
        while k >= 0 and k not in vis:
            vis.add(k)
            k = nodes[k].parent
    return vis


def root_to_leaves(N: int, nodes, phi, visit=None):
    """"Root to Leaves" (Sec. 3.4): u on gamma of each visited node, u_gamma = Phi(d).

    visit=None descends everywhere (the full solution); otherwise only the given set.
    Returns u at all N*N vertices (NaN where not computed; 0 on the Dirichlet boundary).
    """
    u = np.full(N * N, np.nan)
    for j in range(N):
        for i in range(N):
            if not _unknown(N, i, j):
                u[j * N + i] = 0.0
    order = sorted(range(len(nodes)), key=lambda k: nodes[k].depth)
    for k in order:
        if visit is not None and k not in visit:
            continue
        nd = nodes[k]
        g = np.array([u[v] for v in nd.bnd])
        assert not np.isnan(g).any(), "boundary data not yet known"
        phi_g, phi_f = phi[k]
        u[nd.gamma] = phi_g @ g + phi_f
    return u


def solve(N: int, kappa: np.ndarray, leaf: int, f: float = 1.0, obs=None):
    """Full HDD solve: (u, nodes, psi, phi).  With obs, only the pruned descent runs."""
    nodes = build_tree(N, leaf)
    h = 1.0 / (N - 1)
    load = np.full(N * N, h * h * f)     # vertex quadrature of a constant f on this mesh
    psi, phi = leaves_to_root(N, kappa, load, nodes)
    visit = None if obs is None else visited_nodes(nodes, obs)
    u = root_to_leaves(N, nodes, phi, visit)
    return u, nodes, psi, phi
