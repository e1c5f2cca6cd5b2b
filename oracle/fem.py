"""Plain FP64 P1 finite elements + banded Cholesky (test infrastructure only).

What the HDD path computes, written as its plain definition.  The paper states
that, up to the H-matrix error (absent here: every matrix is dense), HDD returns
the exact FE solution (abstract; end of Sec. 3.4: the values on all interfaces
form the solution of the initial problem).  So the oracle is the global FE solve:

  1. kappa_t = exp(q_t), q_t = sum_k Phi[t,k] Z_k          (notation table, kappa=e^q)
  2. element stiffness A_ij = int_t kappa grad b_i . grad b_j  (Sec. 3.1, Eq. coefA)
     with kappa constant on t: A_ij = kappa_t |t| grad b_i . grad b_j
  3. load by vertex quadrature c_i = sum_t |t|/3 f(x_i)     (Sec. 3.1, Eq. coefc;
     the area factor |omega| of Eq. coefc is kept, Eq. coefF's F = I/3 omits it)
  4. homogeneous Dirichlet data g = 0: boundary vertices are not unknowns
     (Eq. elliptic)
  5. solve A u = c by LAPACK banded Cholesky (bandwidth N-1: the "/" diagonals
     couple (i,j) with (i+1,j+1), N-1 apart in natural order)
  6. restrict u to the observation vertices; Gaussian log-likelihood
     L(z) = prod_i pi_eps(y_i - S_i(z)) (Sec. 1.2) with eps_i ~ N(0, sigma^2):
     log L = -1/2 sum_i (y_i - u_i)^2 / sigma^2 - (n_y/2) log(2 pi sigma^2).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def mesh(N: int):
    """Vertex coordinates [N*N, 2] and triangles [n_t, 3] (vertex ids).

    Vertex (i, j) -> id j*N+i at (i h, j h).  Cell (i, j) is cut by its "/"
    diagonal; triangle 2*(j*(N-1)+i) is the lower-right one (i,j),(i+1,j),(i+1,j+1),
    triangle 2*(j*(N-1)+i)+1 the upper-left one (i,j),(i+1,j+1),(i,j+1).  Both are
    listed counter-clockwise.
    """
    h = 1.0 / (N - 1)
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    coords = np.stack([ii.ravel() * h, jj.ravel() * h], axis=1)
    cj, ci = np.meshgrid(np.arange(N - 1), np.arange(N - 1), indexing="ij")
    ci, cj = ci.ravel(), cj.ravel()
    v00 = cj * N + ci
    v10 = v00 + 1
    v11 = v00 + N + 1
    v01 = v00 + N
    tris = np.empty((2 * ci.size, 3), dtype=np.int64)
    tris[0::2] = np.stack([v00, v10, v11], axis=1)
    tris[1::2] = np.stack([v00, v11, v01], axis=1)
    return coords, tris


def element_matrices(coords: np.ndarray, tris: np.ndarray, kappa: np.ndarray):
    """Per-triangle 3x3 stiffness kappa_t |t| grad b_i . grad b_j and areas |t|.

    grad b_0 = (y1 - y2, x2 - x1) / (2|t|), cyclically for b_1, b_2, with
    2|t| = (p1 - p0) x (p2 - p0) (Eq. coefA for P1 basis functions).
    """
    p0, p1, p2 = coords[tris[:, 0]], coords[tris[:, 1]], coords[tris[:, 2]]
    det = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0])
    area = 0.5 * np.abs(det)
    g = np.empty((tris.shape[0], 3, 2))
    g[:, 0, 0], g[:, 0, 1] = p1[:, 1] - p2[:, 1], p2[:, 0] - p1[:, 0]
    g[:, 1, 0], g[:, 1, 1] = p2[:, 1] - p0[:, 1], p0[:, 0] - p2[:, 0]
    g[:, 2, 0], g[:, 2, 1] = p0[:, 1] - p1[:, 1], p1[:, 0] - p0[:, 0]
    g /= det[:, None, None]
    Ke = np.einsum("tid,tjd->tij", g, g) * (kappa * area)[:, None, None]
    return Ke, area


def assemble(N: int, kappa: np.ndarray, f: float | np.ndarray = 1.0):
    """Global stiffness (CSR, all N*N vertices) and load vector by a generic element loop.

    f is a constant or a per-vertex array of nodal values f(x_i).
    """
    coords, tris = mesh(N)
    Ke, area = element_matrices(coords, tris, np.asarray(kappa, dtype=np.float64))
    rows = np.repeat(tris, 3, axis=1).ravel()
    cols = np.tile(tris, (1, 3)).ravel()
    A = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(N * N, N * N)).tocsr()
    fv = np.broadcast_to(np.asarray(f, dtype=np.float64), (N * N,))
    c = np.zeros(N * N)
    for k in range(3):  # Eq. coefc: c_i += |t|/3 f(x_i) for each triangle t containing x_i
        np.add.at(c, tris[:, k], area / 3.0 * fv[tris[:, k]])
    return A, c


def interior_ids(N: int) -> np.ndarray:
    """Flat ids of the (N-2)^2 unknowns, in natural (row-major) order."""
    jj, ii = np.meshgrid(np.arange(1, N - 1), np.arange(1, N - 1), indexing="ij")
    return (jj * N + ii).ravel()


def reduced_system(N: int, kappa: np.ndarray, f=1.0):
    """Drop the Dirichlet vertices (g = 0): A_II, c_I over the unknowns."""
    A, c = assemble(N, kappa, f)
    I = interior_ids(N)
    return A[I][:, I].tocsr(), c[I], I


def banded_lower(A: sp.csr_matrix, bw: int) -> np.ndarray:
    """LAPACK lower band storage ab[d, k] = A[k+d, k], d = 0..bw."""
    n = A.shape[0]
    coo = sp.tril(A).tocoo()
    d = coo.row - coo.col
    if d.max(initial=0) > bw:
        raise ValueError("matrix wider than the stated band")
    ab = np.zeros((bw + 1, n))
    ab[d, coo.col] = coo.data
    return ab


def solve_banded_cholesky(A: sp.csr_matrix, c: np.ndarray, bw: int) -> np.ndarray:
    """Banded Cholesky solve (LAPACK ?pbsv via scipy.linalg.solveh_banded)."""
    return sla.solveh_banded(banded_lower(A, bw), c, lower=True)


def refine_longdouble(A: sp.csr_matrix, c: np.ndarray, u: np.ndarray, bw: int) -> np.ndarray:
    """One refinement step with the residual c - A u accumulated in long double."""
    ld = np.longdouble
    r = c.astype(ld).copy()
    Ac = A.tocoo()
    np.subtract.at(r, Ac.row, Ac.data.astype(ld) * u.astype(ld)[Ac.col])
    return u + solve_banded_cholesky(A, r.astype(np.float64), bw)


def kappa_from_kl(phi: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """kappa_t = exp(sum_k phi[t,k] Z_k) (notation table: kappa = e^q)."""
    return np.exp(phi @ np.asarray(Z, dtype=np.float64))


def solve_full(N: int, kappa: np.ndarray, f=1.0, refine: bool = False) -> np.ndarray:
    """FE solution at all N*N vertices (zero on the boundary)."""
    A, c, I = reduced_system(N, kappa, f)
    u = solve_banded_cholesky(A, c, N - 1)
    if refine:
        u = refine_longdouble(A, c, u, N - 1)
    full = np.zeros(N * N)
    full[I] = u
    return full


def solve_load(N: int, kappa: np.ndarray, c: np.ndarray, refine: bool = False) -> np.ndarray:
    """FE solution for an assembled load vector c [N*N] (entries at boundary vertices
    ignored): A_II u_I = c_I, zero on the boundary.  The operators are independent of
    the load, so one factorisation serves many right-hand sides (Sec. 2); here every
    call simply solves again."""
    A, _ = assemble(N, kappa)
    I = interior_ids(N)
    AI = A[I][:, I].tocsr()
    cI = np.asarray(c, dtype=np.float64)[I]
    u = solve_banded_cholesky(AI, cI, N - 1)
    if refine:
        u = refine_longdouble(AI, cI, u, N - 1)
    full = np.zeros(N * N)
    full[I] = u
    return full


def prolongate(N: int, f_coarse: np.ndarray) -> np.ndarray:
    """Nodal values on the fine N x N grid of the coarse P1 function with nodal values
    f_coarse [NH*NH], NH = (N+1)/2, H = 2h (Sec. 3.5: a right-hand side in V_H, a subspace
    of V_h).  Evaluated at each fine vertex from the coarse triangle that contains it, by its
    barycentric coordinates (the coarse mesh is the same "/" triangulation with step H)."""
    if N % 2 == 0:
        raise ValueError("the two-grid load needs an odd N (the coarse grid has (N+1)/2 vertices per side)")
    NH = (N + 1) // 2
    fH = np.asarray(f_coarse, dtype=np.float64).reshape(NH * NH)
    cc, ct = mesh(NH)
    out = np.empty(N * N)
    hH = 1.0 / (NH - 1)
    for j in range(N):
        for i in range(N):
            x, y = i / (N - 1), j / (N - 1)
            ci, cj = min(int(x / hH), NH - 2), min(int(y / hH), NH - 2)
            fx, fy = x / hH - ci, y / hH - cj
            t = 2 * (cj * (NH - 1) + ci) + (0 if fx >= fy else 1)   # lower-right below the "/" diagonal
            p = cc[ct[t]]
            T = np.array([[p[0, 0], p[1, 0], p[2, 0]], [p[0, 1], p[1, 1], p[2, 1]], [1.0, 1.0, 1.0]])
            lam = np.linalg.solve(T, np.array([x, y, 1.0]))
            out[j * N + i] = lam @ fH[ct[t]]
    return out


def solve_data(N: int, kappa: np.ndarray, c=None, f_coarse=None, g=None, refine: bool = False) -> np.ndarray:
    """FE solution for one load and Dirichlet data (Sec. 2: the solution as a function of the
    right-hand side and of the boundary values, u|_gamma = Phi(u|_dOmega, f)): the load is
    the assembled vector c [N*N] (interior entries used) or, for f given on the coarse grid
    (Sec. 3.5), the vertex-quadrature load of its fine interpolant, c_i = sum_t |t|/3 f(x_i);
    g [N*N] gives u on the boundary vertices (interior entries ignored; None = 0).  Solves
    A_II u_I = c_I - A_IB g_B by banded Cholesky and returns u at every vertex."""
    A, _ = assemble(N, kappa)
    if (c is None) == (f_coarse is None):
        raise ValueError("give exactly one of c and f_coarse")
    if f_coarse is not None:
        _, c = assemble(N, np.ones(2 * (N - 1) ** 2), prolongate(N, f_coarse))
    I = interior_ids(N)
    Bd = np.setdiff1d(np.arange(N * N), I)
    gv = np.zeros(N * N) if g is None else np.asarray(g, dtype=np.float64)
    AII = A[I][:, I].tocsr()
    rhs = np.asarray(c, dtype=np.float64)[I] - A[I][:, Bd] @ gv[Bd]
    u = solve_banded_cholesky(AII, rhs, N - 1)
    if refine:
        u = refine_longdouble(AII, rhs, u, N - 1)
    full = np.zeros(N * N)
    full[I] = u
    full[Bd] = gv[Bd]
    return full


def subdomain_mean(N: int, u: np.ndarray, x0: int, x1: int, y0: int, y1: int) -> float:
    """Mean of the piecewise linear u over the rectangle [x0, x1] x [y0, y1] (vertex
    indices), Sec. 5, Eq. mean: sum over its triangles of |t|/3 (u_1 + u_2 + u_3),
    divided by the summed area of those triangles."""
    coords, tris = mesh(N)
    _, area = element_matrices(coords, tris, np.ones(tris.shape[0]))
    cj, ci = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    cell = (cj * (N - 1) + ci).ravel()
    t = np.concatenate([2 * cell, 2 * cell + 1])
    u = np.asarray(u, dtype=np.float64)
    integral = np.sum(area[t] / 3.0 * u[tris[t]].sum(axis=1))
    return float(integral / np.sum(area[t]))


def loglik(u_obs: np.ndarray, y: np.ndarray, sigma: float) -> float:
    """Gaussian log-likelihood of Sec. 1.2 with i.i.d. N(0, sigma^2) noise."""
    r = np.asarray(y, dtype=np.float64) - np.asarray(u_obs, dtype=np.float64)
    n = r.size
    return float(-0.5 * np.dot(r, r) / sigma ** 2 - 0.5 * n * np.log(2.0 * np.pi * sigma ** 2))


def evaluate(N: int, phi: np.ndarray, Z: np.ndarray, obs: np.ndarray, y: np.ndarray,
             sigma: float, f=1.0, refine: bool = False):
    """One likelihood evaluation: (u at obs, log-likelihood)."""
    u = solve_full(N, kappa_from_kl(phi, Z), f, refine=refine)
    u_obs = u[np.asarray(obs)]
    return u_obs, loglik(u_obs, y, sigma)


def _worker(args):
    N, phi, Z, obs, y, sigma, f = args
    return evaluate(N, phi, Z, obs, y, sigma, f)


def evaluate_batch(N, phi, Zs, obs, y, sigma, f=1.0, processes: int = 1):
    """Evaluate many samples; processes > 1 uses a spawn-started pool."""
    args = [(N, phi, Z, obs, y, sigma, f) for Z in Zs]
    if processes <= 1:
        res = [_worker(a) for a in args]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            res = pool.map(_worker, args)
    u_obs = np.stack([r[0] for r in res])
    ll = np.array([r[1] for r in res])
    return u_obs, ll
