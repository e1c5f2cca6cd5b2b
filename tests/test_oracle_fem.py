"""Pins of the FP64 oracle (oracle/fem.py) against what the paper and mathematics fix.

Each test ties the oracle to something other than itself: closed forms of the
discrete problem, a spectral (DST-I) solve, brute-force dense inversion, a second
route to the P1 element matrix, a library log-density, invariances.
"""
import numpy as np
import pytest
import scipy.fft
import scipy.sparse.linalg as spla
import scipy.stats

import workload as w
from oracle import fem


def _kappa_random(N, seed=0, amp=1.0):
    rng = np.random.default_rng(seed)
    return np.exp(amp * rng.standard_normal(2 * (N - 1) ** 2))


def test_mesh_matches_workload_triangle_order():
    # the oracle's triangle t must be the triangle whose centroid the KL basis row t uses
    for N in (3, 5, 17):
        coords, tris = fem.mesh(N)
        cent = coords[tris].mean(axis=1)
        assert np.allclose(cent, w.triangle_centroids(N), atol=1e-15)
        # counter-clockwise, area h^2/2
        _, area = fem.element_matrices(coords, tris, np.ones(len(tris)))
        assert np.allclose(area, 0.5 / (N - 1) ** 2)


def test_element_matrix_vs_vandermonde_gradients():
    # Eq. coefA: A_ij = kappa |t| grad b_i . grad b_j; gradients re-derived by solving
    # the Vandermonde system [1 x y] c = e_i for the affine basis functions.
    rng = np.random.default_rng(1)
    for _ in range(20):
        p = rng.random((3, 2))
        d = p[1] - p[0]; e = p[2] - p[0]
        if d[0] * e[1] - d[1] * e[0] < 0:
            p = p[[0, 2, 1]]
        kap = float(np.exp(rng.standard_normal()))
        Ke, area = fem.element_matrices(p, np.array([[0, 1, 2]]), np.array([kap]))
        V = np.column_stack([np.ones(3), p])
        grads = np.linalg.solve(V, np.eye(3))[1:, :].T          # row i = grad b_i
        area_ref = 0.5 * abs(np.linalg.det(np.column_stack([p[1] - p[0], p[2] - p[0]])))
        assert np.isclose(area[0], area_ref)
        assert np.allclose(Ke[0], kap * area_ref * grads @ grads.T, rtol=1e-12, atol=1e-12)


def test_right_triangle_element_values():
    # right isosceles triangle with legs h: right-angle vertex kappa, legs -kappa/2,
    # hypotenuse coupling 0 (independent of h in 2D)
    h = 0.25
    p = np.array([[0, 0], [h, 0], [h, h]])      # right angle at vertex 1
    Ke, _ = fem.element_matrices(p, np.array([[0, 1, 2]]), np.array([3.0]))
    ref = 3.0 * np.array([[0.5, -0.5, 0.0], [-0.5, 1.0, -0.5], [0.0, -0.5, 0.5]])
    assert np.allclose(Ke[0], ref, atol=1e-14)


def test_assembly_vs_bruteforce_loop():
    # scatter-add of the oracle vs a plain Python loop over triangles (tiny grids)
    for N in (4, 6):
        kap = _kappa_random(N, 2)
        A, c = fem.assemble(N, kap, 1.0)
        coords, tris = fem.mesh(N)
        D = np.zeros((N * N, N * N))
        cc = np.zeros(N * N)
        for t, tri in enumerate(tris):
            P = coords[tri]
            V = np.column_stack([np.ones(3), P])
            G = np.linalg.solve(V, np.eye(3))[1:, :].T
            ar = 0.5 * abs(np.linalg.det(np.column_stack([P[1] - P[0], P[2] - P[0]])))
            for a in range(3):
                cc[tri[a]] += ar / 3.0
                for b in range(3):
                    D[tri[a], tri[b]] += kap[t] * ar * G[a] @ G[b]
        assert np.allclose(A.toarray(), D, atol=1e-13)
        assert np.allclose(c, cc, atol=1e-16)


def test_five_point_edge_weights():
    # with "/" diagonals the P1 matrix is a 5-point stencil whose axis coupling is
    # minus the mean kappa of the two triangles having that edge as a leg
    N = 9
    kap = _kappa_random(N, 3)
    A, _ = fem.assemble(N, kap, 1.0)
    A = A.toarray()
    cell = lambda i, j: 2 * (j * (N - 1) + i)
    for j in range(1, N - 1):
        for i in range(0, N - 1):
            # horizontal edge (i,j)-(i+1,j): lower-right of cell (i,j), upper-left of cell (i,j-1)
            wgt = 0.5 * (kap[cell(i, j)] + kap[cell(i, j - 1) + 1])
            assert np.isclose(A[j * N + i, j * N + i + 1], -wgt, rtol=1e-13)
    for j in range(0, N - 1):
        for i in range(1, N - 1):
            # vertical edge (i,j)-(i,j+1): upper-left of cell (i,j), lower-right of cell (i-1,j)
            wgt = 0.5 * (kap[cell(i, j) + 1] + kap[cell(i - 1, j)])
            assert np.isclose(A[j * N + i, (j + 1) * N + i], -wgt, rtol=1e-13)
    # diagonal couplings vanish, rows sum to zero
    for j in range(N - 1):
        for i in range(N - 1):
            assert abs(A[j * N + i, (j + 1) * N + i + 1]) < 1e-14
            assert A[j * N + i + 1, (j + 1) * N + i] == 0.0
    assert np.allclose(A.sum(axis=1), 0.0, atol=1e-12)


def test_load_vertex_quadrature():
    # Eq. coefc with the area factor: sum over the 6 triangles of |t|/3 f = h^2 f
    for N in (5, 33):
        h = 1.0 / (N - 1)
        _, c, _ = fem.reduced_system(N, np.ones(2 * (N - 1) ** 2), 1.0)
        assert np.allclose(c, h * h, rtol=1e-14)
        fx = np.linspace(0, 1, N * N)
        _, c2, I = fem.reduced_system(N, np.ones(2 * (N - 1) ** 2), fx)
        assert np.allclose(c2, h * h * fx[I], rtol=1e-13)


@pytest.mark.parametrize("N", [5, 9, 17])
def test_banded_vs_dense_inverse(N):
    # T1: brute-force dense inverse of the same system
    kap = _kappa_random(N, N)
    A, c, _ = fem.reduced_system(N, kap, 1.0)
    u_band = fem.solve_banded_cholesky(A, c, N - 1)
    u_inv = np.linalg.inv(A.toarray()) @ c
    assert np.allclose(u_band, u_inv, rtol=1e-12, atol=0)


def test_banded_vs_superlu():
    N = 65
    kap = _kappa_random(N, 7, amp=2.0)
    A, c, _ = fem.reduced_system(N, kap, 1.0)
    u_band = fem.solve_banded_cholesky(A, c, N - 1)
    u_lu = spla.splu(A.tocsc()).solve(c)
    assert np.max(np.abs(u_band - u_lu)) / np.max(np.abs(u_lu)) < 1e-12


@pytest.mark.parametrize("N", [9, 17, 33])
def test_eigenvector_closed_form(N):
    # T2: kappa = 1, nodal f = sin(pi x) sin(pi y) is the (1,1) eigenvector of the
    # 5-point matrix with eigenvalue 4 - 4 cos(pi h), so u = h^2 f / (4 - 4 cos(pi h))
    h = 1.0 / (N - 1)
    x = np.arange(N) * h
    F = np.outer(np.sin(np.pi * x), np.sin(np.pi * x)).ravel()   # F[j*N+i] = sin(pi y_j) sin(pi x_i)
    u = fem.solve_full(N, np.ones(2 * (N - 1) ** 2), F)
    ref = h * h * F / (4.0 - 4.0 * np.cos(np.pi * h))
    assert np.max(np.abs(u - ref)) < 1e-13 * np.max(np.abs(ref))


def test_manufactured_solution_second_order():
    # T3: u = sin(pi x) sin(pi y), kappa = 1, f = 2 pi^2 u.  Nodal error ratio is
    # 2 pi^2 h^2 / (4 - 4 cos(pi h)) - 1 = pi^2 h^2 / 12 + O(h^4)
    errs = []
    for N in (33, 65):
        h = 1.0 / (N - 1)
        x = np.arange(N) * h
        U = np.outer(np.sin(np.pi * x), np.sin(np.pi * x)).ravel()
        u = fem.solve_full(N, np.ones(2 * (N - 1) ** 2), 2 * np.pi ** 2 * U)
        err = np.max(np.abs(u - U)) / np.max(U)
        assert np.isclose(err, 2 * np.pi ** 2 * h * h / (4 - 4 * np.cos(np.pi * h)) - 1, rtol=1e-9)
        assert abs(err - np.pi ** 2 * h * h / 12) < 0.01 * np.pi ** 2 * h * h / 12
        errs.append(err)
    assert np.isclose(errs[0] / errs[1], 4.0, rtol=0.01)


@pytest.mark.parametrize("N", [17, 33, 65])
def test_dst_spectral_solve(N):
    # T4: kappa = 1, f = 1 equals the 5-point Poisson problem, diagonalised by DST-I
    h = 1.0 / (N - 1)
    n = N - 2
    u = fem.solve_full(N, np.ones(2 * (N - 1) ** 2), 1.0).reshape(N, N)[1:-1, 1:-1]
    k = np.arange(1, n + 1)
    lam = (4 - 2 * np.cos(np.pi * k * h))[:, None] - 2 * np.cos(np.pi * k * h)[None, :]
    rhs = np.full((n, n), h * h)
    u_dst = scipy.fft.idstn(scipy.fft.dstn(rhs, type=1) / lam, type=1)
    assert np.max(np.abs(u - u_dst)) < 1e-13 * np.max(np.abs(u_dst))


def test_center_value_converges_to_continuum():
    # -Laplace u = 1 on the unit square: u(1/2,1/2) = 0.0736713532814...; O(h^2)
    N = 129
    u = fem.solve_full(N, np.ones(2 * (N - 1) ** 2), 1.0).reshape(N, N)
    assert abs(u[64, 64] - 0.07367135328) < 2e-5


def test_kappa_scaling_and_transpose_symmetry():
    N = 17
    base = fem.solve_full(N, np.ones(2 * (N - 1) ** 2), 1.0)
    assert np.allclose(fem.solve_full(N, np.full(2 * (N - 1) ** 2, 4.0), 1.0), base / 4.0, rtol=1e-13)
    # a kappa field invariant under (x,y) -> (y,x): the lower-right triangle of cell
    # (i,j) maps onto the upper-left triangle of cell (j,i)
    rng = np.random.default_rng(5)
    kap = np.empty(2 * (N - 1) ** 2)
    for j in range(N - 1):
        for i in range(N - 1):
            a = np.exp(rng.standard_normal())
            if i <= j:
                kap[2 * (j * (N - 1) + i)] = a
                kap[2 * (i * (N - 1) + j) + 1] = a
            if i < j:
                b = np.exp(rng.standard_normal())
                kap[2 * (j * (N - 1) + i) + 1] = b
                kap[2 * (i * (N - 1) + j)] = b
    U = fem.solve_full(N, kap, 1.0).reshape(N, N)
    assert np.allclose(U, U.T, rtol=1e-12, atol=1e-16)
    assert not np.allclose(U, U[::-1, :], rtol=1e-6)


def test_loglik_vs_scipy_logpdf():
    rng = np.random.default_rng(9)
    u = rng.standard_normal(37)
    y = u + 0.01 * rng.standard_normal(37)
    ref = scipy.stats.norm.logpdf(y, loc=u, scale=0.01).sum()
    assert np.isclose(fem.loglik(u, y, 0.01), ref, rtol=1e-13)
    assert np.isclose(fem.loglik(u, u, 0.5), -0.5 * 37 * np.log(2 * np.pi * 0.25), rtol=1e-14)


def test_refinement_does_not_move_an_accurate_solve():
    N = 33
    kap = _kappa_random(N, 11, amp=2.0)
    u0 = fem.solve_full(N, kap)
    u1 = fem.solve_full(N, kap, refine=True)
    assert np.max(np.abs(u1 - u0)) < 1e-12 * np.max(np.abs(u0))


@pytest.mark.parametrize("N", [17, 65])
def test_refinement_step_removes_a_known_perturbation(N):
    # One step u <- u + A^-1 (c - A u) maps u* + e to u* exactly in exact arithmetic (and a
    # residual of the wrong sign, A u - c, would give u* + 2e).  kappa spans four decades.
    rng = np.random.default_rng(N)
    kap = np.exp(rng.uniform(0.0, np.log(1e4), 2 * (N - 1) ** 2))
    assert kap.max() / kap.min() > 1e3
    A, c, _ = fem.reduced_system(N, kap)
    u_star = fem.solve_banded_cholesky(A, c, N - 1)
    scale = np.max(np.abs(u_star))
    e = 1e-3 * scale * rng.standard_normal(u_star.size)
    u1 = fem.refine_longdouble(A, c, u_star + e, N - 1)
    assert np.max(np.abs(u1 - u_star)) <= 1e-12 * scale
    # the step shrinks the long-double residual by the size of the perturbation
    def res(u):
        return np.max(np.abs(c - A @ u))
    assert res(u1) <= 1e-6 * res(u_star + e)


@pytest.mark.parametrize("N", [9, 17, 33])
def test_solve_load_eigenvector_closed_form(N):
    # an assembled load c = h^2 sin(pi x) sin(pi y) at kappa = 1 gives
    # u = c / (4 - 4 cos(pi h)) (the (1,1) eigenvector of the 5-point matrix);
    # values at boundary vertices are not part of the load and must be ignored
    h = 1.0 / (N - 1)
    x = np.arange(N) * h
    F = np.outer(np.sin(np.pi * x), np.sin(np.pi * x)).ravel()
    c = h * h * F
    bnd = np.setdiff1d(np.arange(N * N), fem.interior_ids(N))
    c_noisy = c.copy()
    c_noisy[bnd] = np.random.default_rng(N).standard_normal(bnd.size)
    u = fem.solve_load(N, np.ones(2 * (N - 1) ** 2), c_noisy)
    ref = c / (4.0 - 4.0 * np.cos(np.pi * h))
    ref[bnd] = 0.0
    assert np.max(np.abs(u - ref)) < 1e-13 * np.max(np.abs(ref))


def test_solve_load_superposition_and_vertex_quadrature():
    # the load of f = 1 by vertex quadrature (Eq. coefc) reproduces the constant-f
    # solve; the solve is linear in c
    N = 17
    kap = _kappa_random(N, 3, amp=1.5)
    _, c1 = fem.assemble(N, kap, 1.0)
    u1 = fem.solve_load(N, kap, c1)
    assert np.max(np.abs(u1 - fem.solve_full(N, kap))) < 1e-14 * np.max(np.abs(u1))
    c2 = np.random.default_rng(4).random(N * N) / (N - 1) ** 2
    u2 = fem.solve_load(N, kap, c2)
    u12 = fem.solve_load(N, kap, c1 - 3.0 * c2)
    assert np.max(np.abs(u12 - (u1 - 3.0 * u2))) < 1e-12 * np.max(np.abs(u12))


def test_subdomain_mean_of_an_affine_field():
    # P1 reproduces affine functions: the mean over a rectangle is the value at its centre
    N = 17
    h = 1.0 / (N - 1)
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    u = (0.3 + 1.7 * ii * h - 0.9 * jj * h).ravel()
    for x0, x1, y0, y1 in [(0, 16, 0, 16), (3, 7, 2, 11), (5, 6, 9, 10), (0, 8, 8, 16)]:
        ref = 0.3 + 1.7 * 0.5 * (x0 + x1) * h - 0.9 * 0.5 * (y0 + y1) * h
        assert abs(fem.subdomain_mean(N, u, x0, x1, y0, y1) - ref) < 1e-14


def test_subdomain_mean_of_the_domain_is_the_load_pairing():
    # int_Omega u_h = sum_i u_i int b_i = sum_i u_i sum_{t containing i} |t|/3 = c . u with
    # c the f = 1 load by vertex quadrature (Eq. coefc), whatever u is (boundary included)
    N = 13
    u = np.random.default_rng(5).standard_normal(N * N)
    _, c = fem.assemble(N, np.ones(2 * (N - 1) ** 2), 1.0)
    assert abs(fem.subdomain_mean(N, u, 0, N - 1, 0, N - 1) - np.dot(c, u)) < 1e-14 * np.abs(u).sum()


def test_subdomain_means_follow_the_tree_recursion():
    # Sec. 5.1: the mean over a father is c_1 mean_1 + c_2 mean_2 with c_i = |omega_i| / |omega|
    from oracle import hdd_dense
    N = 21
    u = np.random.default_rng(6).standard_normal(N * N)
    nodes = hdd_dense.build_tree(N, 4)
    area = lambda nd: (nd.x1 - nd.x0) * (nd.y1 - nd.y0)
    mean = [fem.subdomain_mean(N, u, nd.x0, nd.x1, nd.y0, nd.y1) for nd in nodes]
    for k, nd in enumerate(nodes):
        if nd.leaf:
            continue
        a, b = nd.children
        ref = (area(nodes[a]) * mean[a] + area(nodes[b]) * mean[b]) / area(nd)
        assert abs(mean[k] - ref) < 1e-14 * max(1.0, abs(ref))


# --- Dirichlet data and coarse-grid loads (Sec. 2, Sec. 3.5) ---------------------------------

def _bnd(N):
    return np.setdiff1d(np.arange(N * N), fem.interior_ids(N))


def test_constant_dirichlet_data_gives_a_constant_for_any_kappa():
    # constants are in the kernel of every stiffness (rows of A sum to zero), so g = 1, c = 0
    # gives u = 1 whatever kappa is
    N = 17
    u = fem.solve_data(N, _kappa_random(N, 21, amp=2.0), c=np.zeros(N * N), g=np.ones(N * N))
    assert np.abs(u - 1.0).max() < 1e-12


def test_linear_dirichlet_data_is_reproduced_at_constant_kappa():
    # at constant kappa the P1 (five-point) operator annihilates affine functions
    N = 21
    coords, _ = fem.mesh(N)
    gl = 0.3 + 1.7 * coords[:, 0] - 0.9 * coords[:, 1]
    u = fem.solve_data(N, np.full(2 * (N - 1) ** 2, 2.5), c=np.zeros(N * N), g=gl)
    assert np.abs(u - gl).max() < 1e-12


def test_data_superposition_and_maximum_principle():
    N = 17
    kap = _kappa_random(N, 22, amp=1.5)
    rng = np.random.default_rng(23)
    c = rng.random(N * N) / (N - 1) ** 2
    g = rng.random(N * N)
    u = fem.solve_data(N, kap, c=c, g=g)
    u0 = fem.solve_data(N, kap, c=c)
    ug = fem.solve_data(N, kap, c=np.zeros(N * N), g=g)
    assert np.abs(u - (u0 + ug)).max() < 1e-12 * np.abs(u).max()
    assert np.array_equal(u[_bnd(N)], g[_bnd(N)])
    # an M-matrix: harmonic data stay within the range of their boundary values
    B = _bnd(N)
    assert ug.min() >= g[B].min() - 1e-13 and ug.max() <= g[B].max() + 1e-13


def test_prolongation_is_exact_for_affine_coarse_functions():
    N, NH = 17, 9
    cH, _ = fem.mesh(NH)
    cF, _ = fem.mesh(N)
    a = lambda xy: 0.5 - 2.0 * xy[:, 0] + 3.0 * xy[:, 1]
    assert np.abs(fem.prolongate(N, a(cH)) - a(cF)).max() < 1e-13


def test_prolongation_matches_the_coarse_function_between_coarse_vertices():
    # coarse vertices keep their values; a fine vertex on a coarse edge (axis or "/" diagonal)
    # is the mean of the edge's two coarse ends
    N, NH = 9, 5
    fH = np.random.default_rng(24).standard_normal(NH * NH)
    f = fem.prolongate(N, fH)
    F = lambda i, j: f[j * N + i]
    C = lambda a, b: fH[b * NH + a]
    for b in range(NH):
        for a in range(NH):
            assert F(2 * a, 2 * b) == pytest.approx(C(a, b), abs=1e-14)
    for b in range(NH - 1):
        for a in range(NH - 1):
            assert F(2 * a + 1, 2 * b) == pytest.approx(0.5 * (C(a, b) + C(a + 1, b)), abs=1e-14)
            assert F(2 * a, 2 * b + 1) == pytest.approx(0.5 * (C(a, b) + C(a, b + 1)), abs=1e-14)
            assert F(2 * a + 1, 2 * b + 1) == pytest.approx(0.5 * (C(a, b) + C(a + 1, b + 1)), abs=1e-14)


def test_coarse_constant_load_is_the_fine_constant_load():
    N = 17
    kap = _kappa_random(N, 25)
    NH = (N + 1) // 2
    u1 = fem.solve_data(N, kap, f_coarse=np.full(NH * NH, 1.0))
    u2 = fem.solve_full(N, kap, 1.0)
    assert np.abs(u1 - u2).max() < 1e-13 * np.abs(u2).max()
