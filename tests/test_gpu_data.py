"""GPU parity of hdd_solve_data: many loads with Dirichlet data (Sec. 2) and loads given on
the coarse grid H = 2h (Sec. 3.5), four right-hand sides per sweep through the stored factors,
against the oracle's banded-Cholesky solve of A_II u_I = c_I - A_IB g_B (oracle/fem.py,
solve_data).  Tolerances: 1e-11 relative (FP64 plans), 1e-8 after refinement (mixed plans).
"""
import numpy as np
import pytest

from oracle import fem
from tests.gpu_common import rel_err_field, small_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hdd():
    from paper_1708_02207_gb300 import build, hdd as binding
    build.build()
    return binding


def solve(hdd, N, leaf, phi, Z, c=None, fH=None, g=None, **kw):
    plan = hdd.Plan(N, leaf, phi, np.array([N * (N // 2) + N // 2], dtype=np.int32), 0.1, **kw)
    B = Z.shape[0]
    ws = plan.workspace(B)
    plan.assemble(torch.from_numpy(Z).cuda(), ws)
    plan.upsweep(B, ws)
    nl = (c if c is not None else fH).shape[1]
    u = torch.empty(B, nl, N * N, dtype=torch.float64, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    cuda = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    plan.solve_data(B, ws, u, c=cuda(c), f_coarse=cuda(fH), g=cuda(g), status=st)
    torch.cuda.synchronize()
    return u.cpu().numpy(), st.cpu().numpy(), plan, ws


def reference(N, phi, Z, c=None, fH=None, g=None):
    B, nl = Z.shape[0], (c if c is not None else fH).shape[1]
    out = np.empty((B, nl, N * N))
    for s in range(B):
        kap = fem.kappa_from_kl(phi, Z[s])
        for k in range(nl):
            out[s, k] = fem.solve_data(N, kap, c=None if c is None else c[s, k], f_coarse=None if fH is None else fH[s, k],
                                       g=None if g is None else g[s, k], refine=True)
    return out


def data(N, B, nl, seed, coarse=False):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((B, nl, N * N))
    if coarse:
        NH = (N + 1) // 2
        return None, rng.standard_normal((B, nl, NH * NH)), g
    return rng.standard_normal((B, nl, N * N)) / (N - 1) ** 2, None, g


@pytest.mark.parametrize("N,leaf", [(33, 8), (33, 4), (50, 5), (17, 1)])
def test_fp64_loads_and_dirichlet_data(hdd, N, leaf):
    # six data sets per sample: a full group of four and a partial group of two
    phi, Z = small_problem(N, batch=2, seed=N + leaf)
    c, _, g = data(N, 2, 6, N)
    u, st, _, _ = solve(hdd, N, leaf, phi, Z, c=c, g=g)
    ref = reference(N, phi, Z, c=c, g=g)
    assert (st == 0).all()
    assert rel_err_field(u.reshape(-1, N * N), ref.reshape(-1, N * N)).max() <= 1e-11


@pytest.mark.parametrize("N,leaf", [(33, 4), (65, 8)])
def test_fp64_coarse_grid_loads(hdd, N, leaf):
    phi, Z = small_problem(N, batch=2, seed=3 * N)
    _, fH, g = data(N, 2, 3, 5 * N, coarse=True)
    u, st, _, _ = solve(hdd, N, leaf, phi, Z, fH=fH, g=g)
    ref = reference(N, phi, Z, fH=fH, g=g)
    assert (st == 0).all()
    assert rel_err_field(u.reshape(-1, N * N), ref.reshape(-1, N * N)).max() <= 1e-11
    # without Dirichlet data, a coarse constant f is the plan's own constant load
    NH = (N + 1) // 2
    u1, _, _, _ = solve(hdd, N, leaf, phi, Z, fH=np.ones((2, 1, NH * NH)))
    ref1 = np.array([fem.solve_full(N, fem.kappa_from_kl(phi, z), 1.0, refine=True) for z in Z])
    assert rel_err_field(u1[:, 0], ref1).max() <= 1e-11


def test_constant_boundary_data_give_a_constant(hdd):
    N = 33
    phi, Z = small_problem(N, batch=2, seed=11)
    u, st, _, _ = solve(hdd, N, 4, phi, Z, c=np.zeros((2, 1, N * N)), g=np.ones((2, 1, N * N)))
    assert (st == 0).all() and np.abs(u - 1.0).max() <= 1e-12


def test_data_equals_solve_loads_without_boundary_data(hdd):
    N = 65
    phi, Z = small_problem(N, batch=2, seed=12)
    c, _, _ = data(N, 2, 4, 13)
    u, _, plan, ws = solve(hdd, N, 8, phi, Z, c=c)
    ul = torch.empty(2, 4, N * N, dtype=torch.float64, device="cuda")
    plan.solve_loads(2, ws, torch.from_numpy(c).cuda(), ul)
    torch.cuda.synchronize()
    assert rel_err_field(u.reshape(-1, N * N), ul.cpu().numpy().reshape(-1, N * N)).max() <= 1e-12


@pytest.mark.parametrize("N,leaf,top", [(65, 4, 0), (129, 8, 2), (257, 16, 0)])
def test_mixed_refined_data(hdd, N, leaf, top):
    # 257 with 16 x 16-cell leaves: tensor-core fronts; three refinement steps
    phi, Z = small_problem(N, n_z=20, corr_len=0.2, variance=2.0, batch=2, seed=N + top)
    coarse = N % 2 == 1 and N <= 129
    c, fH, g = data(N, 2, 5, 7 * N, coarse=coarse)
    u, st, _, _ = solve(hdd, N, leaf, phi, Z, c=c, fH=fH, g=g, precision=hdd.HDD_MIXED_FP32, ir_max_iter=3,
                        ir_tol=1e-9, fp64_top_levels=top)
    ref = reference(N, phi, Z, c=c, fH=fH, g=g)
    assert (st == 0).all()
    assert rel_err_field(u.reshape(-1, N * N), ref.reshape(-1, N * N)).max() <= 1e-8
