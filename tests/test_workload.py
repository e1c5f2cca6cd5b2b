"""Pins of the synthetic input recipe (KL basis, observation lattice, seeds)."""
import numpy as np

import workload as w


def test_kl_dense_eigenpairs():
    N, nz, lc, var = 17, 8, 0.3, 1.0
    phi = w.kl_basis(N, nz, lc, var, method="dense")
    c = w.triangle_centroids(N)
    C = w._cov(c, c, lc, var)
    lam = (phi ** 2).sum(axis=0)
    V = phi / np.sqrt(lam)
    assert np.allclose(V.T @ V, np.eye(nz), atol=1e-12)                       # orthonormal
    assert np.linalg.norm(C @ V - V * lam) <= 1e-10 * np.linalg.norm(C)       # eigen-residual
    assert np.all(np.diff(lam) <= 1e-12)                                      # descending
    assert lam.sum() <= np.trace(C) + 1e-9                                    # trace bound
    ref = np.linalg.eigvalsh(C)[::-1][:nz]
    assert np.allclose(lam, ref, rtol=1e-10)


def test_kl_nystrom_reproduces_dense_on_coarse_set():
    # on the Nystrom point set itself (32 x 32 cells = N 33) the extension returns
    # the dense eigenvectors exactly: psi_k(c_i) = sqrt(M) v_k[i]
    a = w.kl_basis(33, 10, 0.3, 1.0, method="dense")
    b = w.kl_basis(33, 10, 0.3, 1.0, method="nystrom")
    assert np.allclose(a, b, atol=1e-10)


def test_kl_nystrom_agrees_with_dense_at_65():
    # At N = 65 (8,192 triangles) the dense covariance over every centroid is still
    # tractable, so the Nystrom basis used above 33^2 (32 x 32-cell coarse set) can be set
    # against it, with the 513^2 workload's field parameters (40 terms, corr. length 0.1,
    # variance 2).  Pairs of eigenvalues are degenerate (the square's symmetry), so the
    # subspaces and the rank-40 covariances are compared, not single columns.
    N, nz, lc, var = 65, 40, 0.1, 2.0
    a = w.kl_basis(N, nz, lc, var, method="dense")
    b = w.kl_basis(N, nz, lc, var, method="nystrom")
    la, lb = (a ** 2).sum(axis=0), (b ** 2).sum(axis=0)
    assert np.max(np.abs(la - lb) / la) < 1e-2                     # eigenvalues within 1%
    Qa, _ = np.linalg.qr(a)
    Qb, _ = np.linalg.qr(b)
    cosines = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
    assert cosines.min() > 0.9999                                   # same 40-dim subspace
    Ca, Cb = a @ a.T, b @ b.T
    assert np.linalg.norm(Ca - Cb) <= 5e-3 * np.linalg.norm(Ca)     # rank-40 covariance
    assert np.max(np.abs(np.diag(Ca) - np.diag(Cb))) <= 1e-2 * np.max(np.diag(Ca))


def test_obs_lattice():
    assert list(w.obs_lattice_indices(33, 3)) == [8, 16, 24]
    from fractions import Fraction
    for N, m in ((513, 16), (257, 8), (129, 5)):
        ref = [int(Fraction(k * (N - 1), m + 1) + Fraction(1, 2)) for k in range(1, m + 1)]
        assert list(w.obs_lattice_indices(N, m)) == ref
    ids = w.obs_vertices(33, 3)
    assert ids[1] == 8 * 33 + 16


def test_seeded_streams_are_reproducible_and_independent():
    cfg = w.CONFIGS["grid33"]
    assert np.array_equal(w.draw_Z(cfg, 4), w.draw_Z(cfg, 4))
    assert not np.allclose(w.draw_Z(cfg, 1)[0], w.draw_Z_true(cfg))
    assert w.draw_noise(cfg).shape == (9,)
