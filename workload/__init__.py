"""Seeded synthetic inputs for the HDD likelihood path.

This module is shared by the FP64 CPU oracle and by the GPU library's tests and
benchmark.  It draws random numbers and builds input arrays only: the mesh
numbering, the Karhunen-Loeve (KL) basis of the log-permeability field, the
observation lattice, the parameter samples Z and the stored observation data y.
It holds none of the method's arithmetic (no assembly, no elimination, no solve,
no likelihood).

Conventions (the paper leaves these open, Sec. 1.1 and Sec. 5):
  * Omega = [0,1]^2 with an N x N vertex grid, h = 1/(N-1); vertex (i, j) sits at
    (i h, j h) and has the flat id v = j*N + i.
  * Each cell (i, j) = [ih,(i+1)h] x [jh,(j+1)h] is split by its "/" diagonal
    (i,j)-(i+1,j+1) into a lower-right triangle (right angle at (i+1, j)) and an
    upper-left triangle (right angle at (i, j+1)).  Triangle t = 2*(j*(N-1)+i)+s,
    s = 0 for the lower-right and s = 1 for the upper-left one.
  * kappa = exp(q) (notation table of the paper), q(x_t, Z) = sum_k Phi[t, k] Z_k
    with Phi already scaled by sqrt(lambda_k); q is constant on each triangle and
    is evaluated at the triangle centroid.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

ROOT_SEED = 1708_02207
_DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


@dataclass(frozen=True)
class Config:
    """One synthetic workload: grid, decomposition, field and observation recipe."""
    name: str
    N: int                 # vertices per side
    leaf: int              # leaf size in cells per side
    batch: int             # number of Z samples per step
    n_z: int               # KL terms
    corr_len: float        # correlation length of exp(-|x-y|/corr_len)
    variance: float        # field variance
    obs_side: int          # m: observations on an m x m interior vertex lattice
    sigma: float           # noise standard deviation
    f: float = 1.0         # constant right-hand side
    spawn_key: int = 0     # child index of the root SeedSequence


CONFIGS = {
    "grid33": Config("grid33", N=33, leaf=8, batch=1, n_z=10, corr_len=0.3, variance=1.0,
                     obs_side=3, sigma=0.01, spawn_key=0),
    "grid257": Config("grid257", N=257, leaf=16, batch=1024, n_z=20, corr_len=0.2, variance=1.0,
                      obs_side=8, sigma=0.01, spawn_key=1),
    "grid513": Config("grid513", N=513, leaf=4, batch=256, n_z=40, corr_len=0.1, variance=2.0,
                      obs_side=16, sigma=0.01, spawn_key=2),
}


def _streams(cfg: Config):
    """Independent child streams for (Z, Z_true, noise) of one config."""
    root = np.random.SeedSequence(ROOT_SEED)
    cfg_seq = root.spawn(cfg.spawn_key + 1)[cfg.spawn_key]
    z_seq, ztrue_seq, noise_seq = cfg_seq.spawn(3)
    return (np.random.default_rng(z_seq), np.random.default_rng(ztrue_seq),
            np.random.default_rng(noise_seq))


def n_triangles(N: int) -> int:
    return 2 * (N - 1) * (N - 1)


def triangle_centroids(N: int) -> np.ndarray:
    """Centroids [n_t, 2] in triangle order t = 2*(j*(N-1)+i)+s."""
    h = 1.0 / (N - 1)
    j, i = np.meshgrid(np.arange(N - 1), np.arange(N - 1), indexing="ij")
    i = i.ravel().astype(np.float64)
    j = j.ravel().astype(np.float64)
    c = np.empty((2 * i.size, 2))
    c[0::2, 0] = (i + 2.0 / 3.0) * h   # lower-right: vertices (i,j),(i+1,j),(i+1,j+1)
    c[0::2, 1] = (j + 1.0 / 3.0) * h
    c[1::2, 0] = (i + 1.0 / 3.0) * h   # upper-left: vertices (i,j),(i+1,j+1),(i,j+1)
    c[1::2, 1] = (j + 2.0 / 3.0) * h
    return c


def _cov(a: np.ndarray, b: np.ndarray, corr_len: float, variance: float) -> np.ndarray:
    """variance * exp(-|a_i - b_j|_2 / corr_len) for point sets a [n,2], b [m,2]."""
    try:
        import torch
        ta, tb = torch.from_numpy(np.ascontiguousarray(a)), torch.from_numpy(np.ascontiguousarray(b))
        d = (ta[:, None, 0] - tb[None, :, 0]) ** 2 + (ta[:, None, 1] - tb[None, :, 1]) ** 2
        return d.sqrt_().mul_(-1.0 / corr_len).exp_().mul_(variance).numpy()
    except ImportError:
        dx = a[:, 0:1] - b[None, :, 0]
        dx *= dx
        dy = a[:, 1:2] - b[None, :, 1]
        dy *= dy
        dx += dy
        np.sqrt(dx, out=dx)
        dx *= -1.0 / corr_len
        np.exp(dx, out=dx)
        dx *= variance
        return dx


def _fix_sign(v: np.ndarray) -> np.ndarray:
    idx = np.argmax(np.abs(v), axis=0)
    s = np.sign(v[idx, np.arange(v.shape[1])])
    s[s == 0] = 1.0
    return v * s


DENSE_KL_MAX_TRIANGLES = 2048
NYSTROM_CELLS = 32


def kl_basis(N: int, n_z: int, corr_len: float, variance: float, method: str = "auto") -> np.ndarray:
    """KL basis Phi[n_t, n_z] of exp(-|x-y|_2/corr_len)*variance, scaled by sqrt(lambda).

    method "dense", "nystrom" or "auto".  With "auto", grids with at most 2048
    triangles (N <= 33) use the dense covariance over all triangle
    centroids.  Larger grids use the Nystrom extension from the centroid set of a
    32 x 32-cell grid (2048 points): with (mu_k, v_k) the top eigenpairs of the
    coarse covariance divided by M = 2048, psi_k(x) = sum_j C(x, c_j) sqrt(M) v_k[j]
    / (M mu_k) and Phi[:, k] = sqrt(mu_k) psi_k.  Each column's entry of largest
    magnitude is made positive.  Degenerate eigenpairs (the square's symmetry) make
    the basis depend on the LAPACK build, so a caller computes it once and feeds
    the same array to every consumer.
    """
    import scipy.linalg as sla

    cent = triangle_centroids(N)
    n_t = cent.shape[0]
    if method == "auto":
        method = "dense" if n_t <= DENSE_KL_MAX_TRIANGLES else "nystrom"
    if method == "dense":
        C = _cov(cent, cent, corr_len, variance)
        lam, V = sla.eigh(C, subset_by_index=[n_t - n_z, n_t - 1])
        lam, V = lam[::-1], _fix_sign(V[:, ::-1])
        return np.ascontiguousarray(V * np.sqrt(np.maximum(lam, 0.0))[None, :])
    coarse = triangle_centroids(NYSTROM_CELLS + 1)
    M = coarse.shape[0]
    Cc = _cov(coarse, coarse, corr_len, variance)
    lam, V = sla.eigh(Cc, subset_by_index=[M - n_z, M - 1])
    lam, V = lam[::-1], _fix_sign(V[:, ::-1])
    mu = np.maximum(lam, 1e-300) / M
    W = V * (np.sqrt(M) / (M * mu))[None, :]           # [M, n_z]
    out = np.empty((n_t, n_z))
    chunk = 16384
    for s in range(0, n_t, chunk):
        out[s:s + chunk] = _cov(cent[s:s + chunk], coarse, corr_len, variance) @ W
    out *= np.sqrt(mu)[None, :]
    return out


def obs_lattice_indices(N: int, m: int) -> np.ndarray:
    """Lattice coordinates round(k (N-1)/(m+1)), k = 1..m, in integer arithmetic."""
    k = np.arange(1, m + 1, dtype=np.int64)
    return (2 * k * (N - 1) + m + 1) // (2 * (m + 1))


def obs_vertices(N: int, m: int) -> np.ndarray:
    """Flat ids j*N+i of the m x m observation lattice, row-major (j outer)."""
    ix = obs_lattice_indices(N, m)
    jj, ii = np.meshgrid(ix, ix, indexing="ij")
    return (jj * N + ii).ravel().astype(np.int32)


def draw_Z(cfg: Config, batch: int | None = None) -> np.ndarray:
    """Prior samples Z ~ N(0, I), shape [batch, n_z], FP64."""
    rz, _, _ = _streams(cfg)
    return rz.standard_normal((cfg.batch if batch is None else batch, cfg.n_z))


def draw_Z_true(cfg: Config) -> np.ndarray:
    _, rt, _ = _streams(cfg)
    return rt.standard_normal(cfg.n_z)


def draw_noise(cfg: Config) -> np.ndarray:
    _, _, rn = _streams(cfg)
    return cfg.sigma * rn.standard_normal(cfg.obs_side * cfg.obs_side)


def observations(cfg: Config) -> np.ndarray:
    """Stored data y = u(Z_true)[obs] + noise, written by the oracle's data script."""
    path = os.path.join(_DATA_DIR, "observations.json")
    with open(path) as fh:
        data = json.load(fh)
    if cfg.name not in data:
        raise KeyError(f"no stored observations for {cfg.name} in {path}")
    y = np.asarray(data[cfg.name]["y"], dtype=np.float64)
    assert y.size == cfg.obs_side ** 2
    return y


@dataclass
class Problem:
    """All arrays of one workload (host, FP64/int32)."""
    cfg: Config
    phi: np.ndarray          # [n_t, n_z]
    obs: np.ndarray          # [n_obs] int32 flat vertex ids
    Z: np.ndarray            # [batch, n_z]
    y: np.ndarray | None = field(default=None)


def make_problem(cfg: Config, batch: int | None = None, with_y: bool = True) -> Problem:
    phi = kl_basis(cfg.N, cfg.n_z, cfg.corr_len, cfg.variance)
    obs = obs_vertices(cfg.N, cfg.obs_side)
    Z = draw_Z(cfg, batch)
    y = observations(cfg) if with_y else None
    return Problem(cfg, phi, obs, Z, y)
