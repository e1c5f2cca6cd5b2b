"""Shared helpers of the GPU parity tests (inputs and the oracle reference)."""
import numpy as np

import workload as w
from oracle import fem


def oracle_eval(N, phi, Z, obs, y, sigma, f=1.0):
    """Oracle u at obs and log-likelihood per sample (long-double refined solve)."""
    U, L = [], []
    for z in np.atleast_2d(Z):
        u_obs, ll = fem.evaluate(N, phi, z, obs, y, sigma, f, refine=True)
        U.append(u_obs)
        L.append(ll)
    return np.array(U), np.array(L)


def oracle_full(N, phi, Z, f=1.0):
    """Oracle solution at every vertex, per sample."""
    return np.array([fem.solve_full(N, fem.kappa_from_kl(phi, z), f, refine=True) for z in np.atleast_2d(Z)])


def rel_err_field(u, ref):
    """max_k |u_k - ref_k| / max_k |ref_k| per sample."""
    return np.max(np.abs(u - ref), axis=-1) / np.max(np.abs(ref), axis=-1)


def rel_err_scalar(a, ref):
    return np.abs(a - ref) / np.abs(ref)


def interior(N):
    return fem.interior_ids(N).astype(np.int32)


def small_problem(N, n_z=10, corr_len=0.3, variance=1.0, batch=3, seed=0):
    phi = w.kl_basis(N, n_z, corr_len, variance)
    Z = np.random.default_rng(seed).standard_normal((batch, n_z))
    return phi, Z
