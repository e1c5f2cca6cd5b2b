"""Write the stored observation data y = u(Z_true)[obs] + noise (test infrastructure).

y is the oracle's FP64 solution at the seeded Z_true (with one long-double
refinement step) restricted to the observation lattice, plus seeded N(0, sigma^2)
noise.  Run:  python -m oracle.make_observations [config ...]
It writes workload/data/observations.json, which the benchmark and the tests read
as plain data.
"""
import json
import os
import sys

import numpy as np

import workload as w
from oracle import fem


def make(name: str) -> dict:
    cfg = w.CONFIGS[name]
    phi = w.kl_basis(cfg.N, cfg.n_z, cfg.corr_len, cfg.variance)
    obs = w.obs_vertices(cfg.N, cfg.obs_side)
    kap = fem.kappa_from_kl(phi, w.draw_Z_true(cfg))
    u = fem.solve_full(cfg.N, kap, cfg.f, refine=True)
    y = u[obs] + w.draw_noise(cfg)
    return {"y": [float(v) for v in y], "sigma": cfg.sigma, "N": cfg.N,
            "n_obs": int(obs.size), "kappa_min": float(kap.min()), "kappa_max": float(kap.max())}


def main(argv):
    names = argv or list(w.CONFIGS)
    path = os.path.join(os.path.dirname(os.path.abspath(w.__file__)), "data", "observations.json")
    data = {}
    if os.path.exists(path):
        with open(path) as fh:
            data = json.load(fh)
    for n in names:
        data[n] = make(n)
        print(n, "kappa range", data[n]["kappa_min"], data[n]["kappa_max"])
    with open(path, "w") as fh:
        json.dump(data, fh, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
