"""FP64 CPU oracle for the HDD likelihood path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The GPU library never calls it and shares no code with it;
the two meet only in the seeded input arrays of the ``workload`` package.

  fem.py        plain P1 finite elements + banded Cholesky: the definition of
                what the HDD path computes (u at the observation vertices and the
                Gaussian log-likelihood).  Sec. 1.1 (Eq. elliptic), Sec. 3.1
                (Eq. coefA, Eq. coefc), Sec. 1.2 (likelihood).
  hdd_dense.py  the HDD method itself written out densely in NumPy (tree of
                Sec. 2.1, Schur maps of Sec. 2.4, father system of Sec. 3.3,
                "Leaves to Root" / "Root to Leaves" of Sec. 3.4, pruned descent
                of Sec. 5.3).  Used to pin the tree bookkeeping, the Schur
                complements and the equivalence of HDD with the global solve.
  make_observations.py  writes the stored observation data y (oracle solution
                at Z_true plus seeded noise).

Every function here is pinned by the ``-m "not gpu"`` tests against closed forms,
spectral solves, brute-force dense inversion, invariants and the paper's
appendix sizes.  Nothing here is "parity unpinned".
"""
