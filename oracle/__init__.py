"""FP64 CPU oracle for kernel columns phi(L) E_W (arXiv 2301.06384).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may call it.  It shares no code with the CUDA path: it is written in plain
numpy / scipy FP64 from the paper's statements, with library primitives (sparse
mat-mul, dense mat-mul, Householder QR, symmetric eigendecomposition, matrix exponential)
as single steps and no blocking, fusion or reordering beyond what the paper states.

Modules
-------
dense   -- the naive two-step spectral evaluation V phi(Lambda) V^T E_W (Section 3,
           Eq. (GBFcompute)) and textbook closed forms (path, cycle, grids) that pin it.
krylov  -- the five block Krylov approximations: classical block Lanczos (Algorithm 1),
           global block Lanczos (Algorithm 2), sequential Lanczos (Section 3.3),
           Chebyshev interpolation (Section 3.4, Eqs. (apprchebyshevseries), (chebcoeff))
           and squared Chebyshev (Section 3.4.1).
bounds  -- the a-priori error bounds of Theorem 4.2 with Eq. (boundapproximation).

Readings of the paper where it is silent or garbled are stated where they are used:
A1 H_{k,k+1} = H_{k+1,k}^T (Algorithm 1 sets them equal, the text says transpose);
A2 the sequential formula applies phi to H^{(w_i)}; A3 Lobatto interpolation
coefficients with endpoint halving; A4 T_0 = 1, T_1 = lambda; A5 Lambda = Gershgorin
bound; A6 breakdown handling; A9 the QR at k = m is skipped.

Every function is pinned by tests in ``tests/test_oracle_pins.py``; none is "parity
unpinned".
"""
from . import dense, krylov, bounds  # noqa: F401
