"""Plain, slow, FP64 CPU oracle for the REXI time step of the rotating shallow-water
equations (Schreiber, Schaeffer & Loft, arXiv 1805.06557).

TEST INFRASTRUCTURE ONLY.  Nothing in the product imports this package: only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import or run it.  It shares no code, table, constant or helper with the
CUDA library; both sides receive the same seeded inputs from
``paper_1805_06557_gb300.synthetic``, which holds none of the method's arithmetic.

Every function states the passage of the paper it follows.  Where the paper is silent the
docstring states the reading that is taken.  Library primitives used as single steps:
``numpy.polynomial.legendre.leggauss`` (Gauss nodes; the weights follow their definition),
``numpy.fft`` (longitude DFT),
``scipy.linalg.solve_banded`` (pivoted banded LU), ``scipy.linalg.expm`` / ``numpy.linalg.eig``
(exact exponential for the pins).

Modules
-------
coeffs  : Cauchy-contour REXI poles and weights (Sec. 4.2.1-4.2.2, Eq. cauchy_alpha/beta).
sht     : Gauss grid, orthonormal associated Legendre functions, scalar and vector
          spherical-harmonic analysis/synthesis (Sec. 3.2).
linop   : spectral form of the linear operator L = L_g + L_c per zonal order (Sec. 3, Eq. 1-3
          and the L_g / L_c split), its grid-space form, the linear energy.
rexi    : the REXI step  U(dt) ~ sum_n beta_n (dt L + alpha_n)^-1 U(0)  (Eq. rexi), solved per
          pole and zonal order with a pivoted banded LU, plus the exact exponential.
rexi_lg : REXI of the gravity operator L_g alone (the lg_* methods of Table 2): a per-degree
          2 x 2 solve per pole, and its closed-form exponential.
swe     : nonlinear term N(U) on the Gauss grid (Sec. 3, the N column of the split), RK2 (with
          optional sub-steps), RK4, the Strang, ETD2RK and Crank-Nicolson steps (Sec. 4.1-4.4),
          and the exact flow of a del^{2q} hyper-diffusion term split off around a step.
"""
