"""Pins of the oracle's nonlinear term and Strang step (Sec. 3 Eq. 1-3, Sec. 4.4).

* Steady zonal flow in gradient-wind balance (the standard solid-body-rotation state,
  u = u0 cos(lat), g h = g h0 - (a Omega u0 + u0^2/2) sin^2(lat)) is a fixed point of the
  full tendency L U + N(U): this pins the curl / kinetic-energy part of N_delta with a
  closed form.
* The flux forms -div(Phi' V), -div(zeta V), k.curl(zeta V) equal their advective forms
  -(V.grad q + q delta) and zeta^2 + (dq/dx v - dq/dy u), computed through a different
  route (scalar gradients on the grid), to rounding.
* Strang ver1 and ver0 with REXI converge at 2nd order to a small-step RK4 reference (the
  paper's own reference is RK4 with a tiny step, Sec. 5).
"""
import math

import numpy as np
import pytest

from oracle import coeffs, linop, rexi, sht, swe
from paper_1805_06557_gb300 import synthetic as syn

OM, A, PB = syn.OMEGA, syn.RADIUS, syn.PHIBAR


def _tc2(T, grid, u0=38.61):
    U = np.zeros((3, sht.nlm(T)), complex)
    U[1, sht.idx(T, 0, 1)] = 2 * u0 / A / math.sqrt(3 / (4 * math.pi))
    phi = -(A * OM * u0 + 0.5 * u0 * u0) * (grid.mu[:, None] ** 2) * np.ones((1, grid.nlon))
    U[0] = grid.analys(phi)
    return U


def test_steady_zonal_flow_full_tendency():
    T, nlat, nlon = 15, 24, 48
    g = sht.Grid(T, nlat, nlon, A)
    U = _tc2(T, g)
    L = linop.apply_L(U, T, OM, A, PB)
    N = swe.nonlinear(U, g)
    tot = L + N
    for f in (0, 2):
        scale = max(np.max(np.abs(L[f])), np.max(np.abs(N[f])), 1e-300)
        assert np.max(np.abs(tot[f])) < 1e-10 * scale
    assert np.max(np.abs(tot[1])) < 1e-10 * np.max(np.abs(L[2]))
    # the nonlinear part alone is not zero: the balance needs the u0^2/2 term
    assert np.max(np.abs(N[2])) > 1e-3 * np.max(np.abs(L[2]))


def _grad_grid(grid, q):
    """(1 - mu^2) dq/dmu and dq/dlambda on the grid, through synth_uv(-a q, 0)."""
    Uq, Vq = grid.synth_uv(-grid.a * q, np.zeros_like(q))
    return Uq, -Vq


@pytest.mark.parametrize("T,nlat,nlon", [(15, 24, 48), (21, 33, 66)])
def test_flux_vs_advective_forms(T, nlat, nlon):
    g = sht.Grid(T, nlat, nlon, A)
    U = syn.gaussian_state(T, 5, scales=(1e3, 2e-5, 5e-6))
    N = swe.nonlinear(U, g)
    Phi, zeta, delta = U
    psi = sht.inv_laplacian(zeta, T, A)
    chi = sht.inv_laplacian(delta, T, A)
    Ug, Vg = g.synth_uv(psi, chi)
    c2 = g.coslat2[:, None]
    Dg = g.synth(delta)
    lap = sht.laplacian_eig(T, A)
    for f, q in ((0, Phi), (1, zeta)):
        qg = g.synth(q)
        dmu, dlam = _grad_grid(g, q)
        adv = (Ug * dlam + Vg * dmu) / (A * c2)
        ref = -g.analys(adv + qg * Dg)
        ref[0] = N[f][0]
        assert np.linalg.norm(N[f] - ref) <= 1e-11 * np.linalg.norm(ref)
    Zg = g.synth(zeta)
    dmu, dlam = _grad_grid(g, zeta)
    curl = Zg * Zg + (dlam * Vg - dmu * Ug) / (A * c2)
    ke = (Ug * Ug + Vg * Vg) / (2 * c2)
    ref = g.analys(curl) - lap * g.analys(ke)
    ref[0] = 0
    assert np.linalg.norm(N[2] - ref) <= 1e-11 * np.linalg.norm(ref)


def test_mass_conservation():
    T = 15
    g = sht.Grid(T, 24, 48, A)
    N = swe.nonlinear(syn.balanced_state(T, 2), g)
    assert abs(N[0][0]) < 1e-12 * np.max(np.abs(N[0]))


def test_strang_ver1_second_order():
    T, nlat, nlon = 15, 24, 48
    g = sht.Grid(T, nlat, nlon, A)
    U0 = syn.balanced_state(T, 2, urms=40.0)
    U0[2] = syn.gaussian_state(T, 8, scales=(0, 0, 2e-6))[2]   # add some divergence
    t_end = 4 * 1800.0
    ref = swe.rk4_full(U0, g, t_end, 240, OM, PB)
    errs = []
    for dt in (1800.0, 900.0, 450.0):
        X = rexi.spectrum_bound(T, dt, OM, A, PB)
        # the circle through p0 and +-iXc must not pass close to the origin: p0 <= Xc
        z, w = coeffs.rexi_coefficients(128, min(6.0, 1.6 * X), 1.6 * X)
        U = U0
        for _ in range(int(round(t_end / dt))):
            U = swe.strang_ver1(U, g, dt, OM, PB, z, w)
        errs.append(float(np.max(rexi.rel_l2(U, ref, T))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.7 < r < 2.5 for r in rates), (errs, rates)


def test_strang_ver0_second_order():
    """Version 0 of the split (Sec. 4.4: L^{dt/2} N^{dt} L^{dt/2}, REXI coefficients for dt/2)
    converges at 2nd order to the same RK4 reference as version 1."""
    T, nlat, nlon = 15, 24, 48
    g = sht.Grid(T, nlat, nlon, A)
    U0 = syn.balanced_state(T, 2, urms=40.0)
    U0[2] = syn.gaussian_state(T, 8, scales=(0, 0, 2e-6))[2]
    t_end = 4 * 1800.0
    ref = swe.rk4_full(U0, g, t_end, 240, OM, PB)
    errs = []
    for dt in (1800.0, 900.0, 450.0):
        X = rexi.spectrum_bound(T, 0.5 * dt, OM, A, PB)
        z, w = coeffs.rexi_coefficients(128, min(6.0, 1.6 * X), 1.6 * X)
        U = U0
        for _ in range(int(round(t_end / dt))):
            U = swe.strang_ver0(U, g, dt, OM, PB, z, w)
        errs.append(float(np.max(rexi.rel_l2(U, ref, T))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.7 < r < 2.5 for r in rates), (errs, rates)


def _rk4_nonlinear(U, g, tau, n):
    """n classical RK4 steps of dU/dt = N(U) over tau: an independent reference for the
    sub-stepped midpoint rule."""
    h = tau / n
    for _ in range(n):
        k1 = swe.nonlinear(U, g)
        k2 = swe.nonlinear(U + 0.5 * h * k1, g)
        k3 = swe.nonlinear(U + 0.5 * h * k2, g)
        k4 = swe.nonlinear(U + h * k3, g)
        U = U + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return U


def test_substepped_erk_second_order_in_substep():
    """N^{tau} by nsub midpoint steps of tau / nsub converges at 2nd order in tau / nsub to the
    exact nonlinear flow (RK4 with many steps): doubling nsub divides the error by ~4.  A
    sub-step that used tau instead of tau / nsub, or left the loop after one pass, fails."""
    T, nlat, nlon = 15, 24, 48
    g = sht.Grid(T, nlat, nlon, A)
    U0 = syn.balanced_state(T, 2, urms=40.0)
    U0[2] = syn.gaussian_state(T, 8, scales=(0, 0, 2e-6))[2]
    tau = 6 * 3600.0
    ref = _rk4_nonlinear(U0, g, tau, 96)
    errs = [float(np.max(rexi.rel_l2(swe.rk2_nonlinear(U0, g, tau, n), ref, T))) for n in (2, 4, 8)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < r < 2.3 for r in rates), (errs, rates)


def test_strang_ver1_substepped_second_order():
    """l_rexi_n_erk_ver1 with N sub-stepped (nsub = 3 midpoint steps per half step) still
    converges at 2nd order in dt to a small-step RK4 reference, and its sub-steps make the
    explicit part closer to the exact N flow than one midpoint step at the largest dt."""
    T, nlat, nlon = 15, 24, 48
    g = sht.Grid(T, nlat, nlon, A)
    U0 = syn.balanced_state(T, 2, urms=40.0)
    U0[2] = syn.gaussian_state(T, 8, scales=(0, 0, 2e-6))[2]
    t_end = 4 * 1800.0
    ref = swe.rk4_full(U0, g, t_end, 240, OM, PB)
    errs = []
    for dt in (1800.0, 900.0, 450.0):
        X = rexi.spectrum_bound(T, dt, OM, A, PB)
        z, w = coeffs.rexi_coefficients(128, min(6.0, 1.6 * X), 1.6 * X)
        U = U0
        for _ in range(int(round(t_end / dt))):
            U = swe.strang_ver1(U, g, dt, OM, PB, z, w, nsub=3)
        errs.append(float(np.max(rexi.rel_l2(U, ref, T))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.7 < r < 2.5 for r in rates), (errs, rates)
    tau = 1800.0
    exact = _rk4_nonlinear(U0, g, tau, 64)
    e1 = float(np.max(rexi.rel_l2(swe.rk2_nonlinear(U0, g, tau, 1), exact, T)))
    e3 = float(np.max(rexi.rel_l2(swe.rk2_nonlinear(U0, g, tau, 3), exact, T)))
    assert e3 < e1 / 6, (e1, e3)


def _grid_laplacian(c, g):
    """lap f by the grid route: V = grad f from the vector synthesis (psi = 0, chi = f), then
    the divergence analysis; independent of the spectral eigenvalues -n(n+1)/a^2."""
    U, V = g.synth_uv(np.zeros_like(c), c)
    div, _ = g.analys_divcurl(U, V)
    return div


def test_diffusion_generator_is_grid_bilaplacian():
    """The exact diffusion flow over a short tau moves U by -tau nu lap^2 U to first order:
    checked against lap applied twice on the Gauss grid (q = 2), and for q = 1 against one
    grid Laplacian.  n = 0 stays unchanged and no coefficient grows."""
    T, nlat, nlon = 15, 24, 48
    g = sht.Grid(T, nlat, nlon, A)
    U = syn.gaussian_state(T, 41)
    # central differences over +-tau: the generator to O((tau nu k^4)^2), tau nu k_T^4 ~ 1e-4
    nu4, tau = 1e15, 3000.0
    gen = (swe.diffuse(U, T, A, tau, nu4, 2) - swe.diffuse(U, T, A, -tau, nu4, 2)) / (2 * tau)
    for f in range(3):
        ref = -nu4 * _grid_laplacian(_grid_laplacian(U[f], g), g)
        assert np.linalg.norm(gen[f] - ref) < 1e-7 * np.linalg.norm(ref)
    nu2 = 1e2
    gen1 = (swe.diffuse(U, T, A, tau, nu2, 1) - swe.diffuse(U, T, A, -tau, nu2, 1)) / (2 * tau)
    ref1 = nu2 * _grid_laplacian(U[1], g)
    assert np.linalg.norm(gen1[1] - ref1) < 1e-7 * np.linalg.norm(ref1)
    big = swe.diffuse(U, T, A, 3600.0, nu4, 2)
    assert np.all(np.abs(big) <= np.abs(U) + 1e-300)
    assert np.array_equal(big[:, 0], U[:, 0])


def test_strang_ver1_with_diffusion_second_order():
    """D^{dt/2} o (N^{dt/2} L^{dt} N^{dt/2} with nsub = 2) o D^{dt/2} converges at 2nd order
    to a small-step RK4 solution of dU/dt = L U + N(U) - nu lap^2 U."""
    T, nlat, nlon = 15, 24, 48
    g = sht.Grid(T, nlat, nlon, A)
    U0 = syn.balanced_state(T, 2, urms=40.0)
    U0[2] = syn.gaussian_state(T, 8, scales=(0, 0, 2e-6))[2]
    lam2 = sht.laplacian_eig(T, A) ** 2
    nu = 0.3 / (3600.0 * (T * (T + 1) / A ** 2) ** 2)   # degree T e-folds in about 3 h
    t_end = 4 * 1800.0
    h, U = t_end / 240, U0
    for _ in range(240):
        f = lambda V: swe.full_tendency(V, g, OM, PB) - nu * lam2[None, :] * V
        k1 = f(U); k2 = f(U + 0.5 * h * k1); k3 = f(U + 0.5 * h * k2); k4 = f(U + h * k3)
        U = U + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    ref = U
    errs = []
    for dt in (1800.0, 900.0, 450.0):
        X = rexi.spectrum_bound(T, dt, OM, A, PB)
        z, w = coeffs.rexi_coefficients(128, min(6.0, 1.6 * X), 1.6 * X)
        U = U0
        step = lambda V: swe.strang_ver1(V, g, dt, OM, PB, z, w, nsub=2)
        for _ in range(int(round(t_end / dt))):
            U = swe.with_diffusion(step, U, T, A, dt, nu)
        errs.append(float(np.max(rexi.rel_l2(U, ref, T))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.7 < r < 2.5 for r in rates), (errs, rates)


# ---- ETD2RK (Sec. 4.3) ------------------------------------------------------------------
def _psi_weights(N, p0, Xc):
    z, w0 = coeffs.rexi_coefficients(N, p0, Xc, k=0)
    _, w1 = coeffs.rexi_coefficients(N, p0, Xc, k=1)
    _, w2 = coeffs.rexi_coefficients(N, p0, Xc, k=2)
    return z, w0, w1, w2


def test_exact_phi_defining_identities():
    """psi_1(K) and psi_2(K) of K = dt L satisfy K psi_1(K) = e^K - I and
    K psi_2(K) = psi_1(K) - I; psi_0 equals exp."""
    T, dt = 15, 3600.0
    U = syn.gaussian_state(T, 21)
    e = rexi.exact_step(U, T, dt, OM, A, PB)
    p0_ = rexi.exact_phi(U, T, dt, OM, A, PB, 0)
    p1 = rexi.exact_phi(U, T, dt, OM, A, PB, 1)
    p2 = rexi.exact_phi(U, T, dt, OM, A, PB, 2)
    KL = lambda V: dt * linop.apply_L(V, T, OM, A, PB)
    assert np.max(rexi.rel_l2(p0_, e, T)) < 1e-12
    assert np.max(rexi.rel_l2(KL(p1), e - U, T)) < 1e-10
    assert np.max(rexi.rel_l2(KL(p2), p1 - U, T)) < 1e-10


@pytest.mark.parametrize("k", [1, 2])
def test_rexi_psi_weights_vs_exact(k):
    """REXI with the psi_k weights of the same poles applies psi_k(dt L) to within its scalar
    error (energy norm; the operator is normal in the energy inner product)."""
    T, dt, N = 15, 3600.0, 128
    X = rexi.spectrum_bound(T, dt, OM, A, PB)
    p0, Xc = min(6.0, 1.6 * X), 1.6 * X
    z, w = coeffs.rexi_coefficients(N, p0, Xc, k=k)
    x = 1j * np.linspace(-X, X, 4001)
    x = x[np.abs(x) > 1e-6]
    ref = (np.expm1(x) / x) if k == 1 else ((np.expm1(x) - x) / x ** 2)
    es = float(np.max(np.abs(coeffs.rational_eval(z, w, x) - ref)))
    U = syn.gaussian_state(T, 22)
    Ur = rexi.rexi_step(U, T, dt, OM, A, PB, z, w)
    Ue = rexi.exact_phi(U, T, dt, OM, A, PB, k)
    err = math.sqrt(linop.energy(Ur - Ue, T, A, PB) / linop.energy(U, T, A, PB))
    assert err <= es + 1e-12, (err, es)


def test_etd2rk_exact_for_constant_forcing():
    """For N(U) = F constant the ETD2RK step is exact: U+ = e^{dt L} U + dt psi_1(dt L) F
    (the psi_2 term vanishes); checked against the eigen-decomposition."""
    T, dt, N = 15, 3600.0, 128
    g = sht.Grid(T, 24, 48, A)
    X = rexi.spectrum_bound(T, dt, OM, A, PB)
    z, w0, w1, w2 = _psi_weights(N, min(6.0, 1.6 * X), 1.6 * X)
    U = syn.gaussian_state(T, 23)
    F = syn.gaussian_state(T, 24, scales=(1e-2, 1e-10, 1e-10))
    out = swe.etd2rk(U, g, dt, OM, PB, z, w0, w1, w2, nonlin=lambda V: F)
    ref = rexi.exact_step(U, T, dt, OM, A, PB) + dt * rexi.exact_phi(F, T, dt, OM, A, PB, 1)
    assert np.max(rexi.rel_l2(out, ref, T)) < 1e-9


def test_etd2rk_second_order():
    """ETD2RK (l_rexi_n_etdrk) converges at 2nd order to a small-step RK4 reference."""
    T, nlat, nlon = 15, 24, 48
    g = sht.Grid(T, nlat, nlon, A)
    U0 = syn.balanced_state(T, 2, urms=40.0)
    U0[2] = syn.gaussian_state(T, 8, scales=(0, 0, 2e-6))[2]
    t_end = 4 * 1800.0
    ref = swe.rk4_full(U0, g, t_end, 240, OM, PB)
    errs = []
    for dt in (1800.0, 900.0, 450.0):
        X = rexi.spectrum_bound(T, dt, OM, A, PB)
        z, w0, w1, w2 = _psi_weights(128, min(6.0, 1.6 * X), 1.6 * X)
        U = U0
        for _ in range(int(round(t_end / dt))):
            U = swe.etd2rk(U, g, dt, OM, PB, z, w0, w1, w2)
        errs.append(float(np.max(rexi.rel_l2(U, ref, T))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.7 < r < 2.6 for r in rates), (errs, rates)


# ---- Crank-Nicolson (Sec. 4.1, irk) -------------------------------------------------------
def test_cn_step_matches_cayley_and_conserves_energy():
    """CN with a = 1/2 is the Cayley map of dt L: equal to the eigen-decomposition route, and,
    L being skew-adjoint in the energy inner product, it conserves the linear energy exactly."""
    T, dt = 15, 3600.0
    U = syn.gaussian_state(T, 31)
    cn = rexi.cn_step(U, T, dt, OM, A, PB)
    ref = rexi.exact_cayley(U, T, dt, OM, A, PB)
    assert np.max(rexi.rel_l2(cn, ref, T)) < 1e-11
    E0, E1 = linop.energy(U, T, A, PB), linop.energy(cn, T, A, PB)
    assert abs(E1 / E0 - 1.0) < 1e-12


def test_cn_step_third_order_local_error():
    """One CN step differs from exp(dt L) by O(dt^3): halving dt divides the gap by ~8."""
    T = 15
    U = syn.gaussian_state(T, 32)
    gaps = []
    for dt in (400.0, 200.0, 100.0):
        gaps.append(float(np.max(rexi.rel_l2(rexi.cn_step(U, T, dt, OM, A, PB),
                                             rexi.exact_step(U, T, dt, OM, A, PB), T))))
    rates = [math.log2(gaps[i] / gaps[i + 1]) for i in range(2)]
    assert all(2.7 < r < 3.3 for r in rates), (gaps, rates)


def test_cn_ver1_second_order():
    """l_irk_n_erk_ver1 converges at 2nd order to a small-step RK4 reference."""
    T, nlat, nlon = 15, 24, 48
    g = sht.Grid(T, nlat, nlon, A)
    U0 = syn.balanced_state(T, 2, urms=40.0)
    U0[2] = syn.gaussian_state(T, 8, scales=(0, 0, 2e-6))[2]
    t_end = 4 * 1800.0
    ref = swe.rk4_full(U0, g, t_end, 240, OM, PB)
    errs = []
    for dt in (1800.0, 900.0, 450.0):
        U = U0
        for _ in range(int(round(t_end / dt))):
            U = swe.cn_ver1(U, g, dt, OM, PB)
        errs.append(float(np.max(rexi.rel_l2(U, ref, T))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.7 < r < 2.6 for r in rates), (errs, rates)
