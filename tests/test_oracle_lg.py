"""Pins of the oracle's gravity-only REXI and the lg schemes (Sec. 3, the L_g / L_c split;
Sec. 5.3 diagonal solve; Table 2 lg_rexi_lc_n_erk_ver1 and lg_rexi_lc_n_etdrk).

* L_c alone evaluated spectrally equals the Coriolis terms evaluated through the Gauss grid
  (-div(f V), k.curl(f V) with f = 2 Omega mu; an independent route, as pin P2).
* The closed-form exp(dt L_g) equals the eigen-decomposition of the full operator at Omega = 0
  and scipy's expm (two independent routes).
* The per-coefficient 2 x 2 REXI solve equals the pivoted banded LU of the full operator at
  Omega = 0 (no Coriolis: L = L_g), and lies within the scalar error of the closed form.
* psi_1 / psi_2 weights of the same poles apply psi_k(dt L_g) (Sec. 4.3).
* lg ver1 and lg ETD2RK converge at 2nd order to a small-step RK4 reference of the same PDE.
* Crank-Nicolson of L_g alone is the Cayley map of dt L_g (eigen route at Omega = 0) and its
  ver0 split (lg_irk_lc_n_erk_ver0) converges at 2nd order.
"""
import math

import numpy as np
import pytest

from oracle import coeffs, linop, rexi, rexi_lg, sht, swe
from paper_1805_06557_gb300 import synthetic as syn

OM, A, PB = syn.OMEGA, syn.RADIUS, syn.PHIBAR


def _X_lg(T, dt):
    """Spectral bound of dt L_g: the gravity-wave frequency of degree T."""
    return dt * math.sqrt(PB * T * (T + 1.0)) / A


def test_split_sums_to_L_and_Lc_on_the_grid():
    for T, nlat, nlon in [(15, 24, 48), (31, 48, 96)]:
        g = sht.Grid(T, nlat, nlon, A)
        U = syn.gaussian_state(T, 41)
        Lg = linop.apply_L(U, T, OM, A, PB, part="Lg")
        Lc = linop.apply_L(U, T, OM, A, PB, part="Lc")
        assert np.max(rexi.rel_l2(Lg + Lc, linop.apply_L(U, T, OM, A, PB), T)) < 1e-14
        # with Phi' = 0 and Phibar = 0 the grid route of L reduces to the Coriolis terms
        V = U.copy()
        V[0] = 0.0
        grid = linop.apply_L_grid(V, g, OM, 0.0)
        assert np.max(rexi.rel_l2(Lc[1:], grid[1:], T)) < 1e-11   # the tolerance of pin P2
        assert np.all(Lc[0] == 0)
        # L_g has no Omega in it
        assert np.max(rexi.rel_l2(Lg, linop.apply_L(U, T, 0.0, A, PB), T)) == 0.0


@pytest.mark.parametrize("dt", [600.0, 3600.0, 14400.0])
def test_exact_lg_closed_form(dt):
    T = 15
    U = syn.gaussian_state(T, 42)
    cf = rexi_lg.exact_lg(U, T, dt, A, PB)
    eig = rexi.exact_step(U, T, dt, 0.0, A, PB)
    assert np.max(rexi.rel_l2(cf, eig, T)) < 1e-12
    ex = rexi.exact_step_expm(U, T, dt, 0.0, A, PB)
    assert np.max(rexi.rel_l2(cf, ex, T)) < 1e-11
    # the gravity wave energy is conserved exactly
    assert abs(linop.energy(cf, T, A, PB) / linop.energy(U, T, A, PB) - 1.0) < 1e-13


@pytest.mark.parametrize("T,dt,N", [(7, 3600.0, 64), (15, 3600.0, 128), (21, 14400.0, 256)])
def test_diagonal_solve_equals_banded_lu(T, dt, N):
    X = _X_lg(T, dt)
    z, w = coeffs.rexi_coefficients(N, min(6.0, 1.6 * X), 1.6 * X)
    U = syn.gaussian_state(T, 43)
    d = rexi_lg.rexi_step_lg(U, T, dt, A, PB, z, w)
    b = rexi.rexi_step(U, T, dt, 0.0, A, PB, z, w)
    amp = coeffs.amplification(z, w, X)
    assert np.max(rexi.rel_l2(d, b, T)) < max(1e-13, 16 * amp * 2.0 ** -53)


@pytest.mark.parametrize("T,dt,N,p0,marg", [(15, 3600.0, 128, 6.0, 1.6), (31, 14400.0, 256, 8.0, 1.5)])
def test_rexi_lg_within_scalar_error(T, dt, N, p0, marg):
    """L_g is normal in the energy inner product, so the REXI error in that norm is bounded by
    the scalar error on [-iX, iX] (as pin P4 for the full operator)."""
    X = _X_lg(T, dt)
    z, w = coeffs.rexi_coefficients(N, min(p0, marg * X), marg * X)
    es = coeffs.scalar_error(z, w, X, npts=4001)
    U = syn.gaussian_state(T, 44)
    Ur = rexi_lg.rexi_step_lg(U, T, dt, A, PB, z, w)
    Ue = rexi_lg.exact_lg(U, T, dt, A, PB)
    err = math.sqrt(linop.energy(Ur - Ue, T, A, PB) / linop.energy(U, T, A, PB))
    amp = coeffs.amplification(z, w, X)
    assert err <= es + 50 * amp * 2.0 ** -53, (err, es)
    # zeta is only divided by each pole: it comes back scaled by sum_p w_p / z_p ~ e^0
    s0 = np.sum(w / z)
    assert np.max(np.abs(Ur[1] - s0 * U[1])) <= 1e-14 * np.max(np.abs(U[1])) * np.sum(np.abs(w / z))


@pytest.mark.parametrize("k", [1, 2])
def test_rexi_lg_psi_weights(k):
    T, dt, N = 15, 3600.0, 128
    X = _X_lg(T, dt)
    z, w = coeffs.rexi_coefficients(N, min(6.0, 1.6 * X), 1.6 * X, k=k)
    x = 1j * np.linspace(-X, X, 4001)
    x = x[np.abs(x) > 1e-6]
    ref = (np.expm1(x) / x) if k == 1 else ((np.expm1(x) - x) / x ** 2)
    es = float(np.max(np.abs(coeffs.rational_eval(z, w, x) - ref)))
    U = syn.gaussian_state(T, 45)
    Ur = rexi_lg.rexi_step_lg(U, T, dt, A, PB, z, w)
    Ue = rexi.exact_phi(U, T, dt, 0.0, A, PB, k)
    err = math.sqrt(linop.energy(Ur - Ue, T, A, PB) / linop.energy(U, T, A, PB))
    assert err <= es + 1e-12, (err, es)


def _converges(step, rate_lo=1.7, rate_hi=2.6):
    T, nlat, nlon = 15, 24, 48
    g = sht.Grid(T, nlat, nlon, A)
    U0 = syn.balanced_state(T, 2, urms=40.0)
    U0[2] = syn.gaussian_state(T, 8, scales=(0, 0, 2e-6))[2]
    t_end = 4 * 1800.0
    ref = swe.rk4_full(U0, g, t_end, 240, OM, PB)
    errs = []
    for dt in (1800.0, 900.0, 450.0):
        X = _X_lg(T, dt)
        U = U0
        for _ in range(int(round(t_end / dt))):
            U = step(U, g, dt, X)
        errs.append(float(np.max(rexi.rel_l2(U, ref, T))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(rate_lo < r < rate_hi for r in rates), (errs, rates)


def test_strang_lg_ver1_second_order():
    def step(U, g, dt, X):
        z, w = coeffs.rexi_coefficients(128, min(6.0, 1.6 * X), 1.6 * X)
        return swe.strang_lg_ver1(U, g, dt, OM, PB, z, w)
    _converges(step)


def test_etd2rk_lg_second_order():
    def step(U, g, dt, X):
        p0, Xc = min(6.0, 1.6 * X), 1.6 * X
        z, w0 = coeffs.rexi_coefficients(128, p0, Xc, k=0)
        w1 = coeffs.rexi_coefficients(128, p0, Xc, k=1)[1]
        w2 = coeffs.rexi_coefficients(128, p0, Xc, k=2)[1]
        return swe.etd2rk_lg(U, g, dt, OM, PB, z, w0, w1, w2)
    _converges(step)


def test_cn_of_lg_is_the_cayley_map():
    T, dt = 15, 3600.0
    U = syn.gaussian_state(T, 46)
    cn = rexi.cn_step(U, T, dt, OM, A, PB, part="Lg")
    ref = rexi.exact_cayley(U, T, dt, 0.0, A, PB)
    assert np.max(rexi.rel_l2(cn, ref, T)) < 1e-12
    # L_g has no zeta terms: zeta passes through unchanged
    assert np.max(np.abs(cn[1] - U[1])) == 0.0


def test_cn_lg_ver0_second_order():
    _converges(lambda U, g, dt, X: swe.cn_lg_ver0(U, g, dt, OM, PB))
