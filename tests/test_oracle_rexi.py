"""Pins of the oracle's linear operator and REXI step (Sec. 3 Eq. 1-3, Sec. 4.2 Eq. rexi).

P2  spectral L equals L evaluated through the Gauss grid (independent route).
P3  with Omega = 0 the eigenvalues are 0 and +-i sqrt(Phibar n(n+1))/a (gravity waves);
    W L is skew-symmetric in the linear-energy weights.
P4  the REXI result is within e_s of the exact exponential in the energy norm (L is normal in
    that norm, so the operator error equals the scalar error on the spectrum).
P5  linear energy is conserved to within 2 e_s.
P6  k-substep RK4 converges to the REXI result like k^-4 down to e_s.
P7  a zonal flow in linear balance is a fixed point of L and of the REXI step.
P9  dense numpy.linalg.solve per pole equals the banded LU.
"""
import math

import numpy as np
import pytest

from oracle import coeffs, linop, rexi, sht, swe
from paper_1805_06557_gb300 import synthetic as syn

OM, A, PB = syn.OMEGA, syn.RADIUS, syn.PHIBAR


def _state(T, seed=1):
    return syn.gaussian_state(T, seed)


def test_spectral_vs_grid_L_P2():
    for T, nlat, nlon in [(15, 24, 48), (31, 48, 96)]:
        g = sht.Grid(T, nlat, nlon, A)
        U = _state(T, 2)
        L1 = linop.apply_L(U, T, OM, A, PB)
        L2 = linop.apply_L_grid(U, g, OM, PB)
        for f in range(3):
            assert np.linalg.norm(L1[f] - L2[f]) <= 1e-11 * np.linalg.norm(L1[f])


@pytest.mark.parametrize("m", [0, 1, 5, 14])
def test_gravity_wave_eigenvalues_P3(m):
    T = 15
    ev = np.linalg.eigvals(linop.operator_m(T, m, 0.0, A, PB))
    freqs = sorted(np.abs(ev.imag))
    expect = [0.0] * (T + 1 - m) + sorted(
        [math.sqrt(PB * n * (n + 1)) / A for n in range(max(m, 1), T + 1)] * 2)
    if m == 0:  # the n = 0 rows are zero: three zero eigenvalues, no wave at n = 0
        expect = [0.0] * (T + 3) + sorted(
            [math.sqrt(PB * n * (n + 1)) / A for n in range(1, T + 1)] * 2)
    assert np.max(np.abs(np.array(freqs) - np.array(expect))) < 1e-12 * max(expect)
    assert np.max(np.abs(ev.real)) < 1e-12 * max(expect)


@pytest.mark.parametrize("m", [0, 2, 9])
def test_energy_skew_symmetry_P3(m):
    T = 15
    Lm = linop.operator_m(T, m, OM, A, PB)
    W = np.diag(linop.energy_weights_m(T, m, A, PB))
    S = W @ Lm
    assert np.max(np.abs(S + S.conj().T)) <= 1e-14 * np.max(np.abs(S))


def test_spectrum_bound():
    for T, dt in [(7, 3600.0), (15, 1800.0), (21, 7200.0)]:
        assert rexi.spectral_radius(T, dt, OM, A, PB) <= rexi.spectrum_bound(T, dt, OM, A, PB)


CONTOURS = [(7, 3600.0, 64, 4.0, 1.8), (15, 3600.0, 128, 6.0, 1.6), (15, 14400.0, 256, 8.0, 1.5)]


@pytest.mark.parametrize("T,dt,N,p0,marg", CONTOURS)
def test_rexi_vs_exact_P4_P5(T, dt, N, p0, marg):
    X = rexi.spectrum_bound(T, dt, OM, A, PB)
    z, w = coeffs.rexi_coefficients(N, p0, marg * X)
    es = coeffs.scalar_error(z, w, X, npts=4001)
    U = _state(T, 7)
    U1 = rexi.rexi_step(U, T, dt, OM, A, PB, z, w)
    Ue = rexi.exact_step(U, T, dt, OM, A, PB)
    E0 = linop.energy(U, T, A, PB)
    err = math.sqrt(linop.energy(U1 - Ue, T, A, PB) / E0)
    # the bound is exact up to the rounding of the solves (amplification * eps)
    amp = coeffs.amplification(z, w, X)
    assert err <= es + 50 * amp * 2.0 ** -53
    drift = abs(linop.energy(U1, T, A, PB) / E0 - 1.0)
    assert drift <= 2 * es + es * es + 100 * amp * 2.0 ** -53
    # both exact routes agree
    Ue2 = rexi.exact_step_expm(U, T, dt, OM, A, PB)
    assert np.max(rexi.rel_l2(Ue2, Ue, T)) < 1e-12


def test_rexi_long_step_independent_of_dt():
    """REXI integrates the linear part with arbitrarily long steps (Sec. 2.2 / 6): one step
    of 12 h equals twelve steps of 1 h to within the scalar errors."""
    T = 10
    U = _state(T, 11)
    Xl = rexi.spectrum_bound(T, 43200.0, OM, A, PB)
    zl, wl = coeffs.rexi_coefficients(256, 10.0, 1.4 * Xl)
    Xs = rexi.spectrum_bound(T, 3600.0, OM, A, PB)
    zs, ws = coeffs.rexi_coefficients(128, 6.0, 1.6 * Xs)
    one = rexi.rexi_step(U, T, 43200.0, OM, A, PB, zl, wl)
    many = U
    for _ in range(12):
        many = rexi.rexi_step(many, T, 3600.0, OM, A, PB, zs, ws)
    assert np.max(rexi.rel_l2(one, many, T)) < 1e-9


def test_rk4_convergence_P6():
    T, dt = 7, 3600.0
    X = rexi.spectrum_bound(T, dt, OM, A, PB)
    z, w = coeffs.rexi_coefficients(128, 6.0, 1.6 * X)
    U = _state(T, 3)
    ref = rexi.rexi_step(U, T, dt, OM, A, PB, z, w)
    errs = []
    for k in [4, 8, 16]:
        u = swe.rk4_linear(U, T, dt, k, OM, A, PB)
        errs.append(math.sqrt(linop.energy(u - ref, T, A, PB) / linop.energy(U, T, A, PB)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.6 < r < 4.4 for r in rates), (errs, rates)
    u = swe.rk4_linear(U, T, dt, 400, OM, A, PB)
    assert math.sqrt(linop.energy(u - ref, T, A, PB) / linop.energy(U, T, A, PB)) < 1e-11


def _balanced_zonal(T, u0=20.0):
    """u = u0 cos(lat): zeta = 2 u0 mu / a (n = 1); Phi' from f zeta - (2 Omega/a) U = lap Phi',
    Phi' = -a Omega u0 (mu^2 - 1/3)  (closed form)."""
    U = np.zeros((3, sht.nlm(T)), complex)
    U[1, sht.idx(T, 0, 1)] = 2 * u0 / A / math.sqrt(3 / (4 * math.pi))
    # mu^2 - 1/3 = (2/3) P_2(mu) = (2/3) Pt_2^0 / sqrt(5/(4 pi))
    U[0, sht.idx(T, 0, 2)] = -A * OM * u0 * (2.0 / 3.0) / math.sqrt(5 / (4 * math.pi))
    return U


def test_balanced_fixed_point_P7():
    T, dt = 15, 7200.0
    U = _balanced_zonal(T)
    LU = linop.apply_L(U, T, OM, A, PB)
    scale = abs(PB * 6 / A ** 2 * U[0, sht.idx(T, 0, 2)])
    assert np.max(np.abs(LU)) < 1e-13 * scale
    X = rexi.spectrum_bound(T, dt, OM, A, PB)
    z, w = coeffs.rexi_coefficients(256, 6.0, 1.6 * X)
    es = coeffs.scalar_error(z, w, X)
    U1 = rexi.rexi_step(U, T, dt, OM, A, PB, z, w)
    assert np.max(rexi.rel_l2(U1, U, T)[:2]) < 10 * es + 1e-12


def test_dense_vs_banded_P9():
    T, dt = 5, 3600.0
    X = rexi.spectrum_bound(T, dt, OM, A, PB)
    z, w = coeffs.rexi_coefficients(8, 3.0, 1.5 * X)
    U = _state(T, 4)
    a = rexi.rexi_step(U, T, dt, OM, A, PB, z, w)
    b = rexi.rexi_step_dense(U, T, dt, OM, A, PB, z, w)
    assert np.max(rexi.rel_l2(a, b, T)) < 1e-14


def test_real_field_symmetry():
    """With conjugate pole pairs the m = 0 output of a real field is real to rounding
    (Im / Re ~ amplification * eps)."""
    T, dt = 15, 3600.0
    X = rexi.spectrum_bound(T, dt, OM, A, PB)
    z, w = coeffs.rexi_coefficients(128, 6.0, 1.6 * X)
    U1 = rexi.rexi_step(_state(T, 9), T, dt, OM, A, PB, z, w)
    for f in range(3):
        m0 = U1[f, : T + 1]
        assert np.max(np.abs(m0.imag)) < 1e-12 * np.max(np.abs(m0))
