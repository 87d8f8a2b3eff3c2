"""Pins of the oracle's spherical-harmonic transforms (Sec. 3.2), pin P8.

Checked against scipy's independent spherical harmonics and associated Legendre functions,
against 40-digit mpmath values deep in the underflow region, and through identities of the
vector transforms (div of grad chi = lap chi, curl of k x grad psi = lap psi)."""
import math

import mpmath
import numpy as np
import pytest
import scipy.special as sp

from oracle import sht
from paper_1805_06557_gb300 import synthetic


def test_gauss_grid():
    mu, w = sht.gauss_grid(48)
    assert abs(w.sum() - 2.0) < 1e-14
    assert np.all(np.diff(mu) < 0)          # north to south
    assert np.allclose(mu, -mu[::-1], atol=1e-15)
    # exact for polynomials up to degree 2*48-1
    assert abs(np.sum(w * mu ** 94) - 2.0 / 95.0) < 1e-12 * (2.0 / 95.0)


def test_gauss_weights_vs_high_precision():
    """The Gauss-Legendre weights against 40-digit ones at the polar, near-polar and
    mid-latitude nodes of a 384-point grid (the weights next to the poles carry the vector
    analysis, weighted there by 1 / (1 - mu^2)).  Reference: Newton on mpmath's P_n from the
    stored node to the true root z, then w(z) = 2 / ((1 - z^2) P_n'(z)^2).  The stored node
    mu is the root rounded to double, and the weight belongs to mu: from the Legendre equation,
    d ln w / dx = -2x / (1 - x^2) at a root (about 5e4 at the polar node here), so the check
    is w(mu) = w(z) (1 - 2z (mu - z) / (1 - z^2)) to 2e-13 relative."""
    n = 384
    mu, w = sht.gauss_grid(n)
    mpmath.mp.dps = 40
    for i in (0, 1, 5, n // 4, n - 1):
        x = mpmath.mpf(float(mu[i]))
        z = x
        for _ in range(6):
            dp = n * (z * mpmath.legendre(n, z) - mpmath.legendre(n - 1, z)) / (z * z - 1)
            z -= mpmath.legendre(n, z) / dp
        dp = n * (z * mpmath.legendre(n, z) - mpmath.legendre(n - 1, z)) / (z * z - 1)
        wr = 2 / ((1 - z * z) * dp * dp) * (1 - 2 * z * (x - z) / (1 - z * z))
        assert abs(float(x - z)) < 2e-16, i
        err = float(mpmath.mpf(float(w[i])) / wr - 1)
        assert abs(err) < 2e-13, (i, err)


def test_legendre_vs_scipy():
    T = 12
    mu, _ = sht.gauss_grid(20)
    P = sht.legendre_table(T, mu)
    H = sht.legendre_H(T, P, mu)
    theta = np.arccos(mu)
    for m in range(T + 1):
        for n in range(m, T + 1):
            Y = sp.sph_harm_y(n, m, theta, 0.0).real * (-1) ** m   # remove Condon-Shortley
            assert np.max(np.abs(P[m][:, n - m] - Y)) < 1e-14
            val, der = sp.assoc_legendre_p(n, m, mu, norm=True, diff_n=1)
            scale = P[m][:, n - m] / np.where(np.abs(val) > 1e-8, val, np.nan)
            c = np.nanmedian(scale)
            assert abs(abs(c) - 1 / math.sqrt(2 * math.pi)) < 1e-12
            assert np.max(np.abs(H[m][:, n - m] - c * (1 - mu ** 2) * der)) < 1e-13


def test_legendre_underflow_region_mpmath():
    """High m near the pole: the scaled recurrence against 40-digit values from the Jacobi
    form  Pt_n^m = sqrt((2n+1)/(4pi) (n-m)!/(n+m)!) (1-x^2)^{m/2} (n+m)!/(2^m n!) P^{(m,m)}_{n-m}(x)
    (a route that shares nothing with the three-term recurrence)."""
    T = 511
    mu = np.array([0.999, 0.9, 0.3])
    P = sht.legendre_table(T, mu)
    mpmath.mp.dps = 40
    for (m, n) in [(300, 300), (300, 320), (500, 511), (450, 460), (100, 400)]:
        for j, xf in enumerate(mu):
            x = mpmath.mpf(xf)
            ref = (mpmath.sqrt((2 * n + 1) / (4 * mpmath.pi) * mpmath.factorial(n - m)
                               / mpmath.factorial(n + m))
                   * (1 - x * x) ** (mpmath.mpf(m) / 2) * mpmath.factorial(n + m)
                   / (2 ** m * mpmath.factorial(n)) * mpmath.jacobi(n - m, m, m, x))
            refv = float(ref)
            got = P[m][j, n - m]
            if abs(ref) < mpmath.mpf("1e-300"):
                assert abs(got) < 1e-290
            else:
                assert abs(got - refv) <= 1e-12 * abs(refv)


def _band_limited(T, seed):
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(sht.nlm(T)) + 1j * rng.standard_normal(sht.nlm(T))
    c[: T + 1] = c[: T + 1].real
    return c


@pytest.mark.parametrize("T,nlat,nlon", [(7, 12, 24), (31, 48, 96), (63, 96, 192)])
def test_roundtrip_P8(T, nlat, nlon):
    g = sht.Grid(T, nlat, nlon, 1.0)
    c = _band_limited(T, T)
    assert np.max(np.abs(g.analys(g.synth(c)) - c)) < 1e-12


def test_synthesis_dense_sum_P8():
    """Synthesis equals the dense sum  c^0 Y^0 + 2 Re sum c^m Y^m  with scipy's Y (T7)."""
    T, nlat, nlon = 7, 12, 24
    g = sht.Grid(T, nlat, nlon, 1.0)
    c = _band_limited(T, 3)
    f = g.synth(c)
    theta = np.arccos(g.mu)[:, None]
    lam = g.lam[None, :]
    ref = np.zeros((nlat, nlon))
    for m in range(T + 1):
        for n in range(m, T + 1):
            Y = sp.sph_harm_y(n, m, theta, lam) * (-1) ** m
            v = c[sht.idx(T, m, n)] * Y
            ref += v.real if m == 0 else 2.0 * v.real
    assert np.max(np.abs(f - ref)) < 1e-12


def test_vector_transforms_laplacian():
    """div(k x grad psi + grad chi) = lap chi and curl(...) = lap psi, through synth_uv and
    analys_divcurl (exact Gauss quadrature for these degrees)."""
    T, nlat, nlon, a = 21, 33, 66, 6.37122e6
    g = sht.Grid(T, nlat, nlon, a)
    psi = _band_limited(T, 5)
    chi = _band_limited(T, 6)
    psi[0] = chi[0] = 0
    U, V = g.synth_uv(psi, chi)
    d, c = g.analys_divcurl(U, V)
    lap = sht.laplacian_eig(T, a)
    assert np.max(np.abs(d - lap * chi)) < 1e-13 * np.max(np.abs(lap * chi))
    assert np.max(np.abs(c - lap * psi)) < 1e-13 * np.max(np.abs(lap * psi))


def test_velocity_solid_body():
    """psi = -a u0 mu gives u = u0 cos(lat), v = 0 (closed form)."""
    T, nlat, nlon, a, u0 = 10, 16, 32, 6.37122e6, 20.0
    g = sht.Grid(T, nlat, nlon, a)
    psi = np.zeros(sht.nlm(T), complex)
    psi[sht.idx(T, 0, 1)] = -a * u0 / math.sqrt(3 / (4 * math.pi))   # Pt_1^0 = sqrt(3/4pi) mu
    U, V = g.synth_uv(psi, np.zeros_like(psi))
    cos = np.sqrt(g.coslat2)[:, None]
    assert np.max(np.abs(U / cos - u0 * cos)) < 1e-12 * u0
    assert np.max(np.abs(V)) < 1e-12 * u0


def test_synthetic_inputs_shape():
    U = synthetic.gaussian_state(15, 1)
    assert U.shape == (3, sht.nlm(15))
    assert np.all(U[:, 0] == 0)
    assert np.all(U[:, :16].imag == 0)
