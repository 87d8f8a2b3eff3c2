"""Pins of the oracle's REXI coefficients (Sec. 4.2.1-4.2.2, Eq. cauchy_alpha/beta).

Each check is tied to something other than the formula itself: the function the rational
sum must reproduce (e^{ix}, psi_1, psi_2 in closed form), the geometry of the contour
(the circle through p0 and +-iX), the conjugate symmetry that makes the REXI sum of a real
field real, and an independent 30-digit evaluation of the exponential."""
import math

import mpmath
import numpy as np
import pytest

from oracle import coeffs

# contour choices per workload (chosen by a search minimising max(e_s, amplification*eps))
CASES = [
    # N, p0, Xc, X (covered half-width), bound on e_s
    (256, 6.0, 1.6 * 11.765, 11.765, 1e-12),     # T63,  dt = 3600 s
    (512, 6.0, 1.4 * 11.54, 11.54, 1e-12),       # T127, dt = 1800 s
    (512, 14.0, 1.4 * 45.73, 45.73, 2e-9),       # T255, dt = 3600 s
]


@pytest.mark.parametrize("N,p0,Xc,X,bound", CASES)
def test_scalar_error_P1(N, p0, Xc, X, bound):
    z, w = coeffs.rexi_coefficients(N, p0, Xc)
    es = coeffs.scalar_error(z, w, X, npts=6001)
    assert es < bound


def test_scalar_error_mpmath_crosscheck():
    """r(ix) at a few points evaluated in 30-digit arithmetic agrees with FP64 r(ix)."""
    N, p0, Xc = 64, 4.0, 8.0
    z, w = coeffs.rexi_coefficients(N, p0, Xc)
    mpmath.mp.dps = 30
    R = mpmath.mpf(p0 * p0 + Xc * Xc) / (2 * p0)
    mu = p0 - R
    for x in [-5.0, -1.3, 0.0, 2.2, 5.0]:
        acc = mpmath.mpc(0)
        for n in range(1, N + 1):
            th = 2 * mpmath.pi * (n - mpmath.mpf(1) / 2) / N
            ring = R * mpmath.exp(1j * th)
            zz = ring + mu
            acc += ring * mpmath.exp(zz) / N / (zz - 1j * x)
        r64 = coeffs.rational_eval(z, w, np.array([1j * x]))[0]
        assert abs(complex(acc) - r64) < 1e-13 * max(1.0, abs(complex(acc)))
        # and both approximate e^{ix}
        assert abs(complex(acc) - complex(mpmath.exp(1j * x))) < 1e-6


def test_contour_geometry():
    """The circle passes through p0 and +-iX (Sec. 4.2.2): |p - mu| = R for the three points,
    and the nodes lie on it."""
    for p0, X in [(10.0, 30.0), (6.0, 18.8), (14.0, 64.0)]:
        R, mu = coeffs.contour(p0, X)
        assert abs(abs(p0 - mu) - R) < 1e-12 * R
        assert abs(abs(1j * X - mu) - R) < 1e-12 * R
        assert abs(abs(-1j * X - mu) - R) < 1e-12 * R
        z, _ = coeffs.rexi_coefficients(32, p0, X)
        assert np.allclose(np.abs(z - mu), R, rtol=1e-14)


def test_conjugate_pairs():
    """Midpoint nodes give conjugate pole/weight pairs and no real pole, so the m >= 0 sum of
    a real field is the half-spectrum of a real field."""
    z, w = coeffs.rexi_coefficients(128, 10.0, 30.0)
    assert np.allclose(z[::-1], np.conj(z), rtol=0, atol=1e-12)
    assert np.allclose(w[::-1], np.conj(w), rtol=1e-13, atol=0)
    assert np.min(np.abs(z.imag)) > 0


def test_paper_parameters_mu0_cancellation():
    """Sec. 4.2.2: with the circle centred at 0 the largest |beta_n| grows like e^R, while the
    shifted circle keeps it near (R/N) e^{p0}."""
    N = 128
    R0 = 30.0
    z0 = R0 * np.exp(2j * np.pi * (np.arange(1, N + 1) - 0.5) / N)
    w0 = z0 * np.exp(z0) / N
    assert np.max(np.abs(w0)) > 0.1 * math.exp(R0) * R0 / N
    z, w = coeffs.rexi_coefficients(N, 10.0, 30.0)
    R, _ = coeffs.contour(10.0, 30.0)
    assert np.max(np.abs(w)) <= (R / N) * math.exp(10.0) * (1 + 1e-12)
    assert np.max(np.abs(w)) > 0.5 * (R / N) * math.exp(10.0)


@pytest.mark.parametrize("k", [1, 2])
def test_phi_functions_P10(k):
    """psi_1, psi_2 (Sec. 4.3) reproduced by the same poles to scalar accuracy; the series
    branch near 0 matches the closed form where both are accurate."""
    z, w = coeffs.rexi_coefficients(256, 6.0, 1.6 * 11.765, k=k)
    x = 1j * np.linspace(-11.765, 11.765, 2001)
    x = x[np.abs(x) > 1e-3]
    ref = (np.expm1(x) / x) if k == 1 else ((np.expm1(x) - x) / x ** 2)
    r = coeffs.rational_eval(z, w, x)
    assert np.max(np.abs(r - ref)) < 1e-11
    small = np.array([0.3 + 0.1j, -0.2j, 0.45])
    ser = coeffs.phi_function(k, small)
    closed = (np.expm1(small) / small) if k == 1 else ((np.expm1(small) - small) / small ** 2)
    assert np.max(np.abs(ser - closed)) < 1e-13
    assert abs(coeffs.phi_function(k, np.array([0.0]))[0] - 1.0 / math.factorial(k)) < 1e-16
