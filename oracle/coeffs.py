"""Cauchy-contour REXI coefficients (paper Sec. 4.2.1 "Cauchy Contour integral" and
Sec. 4.2.2 "Numerical cancellation").

The paper writes the rational approximation as  f(x) ~ sum_n beta_n / (x + alpha_n)  with
(Eq. cauchy_alpha, cauchy_beta)

    alpha_n = -(R e^{i theta_n} + mu),
    beta_n  = -(1/N) R e^{i theta_n} f(R e^{i theta_n} + mu),

obtained from the trapezoidal rule on the circle  Gamma = {R e^{i theta} + mu}.  Writing
z_n = R e^{i theta_n} + mu = -alpha_n and w_n = -beta_n gives the equivalent form used by the
library,  f(x) ~ sum_n w_n / (z_n - x).

Readings taken where the paper is silent:
  * theta_n = 2 pi (n - 1/2) / N, n = 1..N (midpoint nodes: the poles come in conjugate pairs
    and none lies on the real axis);
  * the radius symbol r of the three-point construction and the R of the circle are the
    same quantity;
  * p_{+-1} = +-iX: the circle passes through p0 (real, > 0) and +-iX, so
    R = (p0^2 + X^2) / (2 p0) and the centre is mu = p0 - R (Sec. 4.2.2).
"""
import math

import numpy as np


def contour(p0, X):
    """Radius R and centre mu of the circle through p0 and +-iX (Sec. 4.2.2)."""
    if not (p0 > 0 and X >= 0):
        raise ValueError("need p0 > 0 and X >= 0")
    R = (p0 * p0 + X * X) / (2.0 * p0)
    return R, p0 - R


def phi_function(k, z):
    """psi_0 = exp, psi_1 = (e^z - 1)/z, psi_2 = (e^z - 1 - z)/z^2 (Sec. 4.3, ETD2RK).

    Near z = 0 the closed forms cancel; there the limit (L'Hopital) is taken through the
    Taylor series  psi_k(z) = sum_j z^j / (j + k)!, as the paper prescribes."""
    z = np.asarray(z, dtype=np.complex128)
    if k == 0:
        return np.exp(z)
    out = np.empty_like(z)
    small = np.abs(z) < 0.5
    zs = z[~small]
    if k == 1:
        out[~small] = np.expm1(zs) / zs
    elif k == 2:
        out[~small] = (np.expm1(zs) - zs) / (zs * zs)
    else:
        raise ValueError("k must be 0, 1 or 2")
    zz = z[small]
    acc = np.zeros_like(zz)
    term = np.full_like(zz, 1.0 / math.factorial(k))
    for j in range(0, 30):
        acc = acc + term
        term = term * zz / (j + k + 1)
    out[small] = acc
    return out


def rexi_coefficients(N, p0, X, k=0):
    """Poles z_n and weights w_n of  psi_k(x) ~ sum_n w_n / (z_n - x)  (Eq. cauchy_alpha/beta).

    Returns complex128 arrays z (= -alpha_n) and w (= -beta_n) of length N.

    The circle is symmetric about the real axis and theta_{N+1-n} = 2 pi - theta_n, so node
    N+1-n is the conjugate of node n (psi_k has real Taylor coefficients: psi_k(conj z) =
    conj psi_k(z)).  The nodes n <= N/2 are evaluated and the others set to their exact
    conjugates; for odd N the middle node (theta = pi) is real.  Evaluating every node on its
    own would break the pairing by rounding (the weights carry a relative error of about
    |z| eps through e^z), and the contour's cancellation (|w_n| up to 1e5 summing to O(1))
    would turn that into a spurious imaginary part of the sums."""
    if N < 1:
        raise ValueError("N must be positive")
    R, mu = contour(p0, X)
    h = N // 2
    n = np.arange(1, h + 1, dtype=np.float64)
    theta = 2.0 * np.pi * (n - 0.5) / N
    ring = R * np.exp(1j * theta)
    zh = ring + mu
    wh = ring * phi_function(k, zh) / N
    parts_z, parts_w = [zh], [wh]
    if N % 2:
        zm = np.array([mu - R], dtype=np.complex128)
        parts_z.append(zm)
        parts_w.append((-R * phi_function(k, zm) / N).real.astype(np.complex128))
    parts_z.append(np.conj(zh[::-1]))
    parts_w.append(np.conj(wh[::-1]))
    return np.concatenate(parts_z), np.concatenate(parts_w)


def rational_eval(z, w, x):
    """r(x) = sum_n w_n / (z_n - x) for an array of points x (complex)."""
    x = np.asarray(x, dtype=np.complex128)
    return (w[None, :] / (z[None, :] - x[:, None])).sum(axis=1)


def scalar_error(z, w, X, npts=10001, k=0):
    """max over x in [-iX, iX] of |r(x) - psi_k(x)|  (pin P1: the scalar REXI error e_s)."""
    x = 1j * np.linspace(-X, X, npts)
    return float(np.max(np.abs(rational_eval(z, w, x) - phi_function(k, x))))


def amplification(z, w, X, npts=2001):
    """max over x in [-iX, iX] of sum_n |w_n| / |z_n - x|: the factor by which rounding
    errors of the individual pole solves can grow in the weighted sum (Sec. 4.2.2)."""
    x = 1j * np.linspace(-X, X, npts)
    return float(np.max((np.abs(w)[None, :] / np.abs(z[None, :] - x[:, None])).sum(axis=1)))
