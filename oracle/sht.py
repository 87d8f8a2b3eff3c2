"""Spherical-harmonic transforms on a Gaussian grid (paper Sec. 3.2, "Space discretization
with Spherical Harmonics").  The paper uses SHTns; this module restates the transform from
its definition.

Conventions (the paper leaves them to SHTns; these are the readings taken):
  * mu = sin(latitude); latitudes are the Gauss-Legendre nodes ordered north to south;
    longitudes lambda_k = 2 pi k / nlon.
  * Y_n^m = Pt_n^m(mu) e^{i m lambda} with Pt orthonormal on the sphere
    (integral of |Y|^2 over the unit sphere = 1), no Condon-Shortley phase.
  * A real field is  f = sum_n c_n^0 Y_n^0 + 2 Re sum_{m>=1} sum_n c_n^m Y_n^m, with the m >= 0
    coefficients stored m-major: idx(m, n) = m (2T + 3 - m) / 2 + (n - m).
  * eps_n^m = sqrt((n^2 - m^2) / (4 n^2 - 1)); mu Pt_n = eps_{n+1} Pt_{n+1} + eps_n Pt_{n-1};
    Ht_n^m = (1 - mu^2) dPt_n^m/dmu = -n eps_{n+1} Pt_{n+1} + (n + 1) eps_n Pt_{n-1}.
  * Velocity is carried as U = u cos(lat), V = v cos(lat).  With psi and chi the stream
    function and velocity potential (Sec. 3:  V = k x grad psi + grad chi),
        U = (1/a) [ -(1 - mu^2) d psi/dmu + d chi/dlambda ],
        V = (1/a) [  d psi/dlambda + (1 - mu^2) d chi/dmu ].
"""
import numpy as np


def nlm(T):
    return (T + 1) * (T + 2) // 2


def idx(T, m, n):
    return m * (2 * T + 3 - m) // 2 + (n - m)


def moffset(T, m):
    return m * (2 * T + 3 - m) // 2


def eps(n, m):
    """eps_n^m = sqrt((n^2 - m^2)/(4n^2 - 1)); 0 for n <= m and for n = 0."""
    n = np.asarray(n, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        v = np.sqrt(np.maximum(n * n - m * m, 0.0) / np.maximum(4.0 * n * n - 1.0, 1.0))
    return np.where(n <= m, 0.0, v)


def gauss_grid(nlat):
    """Gauss-Legendre nodes mu_j (north to south) and weights w_j (sum w_j = 2).

    The nodes are numpy's (the roots of P_nlat, to about an ulp).  The weights follow their
    definition, w_j = 2 / ((1 - x_j^2) P_n'(x_j)^2) with n = nlat (the classical Gauss-Legendre
    weight; P_n' (x) = n (x P_n - P_{n-1}) / (x^2 - 1)), i.e.
        w_j = 2 (1 - x_j)(1 + x_j) / (n (x_j P_n(x_j) - P_{n-1}(x_j)))^2,
    with P_n, P_{n-1} by the three-term recurrence and 1 - x^2 formed as (1 - x)(1 + x), which
    keeps its relative accuracy next to the poles.  numpy's own weights are off by up to ~1e-9
    relative there (n = 384 - 768), and the vector analysis weights them by 1 / (1 - x^2)."""
    x, _ = np.polynomial.legendre.leggauss(nlat)
    x = x[::-1].copy()
    p0, p1 = np.ones_like(x), x.copy()   # P_0, P_1
    for k in range(2, nlat + 1):         # k P_k = (2k - 1) x P_{k-1} - (k - 1) P_{k-2}
        p0, p1 = p1, ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k
    w = 2.0 * ((1.0 - x) * (1.0 + x)) / (nlat * (x * p1 - p0)) ** 2
    return x, w


def legendre_table(T, mu, nmax=None):
    """Pt_n^m(mu_j) for 0 <= m <= T, m <= n <= nmax (default T + 1).

    Returns a list P with P[m] of shape (len(mu), nmax + 1 - m).  The three-term recurrence
    runs on a mantissa with a separate power-of-two exponent per node, so that the tiny
    sectoral values near the poles at high m neither underflow nor lose digits; the values
    are converted back at the end (anything below the FP64 range becomes 0)."""
    if nmax is None:
        nmax = T + 1
    mu = np.asarray(mu, dtype=np.float64)
    s = np.sqrt((1.0 - mu) * (1.0 + mu))
    nj = mu.size
    STEP = 256
    P = []
    # sectoral start  Pt_m^m = sqrt((2m+1)/(2m)) * s * Pt_{m-1}^{m-1},  Pt_0^0 = 1/sqrt(4 pi)
    pmm = np.full(nj, 1.0 / np.sqrt(4.0 * np.pi))
    emm = np.zeros(nj, dtype=np.int64)
    for m in range(0, T + 1):
        if m > 0:
            pmm = pmm * (np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s)
            small = np.abs(pmm) < 2.0 ** -STEP
            pmm = np.where(small, pmm * 2.0 ** STEP, pmm)
            emm = np.where(small, emm - STEP, emm)
        out = np.zeros((nj, nmax + 1 - m))
        p_prev = np.zeros(nj)           # Pt_{m-1}^m = 0
        p_cur = pmm.copy()
        e = emm.copy()
        out[:, 0] = np.ldexp(p_cur, e)
        for n in range(m + 1, nmax + 1):
            # mu Pt_{n-1} = eps_n Pt_n + eps_{n-1} Pt_{n-2}
            p_new = (mu * p_cur - float(eps(n - 1, m)) * p_prev) / float(eps(n, m))
            p_prev, p_cur = p_cur, p_new
            big = np.abs(p_cur) > 2.0 ** STEP
            if big.any():
                p_cur = np.where(big, p_cur * 2.0 ** -STEP, p_cur)
                p_prev = np.where(big, p_prev * 2.0 ** -STEP, p_prev)
                e = np.where(big, e + STEP, e)
            out[:, n - m] = np.ldexp(p_cur, e)
        P.append(out)
    return P


def legendre_H(T, P, mu):
    """Ht_n^m = (1 - mu^2) dPt_n^m/dmu for m <= n <= T from the table P (which holds n <= T+1)."""
    H = []
    for m in range(T + 1):
        n = np.arange(m, T + 1, dtype=np.float64)
        Pm = P[m]
        Hm = np.empty((Pm.shape[0], T + 1 - m))
        for k, nn in enumerate(n):
            v = -nn * float(eps(nn + 1, m)) * Pm[:, k + 1]
            if k > 0:
                v = v + (nn + 1) * float(eps(nn, m)) * Pm[:, k - 1]
            Hm[:, k] = v
        H.append(Hm)
    return H


class Grid:
    """Gauss grid plus Legendre tables for truncation T (Sec. 3.2)."""

    def __init__(self, T, nlat, nlon, radius):
        if nlon <= 2 * T:
            raise ValueError("nlon must exceed 2T")
        self.T, self.nlat, self.nlon, self.a = T, nlat, nlon, float(radius)
        self.mu, self.w = gauss_grid(nlat)
        self.P = legendre_table(T, self.mu)
        self.H = legendre_H(T, self.P, self.mu)
        self.lam = 2.0 * np.pi * np.arange(nlon) / nlon
        self.coslat2 = (1.0 - self.mu) * (1.0 + self.mu)

    # --- longitude stage -------------------------------------------------------------
    def _to_grid(self, G):
        """G[j, m] (m = 0..T) -> f[j, k] = G_0 + 2 Re sum_{m>=1} G_m e^{i m lambda_k}."""
        F = np.zeros((self.nlat, self.nlon // 2 + 1), dtype=np.complex128)
        F[:, : self.T + 1] = G
        return np.fft.irfft(F, n=self.nlon, axis=1) * self.nlon

    def _from_grid(self, f):
        """f[j, k] -> F[j, m] = (2 pi / nlon) sum_k f e^{-i m lambda_k}, m = 0..T."""
        return np.fft.rfft(f, axis=1)[:, : self.T + 1] * (2.0 * np.pi / self.nlon)

    # --- scalar transforms ------------------------------------------------------------
    def synth(self, c):
        """Spectral (m-major, nlm complex) -> grid (nlat, nlon) real."""
        T = self.T
        G = np.zeros((self.nlat, T + 1), dtype=np.complex128)
        for m in range(T + 1):
            o = moffset(T, m)
            G[:, m] = self.P[m][:, : T + 1 - m] @ c[o: o + T + 1 - m]
        return self._to_grid(G)

    def analys(self, f):
        """Grid (nlat, nlon) real -> spectral  c_n^m = sum_j w_j Pt_n^m(mu_j) F_m(mu_j)."""
        T = self.T
        F = self._from_grid(f)
        c = np.zeros(nlm(T), dtype=np.complex128)
        for m in range(T + 1):
            o = moffset(T, m)
            c[o: o + T + 1 - m] = self.P[m][:, : T + 1 - m].T @ (self.w * F[:, m])
        return c

    # --- vector transforms ------------------------------------------------------------
    def synth_uv(self, psi, chi):
        """(psi, chi) spectral -> (U, V) = (u cos, v cos) on the grid."""
        T = self.T
        GU = np.zeros((self.nlat, T + 1), dtype=np.complex128)
        GV = np.zeros((self.nlat, T + 1), dtype=np.complex128)
        for m in range(T + 1):
            o = moffset(T, m)
            ps = psi[o: o + T + 1 - m]
            ch = chi[o: o + T + 1 - m]
            Pm = self.P[m][:, : T + 1 - m]
            Hm = self.H[m]
            GU[:, m] = (-(Hm @ ps) + 1j * m * (Pm @ ch)) / self.a
            GV[:, m] = (1j * m * (Pm @ ps) + (Hm @ ch)) / self.a
        return self._to_grid(GU), self._to_grid(GV)

    def analys_divcurl(self, A, B):
        """For a vector field with A = P_u cos, B = P_v cos on the grid, the spectral
        divergence and vertical curl (integration by parts against conj(Y))."""
        T = self.T
        FA = self._from_grid(A)
        FB = self._from_grid(B)
        wq = self.w / self.coslat2
        div = np.zeros(nlm(T), dtype=np.complex128)
        cur = np.zeros(nlm(T), dtype=np.complex128)
        for m in range(T + 1):
            o = moffset(T, m)
            Pm = self.P[m][:, : T + 1 - m]
            Hm = self.H[m]
            a_m = wq * FA[:, m]
            b_m = wq * FB[:, m]
            div[o: o + T + 1 - m] = (1j * m * (Pm.T @ a_m) - Hm.T @ b_m) / self.a
            cur[o: o + T + 1 - m] = (1j * m * (Pm.T @ b_m) + Hm.T @ a_m) / self.a
        return div, cur


def laplacian_eig(T, radius):
    """-n(n+1)/a^2 for every (m, n) in m-major order."""
    out = np.empty(nlm(T))
    for m in range(T + 1):
        n = np.arange(m, T + 1, dtype=np.float64)
        out[moffset(T, m): moffset(T, m) + T + 1 - m] = -n * (n + 1) / radius ** 2
    return out


def inv_laplacian(c, T, radius):
    """nabla^-2 with the n = 0 coefficient set to 0."""
    lam = laplacian_eig(T, radius)
    out = np.zeros_like(c)
    nz = lam != 0
    out[nz] = c[nz] / lam[nz]
    return out
