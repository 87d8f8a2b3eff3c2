"""The REXI linear step (paper Sec. 4.2, Eq. rexi):

    U(dt) = exp(dt L) U(0)  ~  sum_n beta_n (dt L + alpha_n)^-1 U(0)
                            =  sum_n w_n (z_n - dt L)^-1 U(0),   z_n = -alpha_n, w_n = -beta_n.

Each term is an independent solve.  The oracle takes the algorithm as written: for every
pole and every zonal order m it assembles the full interleaved (Phi, zeta, delta) matrix
z_n I - dt L_m (bandwidth 4/4, the Coriolis coupling of Sec. 5.3 makes it banded rather
than diagonal) and solves it with a pivoted banded LU, then sums w_n u_n in FP64 in pole
order.  With m >= 0 storage all N poles are summed and no real part is taken: the poles
come in conjugate pairs, so the sum is already the m >= 0 half of a real field.
"""
import numpy as np
import scipy.linalg

from . import linop, sht


def _band(A, lo=4, up=4):
    n = A.shape[0]
    ab = np.zeros((lo + up + 1, n), dtype=A.dtype)
    for i in range(n):
        for j in range(max(0, i - lo), min(n, i + up + 1)):
            ab[up + i - j, j] = A[i, j]
    return ab


def rexi_step(U0, T, dt, Omega, radius, Phibar, z, w, m_list=None):
    """sum_n w_n (z_n - dt L)^-1 U0 for U0[3, nlm] (Phi', zeta, delta), pivoted banded LU
    per (pole, m).  m_list restricts the zonal orders computed (others are left 0)."""
    U0 = np.asarray(U0, dtype=np.complex128)
    out = np.zeros_like(U0)
    ms = range(T + 1) if m_list is None else m_list
    for m in ms:
        A = dt * linop.operator_m(T, m, Omega, radius, Phibar)
        abL = _band(-A)
        b = linop.split_m(U0, T, m)
        acc = np.zeros_like(b)
        for zp, wp in zip(z, w):
            ab = abL.copy()
            ab[4, :] += zp
            acc += wp * scipy.linalg.solve_banded((4, 4), ab, b)
        linop.merge_m(out, acc, T, m)
    return out


def rexi_step_dense(U0, T, dt, Omega, radius, Phibar, z, w):
    """Same sum with numpy.linalg.solve on the dense matrices (pin P9, tiny T only)."""
    out = np.zeros_like(U0, dtype=np.complex128)
    for m in range(T + 1):
        A = dt * linop.operator_m(T, m, Omega, radius, Phibar)
        b = linop.split_m(U0, T, m)
        I = np.eye(A.shape[0])
        acc = np.zeros_like(b)
        for zp, wp in zip(z, w):
            acc += wp * np.linalg.solve(zp * I - A, b)
        linop.merge_m(out, acc, T, m)
    return out


def exact_step(U0, T, dt, Omega, radius, Phibar):
    """exp(dt L) U0, exact up to rounding (pin P4).

    In the energy-weighted basis  S = D L D^-1,  D = diag(sqrt(W)), the operator is
    skew-Hermitian (linear energy is conserved), so exp(dt S) is computed from the
    eigen-decomposition of the Hermitian matrix i S with numpy.linalg.eigh; this avoids
    the loss of accuracy of a Pade exponential on the badly scaled matrix dt L
    (entries range from Phibar dt ~ 1e8 to n(n+1) dt / a^2 ~ 1e-8)."""
    out = np.zeros_like(U0, dtype=np.complex128)
    for m in range(T + 1):
        A = linop.operator_m(T, m, Omega, radius, Phibar)
        W = linop.energy_weights_m(T, m, radius, Phibar)
        d = np.sqrt(np.where(W > 0, W, 1.0))
        S = (d[:, None] * A) / d[None, :]
        Hm = 1j * S
        Hm = 0.5 * (Hm + Hm.conj().T)
        lam, Q = np.linalg.eigh(Hm)            # S = -i Q diag(lam) Q^H
        b = d * linop.split_m(U0, T, m)
        y = Q @ (np.exp(-1j * dt * lam) * (Q.conj().T @ b))
        linop.merge_m(out, y / d, T, m)
    return out


def exact_phi(U0, T, dt, Omega, radius, Phibar, k):
    """psi_k(dt L) U0 exactly up to rounding (Sec. 4.3: psi_0 = exp, psi_1, psi_2), through the
    same energy-weighted eigen-decomposition as exact_step; psi_k of each eigenvalue comes from
    coeffs.phi_function (Taylor series near 0)."""
    from .coeffs import phi_function
    out = np.zeros_like(U0, dtype=np.complex128)
    for m in range(T + 1):
        A = linop.operator_m(T, m, Omega, radius, Phibar)
        W = linop.energy_weights_m(T, m, radius, Phibar)
        d = np.sqrt(np.where(W > 0, W, 1.0))
        S = (d[:, None] * A) / d[None, :]
        Hm = 1j * S
        Hm = 0.5 * (Hm + Hm.conj().T)
        lam, Q = np.linalg.eigh(Hm)            # S = -i Q diag(lam) Q^H
        b = d * linop.split_m(U0, T, m)
        y = Q @ (phi_function(k, -1j * dt * lam) * (Q.conj().T @ b))
        linop.merge_m(out, y / d, T, m)
    return out


def cn_step(U0, T, dt, Omega, radius, Phibar, a=0.5, part="L"):
    """Crank-Nicolson (Sec. 4.1, the irk scheme):  U+ = (I - a dt L)^-1 (I + (1 - a) dt L) U0,
    a = 1/2; the forward-Euler half by linop.apply_L, the backward-Euler half by the pivoted
    banded LU of every zonal order (the same solver as rexi_step).  part = "Lg" applies it to
    the gravity operator alone (the lg_irk_* methods of Table 2)."""
    V = U0 + (1.0 - a) * dt * linop.apply_L(U0, T, Omega, radius, Phibar, part)
    out = np.zeros_like(U0, dtype=np.complex128)
    for m in range(T + 1):
        A = a * dt * linop.operator_m(T, m, Omega, radius, Phibar, part)
        ab = _band(-A)
        ab[4, :] += 1.0
        linop.merge_m(out, scipy.linalg.solve_banded((4, 4), ab, linop.split_m(V, T, m)), T, m)
    return out


def exact_cayley(U0, T, dt, Omega, radius, Phibar):
    """(I - dt L / 2)^-1 (I + dt L / 2) U0 through the energy-weighted eigen-decomposition
    (each eigenvalue lam of dt L maps to (1 + lam/2) / (1 - lam/2)): pins cn_step."""
    out = np.zeros_like(U0, dtype=np.complex128)
    for m in range(T + 1):
        A = linop.operator_m(T, m, Omega, radius, Phibar)
        W = linop.energy_weights_m(T, m, radius, Phibar)
        d = np.sqrt(np.where(W > 0, W, 1.0))
        S = (d[:, None] * A) / d[None, :]
        Hm = 1j * S
        Hm = 0.5 * (Hm + Hm.conj().T)
        lam, Q = np.linalg.eigh(Hm)            # S = -i Q diag(lam) Q^H
        g = -1j * dt * lam
        b = d * linop.split_m(U0, T, m)
        y = Q @ (((1 + 0.5 * g) / (1 - 0.5 * g)) * (Q.conj().T @ b))
        linop.merge_m(out, y / d, T, m)
    return out


def exact_step_expm(U0, T, dt, Omega, radius, Phibar):
    """exp(dt L) U0 with scipy.linalg.expm applied in the energy-weighted basis (a second,
    independent route to the exact exponential for the pins)."""
    out = np.zeros_like(U0, dtype=np.complex128)
    for m in range(T + 1):
        A = linop.operator_m(T, m, Omega, radius, Phibar)
        W = linop.energy_weights_m(T, m, radius, Phibar)
        d = np.sqrt(np.where(W > 0, W, 1.0))
        S = (d[:, None] * A) / d[None, :]
        y = scipy.linalg.expm(dt * S) @ (d * linop.split_m(U0, T, m))
        linop.merge_m(out, y / d, T, m)
    return out


def spectral_radius(T, dt, Omega, radius, Phibar):
    """max |lambda| over the eigenvalues of dt L (all zonal orders)."""
    r = 0.0
    for m in range(T + 1):
        ev = np.linalg.eigvals(dt * linop.operator_m(T, m, Omega, radius, Phibar))
        r = max(r, float(np.max(np.abs(ev))))
    return r


def spectrum_bound(T, dt, Omega, radius, Phibar):
    """X = dt (sqrt(Phibar T (T+1)) / a + 2 Omega): the gravity-wave frequency of the
    highest degree plus the largest Coriolis frequency, an upper bound on |dt lambda|
    (checked against spectral_radius in the pins)."""
    return dt * (np.sqrt(Phibar * T * (T + 1.0)) / radius + 2.0 * Omega)


def rel_l2(x, ref, T):
    """Per-field relative L2 over all (n, m), m > 0 weighted by 2 (the grid L2 norm)."""
    wts = np.empty(sht.nlm(T))
    for m in range(T + 1):
        o = sht.moffset(T, m)
        wts[o: o + T + 1 - m] = 1.0 if m == 0 else 2.0
    num = np.sqrt(np.sum(wts * np.abs(x - ref) ** 2, axis=-1))
    den = np.sqrt(np.sum(wts * np.abs(ref) ** 2, axis=-1))
    return num / np.where(den > 0, den, 1.0)
