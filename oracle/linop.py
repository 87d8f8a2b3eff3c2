"""The linear part L = L_g + L_c of the shallow-water equations in spectral space
(paper Sec. 3, Eq. 1-3 and the split into L_g U, L_c U, N(U)).

    L_g U = ( -Phibar delta,        0,                  -lap Phi ),
    L_c U = (  0,                   -f delta - V.grad f,  f zeta + k.(grad f x V) ),

with f = 2 Omega mu.  The paper defers the spectral form to a cited paper; it is derived
here from mu Pt_n = eps_{n+1} Pt_{n+1} + eps_n Pt_{n-1} and
(1 - mu^2) dPt_n/dmu = (n + 1) eps_n Pt_{n-1} - n eps_{n+1} Pt_{n+1}.  Using
-f delta - V.grad f = -div(f V) and f zeta + k.(grad f x V) = k.curl(f V), for one zonal
order m (terms with degree > T are dropped by the truncation):

    dPhi_n/dt   = -Phibar delta_n
    dzeta_n/dt  =  i w_n zeta_n - 2 Omega [ (n+1)/n eps_n delta_{n-1} + n/(n+1) eps_{n+1} delta_{n+1} ]
    ddelta_n/dt =  n(n+1)/a^2 Phi_n + i w_n delta_n
                   + 2 Omega [ (n+1)/n eps_n zeta_{n-1} + n/(n+1) eps_{n+1} zeta_{n+1} ]

with w_n = 2 Omega m / (n (n+1)).  Reading taken: the global means zeta_0^0 and delta_0^0
vanish on the sphere; the operator has zero rows and columns for them (they are left
unchanged by exp(dt L)), and the n = 0 Phi row is zero too.

This module also gives the same operator evaluated on the Gauss grid (pin P2) and the
linear energy in which L is skew-adjoint (pin P3)."""
import numpy as np

from . import sht


def operator_m(T, m, Omega, radius, Phibar, part="L"):
    """Dense 3K x 3K matrix of L restricted to zonal order m, K = T + 1 - m, with the
    unknowns interleaved as (Phi_n, zeta_n, delta_n) for n = m..T (bandwidth 4 / 4).
    part = "Lg" keeps only the gravity terms (-Phibar delta_n, n(n+1)/a^2 Phi_n), "Lc" only
    the Coriolis terms (i w_n, the eps couplings); "L" is their sum."""
    if part not in ("L", "Lg", "Lc"):
        raise ValueError(part)
    grav, cor = part in ("L", "Lg"), part in ("L", "Lc")
    K = T + 1 - m
    A = np.zeros((3 * K, 3 * K), dtype=np.complex128)
    a2 = radius * radius
    for k in range(K):
        n = m + k
        iP, iZ, iD = 3 * k, 3 * k + 1, 3 * k + 2
        if n == 0:
            continue
        if grav:
            A[iP, iD] = -Phibar
            A[iD, iP] = n * (n + 1.0) / a2
        if not cor:
            continue
        wn = 2.0 * Omega * m / (n * (n + 1.0))
        A[iZ, iZ] = 1j * wn
        A[iD, iD] = 1j * wn
        if k > 0 and n - 1 > 0:
            cm = 2.0 * Omega * (n + 1.0) / n * float(sht.eps(n, m))
            A[iZ, 3 * (k - 1) + 2] = -cm
            A[iD, 3 * (k - 1) + 1] = +cm
        if k + 1 < K:
            cp = 2.0 * Omega * n / (n + 1.0) * float(sht.eps(n + 1, m))
            A[iZ, 3 * (k + 1) + 2] = -cp
            A[iD, 3 * (k + 1) + 1] = +cp
    return A


def split_m(U, T, m):
    """Interleaved (Phi, zeta, delta) vector of zonal order m from U[3, nlm]."""
    o = sht.moffset(T, m)
    K = T + 1 - m
    v = np.empty(3 * K, dtype=np.complex128)
    v[0::3] = U[0, o: o + K]
    v[1::3] = U[1, o: o + K]
    v[2::3] = U[2, o: o + K]
    return v


def merge_m(out, v, T, m):
    o = sht.moffset(T, m)
    K = T + 1 - m
    out[0, o: o + K] = v[0::3]
    out[1, o: o + K] = v[1::3]
    out[2, o: o + K] = v[2::3]


def apply_L(U, T, Omega, radius, Phibar, part="L"):
    """L U (or L_g U, L_c U with part = "Lg", "Lc") for U[3, nlm] (fields Phi', zeta, delta),
    spectral route."""
    out = np.zeros_like(U, dtype=np.complex128)
    for m in range(T + 1):
        merge_m(out, operator_m(T, m, Omega, radius, Phibar, part) @ split_m(U, T, m), T, m)
    return out


def apply_L_grid(U, grid, Omega, Phibar):
    """L U evaluated through the Gauss grid (pin P2): synthesise V from psi and chi,
    form f U, f V with f = 2 Omega mu, take -div(f V) and k.curl(f V) by analysis, and
    add -Phibar delta and -lap Phi spectrally."""
    T, a = grid.T, grid.a
    Phi, zeta, delta = U
    psi = sht.inv_laplacian(zeta, T, a)
    chi = sht.inv_laplacian(delta, T, a)
    Ug, Vg = grid.synth_uv(psi, chi)
    f = 2.0 * Omega * grid.mu[:, None]
    div, cur = grid.analys_divcurl(f * Ug, f * Vg)
    lap = sht.laplacian_eig(T, a)
    out = np.empty_like(U, dtype=np.complex128)
    out[0] = -Phibar * delta
    out[1] = -div
    out[2] = cur - lap * Phi
    # the global means of zeta and delta are not evolved (see module docstring)
    out[1, 0] = 0.0
    out[2, 0] = 0.0
    out[0, 0] = 0.0
    return out


def energy_weights_m(T, m, radius, Phibar):
    """Diagonal weights W of the linear energy for one zonal order, interleaved order:
    1 for Phi_n and Phibar a^2 / (n (n+1)) for zeta_n, delta_n (n >= 1)."""
    K = T + 1 - m
    W = np.empty(3 * K)
    for k in range(K):
        n = m + k
        W[3 * k] = 1.0
        W[3 * k + 1] = W[3 * k + 2] = Phibar * radius ** 2 / (n * (n + 1.0)) if n > 0 else 0.0
    return W


def energy(U, T, radius, Phibar):
    """E = sum_m w_m [ sum_n |Phi_n|^2 + sum_{n>=1} Phibar a^2/(n(n+1)) (|zeta_n|^2 + |delta_n|^2) ],
    w_0 = 1, w_m = 2 (the m < 0 half of a real field).  Proportional to the integral of
    Phibar |V|^2 + Phi'^2 over the sphere."""
    E = 0.0
    for m in range(T + 1):
        v = split_m(U, T, m)
        W = energy_weights_m(T, m, radius, Phibar)
        E += (1.0 if m == 0 else 2.0) * float(np.sum(W * np.abs(v) ** 2))
    return E
