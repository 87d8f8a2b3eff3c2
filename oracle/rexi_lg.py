"""REXI of the gravity operator L_g alone (paper Sec. 3, the L_g column of the split; the
lg_rexi_* method identifiers of Table 2, where the Coriolis term L_c goes to the explicit
part).  Test infrastructure: plain FP64 CPU code, imported only by tests and the benchmark's
CPU leg.

Without Coriolis the operator does not couple degrees or zonal orders (Sec. 5.3: a diagonal
instead of a banded solve).  For degree n >= 1, with q_n = n(n+1)/a^2,

    dPhi_n/dt = -Phibar delta_n,   dzeta_n/dt = 0,   ddelta_n/dt = q_n Phi_n,

so each REXI term (z - dt L_g)^-1 b is a 2 x 2 solve on (Phi_n, delta_n) and a division of
zeta_n by z:

    det = z^2 + dt^2 Phibar q_n,
    Phi   = (z b_Phi - dt Phibar b_delta) / det,
    delta = (z b_delta + dt q_n b_Phi) / det,
    zeta  = b_zeta / z.

The n = 0 row of the operator is zero (the reading of the full operator: global means are
not evolved), so every field of degree 0 is divided by z.  The terms are summed over the
poles in order, in FP64, with no real part taken (m >= 0 storage, as in rexi.rexi_step).
"""
import numpy as np

from . import sht


def degrees(T):
    """Degree n of every coefficient in the m-major layout."""
    n = np.empty(sht.nlm(T), dtype=np.int64)
    for m in range(T + 1):
        o = sht.moffset(T, m)
        n[o: o + T + 1 - m] = np.arange(m, T + 1)
    return n


def rexi_step_lg(U0, T, dt, radius, Phibar, z, w, idx=None):
    """sum_p w_p (z_p - dt L_g)^-1 U0 for U0[3, nlm] (Phi', zeta, delta): the diagonal solve
    of every pole written out per coefficient, poles summed in order.  idx (optional) restricts
    the computation to those coefficient indices; the result then has shape [3, len(idx)]."""
    U0 = np.asarray(U0, dtype=np.complex128)
    n = degrees(T).astype(np.float64)
    if idx is not None:
        n = n[idx]
        U0 = U0[:, idx]
    q = n * (n + 1.0) / (radius * radius)
    bP, bZ, bD = U0[0], U0[1], U0[2]
    g = n > 0
    out = np.zeros_like(U0)
    for zp, wp in zip(z, w):
        det = zp * zp + dt * dt * Phibar * q
        P = np.where(g, (zp * bP - dt * Phibar * bD) / det, bP / zp)
        D = np.where(g, (zp * bD + dt * q * bP) / det, bD / zp)
        out[0] += wp * P
        out[1] += wp * (bZ / zp)
        out[2] += wp * D
    return out


def exact_lg(U0, T, dt, radius, Phibar):
    """exp(dt L_g) U0 in closed form: on (Phi_n, delta_n) the generator [[0, -Phibar], [q_n, 0]]
    squares to -c_n^2 I with c_n = sqrt(Phibar q_n), so
        exp(dt L_g) = cos(c_n dt) I + sin(c_n dt) / c_n [[0, -Phibar], [q_n, 0]];
    zeta and every degree-0 coefficient are unchanged."""
    U0 = np.asarray(U0, dtype=np.complex128)
    n = degrees(T).astype(np.float64)
    q = n * (n + 1.0) / (radius * radius)
    c = np.sqrt(Phibar * q)
    cs = np.cos(c * dt)
    sc = np.where(n > 0, np.sin(c * dt) / np.where(c > 0, c, 1.0), 0.0)
    out = np.empty_like(U0)
    out[0] = cs * U0[0] - Phibar * sc * U0[2]
    out[1] = U0[1]
    out[2] = q * sc * U0[0] + cs * U0[2]
    out[0] = np.where(n > 0, out[0], U0[0])
    out[2] = np.where(n > 0, out[2], U0[2])
    return out
