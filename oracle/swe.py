"""Nonlinear shallow-water pieces (paper Sec. 3, Eq. 1-3; Sec. 4.4 Strang splitting).

N(U) is the third column of the paper's split (Eq. sw_compact):

    N_Phi   = -V.grad Phi' - Phi' div V     = -div(Phi' V)
    N_zeta  = -div(zeta V)
    N_delta =  k.curl(zeta V) - lap (V.V / 2)

evaluated pseudo-spectrally: V from psi = lap^-1 zeta and chi = lap^-1 delta (Sec. 3), products
on the Gauss grid, divergence / curl / Laplacian by analysis.

Time integrators (Sec. 4.1, 4.4; Table 2):
  * erk  : 2nd-order explicit Runge-Kutta.  Reading taken (the paper does not name the
           variant): the midpoint rule.  Every scheme below that integrates N by erk over an
           interval tau takes `nsub` midpoint steps of tau / nsub (default 1, the paper's
           single step).  Reading taken: the paper treats N explicitly and notes that
           explicitly treated nonlinearities limit the time step (Sec. 2.3); at T511 with
           dt = 7200 s one midpoint step over dt/2 exceeds the advective stability limit, so
           the explicit part is sub-stepped while the linear part keeps the full REXI step.
  * ver1 : T(U) = N^{dt/2} o L^{dt} o N^{dt/2} (U), the linear part L = L_g + L_c by REXI
           (method id l_rexi_n_erk_ver1, Coriolis inside REXI).
  * ver0 : T(U) = L^{dt/2} o N^{dt} o L^{dt/2} (U).
  * etdrk: ETD2RK (Sec. 4.3):  A = psi_0(dt L) U + dt psi_1(dt L) N(U),
           U+ = A + dt psi_2(dt L) (N(A) - N(U)); every psi_k(dt L) applied by REXI with the
           psi_k weights of the same poles (method id l_rexi_n_etdrk).
  * irk  : Crank-Nicolson for the linear part (Sec. 4.1, a = 1/2) inside the Strang ver1 split:
           N^{dt/2} o CN^{dt} o N^{dt/2}  (method id l_irk_n_erk_ver1, Coriolis in L).
  * rk4  : classical 4th-order Runge-Kutta of the full system, used as the small-step
           reference (the paper's reference solution uses RK4 with a tiny step, Sec. 5).
  * lg   : the lg_rexi_lc_n_* identifiers of Table 2: only the gravity operator L_g goes to
           REXI (a diagonal solve, oracle.rexi_lg), the Coriolis term L_c joins N in the
           explicit part:  N'(U) = L_c U + N(U).  lg ver1 is N'^{dt/2} o L_g^{dt} o N'^{dt/2}
           (lg_rexi_lc_n_erk_ver1, the paper's best REXI method, Sec. 5.2); lg etdrk is
           ETD2RK with (L_g, N') in place of (L, N) (lg_rexi_lc_n_etdrk).  lg irk ver0 is
           CN_g^{dt/2} o N'^{dt} o CN_g^{dt/2} with Crank-Nicolson for L_g (lg_irk_lc_n_erk_ver0,
           the paper's best implicit method).
"""
import numpy as np

from . import linop, rexi, rexi_lg, sht


def nonlinear(U, grid):
    """N(U) for U[3, nlm] = (Phi', zeta, delta) on the Gauss grid of `grid`."""
    T, a = grid.T, grid.a
    Phi, zeta, delta = U
    psi = sht.inv_laplacian(zeta, T, a)
    chi = sht.inv_laplacian(delta, T, a)
    Pg = grid.synth(Phi)
    Zg = grid.synth(zeta)
    Ug, Vg = grid.synth_uv(psi, chi)
    div1, _ = grid.analys_divcurl(Pg * Ug, Pg * Vg)
    div2, cur2 = grid.analys_divcurl(Zg * Ug, Zg * Vg)
    ke = (Ug * Ug + Vg * Vg) / (2.0 * grid.coslat2[:, None])
    kes = grid.analys(ke)
    lap = sht.laplacian_eig(T, a)
    out = np.empty_like(U, dtype=np.complex128)
    out[0] = -div1
    out[1] = -div2
    out[2] = cur2 - lap * kes
    out[1, 0] = 0.0
    out[2, 0] = 0.0
    return out


def rk2(U, f, tau):
    """Integrate dU/dt = f(U) over tau with the midpoint rule (erk, 2nd order)."""
    k1 = f(U)
    k2 = f(U + 0.5 * tau * k1)
    return U + tau * k2


def rk2_nonlinear(U, grid, tau, nsub=1):
    """Integrate dU/dt = N(U) over tau with nsub midpoint steps of tau / nsub (erk, 2nd order)."""
    for _ in range(nsub):
        U = rk2(U, lambda V: nonlinear(V, grid), tau / nsub)
    return U


def nonlinear_lc(U, grid, Omega):
    """N'(U) = L_c U + N(U): the explicit part of the lg schemes (Coriolis with N)."""
    return linop.apply_L(U, grid.T, Omega, grid.a, 0.0, part="Lc") + nonlinear(U, grid)


def rk2_sub(U, f, tau, nsub):
    """nsub midpoint steps of tau / nsub for dU/dt = f(U)."""
    for _ in range(nsub):
        U = rk2(U, f, tau / nsub)
    return U


def strang_lg_ver1(U, grid, dt, Omega, Phibar, z, w, nsub=1):
    """One step of lg_rexi_lc_n_erk_ver1:  N'^{dt/2} o L_g^{dt} o N'^{dt/2}  (Sec. 4.4 version 1
    with the Coriolis term in the explicit part)."""
    T, a = grid.T, grid.a
    f = lambda V: nonlinear_lc(V, grid, Omega)
    U1 = rk2_sub(U, f, 0.5 * dt, nsub)
    U2 = rexi_lg.rexi_step_lg(U1, T, dt, a, Phibar, z, w)
    return rk2_sub(U2, f, 0.5 * dt, nsub)


def cn_lg_ver0(U, grid, dt, Omega, Phibar, nsub=1):
    """One step of lg_irk_lc_n_erk_ver0 (the paper's best implicit method, Sec. 5.2):
    CN_g^{dt/2} o N'^{dt} o CN_g^{dt/2}, CN_g the Crank-Nicolson step of the gravity operator
    alone and N' = L_c + N by RK2 (Sec. 4.4 version 0)."""
    T, a = grid.T, grid.a
    U1 = rexi.cn_step(U, T, 0.5 * dt, Omega, a, Phibar, part="Lg")
    U2 = rk2_sub(U1, lambda V: nonlinear_lc(V, grid, Omega), dt, nsub)
    return rexi.cn_step(U2, T, 0.5 * dt, Omega, a, Phibar, part="Lg")


def etd2rk_lg(U, grid, dt, Omega, Phibar, z, w0, w1, w2):
    """One ETD2RK step (Sec. 4.3) of lg_rexi_lc_n_etdrk: psi_k(dt L_g) by the diagonal REXI
    with the psi_k weights of the poles z, nonlinear part N' = L_c + N."""
    T, a = grid.T, grid.a
    R = lambda V, w: rexi_lg.rexi_step_lg(V, T, dt, a, Phibar, z, w)
    NU = nonlinear_lc(U, grid, Omega)
    A = R(U, w0) + dt * R(NU, w1)
    return A + dt * R(nonlinear_lc(A, grid, Omega) - NU, w2)


def strang_ver1(U, grid, dt, Omega, Phibar, z, w, nsub=1):
    """One step of l_rexi_n_erk_ver1:  N^{dt/2} o L^{dt} o N^{dt/2}  (Sec. 4.4, version 1);
    each N^{dt/2} by nsub midpoint steps."""
    T, a = grid.T, grid.a
    U1 = rk2_nonlinear(U, grid, 0.5 * dt, nsub)
    U2 = rexi.rexi_step(U1, T, dt, Omega, a, Phibar, z, w)
    return rk2_nonlinear(U2, grid, 0.5 * dt, nsub)


def strang_ver0(U, grid, dt, Omega, Phibar, z_half, w_half, nsub=1):
    """One step of l_rexi_n_erk_ver0:  L^{dt/2} o N^{dt} o L^{dt/2}  (Sec. 4.4, version 0);
    z_half, w_half are REXI coefficients for a step of dt/2."""
    T, a = grid.T, grid.a
    U1 = rexi.rexi_step(U, T, 0.5 * dt, Omega, a, Phibar, z_half, w_half)
    U2 = rk2_nonlinear(U1, grid, dt, nsub)
    return rexi.rexi_step(U2, T, 0.5 * dt, Omega, a, Phibar, z_half, w_half)


def cn_ver1(U, grid, dt, Omega, Phibar, nsub=1):
    """One step of l_irk_n_erk_ver1:  N^{dt/2} o CN^{dt} o N^{dt/2}."""
    T, a = grid.T, grid.a
    U1 = rk2_nonlinear(U, grid, 0.5 * dt, nsub)
    U2 = rexi.cn_step(U1, T, dt, Omega, a, Phibar)
    return rk2_nonlinear(U2, grid, 0.5 * dt, nsub)


def etd2rk(U, grid, dt, Omega, Phibar, z, w0, w1, w2, nonlin=None):
    """One ETD2RK step (Sec. 4.3) with REXI for psi_0, psi_1, psi_2 (weights w0, w1, w2 of the
    poles z).  nonlin(U) defaults to N(U) on `grid`."""
    T, a = grid.T, grid.a
    N_ = (lambda V: nonlinear(V, grid)) if nonlin is None else nonlin
    NU = N_(U)
    A = rexi.rexi_step(U, T, dt, Omega, a, Phibar, z, w0) + dt * rexi.rexi_step(NU, T, dt, Omega, a, Phibar, z, w1)
    return A + dt * rexi.rexi_step(N_(A) - NU, T, dt, Omega, a, Phibar, z, w2)


def diffuse(U, T, radius, tau, nu, q=2):
    """Exact flow over tau of the hyper-diffusion term (-1)^(q+1) nu lap^q on all three fields:
    lap Y_n = -n(n+1)/a^2 Y_n, so each degree n decays by exp(-tau nu (n(n+1)/a^2)^q).  Not in
    the paper's benchmarks (which run inviscid); the T511 configuration needs it (see strang
    steps with diffusion below)."""
    lam = -sht.laplacian_eig(T, radius)
    return U * np.exp(-tau * nu * lam ** q)[None, :]


def with_diffusion(step, U, T, radius, dt, nu, q=2):
    """D^{dt/2} o step o D^{dt/2} (U): a time step with the diffusion flow D split off
    symmetrically (2nd order like the Strang step itself)."""
    return diffuse(step(diffuse(U, T, radius, 0.5 * dt, nu, q)), T, radius, 0.5 * dt, nu, q)


def full_tendency(U, grid, Omega, Phibar):
    """dU/dt = L U + N(U) (Eq. sw_compact with L = L_g + L_c)."""
    return linop.apply_L(U, grid.T, Omega, grid.a, Phibar) + nonlinear(U, grid)


def rk4_full(U, grid, dt, nsub, Omega, Phibar):
    """nsub classical RK4 steps of the full SWE over a total time dt."""
    h = dt / nsub
    for _ in range(nsub):
        k1 = full_tendency(U, grid, Omega, Phibar)
        k2 = full_tendency(U + 0.5 * h * k1, grid, Omega, Phibar)
        k3 = full_tendency(U + 0.5 * h * k2, grid, Omega, Phibar)
        k4 = full_tendency(U + h * k3, grid, Omega, Phibar)
        U = U + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return U


def rk4_linear(U, T, dt, nsub, Omega, radius, Phibar):
    """nsub classical RK4 steps of dU/dt = L U over a total time dt (pin P6)."""
    h = dt / nsub
    for _ in range(nsub):
        k1 = linop.apply_L(U, T, Omega, radius, Phibar)
        k2 = linop.apply_L(U + 0.5 * h * k1, T, Omega, radius, Phibar)
        k3 = linop.apply_L(U + 0.5 * h * k2, T, Omega, radius, Phibar)
        k4 = linop.apply_L(U + h * k3, T, Omega, radius, Phibar)
        U = U + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return U
