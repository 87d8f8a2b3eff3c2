"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds no arithmetic of the REXI method, the transforms or N(U): it only draws
random spectral coefficients with a prescribed spectrum and the request streams of the
serving workload.  Both the oracle (through the tests) and the library receive exactly the
arrays made here.

Physical constants are those of the linearised rotating shallow-water configuration:
Omega = 7.292e-5 1/s, a = 6.37122e6 m, g = 9.80616 m/s^2, h0 = 1e4 m, Phibar = g h0.

Recipes (the paper's own benchmark, the Galewsky barotropic instability, is replaced by
these seeded states):
  * gaussian_state: c_n^m = s_F n^slope (g1 + i g2)/sqrt(2) for n >= 1 with g1, g2 ~ N(0,1)
    from numpy's default_rng(seed); m = 0 coefficients real; n = 0 set to 0.  Default
    slope -1.5, s_Phi = 1e3 m^2/s^2, s_zeta = s_delta = 1e-5 1/s.
  * balanced_state: delta = 0; zeta with kinetic energy per degree proportional to n^-3,
    scaled to a 20 m/s rms wind; Phi' from the linear balance of the divergence equation
    (the linearised d delta/dt = 0 with delta = 0), solved degree by degree; n = 0 set to 0.
"""
import math

import numpy as np

OMEGA = 7.292e-5
RADIUS = 6.37122e6
GRAVITY = 9.80616
H0 = 1.0e4
PHIBAR = GRAVITY * H0


def nlm(T):
    return (T + 1) * (T + 2) // 2


def _offsets(T):
    m = np.arange(T + 2)
    return m * (2 * T + 3 - m) // 2


def gaussian_state(T, seed, slope=-1.5, scales=(1.0e3, 1.0e-5, 1.0e-5)):
    """U[3, nlm] complex128, m-major, fields (Phi', zeta, delta)."""
    rng = np.random.default_rng(seed)
    off = _offsets(T)
    U = np.zeros((3, nlm(T)), dtype=np.complex128)
    for f, s in enumerate(scales):
        for m in range(T + 1):
            n = np.arange(max(m, 1), T + 1, dtype=np.float64)
            g = rng.standard_normal((2, n.size))
            v = s * n ** slope * (g[0] + 1j * g[1]) / math.sqrt(2.0)
            if m == 0:
                v = v.real + 0j
            U[f, off[m] + (n.astype(np.int64) - m)] = v
    return U


def balanced_state(T, seed, urms=20.0, Omega=OMEGA, radius=RADIUS):
    """Randomly phased, linearly balanced state with a kinetic-energy spectrum ~ n^-3."""
    rng = np.random.default_rng(seed)
    off = _offsets(T)
    zeta = np.zeros(nlm(T), dtype=np.complex128)
    for m in range(T + 1):
        n = np.arange(max(m, 1), T + 1, dtype=np.float64)
        g = rng.standard_normal((2, n.size))
        # KE_n = a^2/(n(n+1)) * sum_m |zeta_n^m|^2 over 2n+1 orders  ~ n^-3
        amp = np.sqrt(n * (n + 1.0) * n ** -3.0 / (2.0 * n + 1.0))
        v = amp * (g[0] + 1j * g[1]) / math.sqrt(2.0)
        if m == 0:
            v = v.real + 0j
        zeta[off[m] + (n.astype(np.int64) - m)] = v
    # rms wind: (1/4pi) * sum_m w_m sum_n a^2/(n(n+1)) |zeta|^2
    ke = 0.0
    for m in range(T + 1):
        n = np.arange(m, T + 1, dtype=np.float64)
        c = zeta[off[m]: off[m] + T + 1 - m]
        with np.errstate(divide="ignore", invalid="ignore"):
            wgt = np.where(n > 0, radius ** 2 / (n * (n + 1.0)), 0.0)
        ke += (1.0 if m == 0 else 2.0) * float(np.sum(wgt * np.abs(c) ** 2))
    zeta *= urms / math.sqrt(ke / (4.0 * math.pi))
    # linear balance of the divergence equation with delta = 0:
    #   n(n+1)/a^2 Phi_n = -2 Omega [ (n+1)/n e_n zeta_{n-1} + n/(n+1) e_{n+1} zeta_{n+1} ]
    phi = np.zeros_like(zeta)
    for m in range(T + 1):
        for n in range(max(m, 1), T + 1):
            s = 0.0 + 0.0j
            if n - 1 >= max(m, 1):
                e_n = math.sqrt((n * n - m * m) / (4.0 * n * n - 1.0))
                s += (n + 1.0) / n * e_n * zeta[off[m] + n - 1 - m]
            if n + 1 <= T:
                e_n1 = math.sqrt(((n + 1) ** 2 - m * m) / (4.0 * (n + 1) ** 2 - 1.0))
                s += n / (n + 1.0) * e_n1 * zeta[off[m] + n + 1 - m]
            phi[off[m] + n - m] = -(radius ** 2 / (n * (n + 1.0))) * 2.0 * Omega * s
    U = np.zeros((3, nlm(T)), dtype=np.complex128)
    U[0] = phi
    U[1] = zeta
    return U


def ensemble_truncations(count=64, seed=3, lo=63, hi=255):
    """Truncations T ~ U{lo..hi} for the uneven ensemble."""
    rng = np.random.default_rng(seed)
    return [int(t) for t in rng.integers(lo, hi + 1, size=count)]


def request_stream(count=2000, seed=5, rate=1.0):
    """Poisson request stream: arrival times, T = round(exp(U[ln 63, ln 511])),
    dt = exp(U[ln 600, ln 14400]) s, N = 256 * 2^round(3 ln(dt/600) / ln 24) (256..2048)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    T = np.rint(np.exp(rng.uniform(math.log(63), math.log(511), size=count))).astype(int)
    dt = np.exp(rng.uniform(math.log(600.0), math.log(14400.0), size=count))
    N = 256 * 2 ** np.rint(3.0 * np.log(dt / 600.0) / math.log(24.0)).astype(int)
    return [dict(arrival=float(t[i]), T=int(T[i]), dt=float(dt[i]), N=int(N[i]), seed=1000 + i)
            for i in range(count)]
