"""GPU parity of the nonlinear term and the Strang-split step (paper Sec. 3, Sec. 4.4)
against the FP64 oracle, through the C ABI (include/swe.h)."""
import math

import numpy as np
import pytest

from oracle import coeffs as oc
from oracle import rexi as orx
from oracle import sht as osht
from oracle import swe as oswe
from paper_1805_06557_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

OM, A, PB = syn.OMEGA, syn.RADIUS, syn.PHIBAR


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_06557_gb300 import rexi
    return torch, rexi


def _state(T, seed):
    U = syn.balanced_state(T, seed, urms=30.0)
    U[2] = syn.gaussian_state(T, seed + 50, scales=(0, 0, 2e-6))[2]
    return U


def _contour(T, dt):
    X = orx.spectrum_bound(T, dt, OM, A, PB)
    return (min(6.0, 1.6 * X), 1.6 * X) if X < 20 else (14.0, 1.4 * X)


@pytest.mark.parametrize("sprec", ["fp64", "df"])
@pytest.mark.parametrize("T,nlat,nlon", [(31, 48, 96), (63, 96, 192), (127, 192, 384)])
@pytest.mark.parametrize("kind,tol", [("gaussian", 2e-9), ("balanced", 5e-9)])
def test_nonlinear_matches_oracle(env, T, nlat, nlon, kind, tol, sprec):
    """N(U) against the oracle.  lap(KE) multiplies the rounding of the kinetic-energy
    analysis by n(n+1)/a^2 (1.6e4 at n = 127 relative to n = 1), which sets the bound of the
    divergence tendency at T127; for the geostrophically balanced state the tendencies are
    also small differences of large terms (|curl(zeta V)| ~ |lap KE| ~ 12 |N_delta|, and
    V.grad Phi' nearly vanishes along isobars).  The double-float Legendre precision meets the
    FP64 bounds."""
    torch, rexi = env
    U = _state(T, 3) if kind == "balanced" else syn.gaussian_state(T, 3, scales=(1e3, 2e-5, 5e-6))
    g = osht.Grid(T, nlat, nlon, A)
    ref = oswe.nonlinear(U, g)
    p0, Xc = _contour(T, 1800.0)
    plan = rexi.SwePlan(T, nlat, nlon, 1800.0, OM, A, PB, 64, p0, Xc, sh_precision=sprec)
    u = torch.from_numpy(U).cuda()
    t = torch.empty_like(u)
    plan.nonlinear(u, t)
    torch.cuda.synchronize()
    err = orx.rel_l2(t.cpu().numpy(), ref, T)
    assert np.all(err < tol), err
    plan.close()


@pytest.mark.parametrize("scheme,rprec,tol,nsub", [("ver1", "fp64", 1e-10, 1), ("ver0", "fp64", 1e-10, 1),
                                                   ("ver1", "mixed", 1e-8, 1), ("etdrk", "fp64", 1e-10, 1),
                                                   ("etdrk", "mixed", 1e-8, 1), ("irk", "fp64", 1e-10, 1),
                                                   ("lg_ver1", "fp64", 1e-10, 1), ("lg_etdrk", "fp64", 1e-10, 1),
                                                   ("lg_irk_ver0", "fp64", 1e-10, 1),
                                                   ("ver1", "fp64", 1e-10, 3), ("ver1", "mixed", 1e-8, 3),
                                                   ("ver0", "fp64", 1e-10, 2), ("irk", "fp64", 1e-10, 2),
                                                   ("lg_ver1", "fp64", 1e-10, 2),
                                                   ("lg_irk_ver0", "fp64", 1e-10, 2)])
def test_strang_steps_match_oracle(env, scheme, rprec, tol, nsub):
    """Strang ver1 / ver0 (Sec. 4.4), ETD2RK (Sec. 4.3), the Crank-Nicolson Strang step
    (Sec. 4.1) and the lg schemes (Coriolis in the explicit part, Table 2) against the oracle,
    with the explicit part in one midpoint step or in nsub sub-steps."""
    torch, rexi = env
    T, nlat, nlon, dt, N, nsteps = 31, 48, 96, 1800.0, 128, 3
    U0 = _state(T, 4)
    g = osht.Grid(T, nlat, nlon, A)
    sub = 0.5 * dt if scheme == "ver0" else dt
    p0, Xc = _contour(T, sub)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    ref = U0
    for _ in range(nsteps):
        if scheme == "ver1":
            ref = oswe.strang_ver1(ref, g, dt, OM, PB, z, w, nsub=nsub)
        elif scheme == "ver0":
            ref = oswe.strang_ver0(ref, g, dt, OM, PB, z, w, nsub=nsub)
        elif scheme == "irk":
            ref = oswe.cn_ver1(ref, g, dt, OM, PB, nsub=nsub)
        elif scheme == "lg_ver1":
            ref = oswe.strang_lg_ver1(ref, g, dt, OM, PB, z, w, nsub=nsub)
        elif scheme == "lg_irk_ver0":
            ref = oswe.cn_lg_ver0(ref, g, dt, OM, PB, nsub=nsub)
        elif scheme == "lg_etdrk":
            w1 = oc.rexi_coefficients(N, p0, Xc, k=1)[1]
            w2 = oc.rexi_coefficients(N, p0, Xc, k=2)[1]
            ref = oswe.etd2rk_lg(ref, g, dt, OM, PB, z, w, w1, w2)
        else:
            w1 = oc.rexi_coefficients(N, p0, Xc, k=1)[1]
            w2 = oc.rexi_coefficients(N, p0, Xc, k=2)[1]
            ref = oswe.etd2rk(ref, g, dt, OM, PB, z, w, w1, w2)
    plan = rexi.SwePlan(T, nlat, nlon, dt, OM, A, PB, N, p0, Xc, rexi_precision=rprec, scheme=scheme,
                        nsub=nsub)
    u = torch.from_numpy(U0).cuda()
    plan.step(u, nsteps)
    torch.cuda.synchronize()
    err = orx.rel_l2(u.cpu().numpy(), ref, T)
    assert np.all(err < tol), err
    plan.close()


@pytest.mark.parametrize("scheme,rprec,tol", [("ver1", "fp64", 1e-10), ("ver1", "mixed", 1e-8),
                                              ("lg_ver1", "fp64", 1e-10), ("etdrk", "fp64", 1e-10)])
def test_steps_with_diffusion_and_substeps_match_oracle(env, scheme, rprec, tol):
    """Three steps with del^4 hyper-diffusion split off symmetrically (D^{dt/2} o step o
    D^{dt/2}) and the explicit part in two sub-steps, against the oracle (T31, dt = 1800 s,
    the truncation degree e-folding in 1 h)."""
    torch, rexi = env
    T, nlat, nlon, dt, N, nsteps, nsub = 31, 48, 96, 1800.0, 128, 3, 2
    nu = 1.0 / (3600.0 * (T * (T + 1) / A ** 2) ** 2)
    U0 = _state(T, 4)
    g = osht.Grid(T, nlat, nlon, A)
    p0, Xc = _contour(T, dt)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    if scheme == "ver1":
        step = lambda V: oswe.strang_ver1(V, g, dt, OM, PB, z, w, nsub=nsub)
    elif scheme == "lg_ver1":
        step = lambda V: oswe.strang_lg_ver1(V, g, dt, OM, PB, z, w, nsub=nsub)
    else:
        w1 = oc.rexi_coefficients(N, p0, Xc, k=1)[1]
        w2 = oc.rexi_coefficients(N, p0, Xc, k=2)[1]
        step = lambda V: oswe.etd2rk(V, g, dt, OM, PB, z, w, w1, w2)
    ref = U0
    for _ in range(nsteps):
        ref = oswe.with_diffusion(step, ref, T, A, dt, nu)
    plan = rexi.SwePlan(T, nlat, nlon, dt, OM, A, PB, N, p0, Xc, rexi_precision=rprec, scheme=scheme,
                        nsub=nsub, visc=nu, visc_order=2)
    u = torch.from_numpy(U0).cuda()
    plan.step(u, nsteps)
    torch.cuda.synchronize()
    err = orx.rel_l2(u.cpu().numpy(), ref, T)
    assert np.all(err < tol), err
    # the diffusion really acts: without it the result differs by far more than the tolerance
    free = U0
    for _ in range(nsteps):
        free = step(free)
    assert np.min(orx.rel_l2(free, ref, T)[1:]) > 1e3 * tol
    plan.close()


def test_steady_zonal_flow_splitting_error_second_order(env):
    """Solid-body rotation in gradient-wind balance (L U + N(U) = 0, closed form) is a fixed
    point of the exact flow; the Strang split moves it by its O(dt^2) splitting error only:
    halving dt over the same 12 h divides the drift by ~4 (2nd order)."""
    torch, rexi = env
    T, nlat, nlon = 31, 48, 96
    g = osht.Grid(T, nlat, nlon, A)
    u0 = 38.61
    U = np.zeros((3, osht.nlm(T)), complex)
    U[1, osht.idx(T, 0, 1)] = 2 * u0 / A / math.sqrt(3 / (4 * math.pi))
    U[0] = g.analys(-(A * OM * u0 + 0.5 * u0 * u0) * g.mu[:, None] ** 2 * np.ones((1, nlon)))
    errs = []
    for dt, n in ((3600.0, 12), (1800.0, 24)):
        p0, Xc = _contour(T, dt)
        plan = rexi.SwePlan(T, nlat, nlon, dt, OM, A, PB, 128, p0, Xc)
        u = torch.from_numpy(U).cuda()
        plan.step(u, n)
        torch.cuda.synchronize()
        errs.append(float(np.max(orx.rel_l2(u.cpu().numpy(), U, T)[:2])))
        plan.close()
    rate = math.log2(errs[0] / errs[1])
    assert errs[0] < 1e-2 and 1.6 < rate < 2.6, (errs, rate)


# Unit of the operands of each tensor-core precision (see test_gpu_sht_tc.py): every transform
# of N(U) then has a relative error of at most 4u of its output's natural scale.
UNIT = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "tf32x3": 2.0 ** -20}
# The split-TF32 path is stated usable inside N(U): every tendency within 1e-3 (relative L2).
TARGET = {"tf32x3": 1e-3}


def nonlinear_error_bound(U, g, eps):
    """First-order bound on the per-field relative error of N(U) (paper Sec. 3, the N column
    of Eq. 1-3) when every SH transform errs by at most eps relative to its natural scale.

    Scales (L2 norms over the sphere, equal on the grid and in spectral space; |.|_inf the
    grid maximum; k = sqrt(T(T+1))/a the norm of divergence and curl on degrees <= T, k^2
    that of the Laplacian):
      synthesis of Phi', zeta:      eps |Phi'|, eps |zeta|
      synthesis of V = (u, v):      eps |V|
      analysis div/curl of F = qV:  eps k |F|, plus the propagated input error
                                    k (|q|_inf eps |V| + |V|_inf eps |q|)
      analysis of KE = V.V/2:       eps k^2 (|KE| + |V|_inf |V|) in the delta tendency.
    N_Phi = -div(Phi' V) and N_zeta = -div(zeta V) take one flux each; N_delta =
    curl(zeta V) - lap(KE) takes the zeta flux and the kinetic energy.  The norms come from
    the oracle's FP64 fields.  Returns the bound for (Phi', zeta, delta) relative to the
    norms of the oracle's tendencies."""
    T, a = g.T, g.a
    Phi, zeta, delta = U
    psi = osht.inv_laplacian(zeta, T, a)
    chi = osht.inv_laplacian(delta, T, a)
    Pg, Zg = g.synth(Phi), g.synth(zeta)
    Ug, Vg = g.synth_uv(psi, chi)
    cos = np.sqrt(g.coslat2)[:, None]
    u, v = Ug / cos, Vg / cos
    wgt = g.w[:, None] * (2.0 * np.pi / g.nlon)
    n2 = lambda f: float(np.sqrt(np.sum(wgt * f * f)))
    sn = lambda c: float(np.sqrt(np.sum(np.where(np.arange(c.shape[-1]) <= T, 1.0, 2.0) * np.abs(c) ** 2)))
    k = math.sqrt(T * (T + 1.0)) / a
    vn = math.hypot(n2(u), n2(v))
    vinf = float(np.max(np.hypot(u, v)))

    def flux(qg, qn):
        return k * (math.hypot(n2(qg * u), n2(qg * v)) + float(np.max(np.abs(qg))) * vn + vinf * qn)

    bP = eps * flux(Pg, sn(Phi))
    bZ = eps * flux(Zg, sn(zeta))
    bD = bZ + eps * k * k * (n2(0.5 * (u * u + v * v)) + vinf * vn)
    N = oswe.nonlinear(U, g)
    return np.array([bP / sn(N[0]), bZ / sn(N[1]), bD / sn(N[2])])


@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3"])
@pytest.mark.parametrize("kind", ["gaussian", "balanced"])
def test_nonlinear_tensor_core_error(env, prec, kind, capsys):
    """N(U) with the Legendre contractions on the tensor cores (and the FP32 FFT of those
    plans) against the FP64 oracle at T127, per field: within the first-order bound derived
    from the operand unit of the precision (nonlinear_error_bound with eps = 4u), and for the
    split-TF32 precision within its stated target of 1e-3.  The delta tendency contains
    -lap(KE), which multiplies the analysis error of KE at degree n by n(n+1)/a^2 (k^2 above):
    plain TF32 and BF16 transforms leave it wrong by O(0.1-1) and are not usable inside N(U);
    split TF32 keeps it near 1e-4."""
    torch, rexi = env
    T, nlat, nlon = 127, 192, 384
    U = _state(T, 3) if kind == "balanced" else syn.gaussian_state(T, 3, scales=(1e3, 2e-5, 5e-6))
    g = osht.Grid(T, nlat, nlon, A)
    ref = oswe.nonlinear(U, g)
    bound = nonlinear_error_bound(U, g, 4 * UNIT[prec])
    p0, Xc = _contour(T, 1800.0)
    plan = rexi.SwePlan(T, nlat, nlon, 1800.0, OM, A, PB, 64, p0, Xc, sh_precision=prec)
    u = torch.from_numpy(U).cuda()
    t = torch.empty_like(u)
    plan.nonlinear(u, t)
    torch.cuda.synchronize()
    err = orx.rel_l2(t.cpu().numpy(), ref, T)
    with capsys.disabled():
        print("\nN(U) %s %s per-field rel L2: %s  bound %s" % (prec, kind, ["%.2e" % e for e in err],
                                                            ["%.2e" % b for b in bound]))
    assert np.all(np.isfinite(err)) and np.all(err < bound), (err, bound)
    if prec in TARGET:
        assert np.all(err < TARGET[prec]), err
    plan.close()


@pytest.mark.parametrize("kind", ["gaussian", "balanced"])
def test_strang_step_split_tf32_matches_oracle(env, kind):
    """One Strang ver1 step at T127 with split-TF32 Legendre (FP64 REXI) against the oracle's
    FP64 step: the four N(U) evaluations of the step enter the state scaled by dt/2, so each
    field stays within the 1e-3 target of the split path (in practice far below it)."""
    torch, rexi = env
    T, nlat, nlon, N, dt = 127, 192, 384, 256, 1800.0
    U = _state(T, 3) if kind == "balanced" else syn.gaussian_state(T, 3, scales=(1e3, 2e-5, 5e-6))
    g = osht.Grid(T, nlat, nlon, A)
    p0, Xc = _contour(T, dt)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    ref = oswe.strang_ver1(U, g, dt, OM, PB, z, w)
    plan = rexi.SwePlan(T, nlat, nlon, dt, OM, A, PB, N, p0, Xc, sh_precision="tf32x3")
    u = torch.from_numpy(U).cuda()
    plan.step(u, 1)
    torch.cuda.synchronize()
    err = orx.rel_l2(u.cpu().numpy(), ref, T)
    assert np.all(err < TARGET["tf32x3"]), err
    plan.close()


@pytest.mark.parametrize("scheme,sprec", [("ver1", "fp64"), ("lg_etdrk", "fp64"), ("ver1", "tf32"),
                                          ("ver1", "tf32x3")])
def test_graph_replay_equals_eager_steps(env, scheme, sprec):
    """swe_step with nsteps >= 2 replays a captured graph of one step: the result equals the
    same steps run one call at a time (eager) bit for bit; a second state recaptures; steps
    with profiling on (always eager) agree as well."""
    torch, rexi = env
    T, nlat, nlon, N, dt = 31, 48, 96, 128, 1800.0
    p0, Xc = _contour(T, dt)
    plan = rexi.SwePlan(T, nlat, nlon, dt, OM, A, PB, N, p0, Xc, sh_precision=sprec, scheme=scheme)
    U0 = torch.from_numpy(syn.balanced_state(T, 2, urms=20.0)).cuda()
    a, b, c = U0.clone(), U0.clone(), U0.clone()
    plan.step(a, 5)          # 1 eager + capture + 4 replays
    for _ in range(5):
        plan.step(b, 1)      # eager
    plan.step(c, 3)          # another state address: recapture
    plan.step(c, 2)          # replays of that capture
    d = U0.clone()
    plan.set_profiling(True)
    plan.step(d, 5)          # eager (profiling)
    plan.set_profiling(False)
    torch.cuda.synchronize()
    assert torch.isfinite(a).all()
    assert torch.equal(a, b) and torch.equal(a, c) and torch.equal(a, d)
    assert not torch.equal(a, U0)
    plan.close()


_T127_REF = []  # the oracle's two steps, computed once for both precisions


@pytest.mark.parametrize("rprec,sprec,tol", [("fp64", "fp64", (1e-10, 1e-10, 5e-9)),
                                             ("mixed", "fp64", (1e-8, 1e-8, 1e-8)),
                                             ("fp64", "df", (1e-10, 1e-10, 5e-9)),
                                             ("mixed", "df", (1e-8, 1e-8, 1e-8))])
def test_config_T127_nonlinear_steps_match_oracle(env, rprec, sprec, tol):
    """The nonlinear configuration at full size: T127 on the 192 x 384 Gauss grid, 512 poles,
    dt = 1800 s, the balanced n^-3 state (seed 2, 20 m/s rms) of the benchmark, two Strang ver1
    steps against the oracle's (FP64 Legendre); the bench times 48 such steps.  The divergence
    starts at 0, so after two steps it is made of dt N_delta and carries the bound of the
    divergence tendency at T127 (5e-9, test_nonlinear_matches_oracle): lap(KE) multiplies the
    analysis rounding by n(n+1)/a^2.  Double-float transforms (SH_DF) meet the same bounds."""
    torch, rexi = env
    T, nlat, nlon, N, dt, nsteps = 127, 192, 384, 512, 1800.0, 2
    U0 = syn.balanced_state(T, 2)
    g = osht.Grid(T, nlat, nlon, A)
    p0, Xc = _contour(T, dt)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    if not _T127_REF:
        ref = U0
        for _ in range(nsteps):
            ref = oswe.strang_ver1(ref, g, dt, OM, PB, z, w)
        _T127_REF.append(ref)
    ref = _T127_REF[0]
    plan = rexi.SwePlan(T, nlat, nlon, dt, OM, A, PB, N, p0, Xc, rexi_precision=rprec, sh_precision=sprec)
    u = torch.from_numpy(U0).cuda()
    plan.step(u, nsteps)
    torch.cuda.synchronize()
    err = orx.rel_l2(u.cpu().numpy(), ref, T)
    assert np.all(err < np.array(tol)), err
    plan.close()
