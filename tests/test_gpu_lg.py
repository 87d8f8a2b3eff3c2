"""GPU parity of the gravity-only REXI step (rexi_lg_*: the lg_rexi_* methods, Sec. 3 split of L
into L_g and L_c, Sec. 5.3 diagonal solve, Eq. rexi) against the FP64 oracle, through the C ABI.

Tolerance (per-field relative L2, m > 0 weighted by 2): max(1e-11, 8 amp 2^-53) with the
contour's amplification amp, as for the full operator."""
import math

import numpy as np
import pytest

from oracle import coeffs as oc
from oracle import rexi as orx
from oracle import rexi_lg as olg
from paper_1805_06557_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

A, PB = syn.RADIUS, syn.PHIBAR


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_06557_gb300 import rexi
    return torch, rexi


def contour(T, dt):
    X = dt * math.sqrt(PB * T * (T + 1.0)) / A
    if X < 20:
        return min(6.0, 1.6 * X), 1.6 * X, X
    return 14.0, 1.4 * X, X


def tol(z, w, X):
    return max(1e-11, 8 * oc.amplification(z, w, X) * 2.0 ** -53)


def run(env, T, N, dt, U0, batch=None, inplace=False, **kw):
    torch, rexi = env
    Ub = U0 if U0.ndim == 3 else U0[None]
    plan = rexi.LgPlan(T, N, dt, A, PB, max_batch=Ub.shape[0], **kw)
    u0 = torch.from_numpy(np.ascontiguousarray(Ub)).cuda()
    u1 = u0 if inplace else torch.empty_like(u0)
    plan.step(u0, u1)
    plan.sync()
    out = u1.cpu().numpy()
    op = plan.operator()
    plan.close()
    return (out if U0.ndim == 3 else out[0]), op


@pytest.mark.parametrize("T,N,dt", [(1, 8, 3600.0), (2, 40, 3600.0), (5, 33, 3600.0), (17, 96, 3600.0),
                                    (63, 256, 3600.0), (127, 512, 1800.0), (255, 512, 3600.0)])
def test_matches_oracle(env, T, N, dt):
    """Tiny truncations, odd pole counts, the T63 / T127 / T255 configurations."""
    p0, Xc, X = contour(T, dt)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    U0 = syn.gaussian_state(T, 60 + T)
    ref = olg.rexi_step_lg(U0, T, dt, A, PB, z, w)
    out, (M, real) = run(env, T, N, dt, U0, p0=p0, Xc=Xc)
    assert real
    err = orx.rel_l2(out, ref, T)
    assert np.all(err < tol(z, w, X)), (err, tol(z, w, X))


@pytest.mark.parametrize("T,N,dt", [(511, 2048, 7200.0), (1023, 1024, 3600.0)])
def test_largest_sizes_sampled(env, T, N, dt):
    """T511 with 2048 poles at dt = 7200 s and the largest truncation: 6000 sampled
    coefficients (first and last included) against the oracle."""
    p0, Xc, X = contour(T, dt)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    U0 = syn.gaussian_state(T, 61)
    nlm = U0.shape[1]
    idx = np.unique(np.concatenate([[0, 1, T, nlm - 2, nlm - 1],
                                    np.random.default_rng(7).choice(nlm, 6000, replace=False)]))
    ref = olg.rexi_step_lg(U0, T, dt, A, PB, z, w, idx=idx)
    out, _ = run(env, T, N, dt, U0, p0=p0, Xc=Xc)
    got = out[:, idx]
    err = np.sqrt(np.sum(np.abs(got - ref) ** 2, axis=1) / np.sum(np.abs(ref) ** 2, axis=1))
    assert np.all(err < tol(z, w, X)), (err, tol(z, w, X))


def test_batch_inplace_and_deterministic(env):
    torch, rexi = env
    T, N, dt = 63, 256, 3600.0
    p0, Xc, X = contour(T, dt)
    U0 = np.stack([syn.gaussian_state(T, 70 + i) for i in range(5)])
    plan = rexi.LgPlan(T, N, dt, A, PB, p0=p0, Xc=Xc, max_batch=5)
    u0 = torch.from_numpy(U0).cuda()
    a = torch.empty_like(u0)
    b = torch.empty_like(u0)
    plan.step(u0, a)
    plan.step(u0, b)
    c = u0.clone()
    plan.step(c, c)  # in place
    plan.sync()
    assert torch.equal(a, b) and torch.equal(a, c)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    for i in (0, 4):
        ref = olg.rexi_step_lg(U0[i], T, dt, A, PB, z, w)
        assert np.all(orx.rel_l2(a[i].cpu().numpy(), ref, T) < tol(z, w, X))
    plan.close()


@pytest.mark.parametrize("k", [1, 2])
def test_psi_weights(env, k):
    """phi = 1, 2 applies the psi_1 / psi_2 weights of the same poles (Sec. 4.3)."""
    T, N, dt = 31, 128, 3600.0
    p0, Xc, X = contour(T, dt)
    z, w = oc.rexi_coefficients(N, p0, Xc, k=k)
    U0 = syn.gaussian_state(T, 80 + k)
    ref = olg.rexi_step_lg(U0, T, dt, A, PB, z, w)
    out, _ = run(env, T, N, dt, U0, p0=p0, Xc=Xc, phi=k)
    assert np.all(orx.rel_l2(out, ref, T) < tol(z, w, X))


def test_crank_nicolson_as_one_pole_plus_identity(env):
    """ident = -1 with the single pole z = 2, w = 4 is Crank-Nicolson of L_g:
    (I - dt L_g / 2)^-1 (I + dt L_g / 2) = 4 (2 - dt L_g)^-1 - I (Sec. 4.1, lg_irk)."""
    T, dt = 63, 1800.0
    U0 = syn.gaussian_state(T, 95)
    ref = orx.cn_step(U0, T, dt, 0.0, A, PB, part="Lg")
    out, (M, real) = run(env, T, 1, dt, U0, z=[2.0], w=[4.0], ident=-1.0)
    assert real
    assert np.all(orx.rel_l2(out, ref, T) < 1e-13)


def test_nonconjugate_poles_use_complex_sums(env):
    """A pole set that is not closed under conjugation (the upper half of a contour) keeps the
    complex per-degree sums."""
    T, N, dt = 31, 128, 3600.0
    p0, Xc, X = contour(T, dt)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    z, w = z[: N // 2], w[: N // 2]
    U0 = syn.gaussian_state(T, 90)
    ref = olg.rexi_step_lg(U0, T, dt, A, PB, z, w)
    out, (M, real) = run(env, T, N // 2, dt, U0, z=z, w=w)
    assert not real
    assert np.max(np.abs(M.imag)) > 1e-3 * np.max(np.abs(M.real))
    assert np.all(orx.rel_l2(out, ref, T) < tol(z, w, X))


def test_operator_is_the_oracle_on_unit_inputs(env):
    """M_n read back from the plan equals the oracle's response to unit coefficients, each entry
    to 64 eps times the sum of the magnitudes of its terms (the rounding bound of the pole
    sum: M_PP from w z / det, M_PD and M_DP from w / det scaled by dt Phibar and dt q_n,
    M_ZZ from w / z)."""
    T, N, dt = 15, 64, 3600.0
    p0, Xc, X = contour(T, dt)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    _, (M, real) = run(env, T, N, dt, syn.gaussian_state(T, 1), p0=p0, Xc=Xc)
    nlm = (T + 1) * (T + 2) // 2
    eps = 2.0 ** -53
    se = np.sum(np.abs(w / z))
    for n in (0, 1, 7, 15):
        q = n * (n + 1.0) / A ** 2
        det = z * z + dt * dt * PB * q
        s1 = np.sum(np.abs(w * z / det)) if n else se
        s0 = np.sum(np.abs(w / det))
        i = n  # m = 0 block: index n
        resp = {}
        for f in (0, 1, 2):
            U = np.zeros((3, nlm), complex)
            U[f, i] = 1.0
            resp[f] = olg.rexi_step_lg(U, T, dt, A, PB, z, w)[:, i]
        checks = [(resp[0][0], M[n, 0], s1), (resp[2][2], M[n, 0], s1), (resp[1][1], M[n, 3], se)]
        if n:
            checks += [(resp[2][0], M[n, 1], dt * PB * s0), (resp[0][2], M[n, 2], dt * q * s0)]
        else:
            checks += [(resp[2][0], M[n, 1], se), (resp[0][2], M[n, 2], se)]
        for got, ref, scale in checks:
            assert abs(got - ref) <= 64 * eps * scale, (n, got, ref, scale)
    assert real


def test_errors(env):
    torch, rexi = env
    T, N, dt = 15, 32, 3600.0
    p0, Xc, _ = contour(T, dt)
    with pytest.raises(rexi.RexiError) as e:
        rexi.LgPlan(0, N, dt, A, PB, p0=p0, Xc=Xc)
    assert e.value.code == rexi.REXI_EINVAL
    with pytest.raises(rexi.RexiError):
        rexi.LgPlan(T, N, dt, A, PB, p0=p0, Xc=Xc, phi=3)
    with pytest.raises(rexi.RexiError):
        rexi.LgPlan(T, 2, dt, A, PB, z=[0.0, 1.0], w=[1.0, 1.0])   # zero pole
    plan = rexi.LgPlan(T, N, dt, A, PB, p0=p0, Xc=Xc, max_batch=2)
    u = torch.zeros(3, 3, rexi.nlm(T), dtype=torch.complex128, device="cuda")
    s = 3 * rexi.nlm(T) * 16
    assert plan.step_raw(u.data_ptr(), u.data_ptr() + s // 2, 1) == rexi.REXI_EINVAL   # partial overlap
    assert plan.step_raw(u.data_ptr(), u[1].data_ptr(), 3) == rexi.REXI_EINVAL        # batch > max
    assert plan.step_raw(u.data_ptr(), u[1].data_ptr(), 0) == rexi.REXI_EINVAL
    assert plan.step_raw(0, u[1].data_ptr(), 1) == rexi.REXI_EINVAL
    assert plan.step_raw(u[0].data_ptr(), u[0].data_ptr(), 1) == rexi.REXI_OK          # in place
    plan.sync()
    plan.close()
