"""GPU parity of rexi_step (paper Eq. rexi) against the FP64 CPU oracle, through the C ABI.

Tolerances (per-field relative L2, m > 0 weighted by 2):
  * FP64 plans: 1e-11, raised to 8 * amp * 2^-53 where the amplification
    amp = max_x sum_n |w_n| / |z_n - ix| of the contour makes FP64 rounding of the
    individual solves larger (T255 at dt = 3600 s: amp = 3.5e5, bound 3.1e-10).
  * mixed plans: 1e-8 (the stated bound of the reduced-precision path).
"""
import numpy as np
import pytest

from oracle import coeffs as oc
from oracle import rexi as orx
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


def contour(T, dt, N):
    X = orx.spectrum_bound(T, dt, OM, A, PB)
    if X < 20:
        return min(6.0, 1.6 * X), 1.6 * X, X
    return 14.0, 1.4 * X, X


def fp64_tol(z, w, X):
    return max(1e-11, 8 * oc.amplification(z, w, X) * 2.0 ** -53)


def run_plan(env, T, N, dt, U0, prec, p0, Xc, batch=None, **kw):
    torch, rexi = env
    Ub = U0 if U0.ndim == 3 else U0[None]
    B = Ub.shape[0]
    plan = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision=prec, max_batch=B, **kw)
    u0 = torch.from_numpy(np.ascontiguousarray(Ub)).cuda()
    u1 = torch.empty_like(u0)
    plan.step(u0, u1)
    plan.sync()
    out = u1.cpu().numpy()
    info = plan.info()
    plan.close()
    return (out if U0.ndim == 3 else out[0]), info


def masked_rel(x, ref, T, ms):
    mask = np.zeros(x.shape[-1], bool)
    for m in ms:
        o = m * (2 * T + 3 - m) // 2
        mask[o: o + T + 1 - m] = True
    w = np.where(np.arange(x.shape[-1]) <= T, 1.0, 2.0)[mask]
    num = np.sqrt(np.sum(w * np.abs(x[..., mask] - ref[..., mask]) ** 2, axis=-1))
    den = np.sqrt(np.sum(w * np.abs(ref[..., mask]) ** 2, axis=-1))
    return num / den


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_config_T63_N256(env, prec):
    """T63, N = 256 poles, dt = 3600 s, n^-1.5 Gaussian coefficients (seed 1)."""
    T, N, dt = 63, 256, 3600.0
    p0, Xc, X = contour(T, dt, N)
    U0 = syn.gaussian_state(T, 1)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    ref = orx.rexi_step(U0, T, dt, OM, A, PB, z, w)
    out, info = run_plan(env, T, N, dt, U0, prec, p0, Xc)
    err = orx.rel_l2(out, ref, T)
    tol = fp64_tol(z, w, X) if prec == "fp64" else 1e-8
    assert np.all(err < tol), (err, tol, info)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_golden_step_on_paper_contour(env, golden_step, prec):
    """The stored T7 step of tests/golden/ (written from the oracle) on the contour that Sec. 5
    starts from: p0 = 10, p_{+-1} = +-30i, N = 128, dt = 21600 s."""
    k, U0, U1 = golden_step("rexi_step_T7_N128.txt")
    assert (k["Omega"], k["radius"], k["Phibar"]) == (OM, A, PB)
    T, N, dt = int(k["T"]), int(k["N"]), k["dt"]
    z, w = oc.rexi_coefficients(N, k["p0"], k["Xc"])
    X = orx.spectrum_bound(T, dt, OM, A, PB)
    out, info = run_plan(env, T, N, dt, U0, prec, k["p0"], k["Xc"])
    err = orx.rel_l2(out, U1, T)
    tol = fp64_tol(z, w, X) if prec == "fp64" else 1e-8
    assert np.all(err < tol), (err, tol, info)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("T,N", [(1, 8), (2, 40), (5, 33), (17, 96), (40, 64), (47, 200)])
def test_small_and_ragged(env, prec, T, N):
    """Tiny truncations (single-element chains), pole counts that are not a multiple of 32,
    chain lengths that are not a multiple of the 16/32-element blocks."""
    dt = 3600.0
    p0, Xc, X = contour(T, dt, N)
    U0 = syn.gaussian_state(T, 10 + T)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    ref = orx.rexi_step(U0, T, dt, OM, A, PB, z, w)
    out, _ = run_plan(env, T, N, dt, U0, prec, p0, Xc)
    err = orx.rel_l2(out, ref, T)
    tol = fp64_tol(z, w, X) if prec == "fp64" else 1e-8
    assert np.all(err < tol), (err, tol)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_T127_N512(env, prec):
    """The linear part of the T127 / dt = 1800 s / 512-pole nonlinear configuration."""
    T, N, dt = 127, 512, 1800.0
    p0, Xc, X = contour(T, dt, N)
    U0 = syn.balanced_state(T, 2)
    U0[2] = syn.gaussian_state(T, 22, scales=(0, 0, 1e-6))[2]
    z, w = oc.rexi_coefficients(N, p0, Xc)
    ms = [0, 1, 2, 3, 31, 64, 100, 126, 127]
    ref = orx.rexi_step(U0, T, dt, OM, A, PB, z, w, m_list=ms)
    out, _ = run_plan(env, T, N, dt, U0, prec, p0, Xc)
    err = masked_rel(out, ref, T, ms)
    tol = fp64_tol(z, w, X) if prec == "fp64" else 1e-8
    assert np.all(err < tol), (err, tol)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_T255_N512_batched_sampled(env, prec):
    """Full benchmark size: a batch of 4 T255 states (seeds 101-104), N = 512, dt = 3600 s,
    in the bench launch configuration; the oracle checks sampled zonal orders."""
    T, N, dt = 255, 512, 3600.0
    p0, Xc, X = contour(T, dt, N)
    U0 = np.stack([syn.gaussian_state(T, 101 + i) for i in range(4)])
    z, w = oc.rexi_coefficients(N, p0, Xc)
    ms = [0, 1, 2, 31, 100, 254, 255]
    out, info = run_plan(env, T, N, dt, U0, prec, p0, Xc)
    tol = fp64_tol(z, w, X) if prec == "fp64" else 1e-8
    for b in (0, 3):
        ref = orx.rexi_step(U0[b], T, dt, OM, A, PB, z, w, m_list=ms)
        err = masked_rel(out[b], ref, T, ms)
        assert np.all(err < tol), (b, err, tol, info)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("T,N,dt,ms", [
    (511, 2048, 7200.0, [0, 1, 2, 255, 510, 511]),      # the high-resolution configuration
    (1023, 1024, 3600.0, [0, 1, 511, 1022, 1023]),      # the largest truncation a plan accepts
])
def test_largest_sizes_sampled(env, prec, T, N, dt, ms):
    """T511 with 2048 poles at dt = 7200 s and T1023 (the plan's maximum truncation, chains of
    up to 512 elements per parity): sampled zonal orders, first and last included."""
    p0, Xc, X = contour(T, dt, N)
    U0 = syn.gaussian_state(T, 7)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    ref = orx.rexi_step(U0, T, dt, OM, A, PB, z, w, m_list=ms)
    out, info = run_plan(env, T, N, dt, U0, prec, p0, Xc)
    err = masked_rel(out, ref, T, ms)
    tol = fp64_tol(z, w, X) if prec == "fp64" else 1e-8
    assert np.all(err < tol), (err, tol, info)


@pytest.mark.parametrize("T,N,dt", [(63, 256, 3600.0), (255, 512, 3600.0)])
def test_fp64_pruned_matches_full_oracle(env, T, N, dt):
    """An FP64 plan that leaves out poles of summed gain <= 2^-60 stays within the FP64
    tolerance of the oracle's sum over all N poles."""
    p0, Xc, X = contour(T, dt, N)
    U0 = syn.gaussian_state(T, 400 + T)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    ms = [0, 1, T // 2, T]
    ref = orx.rexi_step(U0, T, dt, OM, A, PB, z, w, m_list=ms)
    out, info = run_plan(env, T, N, dt, U0, "fp64", p0, Xc, prune_tau=2.0 ** -60)
    assert info["n_pruned"] > 0 and info["pruned_gain"] <= 2.0 ** -60
    err = masked_rel(out, ref, T, ms)
    assert np.all(err < fp64_tol(z, w, X)), (err, info)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_single_and_is_deterministic(env, prec):
    torch, rexi = env
    T, N, dt = 63, 256, 3600.0
    p0, Xc, X = contour(T, dt, N)
    U0 = np.stack([syn.gaussian_state(T, 200 + i) for i in range(5)])
    plan = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision=prec, max_batch=5)
    u0 = torch.from_numpy(U0).cuda()
    u1 = torch.empty_like(u0)
    plan.step(u0, u1)
    u1b = torch.empty_like(u0)
    plan.step(u0, u1b)
    plan.sync()
    assert torch.equal(u1, u1b), "repeated call is not bitwise reproducible"
    tol = 1e-13 if prec == "fp64" else 1e-9
    for b in range(5):
        one = torch.empty_like(u0[b:b + 1])
        plan.step(u0[b:b + 1].contiguous(), one)
        plan.sync()
        err = orx.rel_l2(one.cpu().numpy()[0], u1[b].cpu().numpy(), T)
        assert np.all(err < tol), (b, err)
    plan.close()


@pytest.mark.parametrize("B", [2, 3, 6, 7])
def test_heavy_tile_forms(env, B):
    """Batches that exercise every form of heavy tile: a lone pair (B = 2), a pair and a single
    state (3), two pairs on half-warps and a lone pair (6), and all three (7).  Every state
    matches its one-state result, and the last state of B = 7 the oracle."""
    torch, rexi = env
    T, N, dt = 63, 256, 3600.0
    p0, Xc, X = contour(T, dt, N)
    U0 = np.stack([syn.gaussian_state(T, 500 + i) for i in range(B)])
    plan = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision="mixed", max_batch=8)
    u0 = torch.from_numpy(U0).cuda()
    u1 = torch.empty_like(u0)
    plan.step(u0, u1)
    one = torch.empty_like(u0[:1])
    for b in range(B):
        plan.step(u0[b:b + 1].contiguous(), one)
        plan.sync()
        err = orx.rel_l2(u1[b].cpu().numpy(), one[0].cpu().numpy(), T)
        assert np.all(err < 1e-9), (B, b, err)
    if B == 7:
        z, w = oc.rexi_coefficients(N, p0, Xc)
        ms = [0, 1, 31, 63]
        ref = orx.rexi_step(U0[6], T, dt, OM, A, PB, z, w, m_list=ms)
        assert np.all(masked_rel(u1[6].cpu().numpy(), ref, T, ms) < 1e-8)
    plan.close()


def test_step_host_matches_device(env):
    torch, rexi = env
    T, N, dt = 31, 64, 3600.0
    p0, Xc, _ = contour(T, dt, N)
    U0 = np.stack([syn.gaussian_state(T, 300 + i) for i in range(2)])
    plan = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision="fp64", max_batch=2)
    h = plan.step_host(U0)
    u0 = torch.from_numpy(U0).cuda()
    u1 = torch.empty_like(u0)
    plan.step(u0, u1)
    plan.sync()
    assert np.array_equal(h, u1.cpu().numpy())
    plan.close()


def test_step_host_mixed_pinned_and_pageable(env):
    """Mixed plans read and write pinned (mapped) host buffers in place over the host link and
    stage pageable ones through device copies: both equal the device step bit for bit."""
    torch, rexi = env
    T, N, dt, B = 63, 256, 3600.0, 5
    p0, Xc, _ = contour(T, dt, N)
    U0 = np.stack([syn.gaussian_state(T, 310 + i) for i in range(B)])
    plan = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision="mixed", max_batch=B)
    u0 = torch.from_numpy(U0).cuda()
    u1 = torch.empty_like(u0)
    plan.step(u0, u1, B)
    plan.sync()
    ref = u1.cpu().numpy()
    hin = torch.from_numpy(U0).pin_memory()
    hout = torch.zeros_like(hin).pin_memory()
    plan.step_host_ptr(hin.data_ptr(), hout.data_ptr(), B)  # pinned: in place
    assert np.array_equal(hout.numpy(), ref)
    assert np.array_equal(plan.step_host(U0), ref)            # pageable: staged
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_step_host_async_pipelined(env, prec):
    """rexi_step_host_async: a stream of steps on distinct pinned buffers (copies of the steps
    before and after overlapping each step's kernels, two staging slots in turn), then one
    pair of buffers reused by every call (as a serving loop would), a synchronous host step in
    between, and pageable buffers: every result equals the device step of its input bit for
    bit."""
    torch, rexi = env
    T, N, dt, B, n = 63, 256, 3600.0, 4, 5
    p0, Xc, _ = contour(T, dt, N)
    plan = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision=prec, max_batch=B)
    ins = [np.stack([syn.gaussian_state(T, 400 + 10 * j + i) for i in range(B)]) for j in range(n)]
    refs = []
    for U0 in ins:
        u0 = torch.from_numpy(U0).cuda()
        u1 = torch.empty_like(u0)
        plan.step(u0, u1, B)
        plan.sync()
        refs.append(u1.cpu().numpy())
    hin = [torch.from_numpy(U0).pin_memory() for U0 in ins]
    hout = [torch.full_like(h, float("nan")).pin_memory() for h in hin]
    for j in range(n):
        plan.step_host_async_ptr(hin[j].data_ptr(), hout[j].data_ptr(), B)
    plan.sync()
    for j in range(n):
        assert np.array_equal(hout[j].numpy(), refs[j]), j
    # one buffer pair for every call: the last result stays
    out = torch.full_like(hin[0], float("nan")).pin_memory()
    for j in range(n):
        plan.step_host_async_ptr(hin[j].data_ptr(), out.data_ptr(), B)
    assert np.array_equal(plan.step_host(ins[1]), refs[1])   # a synchronous step in between
    plan.sync()
    assert np.array_equal(out.numpy(), refs[n - 1])
    # pageable buffers: correct, without the overlap
    pg = np.empty_like(ins[2])
    plan.step_host_async_ptr(ins[2].ctypes.data, pg.ctypes.data, B)
    plan.sync()
    assert np.array_equal(pg, refs[2])
    with pytest.raises(rexi.RexiError):
        plan.step_host_async_ptr(hin[0].data_ptr(), hout[0].data_ptr(), B + 1)
    plan.close()


def test_explicit_poles_and_zero_input(env):
    """Poles given explicitly (the oracle's) give the same result; a zero state stays zero."""
    torch, rexi = env
    T, N, dt = 21, 64, 3600.0
    p0, Xc, X = contour(T, dt, N)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    U0 = syn.gaussian_state(T, 5)
    a, _ = run_plan(env, T, N, dt, U0, "fp64", p0, Xc)
    b, _ = run_plan(env, T, N, dt, U0, "fp64", None, None, z=z, w=w)
    assert np.max(orx.rel_l2(a, b, T)) < 1e-14
    zero, _ = run_plan(env, T, N, dt, np.zeros_like(U0), "mixed", p0, Xc)
    assert np.all(zero == 0)


def test_errors(env):
    torch, rexi = env
    T, N, dt = 15, 32, 3600.0
    p0, Xc, _ = contour(T, dt, N)
    with pytest.raises(rexi.RexiError) as e:
        rexi.Plan(0, N, dt, OM, A, PB, p0=p0, Xc=Xc)
    assert e.value.code == rexi.REXI_EINVAL
    with pytest.raises(rexi.RexiError):
        rexi.Plan(T, N, -1.0, OM, A, PB, p0=p0, Xc=Xc)
    with pytest.raises(rexi.RexiError):
        rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision=7)
    plan = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, max_batch=2)
    u = torch.zeros(3, 3, rexi.nlm(T), dtype=torch.complex128, device="cuda")
    assert plan.step_raw(u.data_ptr(), u.data_ptr(), 1) == rexi.REXI_EINVAL      # aliasing
    assert plan.step_raw(u.data_ptr(), u[1].data_ptr(), 3) == rexi.REXI_EINVAL   # batch > max
    assert plan.step_raw(u.data_ptr(), u[1].data_ptr(), 0) == rexi.REXI_EINVAL
    assert plan.step_raw(0, u[1].data_ptr(), 1) == rexi.REXI_EINVAL
    assert "batch" in rexi.last_error() or "null" in rexi.last_error()
    assert plan.step_raw(u[0].data_ptr(), u[1].data_ptr(), 1) == rexi.REXI_OK
    plan.sync()
    plan.close()


def test_mixed_heavy_classification_and_pruning(env):
    """Heavy poles have the largest gains; pruned poles the smallest, their summed gain within
    the default 1e-10; conjugate pairs are kept or pruned together; the largest pruned poles
    fill the last 32-pole light group."""
    torch, rexi = env
    T, N, dt = 255, 512, 3600.0
    p0, Xc, X = contour(T, dt, N)
    plan = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision="mixed")
    z, w, cls = plan.poles()
    info = plan.info()
    assert info["n_heavy"] % 16 == 0 and 0 < info["n_heavy"] < N
    yi = np.clip(z.imag, -X, X)
    gain = np.abs(w) / np.abs(z - 1j * yi)
    heavy, light, pruned = cls == 1, cls == 0, cls == -1
    assert gain[heavy].min() >= gain[light].max()
    assert np.sum(gain > 1e-3) <= info["n_heavy"]
    assert info["n_pruned"] == pruned.sum() > 0
    assert gain[light].min() >= gain[pruned].max()
    assert gain[pruned].sum() <= 1e-10 and abs(gain[pruned].sum() - info["pruned_gain"]) <= 1e-12 * 1e-10
    assert light.sum() % 32 == 0
    assert np.array_equal(np.sort_complex(z[pruned]), np.sort_complex(np.conj(z[pruned])))
    # the oracle's sum over the solved poles alone differs from the full sum by <= the bound
    U = syn.gaussian_state(T, 3)
    zo, wo = oc.rexi_coefficients(N, p0, Xc)
    ref_all = orx.rexi_step(U, T, dt, OM, A, PB, zo, wo, m_list=[0, 200])
    keep = ~pruned
    ref_kept = orx.rexi_step(U, T, dt, OM, A, PB, z[keep], w[keep], m_list=[0, 200])
    # (both FP64 sums, in different pole orders: rounding of order amp * 2^-53)
    assert np.max(masked_rel(ref_kept, ref_all, T, [0, 200])) < fp64_tol(zo, wo, X)
    plan.close()
    fp = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision="fp64")
    assert fp.info()["n_pruned"] == 0          # FP64 plans solve every pole by default
    fp.close()


_PART_REF = []  # the oracle's whole steps of the four states below, computed once


@pytest.mark.parametrize("mode", ["poles", "m"])
@pytest.mark.parametrize("prec,size", [("fp64", 2), ("fp64", 3), ("mixed", 2), ("mixed", 3)])
def test_partitioned_plans_sum_to_the_whole_step(env, mode, prec, size):
    """The multi-GPU partition of one step (paper Sec. 5.3-5.4), run rank by rank on one GPU:
    the sum of the ranks' outputs (what the all-reduce forms) equals the oracle's whole step
    within the precision's tolerance, every rank of the m partition writes exact zeros on the
    orders it does not own, and a batch of 4 (heavy tiles of state pairs) works the same."""
    torch, rexi = env
    T, N, dt, B = 63, 256, 3600.0, 4
    p0, Xc, X = contour(T, dt, N)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    U0 = np.stack([syn.gaussian_state(T, 60 + b) for b in range(B)])
    if not _PART_REF:
        _PART_REF.extend(orx.rexi_step(U0[b], T, dt, OM, A, PB, z, w) for b in range(B))
    u0 = torch.from_numpy(U0).cuda()
    total = torch.zeros_like(u0)
    for r in range(size):
        plan = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision=prec, max_batch=B,
                         partition=(mode, r, size))
        u1 = torch.full_like(u0, float("nan"))
        plan.step(u0, u1)
        plan.sync()
        if mode == "m":
            own = rexi.partition("m", T, N, r, size)
            mask = torch.from_numpy(np.concatenate([np.full(T + 1 - m, own[m]) for m in range(T + 1)])).cuda()
            assert bool((u1[..., ~mask] == 0).all())
        total += u1
        plan.close()
    tot = total.cpu().numpy()
    for b in range(B):
        err = orx.rel_l2(tot[b], _PART_REF[b], T)
        tol = fp64_tol(z, w, X) if prec == "fp64" else 1e-8
        assert np.all(err < tol), (b, err, tol)


def test_mixed_fp64_class_at_large_amplification(env):
    """T511 with 2048 poles at dt = 7200 s on the contour of the library's search (p0 = 20,
    amplification 2.4e8, gains up to 2e7): the mixed plan solves its 64 largest-gain poles in
    FP64, so it is as accurate as the FP64 plan (within a factor of 2 per field, on sampled
    zonal orders against the oracle); without that class, a refined FP32 solve and
    double-float partial sums (about 2^-48 of a partial sum) leave it more than 10x worse."""
    torch, rexi = env
    T, N, dt = 511, 2048, 7200.0
    X = orx.spectrum_bound(T, dt, OM, A, PB)
    p0, Xc = rexi.contour_select(X, N)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    U0 = syn.gaussian_state(T, 7)
    ms = [0, 1, 255, 511]
    ref = orx.rexi_step(U0, T, dt, OM, A, PB, z, w, m_list=ms)
    errs = {}
    for name, kw in (("fp64", dict(precision="fp64")), ("mixed", dict(precision="mixed")),
                     ("mixed_b4", dict(precision="mixed", max_batch=4)),
                     ("mixed_no_fp64_class", dict(precision="mixed", fp64_tau=1e300))):
        kw = dict(kw)
        B = kw.pop("max_batch", 1)
        prec = kw.pop("precision")
        out, info = run_plan(env, T, N, dt, np.stack([U0] * B), prec, p0, Xc, **kw)
        errs[name] = masked_rel(out[0], ref, T, ms)
        if prec == "mixed" and "fp64_tau" not in kw:
            assert info["n_fp64"] == 64, info
    tol = fp64_tol(z, w, X)
    assert np.all(errs["fp64"] < tol), errs
    for name in ("mixed", "mixed_b4"):
        assert np.all(errs[name] < np.maximum(1e-8, 2 * errs["fp64"])), errs
    assert np.max(errs["mixed_no_fp64_class"]) > 10 * np.max(errs["mixed"]), errs
