"""rexi_step_fp64_static: the REXI step for callers that cannot allocate device memory
(a host framework that owns all device memory through its own pool, loops that must not
trigger an allocation's device-wide synchronisation, deployments that fix every byte at
load time).  It must give the same result as the regular FP64 entry point, rexi_step on an
FP64 plan, within the FP64 tolerance of the parity tests, on two calls in a row (the
second call reuses the fixed array the first one left behind), and match the FP64 oracle
(paper Eq. rexi, pivoted banded LU per pole and zonal order) within the same tolerance.

Sizes cover the tile-split edges of the fixed array: T = 1 (the slot count is capped, and
the last slot holds fewer 32-pole groups than the others), pole counts that are not a
multiple of 32, and a call on a non-default stream.

This file is collected last so that a run stopping at its first failure has already run
every other test."""
import numpy as np
import pytest

from oracle import coeffs as oc
from oracle import rexi as orx
from paper_1805_06557_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

OM, A, PB = syn.OMEGA, syn.RADIUS, syn.PHIBAR


def _tol(z, w, X):
    # per-field relative L2, the FP64 parity tolerance: 1e-11, raised to 8 amp 2^-53 where the
    # contour's amplification makes FP64 rounding of the individual solves larger
    return max(1e-11, 8 * oc.amplification(z, w, X) * 2.0 ** -53)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_06557_gb300 import rexi
    return torch, rexi


@pytest.mark.parametrize("T,N,on_stream", [(63, 256, False), (20, 40, False), (1, 270, False),
                                           (5, 300, True), (63, 1024, True)])
def test_static_matches_plan_and_oracle_two_calls(env, T, N, on_stream):
    torch, rexi = env
    dt = 3600.0
    X = rexi.spectrum_bound(T, dt, OM, A, PB)
    p0, Xc = min(6.0, 1.6 * X), 1.6 * X
    z, w = oc.rexi_coefficients(N, p0, Xc)
    tol = _tol(z, w, X)
    stream = torch.cuda.Stream() if on_stream else None
    plan = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision="fp64", max_batch=1)
    for call, seed in enumerate((7, 8)):
        U0 = syn.gaussian_state(T, seed)
        u0 = torch.from_numpy(U0).cuda()
        ref = torch.empty_like(u0)
        plan.step(u0, ref, 1)
        torch.cuda.synchronize()
        out = torch.full_like(u0, float("nan"))
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(stream):
                rexi.step_fp64_static(T, N, dt, OM, A, PB, p0, Xc, u0, out, stream=stream)
        else:
            rexi.step_fp64_static(T, N, dt, OM, A, PB, p0, Xc, u0, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err_plan = orx.rel_l2(got, ref.cpu().numpy(), T)
        assert np.all(err_plan < tol), ("vs plan", call, err_plan, tol)
        oracle = orx.rexi_step(U0, T, dt, OM, A, PB, z, w)
        err_oracle = orx.rel_l2(got, oracle, T)
        assert np.all(err_oracle < tol), ("vs oracle", call, err_oracle, tol)
    plan.close()


def test_static_rejects_sizes_beyond_limit(env):
    torch, rexi = env
    u = torch.zeros(2, 3, rexi.nlm(64), dtype=torch.complex128, device="cuda")
    with pytest.raises(rexi.RexiError) as e:
        rexi.step_fp64_static(64, 64, 3600.0, OM, A, PB, 6.0, 10.0, u[0], u[1])
    assert e.value.code == rexi.REXI_EINVAL and "T = 64" in str(e.value)
    v = torch.zeros(2, 3, rexi.nlm(31), dtype=torch.complex128, device="cuda")
    with pytest.raises(rexi.RexiError) as e:
        rexi.step_fp64_static(31, 2048, 3600.0, OM, A, PB, 6.0, 10.0, v[0], v[1])
    assert e.value.code == rexi.REXI_EINVAL
    assert rexi.static_scratch_bytes() < 32 * 2 ** 20


def test_static_rejects_wrong_tensors(env):
    torch, rexi = env
    T = 15
    good = torch.zeros(3, rexi.nlm(T), dtype=torch.complex128, device="cuda")
    small = torch.zeros(3, rexi.nlm(T - 1), dtype=torch.complex128, device="cuda")
    strided = torch.zeros(3, 2 * rexi.nlm(T), dtype=torch.complex128, device="cuda")[:, ::2]
    single = torch.zeros(3, rexi.nlm(T), dtype=torch.complex64, device="cuda")
    for bad in (small, strided, single, good.cpu()):
        with pytest.raises(ValueError):
            rexi.step_fp64_static(T, 64, 3600.0, OM, A, PB, 6.0, 10.0, bad, good)
