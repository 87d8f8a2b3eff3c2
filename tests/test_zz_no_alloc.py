"""rexi_step_fp64_static: the REXI step for callers that cannot allocate device memory
(a host framework that owns all device memory through its own pool, loops that must not
trigger an allocation's device-wide synchronisation, deployments that fix every byte at
load time).  It must give the same result as the regular FP64 entry point, rexi_step on an
FP64 plan, within the FP64 tolerance of the parity tests, on two calls in a row (the
second call reuses the fixed array the first one left behind).

This file is collected last so that a run stopping at its first failure has already run
every other test."""
import numpy as np
import pytest

from paper_1805_06557_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

OM, A, PB = syn.OMEGA, syn.RADIUS, syn.PHIBAR
TOL = 1e-11  # per-field relative L2, the FP64 parity tolerance


def _rel(x, ref, T):
    w = np.where(np.arange(x.shape[-1]) <= T, 1.0, 2.0)
    num = np.sqrt(np.sum(w * np.abs(x - ref) ** 2, axis=-1))
    return num / np.sqrt(np.sum(w * np.abs(ref) ** 2, axis=-1))


@pytest.mark.parametrize("T,N", [(63, 256), (20, 40)])
def test_static_matches_plan_two_calls(T, N):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_06557_gb300 import rexi
    dt = 3600.0
    X = rexi.spectrum_bound(T, dt, OM, A, PB)
    p0, Xc = min(6.0, 1.6 * X), 1.6 * X
    plan = rexi.Plan(T, N, dt, OM, A, PB, p0=p0, Xc=Xc, precision="fp64", max_batch=1)
    for call, seed in enumerate((7, 8)):
        u0 = torch.from_numpy(syn.gaussian_state(T, seed)).cuda()
        ref = torch.empty_like(u0)
        plan.step(u0, ref, 1)
        out = torch.full_like(u0, float("nan"))
        rexi.step_fp64_static(T, N, dt, OM, A, PB, p0, Xc, u0, out)
        torch.cuda.synchronize()
        err = _rel(out.cpu().numpy(), ref.cpu().numpy(), T)
        assert np.all(err < TOL), (call, err)
    plan.close()


def test_static_rejects_sizes_beyond_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_06557_gb300 import rexi
    u = torch.zeros(2, 3, rexi.nlm(64), dtype=torch.complex128, device="cuda")
    with pytest.raises(rexi.RexiError) as e:
        rexi.step_fp64_static(64, 64, 3600.0, OM, A, PB, 6.0, 10.0, u[0], u[1])
    assert e.value.code == rexi.REXI_EINVAL and "T = 64" in str(e.value)
    with pytest.raises(rexi.RexiError) as e:
        rexi.step_fp64_static(31, 2048, 3600.0, OM, A, PB, 6.0, 10.0, u[0], u[1])
    assert e.value.code == rexi.REXI_EINVAL
    assert rexi.static_scratch_bytes() < 32 * 2 ** 20
