"""Serving loop (continuous batching over ragged REXI launches): each result is the same alone
and in the mix within the mixed-precision bound; invalid or never-fitting requests are
rejected with an error status and leave the others intact; a tight memory budget makes
requests wait for free slots instead of failing."""
import numpy as np
import pytest

from oracle import rexi as orx
from paper_1805_06557_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_06557_gb300 import rexi, serving
    return torch, rexi, serving


SPEC = [(15, 3600.0, 64), (31, 1800.0, 128), (47, 7200.0, 256), (20, 900.0, 64), (63, 3600.0, 256),
        (7, 14400.0, 128), (40, 600.0, 96), (55, 5000.0, 192), (33, 2400.0, 64), (63, 10000.0, 512)]


def _requests(serving, arrivals=None):
    reqs = []
    for k, (T, dt, N) in enumerate(SPEC):
        a = 0.0 if arrivals is None else arrivals[k]
        reqs.append(serving.Request(k, a, T, dt, N, syn.gaussian_state(T, 700 + k)))
    return reqs


def _alone(rexi, serving, r, precision="mixed"):
    """The request stepped alone by a uniform plan on the contour the engine chose for it."""
    import torch
    plan = rexi.Plan(r.T, r.N, r.dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR, p0=r.p0, Xc=r.Xc, precision=precision)
    a = torch.from_numpy(r.state).cuda().reshape(1, 3, -1).contiguous()
    b = torch.empty_like(a)
    plan.step(a, b)
    plan.sync()
    out = b.cpu().numpy()[0]
    plan.close()
    return out


def test_alone_equals_in_mix(env):
    torch, rexi, serving = env
    eng = serving.ServingEngine(Tmax=63, max_slots=16, hbm_bytes=64 << 20, max_poles=4096)
    arrivals = np.linspace(0.0, 0.02, len(SPEC))
    stats = eng.run(_requests(serving, arrivals))
    assert stats["completed"] == len(SPEC) and stats["rejected"] == 0
    for r in eng.done:
        err = orx.rel_l2(r.result, _alone(rexi, serving, r), r.T)
        assert np.all(err < 1e-9), (r.rid, err)
    eng.close()


def test_rejections_leave_others_intact(env):
    torch, rexi, serving = env
    eng = serving.ServingEngine(Tmax=63, max_slots=16, hbm_bytes=64 << 20, max_poles=4096)
    reqs = _requests(serving)
    bad_T = serving.Request(100, 0.0, 127, 3600.0, 64, syn.gaussian_state(127, 1))
    bad_shape = serving.Request(101, 0.0, 31, 3600.0, 64, np.zeros((3, 10), complex))
    eng.run(reqs + [bad_T, bad_shape])
    status = {r.rid: r.status for r in eng.done}
    assert status[100] == serving.REJECTED and status[101] == serving.REJECTED
    assert all(status[k] == serving.OK for k in range(len(SPEC)))
    for r in eng.done:
        if r.rid < len(SPEC):
            assert np.all(orx.rel_l2(r.result, _alone(rexi, serving, r), r.T) < 1e-9)
    eng.close()


def test_memory_budget_admission(env):
    """A budget that holds only ~2 of the largest states at a time: requests wait and are
    admitted as slots free up; a state larger than the whole budget is rejected."""
    torch, rexi, serving = env
    nlm63 = 64 * 65 // 2
    budget = 2 * 16 * (2 * 3 * nlm63 + 100)      # two T63 states (input + output arenas)
    eng = serving.ServingEngine(Tmax=127, max_slots=16, hbm_bytes=budget, max_poles=4096)
    reqs = _requests(serving)
    huge = serving.Request(200, 0.0, 127, 3600.0, 64, syn.gaussian_state(127, 3))
    stats = eng.run(reqs + [huge])
    status = {r.rid: r.status for r in eng.done}
    assert status[200] == serving.REJECTED and "budget" in [r for r in eng.done if r.rid == 200][0].error
    assert stats["completed"] == len(SPEC)
    assert eng.ticks >= 3
    for r in eng.done:
        if r.rid < len(SPEC):
            assert np.all(orx.rel_l2(r.result, _alone(rexi, serving, r), r.T) < 1e-9)
    eng.close()


SPEC_LARGE = [(255, 3600.0, 512), (511, 1800.0, 1024), (127, 1800.0, 512), (300, 2400.0, 512),
              (63, 3600.0, 256), (255, 3600.0, 512), (400, 1200.0, 1024)]


def test_alone_equals_in_mix_up_to_T511(env):
    """The serving sizes (Tmax = 511): requests of T63-T511, two of them identical in
    (T, dt, N) so that the ragged launch pairs their heavy tiles; each result equals the request
    stepped alone within the mixed-precision bound of 1e-8, and the T255 request matches the
    oracle on sampled zonal orders."""
    torch, rexi, serving = env
    from oracle import coeffs as oc
    eng = serving.ServingEngine(Tmax=511, max_slots=16, hbm_bytes=1 << 30, max_poles=1 << 15)
    reqs = [serving.Request(k, 1e-3 * k, T, dt, N, syn.gaussian_state(T, 900 + k))
            for k, (T, dt, N) in enumerate(SPEC_LARGE)]
    stats = eng.run(reqs)
    assert stats["completed"] == len(SPEC_LARGE) and stats["rejected"] == 0
    for r in eng.done:
        err = orx.rel_l2(r.result, _alone(rexi, serving, r), r.T)
        assert np.all(err < 1e-8), (r.rid, r.T, err)
    r0 = [r for r in eng.done if r.rid == 0][0]
    z, w = oc.rexi_coefficients(r0.N, r0.p0, r0.Xc)
    ms = [0, 1, 128, 255]
    ref = orx.rexi_step(r0.state, r0.T, r0.dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR, z, w, m_list=ms)
    mask = np.zeros(r0.result.shape[-1], bool)
    for m in ms:
        o = m * (2 * r0.T + 3 - m) // 2
        mask[o: o + r0.T + 1 - m] = True
    wgt = np.where(np.arange(mask.size) <= r0.T, 1.0, 2.0)[mask]
    num = np.sqrt(np.sum(wgt * np.abs(r0.result[:, mask] - ref[:, mask]) ** 2, axis=-1))
    den = np.sqrt(np.sum(wgt * np.abs(ref[:, mask]) ** 2, axis=-1))
    assert np.all(num / den < 1e-8), num / den
    eng.close()
