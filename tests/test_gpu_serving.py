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
    import torch
    p0, Xc = serving.contour(r.T, r.dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    plan = rexi.Plan(r.T, r.N, r.dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR, p0=p0, Xc=Xc, precision=precision)
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
