"""Ragged REXI launches: instances of different truncation, time step and pole count in one
launch (uneven per-m chain lengths), CUDA-graph replay and the autotuner, against the oracle
and against the same instance solved alone."""
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


def contour(T, dt):
    X = orx.spectrum_bound(T, dt, OM, A, PB)
    return (min(6.0, 1.6 * X), 1.6 * X) if X < 20 else (14.0, 1.4 * X)


INST = [(15, 64, 3600.0), (40, 96, 1800.0), (7, 32, 7200.0), (31, 256, 3600.0), (23, 40, 900.0),
        (47, 128, 5400.0)]


def _run(env, prec, inst, graph=False):
    torch, rexi = env
    Tmax = max(t for t, _, _ in inst)
    elems = sum((t + 1) * (t + 2) // 2 for t, _, _ in inst)
    r = rexi.RaggedPlan(Tmax, len(inst), 4096, elems, OM, A, PB, precision=prec,
                        stream=torch.cuda.Stream())
    full = [(t, n, dt) + contour(t, dt) for t, n, dt in inst]
    off = r.set(full)
    U0 = np.zeros(off[-1], complex)
    states = []
    for i, (t, n, dt) in enumerate(inst):
        s = syn.gaussian_state(t, 500 + i)
        states.append(s)
        U0[off[i]: off[i + 1]] = s.reshape(-1)
    u0 = torch.from_numpy(U0).cuda()
    u1 = torch.empty_like(u0)
    torch.cuda.synchronize()
    if graph:
        r.capture(u0, u1)
    r.step(u0, u1)
    r.sync()
    return r, off, states, u0, u1


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 1e-8)])
def test_ragged_matches_oracle(env, prec, tol):
    torch, rexi = env
    r, off, states, u0, u1 = _run(env, prec, INST)
    out = u1.cpu().numpy()
    for i, (t, n, dt) in enumerate(INST):
        p0, Xc = contour(t, dt)
        z, w = oc.rexi_coefficients(n, p0, Xc)
        ref = orx.rexi_step(states[i], t, dt, OM, A, PB, z, w)
        err = orx.rel_l2(out[off[i]: off[i + 1]].reshape(3, -1), ref, t)
        assert np.all(err < tol), (i, err)
    r.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_alone_equals_in_mix(env, prec):
    """Each instance solved alone (uniform plan) equals its result inside the ragged launch."""
    torch, rexi = env
    r, off, states, u0, u1 = _run(env, prec, INST)
    out = u1.cpu().numpy()
    tol = 1e-13 if prec == "fp64" else 1e-9
    for i, (t, n, dt) in enumerate(INST):
        p0, Xc = contour(t, dt)
        plan = rexi.Plan(t, n, dt, OM, A, PB, p0=p0, Xc=Xc, precision=prec)
        a = torch.from_numpy(states[i]).cuda().reshape(1, 3, -1).contiguous()
        b = torch.empty_like(a)
        plan.step(a, b)
        plan.sync()
        err = orx.rel_l2(out[off[i]: off[i + 1]].reshape(3, -1), b.cpu().numpy()[0], t)
        assert np.all(err < tol), (i, err)
        plan.close()
    r.close()


def test_graph_replay_and_tuner(env):
    torch, rexi = env
    r, off, states, u0, u1 = _run(env, "mixed", INST, graph=True)
    first = u1.clone()
    for _ in range(3):
        r.step(u0, u1)  # graph replays
    r.sync()
    assert torch.equal(first, u1)
    q, ms = r.tune(u0, u1, reps=2)
    assert q in (1, 2, 4, 8) and ms > 0
    r.step(u0, u1)
    r.sync()
    err = np.max(np.abs((u1 - first).cpu().numpy())) / np.max(np.abs(first.cpu().numpy()))
    assert err < 1e-9
    r.close()


def test_ragged_errors(env):
    torch, rexi = env
    r = rexi.RaggedPlan(31, 2, 256, 2000, OM, A, PB, precision="mixed")
    with pytest.raises(rexi.RexiError):
        r.set([(63, 64, 3600.0, 6.0, 10.0)])          # T > Tmax
    with pytest.raises(rexi.RexiError) as e:
        r.set([(31, 64, 3600.0, 6.0, 10.0)] * 3)      # more than max_inst
    assert e.value.code == rexi.REXI_EBUSY
    r.close()


INST_LARGE = [(127, 512, 3600.0)] * 4 + [(255, 512, 3600.0)] * 2 + [(63, 256, 3600.0), (191, 512, 1800.0),
                                                                      (255, 512, 2400.0)]


@pytest.mark.parametrize("prec,tol", [("fp64", None), ("mixed", 1e-8)])
def test_ragged_config_sizes_sampled(env, prec, tol):
    """Ensemble sizes (T63-T255, 256-512 poles) in one ragged launch, with four instances of one
    pole set (heavy tiles of two state pairs) and two of another (a lone pair), against the
    oracle on sampled zonal orders; the launch configuration of the ensemble benchmark."""
    torch, rexi = env
    r, off, states, u0, u1 = _run(env, prec, INST_LARGE)
    out = u1.cpu().numpy()
    for i in (0, 3, 4, 5, 6, 7, 8):
        t, n, dt = INST_LARGE[i]
        p0, Xc = contour(t, dt)
        z, w = oc.rexi_coefficients(n, p0, Xc)
        ms = [0, 1, t // 2, t]
        ref = orx.rexi_step(states[i], t, dt, OM, A, PB, z, w, m_list=ms)
        got = out[off[i]: off[i + 1]].reshape(3, -1)
        mask = np.zeros(got.shape[-1], bool)
        for m in ms:
            o = m * (2 * t + 3 - m) // 2
            mask[o: o + t + 1 - m] = True
        wgt = np.where(np.arange(mask.size) <= t, 1.0, 2.0)[mask]
        num = np.sqrt(np.sum(wgt * np.abs(got[:, mask] - ref[:, mask]) ** 2, axis=-1))
        den = np.sqrt(np.sum(wgt * np.abs(ref[:, mask]) ** 2, axis=-1))
        bound = tol if tol else max(1e-11, 8 * oc.amplification(z, w, orx.spectrum_bound(t, dt, OM, A, PB)) * 2.0 ** -53)
        assert np.all(num / den < bound), (i, num / den, bound)
    r.close()
