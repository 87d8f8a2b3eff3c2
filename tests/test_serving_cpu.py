"""Host logic of the serving loop (paper_1805_06557_gb300/serving.py), without a GPU: the
first-fit state arena, the request contour (quantised spectrum bound, memoised contour search)
and request validation."""
import math
import types

import numpy as np
import pytest

from paper_1805_06557_gb300 import serving, synthetic as syn
from paper_1805_06557_gb300 import rexi


def test_arena_first_fit_against_an_occupancy_model():
    """Random allocations and releases against a per-element occupancy array: every block lies
    inside the arena and overlaps no live block, each allocation starts at the lowest free run
    long enough (first fit), a failed allocation means no such run exists, the free list stays
    sorted and coalesced, and releasing everything leaves one run of the whole arena."""
    rng = np.random.default_rng(3)
    cap = 4000
    a = serving._Arena(cap)
    used = np.zeros(cap, bool)
    live = []
    for _ in range(4000):
        if live and (rng.random() < 0.45 or len(live) > 40):
            s, n = live.pop(rng.integers(len(live)))
            a.release(s, n)
            assert used[s:s + n].all()
            used[s:s + n] = False
        else:
            n = int(rng.integers(1, 400))
            # the lowest start of a free run of length >= n in the model
            runs, i = [], 0
            while i < cap:
                if not used[i]:
                    j = i
                    while j < cap and not used[j]:
                        j += 1
                    runs.append((i, j - i))
                    i = j
                else:
                    i += 1
            expect = next((st for st, ln in runs if ln >= n), None)
            s = a.alloc(n)
            assert s == expect, (n, s, expect)
            if s is not None:
                assert 0 <= s and s + n <= cap and not used[s:s + n].any()
                used[s:s + n] = True
                live.append((s, n))
        # free list: sorted, non-adjacent (coalesced), exactly the free elements of the model
        fl = a.free
        assert all(fl[k][0] + fl[k][1] < fl[k + 1][0] for k in range(len(fl) - 1))
        free_model = np.ones(cap, bool)
        for st, ln in fl:
            free_model[st:st + ln] = False
        assert np.array_equal(free_model, used)
    for s, n in live:
        a.release(s, n)
    assert a.free == [(0, cap)]


@pytest.mark.parametrize("T,dt,N", [(63, 600.0, 256), (127, 1800.0, 512), (255, 3600.0, 512),
                                    (511, 7200.0, 2048), (511, 7000.0, 2048), (1, 100.0, 32)])
def test_request_contour(T, dt, N):
    """Below X = 20 the fixed rule (p0 = min(6, 1.6 X), Xc = 1.6 X); from X = 20 on the library's
    contour search at X rounded up to the 5 % grid 20 * 1.05^q >= X, memoised per (N, q), with
    p0 <= Xc and a covered half-width Xc at or above the grid point."""
    om, a, pb = syn.OMEGA, syn.RADIUS, syn.PHIBAR
    X = rexi.spectrum_bound(T, dt, om, a, pb)
    p0, Xc = serving.contour(T, dt, om, a, pb, N)
    assert 0 < p0 <= Xc
    if X < 20:
        assert p0 == pytest.approx(min(6.0, 1.6 * X)) and Xc == pytest.approx(1.6 * X)
        return
    q = math.ceil(math.log(X / 20.0) / math.log(1.05))
    Xq = 20.0 * 1.05 ** q
    assert X <= Xq < 1.05 * X * (1 + 1e-12)
    assert (p0, Xc) == rexi.contour_select(Xq, N)
    assert Xc >= Xq
    assert serving._CONTOURS[(N, q)] == (p0, Xc)
    # a time step on the same grid point reuses the memoised contour
    assert serving.contour(T, dt * (1 - 1e-9), om, a, pb, N) == (p0, Xc)


def test_request_validation():
    """The engine's admission checks, on a stand-in holding the engine's limits (the engine
    itself allocates its arena on the device): truncation range, pole count and time step,
    state larger than the arena, pole set larger than the pole arena, state shape."""
    eng = types.SimpleNamespace(Tmax=127, cap=3 * rexi.nlm(100), max_poles=1024)
    check = lambda r: serving.ServingEngine._validate(eng, r)
    ok = lambda T, N=256, dt=600.0: serving.Request(0, 0.0, T, dt, N, np.zeros((3, rexi.nlm(T)), complex))
    assert check(ok(63)) is None
    assert check(ok(100)) is None
    assert "outside" in check(ok(0))
    assert "outside" in check(ok(128))
    assert "exceeds the device memory budget" in check(ok(101))
    assert check(ok(63, N=0)) == "bad N or dt"
    assert check(ok(63, N=8193)) == "bad N or dt"
    assert check(ok(63, dt=0.0)) == "bad N or dt"
    assert "pole arena" in check(ok(63, N=1025))
    assert check(ok(63, N=1024)) is None
    r = ok(63)
    r.state = np.zeros((3, rexi.nlm(62)), complex)
    assert check(r) == "state shape mismatch"
    r.state = None
    assert check(r) == "state shape mismatch"
