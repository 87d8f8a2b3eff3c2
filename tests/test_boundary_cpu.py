"""The C ABI on the host: the library builds, loads and exports every function declared in
include/*.h; the host-only coefficient routines agree with the oracle.  No kernel runs."""
import math

import numpy as np
import pytest

from oracle import coeffs as ocoeffs


@pytest.fixture(scope="module")
def rexi():
    import __graft_entry__ as g
    g.build()
    from paper_1805_06557_gb300 import rexi as r
    return r


def test_exports_every_declared_symbol(rexi):
    names = rexi.exported_symbols()
    assert "rexi_step" in names and "rexi_coeffs" in names
    lib = rexi.library()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("N,p0,Xc,phi", [(8, 3.0, 5.0, 0), (256, 6.0, 18.8, 0), (512, 14.0, 64.0, 0),
                                         (128, 6.0, 18.8, 1), (128, 6.0, 18.8, 2)])
def test_coeffs_match_oracle(rexi, N, p0, Xc, phi):
    z, w = rexi.coeffs(N, p0, Xc, phi)
    zo, wo = ocoeffs.rexi_coefficients(N, p0, Xc, k=phi)
    assert np.max(np.abs(z - zo)) <= 1e-13 * np.max(np.abs(zo))
    assert np.max(np.abs(w - wo) / np.maximum(np.abs(wo), 1e-300)) < 1e-12


def test_coeffs_reject_bad_arguments(rexi):
    for args in [(0, 1.0, 1.0, 0), (8, -1.0, 1.0, 0), (8, 1.0, 0.0, 0), (8, 1.0, 1.0, 3)]:
        with pytest.raises(rexi.RexiError) as e:
            rexi.coeffs(*args)
        assert e.value.code == rexi.REXI_EINVAL


def test_spectrum_bound_and_contour_select(rexi):
    from paper_1805_06557_gb300 import synthetic as syn
    X = rexi.spectrum_bound(63, 3600.0, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    assert abs(X - 3600.0 * (math.sqrt(syn.PHIBAR * 63 * 64) / syn.RADIUS + 2 * syn.OMEGA)) < 1e-12 * X
    for X, N in [(0.4, 64), (11.8, 256), (45.7, 512)]:
        p0, Xc = rexi.contour_select(X, N)
        assert 0 < p0 <= Xc and Xc > X
        z, w = ocoeffs.rexi_coefficients(N, p0, Xc)
        es = ocoeffs.scalar_error(z, w, X, npts=2001)
        amp = ocoeffs.amplification(z, w, X)
        assert max(es, amp * 1.1e-16) < 1e-8


def _gains(z, w, X):
    return np.abs(w) / np.abs(z - 1j * np.clip(z.imag, -X, X))


def _pairs_share_class(z, cls):
    for c in (-1, 0, 1):
        s = z[cls == c]
        s = s[np.abs(s.imag) > 0]
        if not np.array_equal(np.sort_complex(s), np.sort_complex(np.conj(s))):
            return False
    return True


@pytest.mark.parametrize("align,nheavy", [(16, 80), (32, 96)])
def test_select_poles_mixed_default(rexi, align, nheavy):
    """Mixed classes at T255, N = 512, dt = 3600 s: heavy poles have the largest gains (every
    gain > 1e-3 among them, rounded up to the alignment), pruned poles the smallest with summed
    gain <= 1e-10, and the largest pruned poles fill the last 32-pole light group."""
    from oracle import rexi as orx
    from paper_1805_06557_gb300 import synthetic as syn
    X = orx.spectrum_bound(255, 3600.0, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    p0, Xc = rexi.contour_select(X, 512)
    z, w = ocoeffs.rexi_coefficients(512, p0, Xc)
    cls, pg = rexi.select_poles(z, w, X, "mixed", heavy_align=align)
    g = _gains(z, w, X)
    heavy, light, pruned = cls == 1, cls == 0, cls == -1
    assert heavy.sum() == nheavy and light.sum() == 32 and pruned.sum() == 512 - nheavy - 32
    assert np.all(g[g > 1e-3] >= g[light].max()) and np.sum(g > 1e-3) <= heavy.sum()
    assert g[heavy].min() >= g[light].max() >= g[light].min() >= g[pruned].max()
    assert g[pruned].sum() <= 1e-10 and abs(g[pruned].sum() - pg) <= 1e-12 * 1e-10
    # without the refill the 1e-10 budget would leave the last light group partly idle
    order = np.sort(g)
    assert np.sum(np.cumsum(order) <= 1e-10) > pruned.sum()
    assert _pairs_share_class(z, cls)


def test_select_poles_fp64_and_options(rexi):
    z, w = ocoeffs.rexi_coefficients(256, 6.0, 18.8)
    X = 11.0
    g = _gains(z, w, X)
    cls, pg = rexi.select_poles(z, w, X, "fp64")
    assert np.all(cls == 1) and pg == 0.0                      # FP64 solves every pole by default
    cls, pg = rexi.select_poles(z, w, X, "fp64", prune_tau=1e-12)
    assert 0 < np.sum(cls == -1) and g[cls == -1].sum() <= 1e-12 and not np.any(cls == 0)
    cls, _ = rexi.select_poles(z, w, X, "mixed", prune_tau=-1.0)
    assert not np.any(cls == -1)                               # pruning off
    cls, _ = rexi.select_poles(z, w, X, "mixed", heavy_tau=0.1, prune_tau=-1.0)
    assert np.all(g[cls == 1].min() >= g[cls == 0].max()) and np.sum(g > 0.1) <= np.sum(cls == 1)
    assert _pairs_share_class(z, cls)


def test_select_poles_reject_bad_arguments(rexi):
    z, w = ocoeffs.rexi_coefficients(16, 3.0, 5.0)
    for kw in (dict(heavy_align=8), dict(precision="fp64", X=-1.0)):
        args = dict(precision="mixed", X=4.0)
        args.update(kw)
        with pytest.raises(rexi.RexiError) as e:
            rexi.select_poles(z, w, args.pop("X"), **args)
        assert e.value.code == rexi.REXI_EINVAL
    z0 = z.copy()
    z0[3] = 0.0
    with pytest.raises(rexi.RexiError):
        rexi.select_poles(z0, w, 4.0)


def test_binding_rejects_wrong_tensors_before_the_call(rexi):
    """The binding checks size, dtype, contiguity and device of every state tensor before its
    address reaches a kernel (no GPU needed: every case fails on the host)."""
    import torch
    T = 15
    n = rexi.nlm(T)
    good_cpu = torch.zeros(3, n, dtype=torch.complex128)
    cases = [torch.zeros(3, n - 1, dtype=torch.complex128),          # too small
             torch.zeros(3, 2 * n, dtype=torch.complex128)[:, ::2],  # strided view
             torch.zeros(3, n, dtype=torch.complex64),               # wrong dtype
             good_cpu]                                               # right shape, on the host
    for bad in cases:
        with pytest.raises(ValueError):
            rexi.step_fp64_static(T, 64, 3600.0, 7.292e-5, 6.37122e6, 9.80616e4, 6.0, 10.0, bad, bad)
    with pytest.raises(ValueError, match="elements"):
        rexi.step_fp64_static(T, 64, 3600.0, 7.292e-5, 6.37122e6, 9.80616e4, 6.0, 10.0, cases[0], good_cpu)


def test_swe_substeps_rule(rexi):
    """Explicit sub-steps of the nonlinear part: the smallest n >= 1 with
    (tau / n) umax sqrt(T (T+1)) / a <= courant (include/swe.h)."""
    a = 6.37122e6
    c = 3600.0 * 40.0 * math.sqrt(511 * 512) / a
    assert rexi.swe_substeps(511, 3600.0, 40.0, a, 1.0) == math.ceil(c) == 12
    assert rexi.swe_substeps(511, 3600.0, 40.0, a, 0.5) == math.ceil(2 * c)
    assert rexi.swe_substeps(127, 900.0, 38.9, a, 1.0) == 1
    assert rexi.swe_substeps(63, 0.0, 40.0, a, 1.0) == 1
    # an exact multiple is not rounded up
    T = 3
    tau = 2.0 * a / math.sqrt(T * (T + 1.0))
    assert rexi.swe_substeps(T, tau, 1.0, a, 1.0) in (2, 3)
    assert rexi.swe_substeps(T, 4.0 * tau, 1.0, a, 8.0) in (1, 2)
    assert rexi.swe_substeps(1023, 1e9, 1e3, a, 1e-3) == 4096
    for args in [(0, 1.0, 1.0, a, 1.0), (5, -1.0, 1.0, a, 1.0), (5, 1.0, -1.0, a, 1.0),
                 (5, 1.0, 1.0, 0.0, 1.0), (5, 1.0, 1.0, a, 0.0)]:
        with pytest.raises(rexi.RexiError):
            rexi.swe_substeps(*args)


def test_mixed_transforms_reject_a_null_plan(rexi):
    """The one-pass scalar + vector transforms check their plan before anything else (no
    kernel runs)."""
    lib = rexi.library()
    assert lib.sh_synthesis_mixed(None, None, None, 1, None, None, None, None, 1) == rexi.REXI_EINVAL
    assert lib.sh_analysis_mixed(None, None, None, None, None, 1, None, None, 1) == rexi.REXI_EINVAL


def test_async_host_step_rejects_a_null_plan(rexi):
    """The pipelined host step checks its plan and buffers before it allocates or enqueues."""
    lib = rexi.library()
    assert lib.rexi_step_host_async(None, None, None, 1) == rexi.REXI_EINVAL


def test_sh_plan_rejects_bad_polar_threshold(rexi):
    """sh_plan_create checks the polar threshold before it touches the device (thresholds of
    1e-3 and above, or NaN, would truncate visibly); the table-use query checks its plan."""
    import ctypes
    lib = rexi.library()
    for thr in (1e-3, 0.5, float("nan")):
        d = rexi.ShDesc()
        d.T, d.nlat, d.nlon, d.radius, d.max_fields = 31, 48, 96, 6.37122e6, 1
        d.precision = rexi.SH_FP64
        d.polar_threshold = thr
        h = ctypes.c_void_p()
        assert lib.sh_plan_create(ctypes.byref(d), ctypes.byref(h)) == rexi.REXI_EINVAL
        assert not h.value
    assert lib.sh_plan_get_table_use(None, None) == rexi.REXI_EINVAL
