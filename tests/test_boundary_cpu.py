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
