"""The vectorised numpy Thomas CPU baseline of bench.py (timed beside the oracle as the fair CPU
comparison) computes the same REXI step as the oracle's pivoted banded LU (Sec. 4.2, Eq. of the
REXI sum): small truncations, with Coriolis, both chain parities and the n = 0 row."""
import math
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from oracle import coeffs as oc  # noqa: E402
from oracle import rexi as orx  # noqa: E402
from paper_1805_06557_gb300 import synthetic as syn  # noqa: E402


@pytest.mark.parametrize("T,N,dt", [(3, 8, 3600.0), (7, 16, 1800.0), (15, 32, 3600.0), (21, 64, 14400.0)])
def test_thomas_baseline_matches_oracle(T, N, dt):
    X = orx.spectrum_bound(T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    p0, Xc = bench.contour(X)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    U0 = syn.gaussian_state(T, 11 + T)
    U0[:, 0] = [3.0, 1e-5, -2e-5]  # the n = 0 row: every field divided by each pole
    ref = orx.rexi_step(U0, T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR, z, w)
    got = bench.thomas_rexi_step(U0, T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR, z, w, chunk=5)
    amp = oc.amplification(z, w, X)
    err = orx.rel_l2(got, ref, T)
    assert np.all(err < max(1e-12, 64 * amp * 2.0 ** -53)), (err, amp)
