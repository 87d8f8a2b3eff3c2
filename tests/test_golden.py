"""Stored fixtures under tests/golden/ against the FP64 oracle.

contour_sec4.txt holds the paper's own numbers: the circle of Sec. 4.2.2 through p0 = 10 and
p_{+-1} = +-30i (the parameters Sec. 5 starts from), radius 50 and centre -40.
rexi_step_T7_N128.txt is one REXI step on that contour, written by make_golden.py from the
oracle; replaying it guards the oracle against silent changes, and its distance to the exact
exponential bounds the REXI error of that contour."""
import os

import numpy as np

from oracle import coeffs as oc
from oracle import rexi as orx


def test_paper_contour_radius_and_centre(golden):
    k, _ = golden("contour_sec4.txt")
    R, mu = oc.contour(k["p0"], k["X"])
    assert (R, mu) == (k["R"], k["mu"])
    z, w = oc.rexi_coefficients(int(k["N"]), k["p0"], k["X"])
    assert len(z) == k["N"]
    assert np.max(np.abs(np.abs(z - k["mu"]) - k["R"])) < 1e-13 * k["R"]
    # no node lies to the right of p0, and the nodes nearest it sit at theta = +-pi / N
    assert np.max(z.real) < k["p0"]
    near = k["mu"] + k["R"] * np.exp(1j * np.pi / k["N"])
    assert np.min(np.abs(z - near)) < 1e-12 * k["R"]
    assert np.min(np.abs(z - np.conj(near))) < 1e-12 * k["R"]


def test_paper_contour_resolves_half_its_width(golden):
    """On the paper's contour, e^{iy} is reproduced to about 2e-11 for |y| <= 10 and to
    about 1e-6 at |y| = 20; near the edge points +-30i the quadrature loses its accuracy."""
    k, _ = golden("contour_sec4.txt")
    z, w = oc.rexi_coefficients(int(k["N"]), k["p0"], k["X"])
    assert oc.scalar_error(z, w, 10.0) < 1e-10
    assert oc.scalar_error(z, w, 20.0) < 1e-5
    assert oc.scalar_error(z, w, 28.0) > 1e-4


def test_oracle_replays_stored_step(golden_step):
    k, U0, U1 = golden_step("rexi_step_T7_N128.txt")
    T = int(k["T"])
    z, w = oc.rexi_coefficients(int(k["N"]), k["p0"], k["Xc"])
    args = (T, k["dt"], k["Omega"], k["radius"], k["Phibar"])
    got = orx.rexi_step(U0, *args, z, w)
    assert np.all(orx.rel_l2(got, U1, T) < 1e-13)
    dense = orx.rexi_step_dense(U0, *args, z, w)
    assert np.all(orx.rel_l2(dense, U1, T) < 1e-11)


def test_stored_step_near_exact_exponential(golden_step):
    """|dt lambda| <= X = 11.1 at T7 and dt = 21600 s.  dt L is skew-adjoint in the energy
    norm, so the REXI step differs from exp(dt L) U0 by at most the contour's scalar error
    over [-iX, iX] (4.5e-11) times |U0|; per field the measured gap is 0.9e-12 to 2.4e-12."""
    k, U0, U1 = golden_step("rexi_step_T7_N128.txt")
    T = int(k["T"])
    args = (T, k["dt"], k["Omega"], k["radius"], k["Phibar"])
    X = orx.spectrum_bound(*args)
    assert 10.0 < X < 11.5
    z, w = oc.rexi_coefficients(int(k["N"]), k["p0"], k["Xc"])
    exact = orx.exact_step(U0, *args)
    assert np.all(orx.rel_l2(U1, exact, T) < oc.scalar_error(z, w, X))


def test_stored_step_is_what_the_script_writes(tmp_path, golden_step):
    """The committed fixture is the output of tests/golden/make_golden.py (oracle only): same
    parameters, same input, and the same result up to the rounding of the host's LAPACK."""
    import subprocess
    import sys
    from conftest import GOLDEN
    subprocess.run([sys.executable, os.path.join(GOLDEN, "make_golden.py"), str(tmp_path)], check=True)
    k, U0, U1 = golden_step("rexi_step_T7_N128.txt")
    k2, V0, V1 = golden_step(str(tmp_path / "rexi_step_T7_N128.txt"))
    assert k == k2
    assert np.max(np.abs(V0 - U0)) <= 1e-15 * np.max(np.abs(U0))
    assert np.all(orx.rel_l2(V1, U1, int(k["T"])) < 1e-13)
