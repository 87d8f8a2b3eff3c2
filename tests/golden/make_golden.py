"""Writes the stored expected values under tests/golden/ from the FP64 oracle alone.

    python tests/golden/make_golden.py [output directory, default: this directory]

rexi_step_T7_N128.txt: one REXI step (Eq. rexi with the Cauchy-contour poles of
Eq. cauchy_alpha / cauchy_beta) of the linear SWE operator at T7, on the contour that Sec. 5
starts from (p0 = 10, p_{+-1} = +-30i, N = 128), dt = 21600 s (|dt lambda| <= 11.1, inside
the well-resolved part of that contour).  U0 is the seeded synthetic Gaussian state; both U0
and the oracle's U1 are stored, so the fixture does not depend on the input generator.
Only the oracle and the seeded input generator are called here.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import coeffs as oc  # noqa: E402
from oracle import rexi as orx  # noqa: E402
from paper_1805_06557_gb300 import synthetic as syn  # noqa: E402

T, N, P0, XC, DT, SEED = 7, 128, 10.0, 30.0, 21600.0, 2018


def main(outdir=HERE):
    z, w = oc.rexi_coefficients(N, P0, XC)
    U0 = syn.gaussian_state(T, SEED)
    U1 = orx.rexi_step(U0, T, DT, syn.OMEGA, syn.RADIUS, syn.PHIBAR, z, w)
    lines = [
        "# One REXI step of the linear SWE operator (Eq. rexi, poles of Eq. cauchy_alpha and",
        "# cauchy_beta on the Sec. 5 contour p0 = 10, p_{+-1} = +-30i, N = 128), written by",
        "# make_golden.py from the FP64 oracle.  Layout: field (0 = Phi', 1 = zeta, 2 = delta),",
        "# m-major index idx(m, n) = m (2T + 3 - m) / 2 + (n - m), then re/im of U0 and of U1.",
        "T %d" % T, "N %d" % N, "p0 %r" % P0, "Xc %r" % XC, "dt %r" % DT,
        "Omega %r" % syn.OMEGA, "radius %r" % syn.RADIUS, "Phibar %r" % syn.PHIBAR,
    ]
    for f in range(3):
        for i in range(U0.shape[1]):
            lines.append("%d %d %.17g %.17g %.17g %.17g" % (f, i, U0[f, i].real, U0[f, i].imag,
                                                         U1[f, i].real, U1[f, i].imag))
    with open(os.path.join(outdir, "rexi_step_T7_N128.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else HERE)
