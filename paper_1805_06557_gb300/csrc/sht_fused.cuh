// Fused spherical-harmonic transforms of the nonlinear shallow-water term (internal to the
// library; not part of the C ABI): the transforms of one N(U) evaluation share one longitude-FFT
// launch per direction, so that the launch covers several fields at once.
#pragma once
#include <cuda_runtime.h>

#include "../../include/sht.h"

// Synthesis of nf scalar spectra S [nf][nlm] to grids G [nf][nlat][nlon], and of nfv vector
// pairs (psi, chi) [nfv][nlm] to U, V [nfv][nlat][nlon] (as sh_synthesis and sh_synthesis_uv).
// Needs nf + 2 nfv <= 2 max_fields.  Errors: REXI_EINVAL, REXI_ECUDA, REXI_ETIMEOUT.
int sh_synth_fused(sh_plan* p, const double2* S, int nf, double* G, const double2* psi, const double2* chi, int nfv,
                   double* U, double* V);

// Analysis of nfv vector pairs (A, B) [nfv][nlat][nlon] to (div, curl) [nfv][nlm] and of nf
// scalar grids G [nf][nlat][nlon] to S [nf][nlm] (as sh_analysis_divcurl and sh_analysis).
// Needs nf + 2 nfv <= 2 max_fields.
int sh_anal_fused(sh_plan* p, const double* A, const double* B, int nfv, double2* dv, double2* cu, const double* G,
                  int nf, double2* S);
