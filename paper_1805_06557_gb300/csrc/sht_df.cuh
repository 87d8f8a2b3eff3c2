// Double-float Legendre contractions for sh_plan precision SH_DF (internal to the library).
#pragma once
#include "sht_tc.cuh"

namespace rexi {

struct DfLegendre;

// P: the FP64 table [moff(m)+k][nh]; Pn: the next degree's row P_{T+1}^m [T+1][nh] (the split
// tables reach n = T + 1; no table of H is needed); w, wq: Gauss weights and w / (1 - mu^2)
// [nh] (device); pb: the plan's polar bounds (device arrays used by the kernels; must outlive
// the state)
int df_legendre_create(DfLegendre** out, const double* P, const double* Pn, const double* w, const double* wq, int T,
                       int nlat, int max_fields, const PolarBounds& pb, cudaStream_t stream);
// table entries (k < T + 1 - m, j < nh) the kernels stream per table: synthesis, analysis
void df_legendre_streamed(const DfLegendre* t, long long* syn, long long* ana);
void df_legendre_destroy(DfLegendre* t);
void df_legendre_set_prof(DfLegendre* t, StageProf* prof);

// Synthesis of nfs scalar spectra spec [nfs][nlm] -> Fourier coefficients F [nfs][T+1][nlat] and
// of nfv (psi, chi) pairs -> FU, FV (either count may be 0), one pass over the tables per group
// of fields.  nfs + 2 nfv <= 2 max_fields.
int df_leg_synth(DfLegendre* t, const double2* spec, double2* F, int nfs, const double2* psi, const double2* chi,
                 double2* FU, double2* FV, int nfv, double inv_a, cudaStream_t s);
// Analysis: divergence and curl of nfv vector fields (Fourier coefficients FA, FB) and the
// spectra of nfs scalar fields (F).
int df_leg_anal(DfLegendre* t, const double2* FA, const double2* FB, double2* dv, double2* cu, int nfv,
                const double2* F, double2* spec, int nfs, double inv_a, cudaStream_t s);

}  // namespace rexi
