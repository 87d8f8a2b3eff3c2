// Tensor-core (tcgen05) Legendre contractions for sh_plan precisions SH_TF32 / SH_BF16.
#pragma once
#include "common.cuh"

namespace rexi {

struct TcLegendre;

int tc_legendre_create(TcLegendre** out, const double* P, const double* H, const double* w,
                       const double* wq, int T, int nlat, int max_fields, bool bf16,
                       cudaStream_t stream);
void tc_legendre_destroy(TcLegendre* t);
int tc_leg_synth(TcLegendre* t, const double2* spec, double2* F, int nf, cudaStream_t s);
int tc_leg_anal(TcLegendre* t, const double2* F, double2* spec, int nf, cudaStream_t s);
int tc_leg_synth_uv(TcLegendre* t, const double2* psi, const double2* chi, double2* FU, double2* FV,
                    int nf, double inv_a, cudaStream_t s);
// reads the device flag set by a tensor-core kernel whose bounded wait gave up (0 = none)
int tc_legendre_error(TcLegendre* t, int* flag);
int tc_leg_anal_divcurl(TcLegendre* t, const double2* FA, const double2* FB, double2* dv,
                        double2* cu, int nf, double inv_a, cudaStream_t s);

}  // namespace rexi
