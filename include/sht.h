/*
 * sht.h -- spherical-harmonic transforms of librexi (paper Sec. 3.2: the pseudo-spectral
 * space discretisation whose transforms serve the nonlinear term N(U); the paper uses SHTns,
 * this is an independent GPU implementation).
 *
 * Grid: nlat Gauss-Legendre latitudes (mu = sin(latitude), north to south; nlat even) times
 * nlon equispaced longitudes lambda_k = 2 pi k / nlon, nlon > 2T.  Grid arrays are
 * [field][nlat][nlon] FP64, row-major.  Spectral arrays use the layout of rexi.h:
 * [field][nlm] complex128, m-major, orthonormal Y_n^m without Condon-Shortley phase,
 * f = sum_n c_n^0 Y_n^0 + 2 Re sum_{m>=1} c_n^m Y_n^m.
 * Every transform is asynchronous on the plan stream and does not allocate.  Status codes
 * and rexi_last_error() as in rexi.h.
 */
#ifndef SHT_H
#define SHT_H

#ifdef __cplusplus
extern "C" {
#endif

#define SH_FP64 0  /* Legendre contraction in FP64 on CUDA cores                           */
#define SH_TF32 1  /* Legendre contraction on tcgen05 tensor cores, TF32 inputs, FP32 sums    */
#define SH_BF16 2  /* Legendre contraction on tcgen05 tensor cores, BF16 inputs, FP32 sums    */
/* Split TF32 on tcgen05 tensor cores: every operand x is carried as x_hi + x_lo with
 * x_hi = tf32(x), x_lo = tf32(x - x_hi), and each product as a_hi b_lo + a_lo b_hi + a_hi b_hi
 * (three MMAs into one FP32 accumulator).  The operand unit is about 3 * 2^-22 instead of
 * TF32's 2^-11, so that the derivatives of N(U) (the Laplacian of the kinetic energy, the
 * divergence of the fluxes) keep a usable accuracy; table bytes are those of FP64 (hi and lo
 * words), still streamed through the tensor cores. */
#define SH_TF32X3 3
/* Double-float on the FP32 CUDA cores: tables, inputs and sums carried as pairs of FP32 words
 * (about 48 significand bits), every contraction a compensated dot product (TwoProduct by FMA,
 * Knuth's TwoSum), the longitude FFT in double-float arithmetic too (FP64 grids and Fourier
 * arrays at its ends).  Close to FP64 accuracy without the FP64 pipe, which
 * GB300 has little of (about 2 FP64 FMAs per clock and SM against 128 FP32 ones).  Tables take
 * twice the memory of SH_FP64 (the FP64 tables and two split layouts of P).  nlat <= 2132.
 * The words are FP32: spectra, grids and the intermediate sums must stay inside the FP32
 * exponent range, with room for the low word below the high one (magnitudes of about 1e-25 to
 * 1e30 keep full accuracy; SH_FP64 has no such limit). */
#define SH_DF 4

typedef struct sh_plan sh_plan;

typedef struct sh_plan_desc {
  int T;            /* triangular truncation, 1 <= T <= 1023                                */
  int nlat, nlon;   /* Gauss grid, nlat even and > T, nlon > 2T, nlon = 2^p 3^q              */
  double radius;    /* sphere radius a [m] (vector transforms)                              */
  int precision;    /* SH_FP64, SH_TF32, SH_BF16, SH_TF32X3 or SH_DF                        */
  int max_fields;   /* largest nfields passed to a transform; tensor-core precisions: <= 8,  */
                    /* the vector operands (8 max_fields columns x nlat/2 latitudes for      */
                    /* analysis, x T+1 degrees for synthesis) must fit in shared memory      */
                    /* (e.g. max_fields <= 4 at T = 1023, nlat = 1536, TF32)                 */
  void* stream;     /* cudaStream_t                                                         */
  int epilogue_wait_polls;  /* 0 (normal use).  For tests of the timeout path of the tensor-core */
                    /* precisions: n > 0 makes the GEMM's epilogue give up waiting for an    */
                    /* accumulator after n non-blocking polls (the copy and MMA roles still  */
                    /* drain everything they issued); that transform's results are invalid  */
                    /* and sh_plan_check then returns REXI_ETIMEOUT                          */
  double polar_threshold;  /* polar truncation of the Legendre sums (below): 0 = the default      */
                    /* SH_POLAR_THRESHOLD_DEFAULT, > 0 (and < 1e-3) = this threshold, < 0 = off */
} sh_plan_desc;

/* Polar truncation.  Pt_n^m and Ht_n^m carry the factor (1 - mu^2)^{m/2}: near the poles, and
 * for m large against n sin(theta), they are smaller than any fixed threshold, so that the
 * leading terms of the sums over degrees (synthesis, per latitude) and over latitudes
 * (analysis, per degree) contribute nothing at FP64 precision.  SHTns, the library the paper
 * computes its transforms with (Sec. 3.2), skips them ("polar optimisation"); so does this
 * plan: per zonal order m it finds, for each group of 32 latitudes, the first degree at which
 * |Pt| or |Ht| exceeds the threshold at one of them, and for each group of 32 degrees the
 * first such latitude, and its kernels start there.  Every skipped table entry is below the
 * threshold in magnitude, so a skipped sum changes a result by at most the threshold times
 * the sum of the magnitudes of the terms it meets (coefficients, or weighted Fourier
 * coefficients).  The default, 1e-19, is about a thousandth of the FP64 rounding unit of the
 * tables' O(1) entries: results equal the untruncated ones to rounding. */
#define SH_POLAR_THRESHOLD_DEFAULT 1e-19

/* Builds the Gauss grid (Newton iteration on P_nlat), the orthonormal associated Legendre
 * table Pt_n^m(mu_j) and Ht_n^m = (1 - mu^2) dPt_n^m/dmu for the northern half (the
 * southern half follows from Pt_n^m(-mu) = (-1)^{n-m} Pt_n^m(mu)), the FFT twiddles and a
 * Fourier-space workspace.  Errors: REXI_EINVAL, REXI_ENOMEM, REXI_ECUDA. */
int sh_plan_create(const sh_plan_desc* desc, sh_plan** out);
int sh_plan_destroy(sh_plan* plan);

/* Gauss nodes mu_j and weights w_j (all nlat, north to south) into host arrays. */
int sh_plan_get_grid(const sh_plan* plan, double* mu, double* w);

/* Scalar synthesis: grid = sum_n c^0 Y^0 + 2 Re sum_{m>=1} c^m Y^m  (Legendre per m, then a
 * complex-to-real FFT of length nlon).  spec: device [nfields][nlm] complex128; grid: device
 * [nfields][nlat][nlon] double. */
int sh_synthesis(sh_plan* plan, const void* spec, void* grid, int nfields);

/* Scalar analysis: c_n^m = sum_j w_j Pt_n^m(mu_j) (2 pi / nlon) sum_k f_jk e^{-i m lambda_k}. */
int sh_analysis(sh_plan* plan, const void* grid, void* spec, int nfields);

/* Velocity synthesis from stream function psi and velocity potential chi (paper Sec. 3:
 * V = k x grad psi + grad chi), returned as U = u cos(lat), V = v cos(lat):
 *   U = (1/a)[-(1-mu^2) dpsi/dmu + dchi/dlambda],  V = (1/a)[dpsi/dlambda + (1-mu^2) dchi/dmu]. */
int sh_synthesis_uv(sh_plan* plan, const void* psi, const void* chi, void* U, void* V,
                    int nfields);

/* Divergence and vertical curl of a vector field given as A = P_u cos(lat), B = P_v cos(lat)
 * on the grid, by integration by parts against conj(Y):
 *   div_n^m  = (1/a) sum_j w_j/(1-mu_j^2) [ i m A_m Pt_n^m - B_m Ht_n^m ]
 *   curl_n^m = (1/a) sum_j w_j/(1-mu_j^2) [ i m B_m Pt_n^m + A_m Ht_n^m ]. */
int sh_analysis_divcurl(sh_plan* plan, const void* A, const void* B, void* div, void* curl,
                        int nfields);

/* Scalar and vector synthesis in one pass (the transforms of the nonlinear term share
 * their inputs' zonal orders): nfields scalar spectra spec -> grid as sh_synthesis, and nvec
 * (psi, chi) pairs -> (U, V) as sh_synthesis_uv, with one longitude-FFT launch for all
 * 2 nvec + nfields grids.  The tensor-core precisions contract the scalar fields beside the
 * vector pairs' columns, so the associated Legendre table Pt is read once (Ht once) instead
 * of once per transform; the results equal those of the separate calls.  Needs nfields >= 1,
 * nvec >= 1 and nfields + 2 nvec <= 2 max_fields.  Errors: REXI_EINVAL, REXI_ECUDA. */
int sh_synthesis_mixed(sh_plan* plan, const void* spec, void* grid, int nfields, const void* psi,
                       const void* chi, void* U, void* V, int nvec);

/* Divergence and curl of nvec vector fields (A, B) as sh_analysis_divcurl, and the analysis
 * of nfields scalar grids as sh_analysis, in one pass: one longitude-FFT launch, and for the
 * tensor-core precisions one read of each table.  Same limits and errors as
 * sh_synthesis_mixed. */
int sh_analysis_mixed(sh_plan* plan, const void* A, const void* B, void* div, void* curl, int nvec,
                      const void* grid, void* spec, int nfields);

/* Table entries per table (Pt, and Ht for vector transforms), to count the Legendre work:
 * total = nlm x nlat/2 (degree, northern latitude) entries; needed_synth / needed_anal = the
 * entries from each latitude's (each degree's) first one above the polar threshold on, the
 * work of the truncated method; streamed_synth / streamed_anal = the entries this plan's
 * kernels stream (whole warps, or whole tensor-core tiles and chunks, from their group's
 * start; padding not counted); threshold = the threshold in use (0: truncation off, every
 * count equal to total).  Errors: REXI_EINVAL. */
typedef struct sh_table_use {
  long long total, needed_synth, needed_anal, streamed_synth, streamed_anal;
  double threshold;
} sh_table_use;
int sh_plan_get_table_use(const sh_plan* plan, sh_table_use* use);

/* Synchronises the plan stream; returns REXI_ETIMEOUT if a tensor-core kernel's bounded
 * wait on its copy / MMA barriers gave up since the plan was created (its results are then
 * invalid), REXI_ECUDA on a CUDA error, REXI_OK otherwise. */
int sh_plan_check(sh_plan* plan);

/*
 * Per-stage timing.  When enabled, every transform records a CUDA event pair on the plan
 * stream around each kernel it launches; sh_plan_get_profile synchronises the stream and
 * returns, per stage, the total milliseconds (ms[k]) and the number of launches
 * (launches[k]) since the last reset (reset = 1 clears them after reading).  Stages:
 * 0 FP64 Legendre contraction (SH_FP64), 1 double-float Legendre contraction with the split
 * of its inputs (SH_DF), 2 tcgen05 Legendre GEMM
 * (its B operands built and its FP64 results written inside the kernel), 3 unused,
 * 4 longitude FFT.  Arrays hold SH_NSTAGES entries; either may be NULL.  Disabled by
 * default.  Errors: REXI_EINVAL, REXI_ECUDA.
 */
#define SH_NSTAGES 5
int sh_plan_set_profiling(sh_plan* plan, int enable);
int sh_plan_get_profile(sh_plan* plan, double* ms, int* launches, int reset);

#ifdef __cplusplus
}
#endif

#endif /* SHT_H */
