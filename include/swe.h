/*
 * swe.h -- nonlinear shallow-water time step of librexi (paper Sec. 3, Eq. 1-3 with the split
 * into L_g, L_c and N; Sec. 4.4 Strang splitting; Table 2 method identifiers).
 *
 * State: device [3][nlm] complex128 (Phi', zeta, delta), layout of rexi.h.
 * N(U) = ( -div(Phi' V), -div(zeta V), k.curl(zeta V) - lap(V.V/2) ) is evaluated
 * pseudo-spectrally: psi = lap^-1 zeta, chi = lap^-1 delta, V from (psi, chi) by the vector
 * synthesis of sht.h, products on the Gauss grid, divergence / curl / scalar analysis.
 * The linear part L = L_g + L_c (Coriolis inside) is integrated by a REXI plan (rexi.h), the
 * nonlinear part by 2nd-order explicit Runge-Kutta (midpoint rule).
 * Status codes and rexi_last_error() as in rexi.h.
 */
#ifndef SWE_H
#define SWE_H

#ifdef __cplusplus
extern "C" {
#endif

#define SWE_L_REXI_N_ERK_VER1 0 /* U+ = N^{dt/2} o L^{dt} o N^{dt/2} (U)  (Sec. 4.4, version 1) */
#define SWE_L_REXI_N_ERK_VER0 1 /* U+ = L^{dt/2} o N^{dt} o L^{dt/2} (U)  (Sec. 4.4, version 0) */
/* ETD2RK (Sec. 4.3, method l_rexi_n_etdrk): A = psi_0(dt L) U + dt psi_1(dt L) N(U),
 * U+ = A + dt psi_2(dt L) (N(A) - N(U)); psi_0 = exp, psi_1(K) = K^-1 (e^K - I),
 * psi_2(K) = K^-2 (e^K - I - K), each applied by REXI with the psi_k weights of the same poles
 * (contour p0, Xc for a step of dt). */
#define SWE_L_REXI_N_ETDRK 2
/* Crank-Nicolson for the linear part inside the Strang ver1 split (Sec. 4.1, irk, a = 1/2;
 * method l_irk_n_erk_ver1): U+ = N^{dt/2} o CN^{dt} o N^{dt/2} (U) with
 * CN^{dt} = (I - dt L / 2)^-1 (I + dt L / 2) = 2 (2 - dt L)^-1 (I + dt L / 2), i.e. the banded
 * solve of one pole z = 2 with weight 2 (FP64); p0 and Xc are not used. */
#define SWE_L_IRK_N_ERK_VER1 3
/* Coriolis in the explicit part (Table 2 lg_rexi_lc_n_*; Sec. 5.2 names lg_rexi_lc_n_erk_ver1 the
 * best REXI method by wallclock time to error): only the gravity operator L_g goes to REXI, by
 * the diagonal gravity-only plan of rexi.h (rexi_lg_*, FP64; rexi_precision is not used), and
 * the explicit part is N'(U) = L_c U + N(U), L_c evaluated spectrally:
 *   zeta_n: i w_n zeta_n - 2 Omega [(n+1)/n eps_n delta_{n-1} + n/(n+1) eps_{n+1} delta_{n+1}]
 *   delta_n: i w_n delta_n + 2 Omega [(n+1)/n eps_n zeta_{n-1} + n/(n+1) eps_{n+1} zeta_{n+1}]
 * LG_..._VER1: U+ = N'^{dt/2} o L_g^{dt} o N'^{dt/2} (U).
 * LG_..._ETDRK: ETD2RK with (L_g, N') in place of (L, N), psi_k(dt L_g) by the diagonal REXI. */
#define SWE_LG_REXI_LC_N_ERK_VER1 4
#define SWE_LG_REXI_LC_N_ETDRK 5
/* The paper's best implicit method (Sec. 5.2, lg_irk_lc_n_erk_ver0): Crank-Nicolson of L_g alone
 * inside the ver0 split, U+ = CN_g^{dt/2} o N'^{dt} o CN_g^{dt/2} (U), N' = L_c + N by RK2;
 * CN_g over a step h is (I - h L_g / 2)^-1 (I + h L_g / 2) = 4 (2 - h L_g)^-1 - I, a gravity-only
 * plan with one pole z = 2, weight 4 and ident = -1 (FP64); N, p0, Xc and rexi_precision are
 * not used. */
#define SWE_LG_IRK_LC_N_ERK_VER0 6

typedef struct swe_plan swe_plan;

typedef struct swe_plan_desc {
  int T, nlat, nlon;        /* truncation and Gauss grid (see sht.h)                       */
  double dt;                /* time step [s]                                                */
  double omega, radius, phibar;
  int N;                    /* REXI poles                                                   */
  double p0, Xc;            /* REXI contour for the linear sub-step (dt for ver1 and etdrk, dt/2 ver0) */
  int rexi_precision;       /* REXI_FP64 or REXI_MIXED                                      */
  int sh_precision;         /* SH_FP64, SH_TF32, SH_BF16, SH_TF32X3 or SH_DF                */
  int scheme;               /* one of the SWE_* scheme identifiers above                    */
  void* stream;             /* cudaStream_t; NULL (the legacy default stream): the plan makes */
                            /* its own blocking stream, implicitly ordered with the default  */
  int nsub;                 /* explicit sub-steps: every RK2 integration of the nonlinear part */
                            /* over an interval tau (the Strang halves of ver1 / irk / lg ver1,  */
                            /* the N step of ver0 / lg irk ver0) takes nsub midpoint steps of    */
                            /* tau / nsub; 0 or 1: one step (the paper's scheme); <= 4096.  The  */
                            /* linear part keeps its full step.  swe_substeps() gives the count */
                            /* for an advective Courant limit.  ETD2RK schemes ignore it.       */
  double visc;              /* hyper-diffusion coefficient nu >= 0 (0: none, the paper's       */
                            /* inviscid runs): the term (-1)^(q+1) nu lap^q on Phi', zeta,      */
                            /* delta, integrated exactly in spectral space (degree n decays by  */
                            /* exp(-t nu (n(n+1)/a^2)^q)) as half steps around every step of    */
                            /* the scheme: U+ = D^{dt/2} o step o D^{dt/2} (U)                  */
  int visc_order;           /* q in [1, 8]; 0: 2 (del^4)                                      */
} swe_plan_desc;

/*
 * swe_substeps -- explicit sub-steps for the nonlinear part over an interval tau (reading of
 * Sec. 2.3 and 4.4: the explicitly treated nonlinear terms limit the time step, the REXI
 * linear step does not): the smallest n >= 1 with
 *     (tau / n) * umax * sqrt(T (T+1)) / radius <= courant,
 * i.e. the advective phase change of the highest resolved degree under the largest wind speed
 * umax [m/s] stays within `courant` radians per midpoint step.  Host only.  Returns n, or
 * REXI_EINVAL for T < 1, tau < 0, umax < 0, radius <= 0 or courant <= 0 (n is capped at 4096).
 */
int swe_substeps(int T, double tau, double umax, double radius, double courant);

/* Creates the REXI plan(s: three for etdrk, gravity-only plans for lg), the SH plan and all
 * work buffers.
 * Errors: REXI_EINVAL, REXI_ENOMEM, REXI_ECUDA. */
int swe_plan_create(const swe_plan_desc* desc, swe_plan** out);
int swe_plan_destroy(swe_plan* plan);

/* Advances `state` (device, [3][nlm] complex128) in place by nsteps steps of the scheme.
 * Asynchronous on the plan stream.  With nsteps >= 2 and profiling off, the first step runs
 * eagerly and the kernels of one step are captured into a CUDA graph that replays the rest
 * (kept per state address: a call on another state recaptures; a stream that cannot capture
 * runs every step eagerly).  Errors: REXI_EINVAL, REXI_ECUDA. */
int swe_step(swe_plan* plan, void* state, int nsteps);

/* tendency = N(state) (device [3][nlm] complex128 each; no aliasing). */
int swe_nonlinear(swe_plan* plan, const void* state, void* tendency);

/*
 * Per-stage timing of swe_step / swe_nonlinear (CUDA events on the plan stream, off by
 * default; see rexi_plan_get_profile and sh_plan_get_profile).  Stages: 0 REXI linear step
 * kernels, 1 Legendre contractions (FP64 or tensor-core, with operand packing and
 * epilogue), 2 longitude FFTs, 3 grid products and spectral assembly of N(U).
 * swe_plan_get_profile synchronises the stream and returns total ms and launches per stage
 * since the last reset (reset = 1 clears them).  Errors: REXI_EINVAL, REXI_ECUDA.
 */
#define SWE_NSTAGES 4
int swe_plan_set_profiling(swe_plan* plan, int enable);
int swe_plan_get_profile(swe_plan* plan, double* ms, int* launches, int reset);

#ifdef __cplusplus
}
#endif

#endif /* SWE_H */
