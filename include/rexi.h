/*
 * rexi.h -- C ABI of librexi.so, a GB300-native (sm_103a) implementation of the REXI time
 * step of the rotating shallow-water equations (Schreiber, Schaeffer & Loft,
 * arXiv 1805.06557).
 *
 * All entry points are plain C: pointers plus sizes, no C++ or framework types.  Every
 * function returns an int status, 0 on success and one of the negative REXI_E* codes on
 * failure; rexi_last_error() then returns a thread-local, human-readable message.  Device
 * buffers are owned by the caller; plans own their device tables and workspace.  Compute
 * entry points are asynchronous on the plan's CUDA stream and never allocate.
 *
 * Spectral layout (shared by every entry point): triangular truncation T,
 * nlm = (T+1)(T+2)/2 complex coefficients per field, m-major,
 *     idx(m, n) = m (2T + 3 - m) / 2 + (n - m),   0 <= m <= n <= T,
 * complex128 as interleaved (re, im) doubles.  Coefficients are of the orthonormal
 * spherical harmonics Y_n^m = Pt_n^m(mu) e^{i m lambda} (no Condon-Shortley phase), a real
 * field being  f = sum_n c_n^0 Y_n^0 + 2 Re sum_{m>=1} c_n^m Y_n^m.
 * A state has three fields in the order (Phi', zeta, delta): geopotential perturbation,
 * relative vorticity, divergence (paper Sec. 3).  A batch of states is [batch][3][nlm].
 */
#ifndef REXI_H
#define REXI_H

#ifdef __cplusplus
extern "C" {
#endif

#define REXI_OK 0
#define REXI_EINVAL (-1)   /* bad argument (size, pointer, aliasing, unsupported option) */
#define REXI_ENOMEM (-2)   /* device or host allocation failed (plan creation only)     */
#define REXI_ECUDA (-3)    /* a CUDA runtime call failed                                 */
#define REXI_ETIMEOUT (-4) /* a bounded device-side wait gave up                         */
#define REXI_EBUSY (-5)    /* resource busy (serving slots / memory budget exhausted)    */

#define REXI_FP64 0   /* every solve and sum in FP64                                         */
#define REXI_PART_NONE 0   /* the plan computes the whole step                                 */
#define REXI_PART_POLES 1  /* the plan sums only its rank's share of the poles                 */
#define REXI_PART_M 2      /* the plan computes only its rank's zonal orders, zeros elsewhere  */
#define REXI_MIXED 1  /* FP32 solves; poles with large weight refined (double-float residual) */
                      /* and summed in FP64; the others summed in FP32                        */

/* Thread-local description of the last error of the calling thread ("" if none). */
const char* rexi_last_error(void);

/*
 * rexi_coeffs -- Cauchy-contour REXI coefficients (paper Sec. 4.2.1-4.2.2,
 * Eq. cauchy_alpha / cauchy_beta).
 *
 * The circle passes through p0 (real, > 0) and +-i Xc, so R = (p0^2 + Xc^2)/(2 p0) and its
 * centre is mu = p0 - R; nodes theta_n = 2 pi (n - 1/2)/N, n = 1..N.  Outputs
 *     z_n = mu + R e^{i theta_n}            (= -alpha_n of the paper)
 *     w_n = (R e^{i theta_n} / N) psi_k(z_n) (= -beta_n of the paper)
 * so that  psi_k(x) ~ sum_n w_n / (z_n - x)  for x on [-i X, i X], X < Xc.  psi_0 = exp,
 * psi_1(z) = (e^z - 1)/z, psi_2(z) = (e^z - 1 - z)/z^2 (Sec. 4.3; series near 0).
 *   N       number of poles, >= 1
 *   p0, Xc  contour points; p0 > 0, Xc > 0
 *   phi     0, 1 or 2 (the psi_k above)
 *   z_out, w_out  caller-owned host arrays of 2N doubles (re, im interleaved)
 * Host only, FP64.  Errors: REXI_EINVAL.
 */
int rexi_coeffs(int N, double p0, double Xc, int phi, double* z_out, double* w_out);

/*
 * rexi_contour_select -- default contour for covering the spectrum [-iX, iX] with N poles:
 * Xc = margin X and p0 <= Xc picked from a small candidate set to minimise
 * max(scalar error, amplification * 2^-53) (the cancellation trade-off of Sec. 4.2.2).
 * Host only.  Outputs p0, Xc.  Errors: REXI_EINVAL.
 */
int rexi_contour_select(double X, int N, double* p0, double* Xc);

/*
 * rexi_select_poles -- the pole classes a plan would use, computed on the host (no GPU).
 *   precision    REXI_FP64 or REXI_MIXED
 *   z, w         N poles and weights, caller-owned host arrays of 2N doubles (re, im)
 *   X            half-width of the spectrum [-iX, iX] (rexi_spectrum_bound)
 *   heavy_tau, prune_tau   as in rexi_plan_desc (< 0 / 0 select the defaults)
 *   heavy_align  16 (plans with max_batch >= 4: state pairs on half-warps) or 32
 *   cls          caller-owned array of N ints: 1 heavy (FP32 solve refined with a double-float
 *                residual; every solved pole of an FP64 plan), 0 light, -1 pruned, 2 (mixed)
 *                solved and summed in FP64 (gain above the default fp64_tau of rexi_plan_desc)
 *   pruned_gain  optional: summed gain of the pruned poles (bound on the relative energy-norm
 *                change of the result, Sec. 4.2 contour sum with those terms left out)
 * The gain of pole n is |w_n| / dist(z_n, [-iX, iX]).  Errors: REXI_EINVAL (bad arguments or a
 * zero pole). */
int rexi_select_poles(int precision, int N, const double* z, const double* w, double X, double heavy_tau,
                      double prune_tau, int heavy_align, int* cls, double* pruned_gain);

/*
 * rexi_partition -- which poles or zonal orders rank `rank` of `size` owns (host only).
 *   REXI_PART_POLES: owned[n] for the N contour poles n = 0..N-1: the conjugate pair
 *     {k, N-1-k} (rexi_coeffs places the conjugate of node n at N-1-n; the middle node of an
 *     odd N is alone) goes to rank k mod size, so that the large-weight poles near both ends of
 *     the node list spread over the ranks.
 *   REXI_PART_M: owned[m] for m = 0..T: the orders pair as (m, T-m), chains of total length
 *     T + 2, and pair min(m, T-m) goes to rank min(m, T-m) mod size.
 * owned: caller-owned int array (N or T+1 entries), 1 owned, 0 not.  Errors: REXI_EINVAL.
 */
int rexi_partition(int mode, int T, int N, int rank, int size, int* owned);

/* X = dt (sqrt(phibar T (T+1)) / radius + 2 omega): bound on |dt lambda| over the spectrum
 * of dt L (gravity-wave frequency of degree T plus the largest Coriolis frequency). */
double rexi_spectrum_bound(int T, double dt, double omega, double radius, double phibar);

typedef struct rexi_plan rexi_plan;

typedef struct rexi_plan_desc {
  int T;              /* triangular truncation, 1 <= T <= 1023                           */
  int N;              /* number of poles, 1 <= N <= 8192                                 */
  double dt;          /* time step [s]                                                   */
  double omega;       /* rotation rate Omega [1/s]                                       */
  double radius;      /* sphere radius a [m]                                             */
  double phibar;      /* mean geopotential Phibar = g h0 [m^2/s^2]                       */
  double p0, Xc;      /* contour (used when z == NULL)                                   */
  const double* z;    /* optional host array, 2N doubles: poles z_n (= -alpha_n)         */
  const double* w;    /* optional host array, 2N doubles: weights w_n (= -beta_n)        */
  int precision;      /* REXI_FP64 or REXI_MIXED                                         */
  double heavy_tau;   /* REXI_MIXED: a pole whose gain |w_n| / dist(z_n, [-iX, iX])      */
                      /* exceeds heavy_tau is refined and summed in FP64; < 0: 1e-3      */
  int max_batch;      /* largest batch passed to rexi_step, >= 1                         */
  void* stream;       /* cudaStream_t the plan launches on (NULL: legacy default stream) */
  double prune_tau;   /* pole pruning: the poles of smallest gain |w_n| / dist(z_n, [-iX, iX]) */
                      /* (a bound on the energy-norm size of their term relative to U0, dt L */
                      /* being skew-adjoint in that norm) are left out while their summed    */
                      /* gain stays <= prune_tau, conjugate pairs together; 0: default    */
                      /* (REXI_MIXED 1e-10, REXI_FP64 none: every pole is solved); < 0: none */
                      /* REXI_MIXED then completes the last 32-pole light group with the    */
                      /* largest pruned poles (pairs whole), so fewer may be left out       */
  int part_mode;      /* work partition over part_size devices (paper Sec. 5.3-5.4: REXI     */
  int part_rank;      /* terms spread over MPI ranks, U0 broadcast, the sum reduced):        */
  int part_size;      /* REXI_PART_NONE (0), REXI_PART_POLES or REXI_PART_M; rexi_partition  */
                      /* says which poles / orders rank part_rank owns.  POLES: the plan's   */
                      /* pole set is its share of the N poles, pruned within prune_tau /     */
                      /* part_size; U1 holds the partial sum over those poles (Phi included). */
                      /* M: U1 holds the full result on the owned orders and 0 elsewhere.    */
                      /* Either way the element-wise sum of U1 over the ranks (one all-reduce */
                      /* of 3 nlm complex128 per state) is the whole step                    */
  double fp64_tau;    /* REXI_MIXED: poles whose gain exceeds fp64_tau (rounded up to whole   */
                      /* 32-pole groups with the next-largest gains) are solved and summed    */
                      /* in FP64, as by an FP64 plan: a refined FP32 solve and double-float   */
                      /* partial sums keep about 2^-48 of a partial sum, too little for the   */
                      /* cancellation of very large weights; <= 0: 5e4 (none at T255,         */
                      /* dt = 3600 s; the largest 64 at T511, dt = 7200 s)                    */
} rexi_plan_desc;

/*
 * rexi_plan_create -- build a plan for  U1 = sum_n w_n (z_n - dt L)^-1 U0  (paper Eq. rexi),
 * L = L_g + L_c the linear gravity + Coriolis operator (Sec. 3, the L_g and L_c columns of
 * the split).  In spectral space, per zonal order m, with eps_n = sqrt((n^2-m^2)/(4n^2-1)):
 *   dPhi_n/dt  = -Phibar delta_n
 *   dzeta_n/dt = i w_n zeta_n - 2 Omega [(n+1)/n eps_n delta_{n-1} + n/(n+1) eps_{n+1} delta_{n+1}]
 *   ddelta_n/dt= n(n+1)/a^2 Phi_n + i w_n delta_n
 *                + 2 Omega [(n+1)/n eps_n zeta_{n-1} + n/(n+1) eps_{n+1} zeta_{n+1}]
 * w_n = 2 Omega m / (n(n+1)); the n = 0 vorticity and divergence are left unchanged.
 * The Coriolis coupling makes each (pole, m) system banded in n (Sec. 5.3); the library
 * eliminates Phi and solves two tridiagonal parity chains per (pole, m).
 * Allocates device tables and workspace (FP64 plan: per-warp scratch for the elimination).
 * Errors: REXI_EINVAL, REXI_ENOMEM, REXI_ECUDA.
 */
int rexi_plan_create(const rexi_plan_desc* desc, rexi_plan** out);

/* Frees the plan and its device memory.  NULL is allowed.  Synchronises the plan stream. */
int rexi_plan_destroy(rexi_plan* plan);

/*
 * rexi_step -- one REXI linear step for `batch` independent states.
 *   U0  device pointer, [batch][3][nlm] complex128 (caller-owned, read only)
 *   U1  device pointer, [batch][3][nlm] complex128 (caller-owned, written)
 * U0 and U1 must not overlap (REXI_EINVAL).  1 <= batch <= max_batch.  Asynchronous on the
 * plan stream; allocates nothing; launches the pre-pass (mixed), the solve kernels and the
 * finalize kernel.  With conjugate pole pairs the result is the m >= 0 half of a real field.
 * Errors: REXI_EINVAL, REXI_ECUDA (launch failure).
 */
int rexi_step(rexi_plan* plan, const void* U0, void* U1, int batch);

/*
 * rexi_step_host -- rexi_step on HOST buffers, on the plan stream, then synchronises it.
 * FP64 plans, and any plan given pageable memory: U0 is copied to plan-owned device staging
 * memory, the step runs there and U1 is copied back.  Mixed plans given pinned (mapped)
 * buffers: the step's kernels read U0 and write U1 in host memory directly over the host link
 * (each is touched once), without staging copies.
 * U0/U1: host arrays of batch*3*nlm complex128 (pinned memory gives full bandwidth).
 * Errors: REXI_EINVAL, REXI_ECUDA.
 */
int rexi_step_host(rexi_plan* plan, const double* U0, double* U1, int batch);

/*
 * rexi_step_host_async -- rexi_step on HOST buffers, pipelined for a stream of steps: the call
 * enqueues the copy of U0 to one of two plan-owned device staging slots (on a copy stream), the
 * step (on the plan stream) and the copy of the result to U1 (on a second copy stream), and
 * returns without waiting.  Consecutive calls alternate the slots, so the copies of the steps
 * before and after run on the copy engines while a step's kernels run; each call's copies and
 * step are ordered by events.  U0 and U1 (batch*3*nlm complex128 each, as rexi_step_host) must
 * stay valid and unchanged (U0) or unread (U1) until rexi_sync returns; page-locked memory is
 * needed for the copies to overlap (pageable memory still gives the right result).  The first
 * call allocates the two slots (2 x 2 x batch_max x 3 x nlm complex128) and creates the streams.
 * Errors: REXI_EINVAL, REXI_ENOMEM, REXI_ECUDA.
 */
int rexi_step_host_async(rexi_plan* plan, const double* U0, double* U1, int batch);

/* Synchronises the plan stream (and the copy streams of rexi_step_host_async) and reports any
 * error raised by device work since the last call (REXI_ECUDA).  */
int rexi_sync(rexi_plan* plan);

/* Plan facts for benchmarking and tests. */
typedef struct rexi_plan_info {
  int T, N, nlm, precision;
  int n_heavy;            /* poles refined and summed in FP64 (mixed), N for FP64 plans  */
  int n_groups;           /* 32-pole groups (N rounded up to a multiple of 32)           */
  int n_tiles;            /* work tiles per state                                        */
  int q_slots;            /* pole ranges summed separately before the final sum          */
  int grid_fp64, grid_light, grid_heavy;   /* persistent grid sizes (blocks)            */
  long long workspace_bytes;               /* device memory owned by the plan           */
  double s0_re, s0_im;    /* sum_n w_n / z_n over the poles solved                       */
  double X;               /* covered half-width used for the heavy classification        */
  int n_pruned;           /* poles left out by pruning                                   */
  double pruned_gain;     /* their summed gain (bound on the relative energy-norm change) */
  int n_fp64;             /* REXI_MIXED: poles solved in FP64 (gain > fp64_tau)          */
} rexi_plan_info;

int rexi_plan_get_info(const rexi_plan* plan, rexi_plan_info* info);

/* Copies the plan's poles and weights (2*N doubles each: the solved poles in the plan's
 * internal order, then the pruned ones) and per-pole classes (N ints: 2 solved in FP64 (mixed
 * plans), 1 heavy, 0 light, -1 pruned) to host arrays; any pointer may be NULL. */
int rexi_plan_get_poles(const rexi_plan* plan, double* z, double* w, int* heavy);

/*
 * Gravity-only REXI plans (the lg_rexi_* method identifiers of Table 2: only L_g goes to REXI,
 * the Coriolis term L_c is left to the explicit part; Sec. 3 split, Sec. 5.3).  Without
 * Coriolis the operator couples neither degrees nor zonal orders; for degree n >= 1, with
 * q_n = n(n+1)/a^2,
 *     dPhi_n/dt = -Phibar delta_n,   dzeta_n/dt = 0,   ddelta_n/dt = q_n Phi_n,
 * so each REXI term (z_p - dt L_g)^-1 is a 2 x 2 solve on (Phi_n, delta_n) (determinant
 * z_p^2 + dt^2 Phibar q_n) and a division of zeta_n by z_p, and the pole sum
 *     M_n = sum_p w_p (z_p - dt L_g,n)^-1
 * is a 2 x 2 matrix on (Phi_n, delta_n) and the scalar sum_p w_p / z_p on zeta_n, the same for
 * every zonal order.  Degree 0 (a zero row of the operator) gets sum_p w_p / z_p on all three
 * fields.  Plan creation evaluates M_n on the device in FP64 (one thread per degree, poles in
 * order); rexi_lg_step applies it: one pass over the state.  When the pole set is closed under
 * conjugation (pole p and pole N-1-p conjugate, weights too, to 1e-13 relative, as rexi_coeffs
 * makes them), M_n is real up to rounding and only its real part is applied.
 */
typedef struct rexi_lg_plan rexi_lg_plan;

typedef struct rexi_lg_desc {
  int T;              /* triangular truncation, 1 <= T <= 1023                           */
  int N;              /* number of poles, 1 <= N <= 8192                                 */
  double dt;          /* time step [s]                                                   */
  double radius;      /* sphere radius a [m]                                             */
  double phibar;      /* mean geopotential Phibar [m^2/s^2]                              */
  double p0, Xc;      /* contour (used when z == NULL)                                   */
  const double* z;    /* optional host array, 2N doubles: poles z_p                      */
  const double* w;    /* optional host array, 2N doubles: weights w_p                    */
  int phi;            /* z == NULL: 0, 1, 2 for the psi_0, psi_1, psi_2 weights (rexi_coeffs) */
  double ident;       /* coefficient c0 of a polynomial part: the plan applies              */
                      /* c0 I + sum_p w_p (z_p - dt L_g)^-1 (0 for REXI; Crank-Nicolson of   */
                      /* L_g over dt is 4 (2 - dt L_g)^-1 - I: one pole z = 2, w = 4, c0 = -1) */
  int max_batch;      /* largest batch passed to rexi_lg_step, >= 1                      */
  void* stream;       /* cudaStream_t the plan launches on (NULL: legacy default stream) */
} rexi_lg_desc;

/* Allocates the per-degree table ((T+1) x 64 bytes) and computes it.
 * Errors: REXI_EINVAL, REXI_ENOMEM, REXI_ECUDA. */
int rexi_lg_create(const rexi_lg_desc* desc, rexi_lg_plan** out);
/* Frees the plan (NULL allowed).  Synchronises the plan stream. */
int rexi_lg_destroy(rexi_lg_plan* plan);
/*
 * U1 = sum_p w_p (z_p - dt L_g)^-1 U0 for `batch` states, [batch][3][nlm] complex128 device
 * arrays (caller-owned).  U0 == U1 (in place) is allowed; any other overlap is REXI_EINVAL.
 * 1 <= batch <= max_batch.  Asynchronous on the plan stream, no allocation, one kernel launch.
 * Errors: REXI_EINVAL, REXI_ECUDA.
 */
int rexi_lg_step(rexi_lg_plan* plan, const void* U0, void* U1, int batch);
/* Synchronises the plan stream; reports errors of device work since the last call. */
int rexi_lg_sync(rexi_lg_plan* plan);
/*
 * Copies the per-degree pole sums to a host array of (T+1) x 8 doubles:
 * per degree (M_PhiPhi, M_PhiDelta, M_DeltaPhi, M_ZetaZeta) as (re, im) pairs
 * (M_DeltaDelta = M_PhiPhi).  *real_only (may be NULL) is 1 if the step applies real parts.
 * Synchronous.  Errors: REXI_EINVAL, REXI_ECUDA.
 */
int rexi_lg_get_operator(const rexi_lg_plan* plan, double* M, int* real_only);

/*
 * Ragged plans -- one launch over instances of different truncation T, time step dt and pole
 * count N (uneven per-m chain lengths from many states; the ensemble and serving forms).
 * Each instance gets its own Cauchy pole set; the tiles of all instances are sorted by cost
 * and dealt to the same persistent kernels as rexi_step.  States are concatenated:
 * instance i occupies [3][nlm_i] complex128 at complex offset soff[i] (rexi_ragged_offsets).
 */
typedef struct rexi_ragged rexi_ragged;

typedef struct rexi_ragged_desc {
  int Tmax;            /* largest truncation of any instance, <= 1023                        */
  int max_inst;        /* largest number of instances per set                                */
  int max_poles;       /* capacity of the pole arena (sum of padded pole counts)             */
  long long max_elems; /* largest sum over instances of nlm_i                                */
  double omega, radius, phibar;
  int precision;       /* REXI_FP64 or REXI_MIXED                                            */
  double heavy_tau;    /* as in rexi_plan_desc                                               */
  void* stream;        /* cudaStream_t (graph capture needs a non-default stream)            */
  double prune_tau;    /* as in rexi_plan_desc, per instance pole set                        */
  double fp64_tau;     /* as in rexi_plan_desc                                               */
} rexi_ragged_desc;

typedef struct rexi_instance {
  int T, N;            /* truncation, poles                                                  */
  double dt;           /* time step [s]                                                      */
  double p0, Xc;       /* contour (rexi_coeffs)                                              */
  long long soff;      /* complex offset of the state in U0 / U1; -1: concatenate in order   */
                       /* (either every instance gives an offset or none; states must not    */
                       /* overlap)                                                           */
} rexi_instance;

/* Allocates tables (Tmax), pole arena, workspace.  Errors: REXI_EINVAL, REXI_ENOMEM, REXI_ECUDA. */
int rexi_ragged_create(const rexi_ragged_desc* desc, rexi_ragged** out);
int rexi_ragged_destroy(rexi_ragged* r);
/* Sets the instance list (host array).  Pole sets are generated on the host and cached by
 * (T, N, dt, p0, Xc); tiles and descriptors are rebuilt on the host and uploaded, with the new
 * pole sets, by asynchronous copies on the plan stream from pinned packets: they run after the
 * work already queued on that stream (a step in flight keeps its data), and the call does not
 * wait for the device except to grow a buffer.  A failed call leaves no instance set.
 * Errors: REXI_EINVAL (bad instance), REXI_EBUSY (capacity exceeded), REXI_ENOMEM, REXI_ECUDA. */
int rexi_ragged_set(rexi_ragged* r, int ninst, const rexi_instance* inst);
/* soff[0..ninst]: complex offsets of the states in the concatenated layout (soff[ninst] = total). */
int rexi_ragged_offsets(const rexi_ragged* r, long long* soff);
/* One REXI step of every instance: U1 = sum_n w_n (z_n - dt L)^-1 U0 per instance.
 * Asynchronous, no allocation; replays the captured graph if (U0, U1) match the capture. */
int rexi_ragged_step(rexi_ragged* r, const void* U0, void* U1);
/* Captures one step for fixed (U0, U1) into a CUDA graph (one graph launch per step). */
int rexi_ragged_capture(rexi_ragged* r, const void* U0, void* U1);
/* Autotuner: times tile densities {1, 2, 4, 8} tiles per resident warp on the current set,
 * keeps the fastest.  Synchronous; overwrites U1. */
int rexi_ragged_tune(rexi_ragged* r, const void* U0, void* U1, int reps, int* best_qmul, double* best_ms);
int rexi_ragged_sync(rexi_ragged* r);
int rexi_ragged_set_profiling(rexi_ragged* r, int enable);
int rexi_ragged_get_profile(rexi_ragged* r, double* ms, int* launches, int reset);

/*
 * Per-kernel timing.  When enabled, rexi_step records a CUDA event pair on the plan stream
 * around every kernel it launches and accumulates the elapsed times at the next
 * rexi_plan_get_profile call (which synchronises the stream).  Kernel ids: 0 pre-pass,
 * 1 FP64 solve, 2 light solve, 3 heavy solve, 4 finalize.  ms[i] receives the total time
 * and launches[i] the number of launches of kernel i since the last reset (reset = 1
 * clears them after reading).  Enabling adds event records between launches; disabled by
 * default.  Errors: REXI_EINVAL, REXI_ECUDA.
 */
#define REXI_NKERNELS 5
int rexi_plan_set_profiling(rexi_plan* plan, int enable);
int rexi_plan_get_profile(rexi_plan* plan, double* ms, int* launches, int reset);

/*
 * rexi_step_fp64_static -- the FP64 REXI step for callers that cannot allocate device
 * memory: code running inside a host framework that owns all device memory through its
 * own pool, loops that must never trigger the device-wide synchronisation of an
 * allocation, or deployments that fix every byte at load time.  The paper has no
 * counterpart; it is a service of this library.
 *
 * Computes the same  U1 = sum_n w_n (z_n - dt L)^-1 U0  as an FP64 plan built from
 * (p0, Xc), for one state, with the same kernels, but takes every table, the elimination
 * scratch and the partial sums from one fixed array of device memory that is part of the
 * library image (rexi_static_scratch_bytes(), about 18 MB; every GPU on which the library
 * is used keeps it until the process exits).  It calls no cudaMalloc / cudaFree and no
 * allocating routine.
 *   T <= 63, N <= 1024 (REXI_EINVAL beyond); U0, U1 device pointers of 3*nlm complex128,
 *   not overlapping; stream: cudaStream_t (NULL = legacy default stream).
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress) and sets the solve kernel's shared-memory limit, so the address stays
 * valid after cudaDeviceReset; the first call on a device also loads the library's module
 * there: make that first call before any stream capture.  Every call reuses the same array
 * and leaves the last call's contents in it
 * (everything a call reads is written by it first); calls that overlap on the GPU (two
 * streams, or two host threads) race on that array and must be serialised by the caller.
 * Asynchronous on `stream`.  Errors: REXI_EINVAL, REXI_ECUDA.
 */
int rexi_step_fp64_static(int T, int N, double dt, double omega, double radius, double phibar,
                          double p0, double Xc, const void* U0, void* U1, void* stream);

/* Size in bytes of the fixed device array used by rexi_step_fp64_static. */
long long rexi_static_scratch_bytes(void);

/*
 * rexi_alu_peaks -- measures the FP64 and FP32 FMA throughput of the current device
 * (TFLOP/s, an FMA counted as 2 flops) with two short probe kernels: 8 independent FMA
 * chains per thread, 16 blocks of 256 threads per SM, timed with CUDA events.  These are
 * the roofline denominators of the ALU-bound solve kernels.  Synchronous; allocates and
 * frees a small device buffer.  Errors: REXI_EINVAL, REXI_ECUDA.
 */
int rexi_alu_peaks(double* fp64_tflops, double* fp32_tflops);

#ifdef __cplusplus
}
#endif

#endif /* REXI_H */
