// Nonlinear shallow-water step (paper Sec. 3 Eq. 1-3, Sec. 4.4): N(U) on the Gauss grid and
// the Strang splittings around the REXI linear step.
#include <cmath>
#include <vector>

#include "../../include/sht.h"
#include "../../include/swe.h"
#include "common.cuh"
#include "sht_tc.cuh"

namespace rexi {
namespace {

// psi = lap^-1 zeta, chi = lap^-1 delta with lap Y_n = -n(n+1)/a^2 Y_n; n = 0 -> 0.
// ilap[n] = -a^2 / (n(n+1)) (0 for n = 0), formed on the host.
__global__ void k_inv_lap(const double2* __restrict__ U, double2* __restrict__ psi,
                          double2* __restrict__ chi, int T, int nlm, const double* __restrict__ ilap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlm) return;
  int m = 0;
  // zonal order of coefficient i (m-major): largest m with moff(m) <= i
  int lo = 0, hi = T;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (moff(T, mid) <= i) lo = mid;
    else hi = mid - 1;
  }
  m = lo;
  const int n = m + (i - moff(T, m));
  const double s = ilap[n];
  const double2 z = U[nlm + i], d = U[2 * nlm + i];
  psi[i] = make_double2(s * z.x, s * z.y);
  chi[i] = make_double2(s * d.x, s * d.y);
}

// grid products: A = (Phi U, zeta U), B = (Phi V, zeta V), KE = (U^2 + V^2) / (2 cos^2);
// block row blockIdx.y = latitude j, ikc[j] = 1 / (2 cos^2 of latitude j), formed on the host
__global__ void k_swe_products(const double* __restrict__ PZ, const double* __restrict__ Ug,
                               const double* __restrict__ Vg, const double* __restrict__ ikc,
                               double* __restrict__ A, double* __restrict__ B, double* __restrict__ KE,
                               int nlat, int nlon) {
  const int npt = nlat * nlon;
  const int j = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nlon) return;
  const int i = j * nlon + k;
  const double u = Ug[i], v = Vg[i], ph = PZ[i], ze = PZ[npt + i];
  A[i] = ph * u;
  A[npt + i] = ze * u;
  B[i] = ph * v;
  B[npt + i] = ze * v;
  KE[i] = (u * u + v * v) * ikc[j];
}

// out = base + tau * N,  N = (-div(Phi V), -div(zeta V), curl(zeta V) + n(n+1)/a^2 KE_s);
// the n = 0 vorticity and divergence tendencies are 0 (global means).  With a Coriolis table
// (the lg schemes) the tendency is N' = L_c U + N, L_c U evaluated spectrally from U:
//   zeta_n: i omega_n zeta_n - (cm_n delta_{n-1} + cp_n delta_{n+1})
//   delta_n: i omega_n delta_n + (cm_n zeta_{n-1} + cp_n zeta_{n+1})
__global__ void k_swe_combine(const double2* __restrict__ base, const double2* __restrict__ dv,
                              const double2* __restrict__ cu, const double2* __restrict__ kes,
                              const double2* __restrict__ U, const D4* __restrict__ ctab,
                              double2* __restrict__ out, double tau, int T, int nlm, double inv_a2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlm) return;
  int lo = 0, hi = T;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (moff(T, mid) <= i) lo = mid;
    else hi = mid - 1;
  }
  const int n = lo + (i - moff(T, lo));
  double2 nP = make_double2(-dv[i].x, -dv[i].y);
  double2 nZ = make_double2(-dv[nlm + i].x, -dv[nlm + i].y);
  const double l = double(n) * (n + 1) * inv_a2;
  double2 nD = make_double2(cu[nlm + i].x + l * kes[i].x, cu[nlm + i].y + l * kes[i].y);
  if (ctab) {
    const int m = lo;
    const D4 t = ctab[i];  // (omega, cm, cp, -)
    const double2* Z = U + nlm;
    const double2* D = U + 2 * nlm;
    const double2 zm = n > m ? Z[i - 1] : make_double2(0.0, 0.0), zp = n < T ? Z[i + 1] : make_double2(0.0, 0.0);
    const double2 dm = n > m ? D[i - 1] : make_double2(0.0, 0.0), dp = n < T ? D[i + 1] : make_double2(0.0, 0.0);
    const double2 z0 = Z[i], d0 = D[i];
    nZ.x += -t.x * z0.y - (t.y * dm.x + t.z * dp.x);
    nZ.y += t.x * z0.x - (t.y * dm.y + t.z * dp.y);
    nD.x += -t.x * d0.y + (t.y * zm.x + t.z * zp.x);
    nD.y += t.x * d0.x + (t.y * zm.y + t.z * zp.y);
  }
  if (i == 0) nZ = nD = make_double2(0.0, 0.0);
  if (tau == 0.0) {  // plain tendency
    out[i] = nP;
    out[nlm + i] = nZ;
    out[2 * nlm + i] = nD;
    return;
  }
  out[i] = make_double2(fma(tau, nP.x, base[i].x), fma(tau, nP.y, base[i].y));
  out[nlm + i] = make_double2(fma(tau, nZ.x, base[nlm + i].x), fma(tau, nZ.y, base[nlm + i].y));
  out[2 * nlm + i] = make_double2(fma(tau, nD.x, base[2 * nlm + i].x), fma(tau, nD.y, base[2 * nlm + i].y));
}

// out = U + s L U (the forward-Euler half of Crank-Nicolson), one thread per (m, n), with the
// per-(m, n) table (omega_n, cm_n, cp_n, n(n+1)/a^2) of the spectral operator L_m:
//   dPhi_n   = -Phibar delta_n
//   dzeta_n  = i omega_n zeta_n  - (cm_n delta_{n-1} + cp_n delta_{n+1})
//   ddelta_n = q_n Phi_n + i omega_n delta_n + (cm_n zeta_{n-1} + cp_n zeta_{n+1})
// (cm_n = 2 Omega (n+1)/n eps_n, cp_n = 2 Omega n/(n+1) eps_{n+1}; entries outside m <= n <= T
// are zero).
__global__ void k_apply_L(const double2* __restrict__ U, const D4* __restrict__ tab, double s,
                          double phibar, double2* __restrict__ out, int T, int nlm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlm) return;
  int lo = 0, hi = T;  // m = largest with moff(m) <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (moff(T, mid) <= i) lo = mid;
    else hi = mid - 1;
  }
  const int m = lo, n = m + (i - moff(T, m));
  const D4 t = tab[i];  // (omega, cm, cp, q)
  const double2* P = U;
  const double2* Z = U + nlm;
  const double2* D = U + 2 * nlm;
  const double2 zm = n > m ? Z[i - 1] : make_double2(0.0, 0.0), zp = n < T ? Z[i + 1] : make_double2(0.0, 0.0);
  const double2 dm = n > m ? D[i - 1] : make_double2(0.0, 0.0), dp = n < T ? D[i + 1] : make_double2(0.0, 0.0);
  const double2 z0 = Z[i], d0 = D[i], p0 = P[i];
  const double2 lP = make_double2(-phibar * d0.x, -phibar * d0.y);
  const double2 lZ = make_double2(-t.x * z0.y - (t.y * dm.x + t.z * dp.x), t.x * z0.x - (t.y * dm.y + t.z * dp.y));
  const double2 lD = make_double2(t.w * p0.x - t.x * d0.y + (t.y * zm.x + t.z * zp.x),
                                  t.w * p0.y + t.x * d0.x + (t.y * zm.y + t.z * zp.y));
  out[i] = make_double2(fma(s, lP.x, p0.x), fma(s, lP.y, p0.y));
  out[nlm + i] = make_double2(fma(s, lZ.x, z0.x), fma(s, lZ.y, z0.y));
  out[2 * nlm + i] = make_double2(fma(s, lD.x, d0.x), fma(s, lD.y, d0.y));
}

// U <- fac[n] U on all three fields: the exact factor exp(-tau nu (n(n+1)/a^2)^q) of the
// hyper-diffusion term, fac formed on the host per degree (fac[0] = 1)
__global__ void k_diffuse(double2* __restrict__ U, const double* __restrict__ fac, int T, int nlm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlm) return;
  int lo = 0, hi = T;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (moff(T, mid) <= i) lo = mid;
    else hi = mid - 1;
  }
  const double f = fac[lo + (i - moff(T, lo))];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double2 u = U[(size_t)k * nlm + i];
    U[(size_t)k * nlm + i] = make_double2(f * u.x, f * u.y);
  }
}

// out = a + s * b over n complex entries (ETD2RK combinations)
__global__ void k_axpy(const double2* __restrict__ a, const double2* __restrict__ b, double s,
                       double2* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = make_double2(fma(s, b[i].x, a[i].x), fma(s, b[i].y, a[i].y));
}

}  // namespace
}  // namespace rexi

using namespace rexi;

struct swe_plan {
  swe_plan_desc d{};
  int nlm = 0, npt = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;             // made here because the caller gave the legacy stream
  cudaGraphExec_t step_graph = nullptr;  // one step's kernels, replayed by swe_step
  const void* graph_state = nullptr;   // the state address the graph was captured for
  bool no_graph = false;               // the stream could not capture: steps run eagerly
  rexi_plan* rp = nullptr;             // REXI of exp (ver1: dt, ver0: dt/2, etdrk: dt)
  rexi_plan *rp1 = nullptr, *rp2 = nullptr;  // etdrk: REXI of psi_1, psi_2 (same poles)
  sh_plan* sp = nullptr;
  double2 *NU = nullptr, *A3 = nullptr;      // etdrk: N(U), A
  D4* Ltab = nullptr;                        // irk, lg: (omega, cm, cp, n(n+1)/a^2) per (m, n)
  rexi_lg_plan* lg[3] = {nullptr, nullptr, nullptr};  // lg: REXI of psi_0, psi_1, psi_2 of dt L_g
  bool is_lg = false;
  double2 *psi = nullptr, *chi = nullptr, *Um = nullptr, *Ut = nullptr, *dv = nullptr, *cu = nullptr,
          *kes = nullptr;
  double *PZ = nullptr, *Ug = nullptr, *Vg = nullptr, *A = nullptr, *B = nullptr, *KE = nullptr,
         *ikc = nullptr, *ilap = nullptr;
  double* dfac = nullptr;  // hyper-diffusion factor per degree over dt/2 (nullptr: none)
  StageProf prof;  // the step's own grid and spectral kernels (stage 0)
};

extern "C" int swe_plan_destroy(swe_plan* p) {
  if (!p) return REXI_OK;
  cudaStreamSynchronize(p->stream);
  if (p->step_graph) cudaGraphExecDestroy(p->step_graph);
  rexi_plan_destroy(p->rp);
  rexi_plan_destroy(p->rp1);
  rexi_plan_destroy(p->rp2);
  for (rexi_lg_plan* q : p->lg) rexi_lg_destroy(q);
  sh_plan_destroy(p->sp);
  p->prof.release();
  for (void* q : {(void*)p->psi, (void*)p->chi, (void*)p->Um, (void*)p->Ut, (void*)p->dv, (void*)p->cu,
                  (void*)p->kes, (void*)p->PZ, (void*)p->Ug, (void*)p->Vg, (void*)p->A, (void*)p->B,
                  (void*)p->KE, (void*)p->ikc, (void*)p->ilap, (void*)p->NU, (void*)p->A3, (void*)p->Ltab,
                  (void*)p->dfac})
    cudaFree(q);
  if (p->own_stream) cudaStreamDestroy(p->stream);
  delete p;
  return REXI_OK;
}

extern "C" int swe_plan_create(const swe_plan_desc* desc, swe_plan** out) {
  if (!desc || !out) return fail(REXI_EINVAL, "swe_plan_create: null argument");
  *out = nullptr;
  const swe_plan_desc& d = *desc;
  if (d.scheme < SWE_L_REXI_N_ERK_VER1 || d.scheme > SWE_LG_IRK_LC_N_ERK_VER0)
    return fail(REXI_EINVAL, "swe_plan_create: unknown scheme %d", d.scheme);
  if (d.nsub < 0 || d.nsub > 4096) return fail(REXI_EINVAL, "swe_plan_create: nsub = %d outside [0, 4096]", d.nsub);
  if (!(d.visc >= 0) || d.visc_order < 0 || d.visc_order > 8)
    return fail(REXI_EINVAL, "swe_plan_create: need visc >= 0 and visc_order in [0, 8]");
  swe_plan* p = new swe_plan();
  p->d = d;
  p->is_lg = d.scheme == SWE_LG_REXI_LC_N_ERK_VER1 || d.scheme == SWE_LG_REXI_LC_N_ETDRK ||
             d.scheme == SWE_LG_IRK_LC_N_ERK_VER0;
  p->stream = (cudaStream_t)d.stream;
  if (!p->stream) {  // the legacy stream cannot capture graphs; a blocking stream orders with it
    cudaError_t es = cudaStreamCreate(&p->stream);
    if (es) {
      delete p;
      return cuda_fail(es, "swe_plan_create: cudaStreamCreate");
    }
    p->own_stream = true;
  }
  p->prof.stream = p->stream;
  p->nlm = (d.T + 1) * (d.T + 2) / 2;
  p->npt = d.nlat * d.nlon;
  auto bail = [&](int code) {
    swe_plan_destroy(p);
    return code;
  };
  sh_plan_desc sd{};
  sd.T = d.T;
  sd.nlat = d.nlat;
  sd.nlon = d.nlon;
  sd.radius = d.radius;
  sd.precision = d.sh_precision;
  sd.max_fields = 3;  // Fourier work slots for the fused analysis: A, B (2 each) and KE
  sd.stream = p->stream;
  int rc = sh_plan_create(&sd, &p->sp);
  if (rc) return bail(rc);
  rexi_plan_desc rd{};
  rd.T = d.T;
  rd.N = d.N;
  rd.dt = d.scheme == SWE_L_REXI_N_ERK_VER0 ? 0.5 * d.dt : d.dt;
  rd.omega = d.omega;
  rd.radius = d.radius;
  rd.phibar = d.phibar;
  rd.p0 = d.p0;
  rd.Xc = d.Xc;
  rd.precision = d.rexi_precision;
  rd.heavy_tau = -1.0;
  rd.max_batch = 1;
  rd.stream = p->stream;
  double cn_z[2] = {2.0, 0.0}, cn_w[2] = {2.0, 0.0};  // irk: one pole z = 2, weight 2, FP64
  if (d.scheme == SWE_L_IRK_N_ERK_VER1) {
    rd.N = 1;
    rd.z = cn_z;
    rd.w = cn_w;
    rd.precision = REXI_FP64;
  }
  double cn_w4[2] = {4.0, 0.0};
  if (p->is_lg) {  // L_g by the diagonal REXI (FP64), psi_1 and psi_2 too for ETD2RK
    const int nk = d.scheme == SWE_LG_REXI_LC_N_ETDRK ? 3 : 1;
    for (int k = 0; k < nk; ++k) {
      rexi_lg_desc ld{};
      ld.T = d.T;
      ld.N = d.N;
      ld.dt = d.dt;
      ld.radius = d.radius;
      ld.phibar = d.phibar;
      ld.p0 = d.p0;
      ld.Xc = d.Xc;
      ld.phi = k;
      ld.max_batch = 1;
      ld.stream = p->stream;
      if (d.scheme == SWE_LG_IRK_LC_N_ERK_VER0) {  // CN_g over dt/2: 4 (2 - (dt/2) L_g)^-1 - I
        ld.N = 1;
        ld.dt = 0.5 * d.dt;
        ld.z = cn_z;
        ld.w = cn_w4;
        ld.ident = -1.0;
      }
      if ((rc = rexi_lg_create(&ld, &p->lg[k]))) return bail(rc);
    }
  } else {
    rc = rexi_plan_create(&rd, &p->rp);
    if (rc) return bail(rc);
  }
  if (d.scheme == SWE_L_IRK_N_ERK_VER1 || p->is_lg) {
    std::vector<D4> t(p->nlm);
    for (int m = 0; m <= d.T; ++m)
      for (int n = m; n <= d.T; ++n) {
        auto eps = [&](int nn) { return nn > m ? std::sqrt((double(nn) * nn - double(m) * m) / (4.0 * nn * nn - 1.0)) : 0.0; };
        const double nn1 = double(n) * (n + 1);
        const double om = n > 0 ? 2.0 * d.omega * m / nn1 : 0.0;
        const double cm = n > m && n - 1 > 0 ? 2.0 * d.omega * (n + 1.0) / n * eps(n) : 0.0;
        const double cp = n > 0 && n < d.T ? 2.0 * d.omega * n / (n + 1.0) * eps(n + 1) : 0.0;
        t[moff(d.T, m) + (n - m)] = D4{om, cm, cp, nn1 / (d.radius * d.radius)};
      }
    cudaError_t e2;
    if ((e2 = cudaMalloc(&p->Ltab, sizeof(D4) * p->nlm)) ||
        (e2 = cudaMemcpy(p->Ltab, t.data(), sizeof(D4) * p->nlm, cudaMemcpyHostToDevice))) {
      cudaGetLastError();
      return bail(fail(REXI_ENOMEM, "swe_plan_create: operator table: %s", cudaGetErrorString(e2)));
    }
  }
  if (d.scheme == SWE_L_REXI_N_ETDRK) {  // psi_1 and psi_2 weights of the same poles
    std::vector<double> zz(2 * (size_t)d.N), ww(2 * (size_t)d.N);
    for (int k = 1; k <= 2; ++k) {
      if ((rc = rexi_coeffs(d.N, d.p0, d.Xc, k, zz.data(), ww.data()))) return bail(rc);
      rexi_plan_desc rk = rd;
      rk.z = zz.data();
      rk.w = ww.data();
      if ((rc = rexi_plan_create(&rk, k == 1 ? &p->rp1 : &p->rp2))) return bail(rc);
    }
  }
  const size_t s3 = sizeof(double2) * 3 * (size_t)p->nlm, s1 = sizeof(double2) * (size_t)p->nlm;
  const size_t g1 = sizeof(double) * (size_t)p->npt;
  cudaError_t e;
  if ((e = cudaMalloc(&p->psi, s1)) || (e = cudaMalloc(&p->chi, s1)) || (e = cudaMalloc(&p->Um, s3)) ||
      (e = cudaMalloc(&p->Ut, s3)) || (e = cudaMalloc(&p->dv, 2 * s1)) || (e = cudaMalloc(&p->cu, 2 * s1)) ||
      (e = cudaMalloc(&p->kes, s1)) || (e = cudaMalloc(&p->PZ, 2 * g1)) || (e = cudaMalloc(&p->Ug, g1)) ||
      (e = cudaMalloc(&p->Vg, g1)) || (e = cudaMalloc(&p->A, 2 * g1)) || (e = cudaMalloc(&p->B, 2 * g1)) ||
      (e = cudaMalloc(&p->KE, g1)) || (e = cudaMalloc(&p->ikc, sizeof(double) * d.nlat)) ||
      (e = cudaMalloc(&p->ilap, sizeof(double) * (d.T + 1))) ||
      ((d.scheme == SWE_L_REXI_N_ETDRK || d.scheme == SWE_LG_REXI_LC_N_ETDRK) &&
       ((e = cudaMalloc(&p->NU, s3)) || (e = cudaMalloc(&p->A3, s3))))) {
    cudaGetLastError();
    return bail(fail(REXI_ENOMEM, "swe_plan_create: cudaMalloc failed: %s", cudaGetErrorString(e)));
  }
  std::vector<double> mu(d.nlat), ikc(d.nlat), ilap(d.T + 1, 0.0);
  sh_plan_get_grid(p->sp, mu.data(), nullptr);
  for (int j = 0; j < d.nlat; ++j) ikc[j] = 1.0 / (2.0 * ((1.0 - mu[j]) * (1.0 + mu[j])));
  for (int n = 1; n <= d.T; ++n) ilap[n] = -(d.radius * d.radius) / (double(n) * (n + 1));
  if ((e = cudaMemcpy(p->ikc, ikc.data(), sizeof(double) * d.nlat, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(p->ilap, ilap.data(), sizeof(double) * (d.T + 1), cudaMemcpyHostToDevice)))
    return bail(cuda_fail(e, "swe_plan_create: cudaMemcpy"));
  if (d.visc > 0) {  // exp(-(dt/2) nu (n(n+1)/a^2)^q) per degree
    const int q = d.visc_order > 0 ? d.visc_order : 2;
    std::vector<double> f(d.T + 1);
    for (int n = 0; n <= d.T; ++n)
      f[n] = std::exp(-0.5 * d.dt * d.visc * std::pow(double(n) * (n + 1) / (d.radius * d.radius), q));
    if ((e = cudaMalloc(&p->dfac, sizeof(double) * (d.T + 1))) ||
        (e = cudaMemcpy(p->dfac, f.data(), sizeof(double) * (d.T + 1), cudaMemcpyHostToDevice))) {
      cudaGetLastError();
      return bail(fail(REXI_ENOMEM, "swe_plan_create: diffusion table: %s", cudaGetErrorString(e)));
    }
  }
  *out = p;
  return REXI_OK;
}

// out = base + tau * N(U)   (tau = 0: out = N(U)); with ctab, N' = L_c U + N(U) instead
static int nonlinear_update(swe_plan* p, const double2* U, const double2* base, double tau, double2* out,
                            const D4* ctab = nullptr) {
  const int T = p->d.T, nlm = p->nlm;
  const int tb = 256;
  {
    const int ph = p->prof.begin(0);
    k_inv_lap<<<(nlm + tb - 1) / tb, tb, 0, p->stream>>>(U, p->psi, p->chi, T, nlm, p->ilap);
    p->prof.end(ph);
  }
  int rc;
  // Phi', zeta and U, V: one pass (one read of each Legendre table, one FFT launch)
  if ((rc = sh_synthesis_mixed(p->sp, U, p->PZ, 2, p->psi, p->chi, p->Ug, p->Vg, 1))) return rc;
  {
    const int ph = p->prof.begin(0);
    k_swe_products<<<dim3((p->d.nlon + tb - 1) / tb, p->d.nlat), tb, 0, p->stream>>>(p->PZ, p->Ug, p->Vg, p->ikc,
                                                                                  p->A, p->B, p->KE,
                                                                p->d.nlat, p->d.nlon);
    p->prof.end(ph);
  }
  // div / curl of A, B (two fields each) and KE: one pass, as the synthesis
  if ((rc = sh_analysis_mixed(p->sp, p->A, p->B, p->dv, p->cu, 2, p->KE, p->kes, 1))) return rc;
  {
    const int ph = p->prof.begin(0);
    k_swe_combine<<<(nlm + tb - 1) / tb, tb, 0, p->stream>>>(base, p->dv, p->cu, p->kes, U, ctab, out, tau, T,
                                                             nlm, 1.0 / (p->d.radius * p->d.radius));
    p->prof.end(ph);
  }
  cudaError_t e = cudaGetLastError();
  return e ? cuda_fail(e, "swe nonlinear kernels") : REXI_OK;
}

// U <- U + h N(U + h/2 N(U)), h = tau / nsub, nsub times   (explicit midpoint rule; N' = L_c + N
// for the lg schemes)
static int rk2_nonlinear(swe_plan* p, double2* U, double tau) {
  const D4* ctab = p->is_lg ? p->Ltab : nullptr;
  const int ns = p->d.nsub > 1 ? p->d.nsub : 1;
  const double h = tau / ns;
  for (int i = 0; i < ns; ++i) {
    int rc = nonlinear_update(p, U, U, 0.5 * h, p->Um, ctab);
    if (rc) return rc;
    if ((rc = nonlinear_update(p, p->Um, U, h, U, ctab))) return rc;
  }
  return REXI_OK;
}

// the gravity-only REXI step, timed as part of the REXI stage
static int lg_step(swe_plan* p, int k, const double2* in, double2* out) {
  const int ph = p->prof.begin(1);
  int rc = rexi_lg_step(p->lg[k], in, out, 1);
  p->prof.end(ph);
  return rc;
}

extern "C" int swe_substeps(int T, double tau, double umax, double radius, double courant) {
  if (T < 1 || !(tau >= 0) || !(umax >= 0) || !(radius > 0) || !(courant > 0))
    return fail(REXI_EINVAL, "swe_substeps: need T >= 1, tau >= 0, umax >= 0, radius > 0, courant > 0");
  const double c = tau * umax * std::sqrt(double(T) * (T + 1.0)) / (radius * courant);
  if (!(c <= 4096.0)) return 4096;
  const int n = (int)std::ceil(c);
  return n < 1 ? 1 : n;
}

extern "C" int swe_nonlinear(swe_plan* p, const void* state, void* tend) {
  if (!p || !state || !tend) return fail(REXI_EINVAL, "swe_nonlinear: null argument");
  if (state == tend) return fail(REXI_EINVAL, "swe_nonlinear: state and tendency alias");
  return nonlinear_update(p, (const double2*)state, nullptr, 0.0, (double2*)tend);
}

static int scheme_step(swe_plan* p, double2* U);

// the hyper-diffusion factor over dt/2 (no-op without diffusion)
static int diffuse_half(swe_plan* p, double2* U) {
  if (!p->dfac) return REXI_OK;
  const int ph = p->prof.begin(0);
  k_diffuse<<<(p->nlm + 255) / 256, 256, 0, p->stream>>>(U, p->dfac, p->d.T, p->nlm);
  p->prof.end(ph);
  REXI_CUDA_TRY(cudaGetLastError());
  return REXI_OK;
}

// One step on U: D^{dt/2} o (the scheme's step) o D^{dt/2} with D the exact hyper-diffusion
// flow (identity without diffusion); kernels and device copies on the plan stream only.
static int step_once(swe_plan* p, double2* U) {
  int rc;
  if ((rc = diffuse_half(p, U))) return rc;
  if ((rc = scheme_step(p, U))) return rc;
  return diffuse_half(p, U);
}

static int scheme_step(swe_plan* p, double2* U) {
  const size_t s3 = sizeof(double2) * 3 * (size_t)p->nlm;
  const double dt = p->d.dt;
  {
    int rc;
    if (p->d.scheme == SWE_L_REXI_N_ERK_VER1) {
      if ((rc = rk2_nonlinear(p, U, 0.5 * dt))) return rc;
      if ((rc = rexi_step(p->rp, U, p->Ut, 1))) return rc;
      REXI_CUDA_TRY(cudaMemcpyAsync(U, p->Ut, s3, cudaMemcpyDeviceToDevice, p->stream));
      if ((rc = rk2_nonlinear(p, U, 0.5 * dt))) return rc;
    } else if (p->d.scheme == SWE_L_REXI_N_ERK_VER0) {
      if ((rc = rexi_step(p->rp, U, p->Ut, 1))) return rc;
      if ((rc = rk2_nonlinear(p, p->Ut, dt))) return rc;
      if ((rc = rexi_step(p->rp, p->Ut, U, 1))) return rc;
    } else if (p->d.scheme == SWE_L_IRK_N_ERK_VER1) {
      if ((rc = rk2_nonlinear(p, U, 0.5 * dt))) return rc;
      k_apply_L<<<(p->nlm + 255) / 256, 256, 0, p->stream>>>(U, p->Ltab, 0.5 * dt, p->d.phibar, p->Ut, p->d.T,
                                                             p->nlm);
      REXI_CUDA_TRY(cudaGetLastError());
      if ((rc = rexi_step(p->rp, p->Ut, U, 1))) return rc;  // 2 (2 - dt L)^-1 (I + dt L / 2) U
      if ((rc = rk2_nonlinear(p, U, 0.5 * dt))) return rc;
    } else if (p->d.scheme == SWE_LG_REXI_LC_N_ERK_VER1) {
      if ((rc = rk2_nonlinear(p, U, 0.5 * dt))) return rc;
      if ((rc = lg_step(p, 0, U, U))) return rc;  // in place
      if ((rc = rk2_nonlinear(p, U, 0.5 * dt))) return rc;
    } else if (p->d.scheme == SWE_LG_IRK_LC_N_ERK_VER0) {
      if ((rc = lg_step(p, 0, U, U))) return rc;  // CN_g^{dt/2}, in place
      if ((rc = rk2_nonlinear(p, U, dt))) return rc;
      if ((rc = lg_step(p, 0, U, U))) return rc;
    } else if (p->d.scheme == SWE_LG_REXI_LC_N_ETDRK) {
      const int n3 = 3 * p->nlm, tb = 256, nb = (n3 + tb - 1) / tb;
      if ((rc = nonlinear_update(p, U, nullptr, 0.0, p->NU, p->Ltab))) return rc;  // N'(U)
      if ((rc = lg_step(p, 0, U, p->Ut))) return rc;                              // psi_0 U
      if ((rc = lg_step(p, 1, p->NU, p->Um))) return rc;                          // psi_1 N'(U)
      k_axpy<<<nb, tb, 0, p->stream>>>(p->Ut, p->Um, dt, p->A3, n3);               // A
      if ((rc = nonlinear_update(p, p->A3, nullptr, 0.0, p->Ut, p->Ltab))) return rc;  // N'(A)
      k_axpy<<<nb, tb, 0, p->stream>>>(p->Ut, p->NU, -1.0, p->Um, n3);             // N'(A) - N'(U)
      if ((rc = lg_step(p, 2, p->Um, p->Ut))) return rc;                          // psi_2 (...)
      k_axpy<<<nb, tb, 0, p->stream>>>(p->A3, p->Ut, dt, U, n3);                   // U+
      REXI_CUDA_TRY(cudaGetLastError());
    } else {  // ETD2RK
      const int n3 = 3 * p->nlm, tb = 256, nb = (n3 + tb - 1) / tb;
      if ((rc = nonlinear_update(p, U, nullptr, 0.0, p->NU))) return rc;          // N(U)
      if ((rc = rexi_step(p->rp, U, p->Ut, 1))) return rc;                       // psi_0 U
      if ((rc = rexi_step(p->rp1, p->NU, p->Um, 1))) return rc;                  // psi_1 N(U)
      k_axpy<<<nb, tb, 0, p->stream>>>(p->Ut, p->Um, dt, p->A3, n3);              // A
      if ((rc = nonlinear_update(p, p->A3, nullptr, 0.0, p->Ut))) return rc;      // N(A)
      k_axpy<<<nb, tb, 0, p->stream>>>(p->Ut, p->NU, -1.0, p->Um, n3);            // N(A) - N(U)
      if ((rc = rexi_step(p->rp2, p->Um, p->Ut, 1))) return rc;                  // psi_2 (...)
      k_axpy<<<nb, tb, 0, p->stream>>>(p->A3, p->Ut, dt, U, n3);                  // U+
      REXI_CUDA_TRY(cudaGetLastError());
    }
  }
  return REXI_OK;
}

// Records one step on U into p->step_graph (stream capture: nothing runs).  A stream or a call
// that cannot be captured leaves no graph and sets no_graph; steps then run eagerly.
static void capture_step(swe_plan* p, double2* U) {
  if (p->step_graph) {
    cudaGraphExecDestroy(p->step_graph);
    p->step_graph = nullptr;
    p->graph_state = nullptr;
  }
  if (cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    p->no_graph = true;
    return;
  }
  const int rc = step_once(p, U);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(p->stream, &g);
  cudaGraphExec_t x = nullptr;
  if (rc || e != cudaSuccess || !g || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
    cudaGetLastError();
    p->no_graph = true;
    x = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  p->step_graph = x;
  p->graph_state = x ? U : nullptr;
}

extern "C" int swe_step(swe_plan* p, void* state, int nsteps) {
  if (!p || !state) return fail(REXI_EINVAL, "swe_step: null argument");
  if (nsteps < 0) return fail(REXI_EINVAL, "swe_step: nsteps < 0");
  double2* U = (double2*)state;
  // a step is ~50 dependent kernels (most of them short at moderate truncations): replaying a
  // captured graph removes their per-launch host work and shortens the gaps between them.  The
  // first step of a new state runs eagerly, so that anything a sub-plan builds on first use
  // exists before the capture; profiling (host-collected event pairs) always runs eagerly.
  const bool graphs = !p->prof.on && !p->no_graph && nsteps >= 2;
  int s = 0;
  if (graphs && (!p->step_graph || p->graph_state != U)) {
    int rc = step_once(p, U);
    if (rc) return rc;
    ++s;
    capture_step(p, U);
  }
  for (; s < nsteps; ++s) {
    if (graphs && p->step_graph && p->graph_state == U) {
      REXI_CUDA_TRY(cudaGraphLaunch(p->step_graph, p->stream));
    } else {
      int rc = step_once(p, U);
      if (rc) return rc;
    }
  }
  return REXI_OK;
}

extern "C" int swe_plan_set_profiling(swe_plan* p, int enable) {
  if (!p) return fail(REXI_EINVAL, "swe_plan_set_profiling: null plan");
  p->prof.on = enable != 0;
  int rc = p->rp ? rexi_plan_set_profiling(p->rp, enable) : REXI_OK;
  for (rexi_plan* q : {p->rp1, p->rp2})
    if (!rc && q) rc = rexi_plan_set_profiling(q, enable);
  return rc ? rc : sh_plan_set_profiling(p->sp, enable);
}

extern "C" int swe_plan_get_profile(swe_plan* p, double* ms, int* launches, int reset) {
  if (!p) return fail(REXI_EINVAL, "swe_plan_get_profile: null plan");
  double rm[REXI_NKERNELS] = {}, sm[SH_NSTAGES];
  int rn[REXI_NKERNELS] = {}, sn[SH_NSTAGES];
  int rc = p->rp ? rexi_plan_get_profile(p->rp, rm, rn, reset) : REXI_OK;
  if (rc) return rc;
  for (rexi_plan* q : {p->rp1, p->rp2}) {
    if (!q) continue;
    double qm[REXI_NKERNELS];
    int qn[REXI_NKERNELS];
    if ((rc = rexi_plan_get_profile(q, qm, qn, reset))) return rc;
    for (int k = 0; k < REXI_NKERNELS; ++k) {
      rm[k] += qm[k];
      rn[k] += qn[k];
    }
  }
  if ((rc = sh_plan_get_profile(p->sp, sm, sn, reset))) return rc;
  REXI_CUDA_TRY(p->prof.collect());
  double out[SWE_NSTAGES] = {0, 0, 0, 0};
  int cnt[SWE_NSTAGES] = {0, 0, 0, 0};
  for (int k = 0; k < REXI_NKERNELS; ++k) {
    out[0] += rm[k];
    cnt[0] += rn[k];
  }
  for (int k = 0; k < 4; ++k) {
    out[1] += sm[k];
    cnt[1] += sn[k];
  }
  out[2] = sm[4];
  cnt[2] = sn[4];
  out[0] += p->prof.ms[1];  // gravity-only REXI launches (lg schemes)
  cnt[0] += p->prof.n[1];
  out[3] = p->prof.ms[0];
  cnt[3] = p->prof.n[0];
  if (reset)
    for (int k = 0; k < 2; ++k) {
      p->prof.ms[k] = 0.0;
      p->prof.n[k] = 0;
    }
  for (int k = 0; k < SWE_NSTAGES; ++k) {
    if (ms) ms[k] = out[k];
    if (launches) launches[k] = cnt[k];
  }
  return REXI_OK;
}
