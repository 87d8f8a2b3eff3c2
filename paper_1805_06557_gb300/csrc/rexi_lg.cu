// Gravity-only REXI (the lg_rexi_* methods: L_g by REXI, Coriolis in the explicit part;
// paper Sec. 3 split of L into L_g and L_c, Sec. 5.3 diagonal solve, Eq. rexi).
//
// Without the Coriolis coupling the operator acts on each coefficient alone and depends on
// the degree n only, so the pole sum  M_n = sum_p w_p (z_p - dt L_g,n)^-1  collapses to a
// 2 x 2 matrix on (Phi_n, delta_n) plus a scalar on zeta_n.  A plan evaluates M_n once per
// degree on the device (FP64, poles summed in order); a step is one pass over the state in
// HBM.  With a conjugate-closed pole set M_n is real up to rounding and the step applies its
// real part: 10 FP64 instructions per coefficient triple instead of 20, which keeps the pass
// near the HBM roof on a part whose FP64 pipe issues about 2 FMAs per clock per SM.
#include <cmath>
#include <complex>
#include <vector>

#include "common.cuh"

using namespace rexi;

namespace {

// Per-degree pole sums (M_PP, M_PD, M_DP, M_ZZ); M_DD = M_PP.
struct LgM {
  double2 pp, pd, dp, zz;
};

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double s = 1.0 / fma(b.x, b.x, b.y * b.y);
  return make_double2(fma(a.x, b.x, a.y * b.y) * s, fma(a.y, b.x, -a.x * b.y) * s);
}

// One thread per degree n: S1 = sum w z / det, S0 = sum w / det, E = sum w / z with
// det = z^2 + dt^2 Phibar q_n; M_PP = S1, M_PD = -dt Phibar S0, M_DP = dt q_n S0, M_ZZ = E.
// Degree 0 (zero operator row): every field gets E.  A polynomial part c0 I is added to the
// diagonal (M_PP, M_DD, M_ZZ).
__global__ void k_lg_sums(const double2* __restrict__ z, const double2* __restrict__ w, int N, int T,
                          double dt, double phibar, double inv_a2, double ident, LgM* __restrict__ M) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n > T) return;
  const double q = double(n) * (n + 1) * inv_a2;
  const double c2 = dt * dt * phibar * q;
  double2 s1 = make_double2(0.0, 0.0), s0 = s1, e = s1;
  for (int p = 0; p < N; ++p) {
    const double2 zp = z[p], wp = w[p];
    const double2 det = make_double2(fma(zp.x, zp.x, -zp.y * zp.y) + c2, 2.0 * zp.x * zp.y);
    const double2 a = cdiv(wp, det);  // w / det
    s0 = cadd(s0, a);
    s1 = cadd(s1, cmul(a, zp));
    e = cadd(e, cdiv(wp, zp));
  }
  LgM r;
  if (n == 0) {
    r.pp = e;
    r.pd = r.dp = make_double2(0.0, 0.0);
  } else {
    r.pp = s1;
    r.pd = make_double2(-dt * phibar * s0.x, -dt * phibar * s0.y);
    r.dp = make_double2(dt * q * s0.x, dt * q * s0.y);
  }
  r.zz = e;
  r.pp.x += ident;  // polynomial part c0 I (M_DD = M_PP carries it too)
  r.zz.x += ident;
  M[n] = r;
}

// Real parts of M_n packed for the real path: (M_PP, M_PD, M_DP, M_ZZ).
__global__ void k_lg_pack_real(const LgM* __restrict__ M, D4* __restrict__ R, int T) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n > T) return;
  const LgM m = M[n];
  R[n] = D4{m.pp.x, m.pd.x, m.dp.x, m.zz.x};
}

// One thread per coefficient (state b, index i) in a grid-stride loop; reads its Phi, zeta,
// delta and writes the three results (in place is safe: nothing else reads them).
template <bool REAL>
__global__ void __launch_bounds__(256) k_lg_apply(const double2* U0, double2* U1, const LgM* __restrict__ M,
                                                  const D4* __restrict__ R, int T, int nlm, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / nlm;
    const int i = (int)(e - b * nlm);
    const int m = m_of(T, i);
    const int n = m + (i - moff(T, m));
    const size_t base = (size_t)b * 3 * nlm + i;
    const double2 bp = U0[base], bz = U0[base + nlm], bd = U0[base + 2 * (size_t)nlm];
    double2 op, oz, od;
    if (REAL) {
      const D4 r = R[n];
      op = make_double2(fma(r.x, bp.x, r.y * bd.x), fma(r.x, bp.y, r.y * bd.y));
      od = make_double2(fma(r.z, bp.x, r.x * bd.x), fma(r.z, bp.y, r.x * bd.y));
      oz = make_double2(r.w * bz.x, r.w * bz.y);
    } else {
      const LgM c = M[n];
      op = cfma(c.pd, bd, cmul(c.pp, bp));
      od = cfma(c.pp, bd, cmul(c.dp, bp));
      oz = cmul(c.zz, bz);
    }
    U1[base] = op;
    U1[base + nlm] = oz;
    U1[base + 2 * (size_t)nlm] = od;
  }
}

bool conj_closed(const std::vector<std::complex<double>>& z, const std::vector<std::complex<double>>& w) {
  const int N = (int)z.size();
  double zs = 0.0, ws = 0.0;
  for (int p = 0; p < N; ++p) {
    zs = std::max(zs, std::abs(z[p]));
    ws = std::max(ws, std::abs(w[p]));
  }
  for (int p = 0; p < N; ++p) {
    const int q = N - 1 - p;
    if (std::abs(z[q] - std::conj(z[p])) > 1e-13 * zs || std::abs(w[q] - std::conj(w[p])) > 1e-13 * ws)
      return false;
  }
  return true;
}

}  // namespace

struct rexi_lg_plan {
  rexi_lg_desc d{};
  int nlm = 0, nsm = 0, real_only = 0;
  cudaStream_t stream = nullptr;
  LgM* M = nullptr;
  D4* R = nullptr;
};

extern "C" int rexi_lg_destroy(rexi_lg_plan* p) {
  if (!p) return REXI_OK;
  cudaStreamSynchronize(p->stream);
  cudaFree(p->M);
  cudaFree(p->R);
  delete p;
  return REXI_OK;
}

extern "C" int rexi_lg_create(const rexi_lg_desc* desc, rexi_lg_plan** out) {
  if (!desc || !out) return fail(REXI_EINVAL, "rexi_lg_create: null argument");
  *out = nullptr;
  const rexi_lg_desc& d = *desc;
  if (d.T < 1 || d.T > 1023) return fail(REXI_EINVAL, "rexi_lg_create: T must be in [1, 1023] (got %d)", d.T);
  if (d.N < 1 || d.N > 8192) return fail(REXI_EINVAL, "rexi_lg_create: N must be in [1, 8192] (got %d)", d.N);
  if (!(d.dt > 0) || !(d.radius > 0) || !(d.phibar > 0) || !std::isfinite(d.ident))
    return fail(REXI_EINVAL, "rexi_lg_create: need dt > 0, radius > 0, phibar > 0, finite ident");
  if (d.max_batch < 1) return fail(REXI_EINVAL, "rexi_lg_create: max_batch must be >= 1");
  if ((d.z == nullptr) != (d.w == nullptr)) return fail(REXI_EINVAL, "rexi_lg_create: give both z and w or neither");
  if (!d.z && (!(d.p0 > 0) || !(d.Xc > 0) || d.phi < 0 || d.phi > 2))
    return fail(REXI_EINVAL, "rexi_lg_create: need p0 > 0, Xc > 0 and phi in {0, 1, 2}");
  std::vector<double> zz(2 * (size_t)d.N), ww(2 * (size_t)d.N);
  if (d.z) {
    for (int k = 0; k < 2 * d.N; ++k) {
      zz[k] = d.z[k];
      ww[k] = d.w[k];
    }
  } else {
    int rc = rexi_coeffs(d.N, d.p0, d.Xc, d.phi, zz.data(), ww.data());
    if (rc) return rc;
  }
  std::vector<std::complex<double>> zc(d.N), wc(d.N);
  for (int p = 0; p < d.N; ++p) {
    zc[p] = {zz[2 * p], zz[2 * p + 1]};
    wc[p] = {ww[2 * p], ww[2 * p + 1]};
    if (std::abs(zc[p]) == 0.0 || !std::isfinite(std::abs(zc[p])) || !std::isfinite(std::abs(wc[p])))
      return fail(REXI_EINVAL, "rexi_lg_create: pole %d is zero or not finite", p);
  }
  rexi_lg_plan* p = new rexi_lg_plan();
  p->d = d;
  p->d.z = p->d.w = nullptr;
  p->nlm = (d.T + 1) * (d.T + 2) / 2;
  p->stream = (cudaStream_t)d.stream;
  p->real_only = conj_closed(zc, wc) ? 1 : 0;
  auto bail = [&](int code) {
    rexi_lg_destroy(p);
    return code;
  };
  int dev = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev)))
    return bail(cuda_fail(e, "rexi_lg_create: device query"));
  double2* dz = nullptr;
  double2* dw = nullptr;
  if ((e = cudaMalloc(&p->M, sizeof(LgM) * (d.T + 1))) || (e = cudaMalloc(&p->R, sizeof(D4) * (d.T + 1))) ||
      (e = cudaMalloc(&dz, sizeof(double2) * d.N)) || (e = cudaMalloc(&dw, sizeof(double2) * d.N))) {
    cudaFree(dz);
    cudaFree(dw);
    cudaGetLastError();
    return bail(fail(REXI_ENOMEM, "rexi_lg_create: cudaMalloc failed: %s", cudaGetErrorString(e)));
  }
  if ((e = cudaMemcpy(dz, zz.data(), sizeof(double2) * d.N, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(dw, ww.data(), sizeof(double2) * d.N, cudaMemcpyHostToDevice))) {
    cudaFree(dz);
    cudaFree(dw);
    return bail(cuda_fail(e, "rexi_lg_create: cudaMemcpy"));
  }
  const int tb = 128, nb = (d.T + 1 + tb - 1) / tb;
  k_lg_sums<<<nb, tb, 0, p->stream>>>(dz, dw, d.N, d.T, d.dt, d.phibar, 1.0 / (d.radius * d.radius), d.ident,
                                      p->M);
  k_lg_pack_real<<<nb, tb, 0, p->stream>>>(p->M, p->R, d.T);
  e = cudaGetLastError();
  if (!e) e = cudaStreamSynchronize(p->stream);
  cudaFree(dz);
  cudaFree(dw);
  if (e) return bail(cuda_fail(e, "rexi_lg_create: pole sums"));
  *out = p;
  return REXI_OK;
}

extern "C" int rexi_lg_step(rexi_lg_plan* p, const void* U0, void* U1, int batch) {
  if (!p || !U0 || !U1) return fail(REXI_EINVAL, "rexi_lg_step: null argument");
  if (batch < 1 || batch > p->d.max_batch)
    return fail(REXI_EINVAL, "rexi_lg_step: batch %d outside [1, %d]", batch, p->d.max_batch);
  const size_t bytes = sizeof(double2) * 3 * (size_t)p->nlm * batch;
  const char* a = (const char*)U0;
  const char* b = (const char*)U1;
  if (a != b && a < b + bytes && b < a + bytes) return fail(REXI_EINVAL, "rexi_lg_step: U0 and U1 overlap");
  const long long total = (long long)p->nlm * batch;
  const int tb = 256;
  const long long need = (total + tb - 1) / tb;
  const int nb = (int)std::min<long long>(need, (long long)p->nsm * 8);
  if (p->real_only)
    k_lg_apply<true><<<nb, tb, 0, p->stream>>>((const double2*)U0, (double2*)U1, p->M, p->R, p->d.T, p->nlm, total);
  else
    k_lg_apply<false><<<nb, tb, 0, p->stream>>>((const double2*)U0, (double2*)U1, p->M, p->R, p->d.T, p->nlm, total);
  cudaError_t e = cudaGetLastError();
  return e ? cuda_fail(e, "rexi_lg_step") : REXI_OK;
}

extern "C" int rexi_lg_sync(rexi_lg_plan* p) {
  if (!p) return fail(REXI_EINVAL, "rexi_lg_sync: null plan");
  REXI_CUDA_TRY(cudaStreamSynchronize(p->stream));
  REXI_CUDA_TRY(cudaGetLastError());
  return REXI_OK;
}

extern "C" int rexi_lg_get_operator(const rexi_lg_plan* p, double* M, int* real_only) {
  if (!p || !M) return fail(REXI_EINVAL, "rexi_lg_get_operator: null argument");
  REXI_CUDA_TRY(cudaStreamSynchronize(p->stream));
  REXI_CUDA_TRY(cudaMemcpy(M, p->M, sizeof(LgM) * (p->d.T + 1), cudaMemcpyDeviceToHost));
  if (real_only) *real_only = p->real_only;
  return REXI_OK;
}
