// Host-side REXI coefficients (paper Sec. 4.2.1-4.2.2, Eq. cauchy_alpha / cauchy_beta),
// contour selection and error reporting of librexi.
#include <complex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace rexi {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(REXI_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

using cplx = std::complex<double>;

// psi_0 = exp, psi_1 = (e^z - 1)/z, psi_2 = (e^z - 1 - z)/z^2; near 0 the limit is taken
// through the Taylor series psi_k(z) = sum_j z^j / (j + k)!  (L'Hopital, Sec. 4.3).
static cplx psi(int k, cplx z) {
  if (k == 0) return std::exp(z);
  if (std::abs(z) >= 0.5) {
    cplx em1 = std::exp(z) - 1.0;
    if (k == 1) return em1 / z;
    return (em1 - z) / (z * z);
  }
  cplx acc = 0.0, term = (k == 1) ? 1.0 : 0.5;
  for (int j = 0; j < 30; ++j) {
    acc += term;
    term *= z / double(j + k + 1);
  }
  return acc;
}

static void contour_coeffs(int N, double p0, double Xc, int k, std::vector<cplx>& z,
                           std::vector<cplx>& w) {
  const double R = (p0 * p0 + Xc * Xc) / (2.0 * p0);
  const double mu = p0 - R;
  z.resize(N);
  w.resize(N);
  // node N+1-n is the conjugate of node n (the circle is symmetric about the real axis and
  // psi_k(conj z) = conj psi_k(z)): evaluate n <= N/2 and mirror, so that the pairs are exact
  // and conjugate sums have no imaginary part from rounding; odd N: the middle node is real
  for (int n = 1; n <= N / 2; ++n) {
    const double th = 2.0 * M_PI * (n - 0.5) / N;
    const cplx ring = R * cplx(std::cos(th), std::sin(th));
    z[n - 1] = ring + mu;
    w[n - 1] = ring * psi(k, z[n - 1]) / double(N);
    z[N - n] = std::conj(z[n - 1]);
    w[N - n] = std::conj(w[n - 1]);
  }
  if (N % 2) {
    z[N / 2] = cplx(mu - R, 0.0);
    w[N / 2] = cplx((-R * psi(k, z[N / 2]) / double(N)).real(), 0.0);
  }
}

}  // namespace rexi

using namespace rexi;

extern "C" const char* rexi_last_error(void) { return g_err.c_str(); }

extern "C" int rexi_coeffs(int N, double p0, double Xc, int phi, double* z_out, double* w_out) {
  if (N < 1 || !(p0 > 0) || !(Xc > 0) || phi < 0 || phi > 2 || !z_out || !w_out)
    return fail(REXI_EINVAL, "rexi_coeffs: need N >= 1, p0 > 0, Xc > 0, phi in {0,1,2}, non-null outputs");
  std::vector<cplx> z, w;
  contour_coeffs(N, p0, Xc, phi, z, w);
  for (int n = 0; n < N; ++n) {
    z_out[2 * n] = z[n].real();
    z_out[2 * n + 1] = z[n].imag();
    w_out[2 * n] = w[n].real();
    w_out[2 * n + 1] = w[n].imag();
  }
  return REXI_OK;
}

extern "C" double rexi_spectrum_bound(int T, double dt, double omega, double radius, double phibar) {
  return dt * (std::sqrt(phibar * T * (T + 1.0)) / radius + 2.0 * omega);
}

// Score of a contour: max over x in [0, X] of |r(ix) - e^{ix}| and of the rounding growth
// sum_n |w_n| / |z_n - ix| times 2^-53 (conjugate symmetry covers [-X, 0]).  The points go
// from the band edge x = X inward, where both terms peak, and the evaluation stops once the
// partial maximum reaches `stop` (the best score so far): such a contour cannot win, so the
// search's choice is the same as with full evaluations.  The conjugate pairs of the node
// list are summed together (w/(z - ix) + conj(w)/(conj(z) - ix)).
static double contour_score(int N, double p0, double Xc, double X, double stop) {
  std::vector<cplx> z, w;
  contour_coeffs(N, p0, Xc, 0, z, w);
  const int npts = 201, half = N / 2;
  double score = 0;
  for (int j = npts - 1; j >= 0; --j) {
    const cplx x(0.0, X * j / (npts - 1));
    cplx r = 0.0;
    double a = 0.0;
    for (int n = 0; n < half; ++n) {
      const cplx t = w[n] / (z[n] - x), u = w[N - 1 - n] / (z[N - 1 - n] - x);
      r += t + u;
      a += std::abs(t) + std::abs(u);
    }
    if (N % 2) {
      const cplx t = w[half] / (z[half] - x);
      r += t;
      a += std::abs(t);
    }
    score = std::max(score, std::max(std::abs(r - std::exp(x)), a * 1.1102230246251565e-16));
    if (score >= stop) break;
  }
  return score;
}

extern "C" int rexi_contour_select(double X, int N, double* p0_out, double* Xc_out) {
  if (!(X > 0) || N < 2 || !p0_out || !Xc_out)
    return fail(REXI_EINVAL, "rexi_contour_select: need X > 0, N >= 2, non-null outputs");
  const double margins[] = {1.4, 1.6};
  const double p0s[] = {1, 2, 3, 4, 6, 8, 10, 12, 14, 16, 20, 24};
  double best = 1e300, bp = 0, bx = 0;
  for (double mg : margins) {
    const double Xc = mg * X;
    for (double p : p0s) {
      const double pp = std::min(p, Xc);  // the circle must not pass near the origin
      const double s = contour_score(N, pp, Xc, X, best);
      if (s < best) {
        best = s;
        bp = pp;
        bx = Xc;
      }
      if (p >= Xc) break;
    }
  }
  *p0_out = bp;
  *Xc_out = bx;
  return REXI_OK;
}
