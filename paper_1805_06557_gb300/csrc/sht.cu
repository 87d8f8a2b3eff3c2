// Spherical-harmonic transforms on a Gaussian grid (paper Sec. 3.2), FP64 path.
//
// Synthesis = Legendre contraction per zonal order m (G_m(mu_j) = sum_n c_n^m Pt_n^m(mu_j))
// followed by a complex-to-real FFT along each latitude; analysis is the reverse.  The
// Legendre tables hold the northern half only: Pt_n^m(-mu) = (-1)^{n-m} Pt_n^m(mu) and
// Ht_n^m(-mu) = -(-1)^{n-m} Ht_n^m(mu), so every contraction forms even and odd partial sums
// over the northern latitudes and combines them for both hemispheres.
//
// Layouts: Legendre tables [moff(m)+k][nh] (nh = nlat/2, latitude fastest: coalesced over
// threads that own latitudes); Fourier workspace [field][m][nlat]; grids [field][nlat][nlon].
// The FFT is a shared-memory Stockham autosort transform with radix-8, 4, 2 and 3 passes
// (register butterflies), two real latitude rows packed into one complex sequence.
#include <algorithm>
#include <cmath>
#include <complex>
#include <initializer_list>
#include <type_traits>
#include <tuple>
#include <vector>

#include "../../include/sht.h"
#include "common.cuh"
#include "cvt.cuh"
#include "df.cuh"
#include "sht_df.cuh"
#include "sht_tc.cuh"

namespace rexi {
namespace {

// ---- Legendre tables (scaled three-term recurrence, one thread per (m, latitude)) -------
__device__ __forceinline__ double eps_d(int n, int m) {
  if (n <= m) return 0.0;
  return sqrt((double(n) * n - double(m) * m) / (4.0 * n * n - 1.0));
}

// P, H: [moff(m)+k][nh]; Pn: the next degree's row P_{T+1}^m [m][nh] (the analysis of vector
// fields forms its H-sums from P-sums of the neighbouring degrees, k_divcurl_from_p)
__global__ void k_legendre_table(const double* __restrict__ mu, double* __restrict__ P,
                                 double* __restrict__ H, double* __restrict__ Pn, int T, int nh) {
  const int jh = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (jh >= nh) return;
  const double x = mu[jh];
  const double s = sqrt((1.0 - x) * (1.0 + x));
  const double TWO256 = 1.157920892373162e77, INV256 = 8.636168555094445e-78;  // 2^256, 2^-256
  double p = 0.28209479177387814;  // 1/sqrt(4 pi)
  int e = 0;
  for (int k = 1; k <= m; ++k) {
    p *= sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
    if (fabs(p) < INV256) {
      p *= TWO256;
      e -= 256;
    }
  }
  const size_t base = (size_t)moff(T, m) * nh + jh;
  // sliding window of converted values v_{n-1}, v_n, v_{n+1}
  double vprev = 0.0, vcur = ldexp(p, e);
  double pprev = 0.0, pcur = p;
  for (int n = m; n <= T; ++n) {
    // advance the recurrence to n + 1
    const double pnew = (x * pcur - eps_d(n, m) * pprev) / eps_d(n + 1, m);
    pprev = pcur;
    pcur = pnew;
    if (fabs(pcur) > TWO256) {
      pcur *= INV256;
      pprev *= INV256;
      e += 256;
    }
    const double vnext = ldexp(pcur, e);
    const size_t o = base + (size_t)(n - m) * nh;
    P[o] = vcur;
    H[o] = -n * eps_d(n + 1, m) * vnext + (n + 1.0) * eps_d(n, m) * vprev;
    vprev = vcur;
    vcur = vnext;
  }
  Pn[(size_t)m * nh + jh] = vcur;  // P_{T+1}^m
}

// Divergence and curl of nfv vector fields from the P-sums of their analysis:
// raw[(2 v) nlme + moff(T+1, m) + k] = sum_j wq_j Pt_n^m(mu_j) A_m(j) and raw[(2 v + 1) nlme + ...]
// the same of B (n = m + k = m .. T + 1; each degree with the hemispheric sums or differences
// of its own parity).  Since Ht_n = (n+1) eps_n Pt_{n-1} - n eps_{n+1} Pt_{n+1} (the relation
// the table kernel builds Ht with), the H-sums are those P-sums of the neighbouring degrees,
// which pair with the other parity's sums exactly as Ht_n does:
//   div_n = (i m PA_n - HB_n) / a,  curl_n = (i m PB_n + HA_n) / a,
//   HX_n = (n+1) eps_n PX_{n-1} - n eps_{n+1} PX_{n+1}   (PX_{m-1} does not enter: eps_m = 0).
__global__ void k_divcurl_from_p(const double2* __restrict__ raw, double2* __restrict__ dv,
                                 double2* __restrict__ cu, int T, int nlm, int nlme, double inv_a) {
  const int m = blockIdx.x, v = blockIdx.y, K = T + 1 - m;
  const double2* PA = raw + (size_t)(2 * v) * nlme + moff(T + 1, m);
  const double2* PB = PA + nlme;
  double2* od = dv + (size_t)v * nlm + moff(T, m);
  double2* oc = cu + (size_t)v * nlm + moff(T, m);
  const double fm = (double)m;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const int n = m + k;
    const double c0 = (n + 1.0) * eps_d(n, m), c1 = (double)n * eps_d(n + 1, m);
    const double2 a0 = PA[k], b0 = PB[k], ap = PA[k + 1], bp = PB[k + 1];
    const double2 am = k > 0 ? PA[k - 1] : make_double2(0.0, 0.0);
    const double2 bm = k > 0 ? PB[k - 1] : make_double2(0.0, 0.0);
    const double hax = c0 * am.x - c1 * ap.x, hay = c0 * am.y - c1 * ap.y;
    const double hbx = c0 * bm.x - c1 * bp.x, hby = c0 * bm.y - c1 * bp.y;
    od[k] = make_double2(inv_a * (-fm * a0.y - hbx), inv_a * (fm * a0.x - hby));
    oc[k] = make_double2(inv_a * (-fm * b0.y + hax), inv_a * (fm * b0.x + hay));
  }
}

// ---- polar bounds (see PolarBounds) ----------------------------------------------------
// One warp per (m, 32-latitude group): each lane scans the degrees of its latitude for the
// first entry of P or H above thr in magnitude; the warp keeps the smallest start and the
// number of entries from each latitude's own start on (the entries the method needs).
__global__ void k_polar_synth(const double* __restrict__ P, const double* __restrict__ H, int T, int nh, double thr,
                              int ngl, int* __restrict__ ks, int* __restrict__ need) {
  const int g = blockIdx.x, m = blockIdx.y, jh = 32 * g + threadIdx.x;
  const int K = T + 1 - m;
  int k = K;
  if (jh < nh) {
    const double* Pm = P + (size_t)moff(T, m) * nh + jh;
    const double* Hm = H + (size_t)moff(T, m) * nh + jh;
    for (k = 0; k < K; ++k)
      if (fabs(Pm[(size_t)k * nh]) > thr || fabs(Hm[(size_t)k * nh]) > thr) break;
  }
  const unsigned kmin = __reduce_min_sync(0xffffffffu, (unsigned)k);
  const unsigned n = __reduce_add_sync(0xffffffffu, jh < nh ? (unsigned)(K - k) : 0u);
  if (threadIdx.x == 0) {
    ks[m * ngl + g] = (int)kmin;
    need[m * ngl + g] = (int)n;
  }
}

// One warp per (m, 32-degree group): each lane scans the latitudes of its degree; degree index
// K (n = T + 1, whose P-sums the vector analysis uses) by its row of P alone.
__global__ void k_polar_anal(const double* __restrict__ P, const double* __restrict__ H, const double* __restrict__ Pn,
                             int T, int nh, double thr, int ngd, int* __restrict__ ja, int* __restrict__ need) {
  const int g = blockIdx.x, m = blockIdx.y, k = 32 * g + threadIdx.x;
  const int K = T + 1 - m;
  int j = nh;
  if (k < K) {
    const double* Pk = P + (size_t)(moff(T, m) + k) * nh;
    const double* Hk = H + (size_t)(moff(T, m) + k) * nh;
    for (j = 0; j < nh; ++j)
      if (fabs(Pk[j]) > thr || fabs(Hk[j]) > thr) break;
  } else if (k == K) {
    const double* Pk = Pn + (size_t)m * nh;
    for (j = 0; j < nh; ++j)
      if (fabs(Pk[j]) > thr) break;
  }
  const unsigned jmin = __reduce_min_sync(0xffffffffu, (unsigned)j);
  const unsigned n = __reduce_add_sync(0xffffffffu, k < K ? (unsigned)(nh - j) : 0u);
  if (threadIdx.x == 0) {
    ja[m * ngd + g] = (int)jmin;
    need[m * ngd + g] = (int)n;
  }
}

// ---- Legendre synthesis ------------------------------------------------------------
// One thread per (m, field, northern latitude): even- and odd-degree partial sums, combined
// for the latitude and its mirror.  Each warp starts at the first degree its 32 latitudes
// need (ks, rounded down to even so that the loop's parity pairing holds).  Latitude tiles
// run equator first (the last tile has the most work left after the polar truncation, and
// the first blocks launched finish last).
constexpr int LTH = 128;

// Scalar fields: coefficients spec [f][cstride] at moff(T, m), degrees n = m .. T (Pn null).
// With Pn given, the coefficients run to n = T + 1 at moff(T + 1, m) (the vector syntheses'
// u and v, below) and the row of n = T + 1 is Pn [m][nh].  Field f < nsplit goes to F, the
// others to F2 (field f - nsplit).
__global__ void __launch_bounds__(LTH) k_leg_synth(const double* __restrict__ P, const double* __restrict__ Pn,
                                                   const double2* __restrict__ spec, double2* __restrict__ F,
                                                   double2* __restrict__ F2, int nsplit, int T, int nlat,
                                                   int cstride, const int* __restrict__ ks, int ngl) {
  const int m = blockIdx.x, f = blockIdx.y;
  const int nh = nlat / 2;
  const int jh = (gridDim.z - 1 - blockIdx.z) * LTH + threadIdx.x;
  if (jh >= nh) return;
  const int K = T + 1 - m, base = moff(T, m);
  const double2* c = spec + (size_t)f * cstride + (Pn ? moff(T + 1, m) : base);
  const double* Pm = P + (size_t)base * nh + jh;
  double2 e = make_double2(0, 0), o = make_double2(0, 0);
  int k = __ldg(ks + m * ngl + (jh >> 5)) & ~1;
  for (; k + 1 < K; k += 2) {
    const double pe = Pm[(size_t)k * nh], po = Pm[(size_t)(k + 1) * nh];
    const double2 ce = c[k], co = c[k + 1];
    e.x = fma(pe, ce.x, e.x);
    e.y = fma(pe, ce.y, e.y);
    o.x = fma(po, co.x, o.x);
    o.y = fma(po, co.y, o.y);
  }
  if (k < K) {
    const double pe = Pm[(size_t)k * nh];
    e.x = fma(pe, c[k].x, e.x);
    e.y = fma(pe, c[k].y, e.y);
  }
  if (Pn) {  // n = T + 1, degree index K
    const double pn = Pn[(size_t)m * nh + jh];
    const double2 cn = c[K];
    double2& acc = (K & 1) ? o : e;
    acc.x = fma(pn, cn.x, acc.x);
    acc.y = fma(pn, cn.y, acc.y);
  }
  double2* out = (f < nsplit ? F + ((size_t)f * (T + 1) + m) * nlat : F2 + ((size_t)(f - nsplit) * (T + 1) + m) * nlat);
  out[jh] = make_double2(e.x + o.x, e.y + o.y);
  out[nlat - 1 - jh] = make_double2(e.x - o.x, e.y - o.y);
}

// Spectra of the velocity components of nf (psi, chi) pairs for n = m .. T + 1 (layout of
// moff(T + 1, m), [f][nlme]): U = (1/a)(-H psi + i m P chi) and V = (1/a)(i m P psi + H chi)
// with Ht_n = (n+1) eps_n Pt_{n-1} - n eps_{n+1} Pt_{n+1} become P-sums,
//   U = sum_p Pt_p u_p,  u_p = (-psi'_p + i m chi_p) / a,
//   V = sum_p Pt_p v_p,  v_p = (i m psi_p + chi'_p) / a,
//   x'_p = (p + 2) eps_{p+1} x_{p+1} - (p - 1) eps_p x_{p-1}   (x_{T+1} = x_{m-1} = 0),
// so a vector synthesis is two scalar ones over one table (the combinations in FP64, before any
// rounding of a transform).
__global__ void k_uv_coeffs(const double2* __restrict__ psi, const double2* __restrict__ chi, double2* __restrict__ u,
                            double2* __restrict__ v, int T, int nlm, int nlme, double inv_a) {
  const int m = blockIdx.x, f = blockIdx.y, K = T + 1 - m;
  const double2* ps = psi + (size_t)f * nlm + moff(T, m);
  const double2* ch = chi + (size_t)f * nlm + moff(T, m);
  double2* uo = u + (size_t)f * nlme + moff(T + 1, m);
  double2* vo = v + (size_t)f * nlme + moff(T + 1, m);
  const double fm = (double)m;
  const double2 z = make_double2(0.0, 0.0);
  for (int k = threadIdx.x; k <= K; k += blockDim.x) {
    const int p = m + k;
    const double a1 = (p + 2.0) * eps_d(p + 1, m), a0 = (p - 1.0) * eps_d(p, m);
    const double2 p0 = k < K ? ps[k] : z, c0 = k < K ? ch[k] : z;
    const double2 pp = k + 1 < K ? ps[k + 1] : z, cp = k + 1 < K ? ch[k + 1] : z;
    const double2 pm = k > 0 ? ps[k - 1] : z, cm = k > 0 ? ch[k - 1] : z;
    const double dpx = a1 * pp.x - a0 * pm.x, dpy = a1 * pp.y - a0 * pm.y;  // psi'
    const double dcx = a1 * cp.x - a0 * cm.x, dcy = a1 * cp.y - a0 * cm.y;  // chi'
    uo[k] = make_double2(inv_a * (-dpx - fm * c0.y), inv_a * (-dpy + fm * c0.x));
    vo[k] = make_double2(inv_a * (-fm * p0.y + dcx), inv_a * (fm * p0.x + dcy));
  }
}

// ---- Legendre analysis -------------------------------------------------------------
constexpr int ATH = 256;


__global__ void __launch_bounds__(ATH) k_leg_anal(const double* __restrict__ P,
                                                  const double* __restrict__ w,
                                                  const double2* __restrict__ F,
                                                  double2* __restrict__ spec, int T, int nlat, int nlm,
                                                  const int* __restrict__ ja, int ngd) {
  extern __shared__ double2 sm2[];
  const int m = blockIdx.x, f = blockIdx.y;
  const int nh = nlat / 2;
  double2* Se = sm2;
  double2* So = sm2 + nh;
  const double2* in = F + ((size_t)f * (T + 1) + m) * nlat;
  for (int j = threadIdx.x; j < nh; j += ATH) {
    const double2 a = in[j], b = in[nlat - 1 - j];
    const double wj = w[j];
    Se[j] = make_double2(wj * (a.x + b.x), wj * (a.y + b.y));
    So[j] = make_double2(wj * (a.x - b.x), wj * (a.y - b.y));
  }
  __syncthreads();
  // one thread per degree: it streams its own table row (32-byte pieces when nh % 4 == 0)
  // against the shared hemispheric sums; no cross-lane reduction.  Each warp (32 consecutive
  // degrees) starts at the first latitude its degrees need (ja).
  const int K = T + 1 - m, base = moff(T, m);
  for (int k = threadIdx.x; k < K; k += ATH) {
    const double* Pk = P + (size_t)(base + k) * nh;
    const double2* src = (k & 1) ? So : Se;
    const int jb = __ldg(ja + m * ngd + (k >> 5));
    double2 acc = make_double2(0, 0);
    if ((nh & 3) == 0) {
      const double2* P2 = reinterpret_cast<const double2*>(Pk);
      for (int j4 = jb >> 2; j4 < nh / 4; ++j4) {
        const double2 pa = __ldg(P2 + 2 * j4), pb = __ldg(P2 + 2 * j4 + 1);  // one 32-byte sector
        const double2 s0 = src[4 * j4], s1 = src[4 * j4 + 1], s2 = src[4 * j4 + 2], s3 = src[4 * j4 + 3];
        acc.x = fma(pa.x, s0.x, acc.x);
        acc.y = fma(pa.x, s0.y, acc.y);
        acc.x = fma(pa.y, s1.x, acc.x);
        acc.y = fma(pa.y, s1.y, acc.y);
        acc.x = fma(pb.x, s2.x, acc.x);
        acc.y = fma(pb.x, s2.y, acc.y);
        acc.x = fma(pb.y, s3.x, acc.x);
        acc.y = fma(pb.y, s3.y, acc.y);
      }
    } else {
      for (int j = jb; j < nh; ++j) {
        const double p = __ldg(Pk + j);
        acc.x = fma(p, src[j].x, acc.x);
        acc.y = fma(p, src[j].y, acc.y);
      }
    }
    spec[(size_t)f * nlm + base + k] = acc;
  }
}

// P-sums of a vector field's A and B for the degrees n = m .. T + 1 (raw layout of
// k_divcurl_from_p, which forms divergence and curl from them): one thread per degree, each
// sum with the hemispheric sums or differences of its own parity; the row of n = T + 1 is Pn.
// Two FP64 FMA pairs per table entry instead of four with the H table.
__global__ void __launch_bounds__(ATH) k_leg_anal_divcurl(const double* __restrict__ P,
                                                          const double* __restrict__ Pn,
                                                          const double* __restrict__ wq,
                                                          const double2* __restrict__ FA,
                                                          const double2* __restrict__ FB,
                                                          double2* __restrict__ raw, int T, int nlat,
                                                          int nlme, const int* __restrict__ ja, int ngd) {
  extern __shared__ double2 sm2[];
  const int m = blockIdx.x, f = blockIdx.y;
  const int nh = nlat / 2;
  const int K = T + 1 - m, k = blockIdx.z * ATH + threadIdx.x;  // degree index, to K (n = T + 1)
  if (blockIdx.z * ATH > K) return;  // uniform over the block
  double2* Ap = sm2;
  double2* Am = sm2 + nh;
  double2* Bp = sm2 + 2 * nh;
  double2* Bm = sm2 + 3 * nh;
  const double2* ia = FA + ((size_t)f * (T + 1) + m) * nlat;
  const double2* ib = FB + ((size_t)f * (T + 1) + m) * nlat;
  for (int j = threadIdx.x; j < nh; j += ATH) {
    const double2 an = ia[j], as = ia[nlat - 1 - j], bn = ib[j], bs = ib[nlat - 1 - j];
    const double q = wq[j];
    Ap[j] = make_double2(q * (an.x + as.x), q * (an.y + as.y));
    Am[j] = make_double2(q * (an.x - as.x), q * (an.y - as.y));
    Bp[j] = make_double2(q * (bn.x + bs.x), q * (bn.y + bs.y));
    Bm[j] = make_double2(q * (bn.x - bs.x), q * (bn.y - bs.y));
  }
  __syncthreads();
  // one thread per degree (see k_leg_anal); the blocks of one zonal order take its degrees ATH
  // at a time (blockIdx.z), so that no block carries more than ATH of them (one block per
  // order left the m = 0 block with two rounds of degrees, the others with one: T511
  // analysis_divcurl 0.479 ms that way, 0.380 ms tiled; the scalar analysis, launched with
  // more fields per order, stays one block per order)
  const int base = moff(T, m);
  double2* oA = raw + (size_t)(2 * f) * nlme + moff(T + 1, m);
  double2* oB = oA + nlme;
  if (k <= K) {
    const double* Pk = k < K ? P + (size_t)(base + k) * nh : Pn + (size_t)m * nh;
    const bool odd = k & 1;
    const int jb = __ldg(ja + m * ngd + (k >> 5));
    // P terms pair with (north + s south), s = (-1)^k
    const double2* AP = odd ? Am : Ap;
    const double2* BP = odd ? Bm : Bp;
    double2 sPA = make_double2(0, 0), sPB = sPA;
    auto step = [&](double p, int j) {
      const double2 ap = AP[j], bp = BP[j];
      sPA.x = fma(p, ap.x, sPA.x);
      sPA.y = fma(p, ap.y, sPA.y);
      sPB.x = fma(p, bp.x, sPB.x);
      sPB.y = fma(p, bp.y, sPB.y);
    };
    if ((nh & 3) == 0) {
      const double2* P2 = reinterpret_cast<const double2*>(Pk);
      for (int j4 = jb >> 2; j4 < nh / 4; ++j4) {
        const double2 pa = __ldg(P2 + 2 * j4), pb = __ldg(P2 + 2 * j4 + 1);
        step(pa.x, 4 * j4);
        step(pa.y, 4 * j4 + 1);
        step(pb.x, 4 * j4 + 2);
        step(pb.y, 4 * j4 + 3);
      }
    } else {
      for (int j = jb; j < nh; ++j) step(__ldg(Pk + j), j);
    }
    oA[k] = sPA;
    oB[k] = sPB;
  }
}

// ---- longitude FFT (Stockham autosort, radix 8, 4, 2 and 3, shared memory) -----------------
// Templated on the arithmetic type: FP64 for SH_FP64 plans, FP32 for the tensor-core plans
// (whose Legendre stage already rounds to TF32 / BF16), double-float for SH_DF plans (FP32
// pipe, about 48 bits); grids and Fourier arrays stay FP64.
struct FftPlan {
  int n, nrad;
  int rad[24];
  unsigned magic[24];  // ceil(2^32 / Ns) of each pass: j / Ns = umulhi(j, magic) for j < n
  int twoff[24];       // first entry of each pass's twiddle table (see fft_twiddle_tables)
};

// row width of a pass's twiddle table: R, or 4 for radix 3 (rows of 16-byte pairs)
__host__ __device__ constexpr int tw_width(int R) { return R == 3 ? 4 : R; }

constexpr int FTH = 256;
constexpr double SQRT3_2 = 0.86602540378443864676;  // sin(2 pi / 3)

template <typename C> struct Cx;
// per arithmetic type: make, and the butterfly constants 1/sqrt(2), 1/2 and sin(2 pi / 3)
template <> struct Cx<double2> {
  using R = double;
  static __device__ __forceinline__ double2 make(double x, double y) { return make_double2(x, y); }
  static __device__ __forceinline__ double rsqrt2() { return 0.70710678118654752440; }
  static __device__ __forceinline__ double half() { return 0.5; }
  static __device__ __forceinline__ double sqrt3_2() { return SQRT3_2; }
};
template <> struct Cx<float2> {
  using R = float;
  static __device__ __forceinline__ float2 make(float x, float y) { return make_float2(x, y); }
  static __device__ __forceinline__ float rsqrt2() { return 0.70710678118654752440f; }
  static __device__ __forceinline__ float half() { return 0.5f; }
  static __device__ __forceinline__ float sqrt3_2() { return (float)SQRT3_2; }
};
// double-float complex (SH_DF plans): about 48 significand bits on the FP32 pipe, the same 16
// bytes as double2 in shared memory and in the twiddle tables
struct dfcx {
  dfr x, y;
};
template <> struct Cx<dfcx> {
  using R = dfr;
  static __device__ __forceinline__ dfcx make(dfr x, dfr y) { return dfcx{x, y}; }
  // the constants as exact (hi, lo) pairs of FP32 literals: no FP64 conversion in the butterflies
  static __device__ __forceinline__ dfr rsqrt2() { return dfr(0x1.6a09e6p-1f, 0x1.9fcef4p-27f); }
  static __device__ __forceinline__ dfr half() { return dfr(0.5f, 0.f); }
  static __device__ __forceinline__ dfr sqrt3_2() { return dfr(0x1.bb67aep-1f, 0x1.0b0996p-26f); }
};
// FP64 grid and Fourier values into the transform's arithmetic and back: FP32 and double-float
// plans convert on the integer pipe (cvt.cuh; the F2F instructions would occupy the scarce FP64
// pipe).  The double-float split is the same as dfr(double): hi = d rounded to FP32, lo = the
// exact FP64 difference d - hi rounded to FP32; one FP64 subtraction each way remains.
template <typename R> __device__ __forceinline__ R from_f64(double d) { return R(d); }
template <> __device__ __forceinline__ float from_f64<float>(double d) { return cvt::f64_to_f32(d); }
template <> __device__ __forceinline__ dfr from_f64<dfr>(double d) {
  const float h = cvt::f64_to_f32(d);
  return dfr(h, cvt::f64_to_f32(d - cvt::f32_to_f64(h)));
}
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return cvt::f32_to_f64(x); }
__device__ __forceinline__ double to_f64(dfr x) { return cvt::f32_to_f64(x.hi) + cvt::f32_to_f64(x.lo); }
// one twiddle-table entry
__device__ __forceinline__ double2 ld_tw(const double2* p) { return __ldg(p); }
__device__ __forceinline__ dfcx ld_tw(const dfcx* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return dfcx{dfr(v.x, v.y), dfr(v.z, v.w)};
}
template <typename C> __device__ __forceinline__ C c_mul(C a, C b) {
  return Cx<C>::make(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C c_add(C a, C b) { return Cx<C>::make(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C c_sub(C a, C b) { return Cx<C>::make(a.x - b.x, a.y - b.y); }

// R-point DFTs in registers, X_k = sum_j v_j w^{jk} with w = e^{sign 2 pi i / R}
template <typename C> __device__ __forceinline__ C c_mul_i(C a, int sign) {  // (sign i) * a
  return sign > 0 ? Cx<C>::make(-a.y, a.x) : Cx<C>::make(a.y, -a.x);
}
template <typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  const C t = c_sub(a, b);
  a = c_add(a, b);
  b = t;
}
template <typename C> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3, int sign) {
  const C a0 = c_add(v0, v2), a1 = c_sub(v0, v2), a2 = c_add(v1, v3);
  const C d = c_mul_i(c_sub(v1, v3), sign);
  v0 = c_add(a0, a2);
  v2 = c_sub(a0, a2);
  v1 = c_add(a1, d);
  v3 = c_sub(a1, d);
}
template <typename C> __device__ __forceinline__ void dft8(C* v, int sign) {
  using R = typename Cx<C>::R;
  const R h = Cx<C>::rsqrt2();
  dft4(v[0], v[2], v[4], v[6], sign);     // even samples -> E_0..E_3 in v[0], v[2], v[4], v[6]
  dft4(v[1], v[3], v[5], v[7], sign);     // odd samples  -> O_0..O_3 in v[1], v[3], v[5], v[7]
  // twiddles w8^k O_k, w8 = (1 + sign i) / sqrt 2
  const C o1 = Cx<C>::make(h * (v[3].x - sign * v[3].y), h * (v[3].y + sign * v[3].x));
  const C o2 = c_mul_i(v[5], sign);
  const C o3 = Cx<C>::make(h * (-v[7].x - sign * v[7].y), h * (-v[7].y + sign * v[7].x));
  const C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
  v[0] = c_add(e0, o0);
  v[4] = c_sub(e0, o0);
  v[1] = c_add(e1, o1);
  v[5] = c_sub(e1, o1);
  v[2] = c_add(e2, o2);
  v[6] = c_sub(e2, o2);
  v[3] = c_add(e3, o3);
  v[7] = c_sub(e3, o3);
}

// Segments of one FFT launch: blockIdx.y in [start[s], start[s + 1]) is field y - start[s] of
// segment s, whose Fourier coefficients are F[s] ([nf_s][T+1][nlat]) and grid rows g[s]
// ([nf_s][nlat][nlon]); unused segments have start[s] = start[s + 1] = the field total.
struct FftSegs {
  double2* F[3];
  double* g[3];
  int start[4];
};

// padded shared-memory index: one spare slot per 8 elements, so that the stride-R stores of
// the early passes spread over the banks
__device__ __forceinline__ int fpad(int i) { return i + (i >> 3); }
__host__ __device__ constexpr int fft_padded(int n) { return n + (n >> 3) + 1; }

// One Stockham pass of radix R (2, 3, 4 or 8): for j < n / R, jm = j mod Ns, q = j / Ns, the
// R inputs src(j + r n/R) times the twiddles w^{r jm stride} are transformed and written to
// dst(q Ns R + jm + r Ns).  twp is the pass's twiddle table, row jm = (w^{r jm stride}, r < R),
// tw_width(R) entries per row, read as 16-byte pairs (FP32) or 16-byte entries (FP64); the
// first pass (Ns = 1) has no twiddles.
template <typename C, int R, typename Src, typename Dst>
__device__ __forceinline__ void fft_pass(Src src, Dst dst, int n, int Ns, unsigned mg, const C* twp, int sign) {
  using Rt = typename Cx<C>::R;
  constexpr int W = tw_width(R);
  const int nb = n / R;
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int q = (Ns == 1) ? j : (int)__umulhi((unsigned)j, mg);  // j / Ns
    const int jm = j - q * Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src(j + r * nb);
    if (Ns > 1) {  // uniform over the block
      auto apply = [&](int r, C tr) {
        if (sign > 0) tr.y = -tr.y;
        v[r] = c_mul(v[r], tr);
      };
      if constexpr (std::is_same<C, float2>::value) {
        const float4* tp = reinterpret_cast<const float4*>(twp + jm * W);
#pragma unroll
        for (int h = 0; h < W / 2; ++h) {  // a 16-byte pair per load, applied as it arrives
          const float4 pr = __ldg(tp + h);
          if (h > 0) apply(2 * h, make_float2(pr.x, pr.y));
          if (2 * h + 1 < R) apply(2 * h + 1, make_float2(pr.z, pr.w));
        }
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) apply(r, ld_tw(twp + jm * W + r));
      }
    }
    if (R == 2) {
      dft2(v[0], v[1]);
    } else if (R == 4) {
      dft4(v[0], v[1], v[2], v[3], sign);
    } else if (R == 8) {
      dft8(v, sign);
    } else {  // R == 3
      const C s1 = c_add(v[1], v[2]);
      const C t2 = Cx<C>::make(v[0].x - Cx<C>::half() * s1.x, v[0].y - Cx<C>::half() * s1.y);
      const C d = c_sub(v[1], v[2]);
      const Rt sg = sign * Cx<C>::sqrt3_2();
      const C x0 = c_add(v[0], s1);
      v[1] = Cx<C>::make(t2.x - sg * d.y, t2.y + sg * d.x);
      v[2] = Cx<C>::make(t2.x + sg * d.y, t2.y - sg * d.x);
      v[0] = x0;
    }
    const int base = q * Ns * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) dst(base + r * Ns, v[r]);
  }
}

template <typename C, typename Src, typename Dst>
__device__ __forceinline__ void fft_pass_r(int R, Src src, Dst dst, int n, int Ns, unsigned mg, const C* tw,
                                           int sign) {
  if (R == 8) fft_pass<C, 8>(src, dst, n, Ns, mg, tw, sign);
  else if (R == 4) fft_pass<C, 4>(src, dst, n, Ns, mg, tw, sign);
  else if (R == 2) fft_pass<C, 2>(src, dst, n, Ns, mg, tw, sign);
  else fft_pass<C, 3>(src, dst, n, Ns, mg, tw, sign);
}

// All passes of one length-n transform (sign = -1 forward, +1 inverse, no scaling; tw holds the
// passes' twiddle tables of e^{-2 pi i k / n}, pass s from fp.twoff[s]).  The first pass reads its inputs through src (global memory); the passes
// in between go through the padded shared buffers a and b; the last pass writes through dst,
// or, with LAST_SMEM, into a shared buffer whose address is returned (padded indices).
template <typename C, bool LAST_SMEM, typename Src, typename Dst>
__device__ C* fft_run(Src src, Dst dst, C* a, C* b, const FftPlan& fp, const C* tw, int sign) {
  const int n = fp.n, S = fp.nrad;
  C* cur = a;  // holds the input of the next pass (after the first)
  C* nxt = b;
  int Ns = 1;
  for (int s = 0; s < S; ++s) {
    const int R = fp.rad[s];
    const unsigned mg = fp.magic[s];
    const C* twp = tw + fp.twoff[s];
    C* const rb = cur;
    C* const wb = nxt;
    auto rd = [rb](int i) { return rb[fpad(i)]; };
    auto wr = [wb](int i, C v) { wb[fpad(i)] = v; };
    const bool last = s == S - 1;
    if (s == 0) {
      if (last && !LAST_SMEM) fft_pass_r<C>(R, src, dst, n, Ns, mg, twp, sign);
      else fft_pass_r<C>(R, src, wr, n, Ns, mg, twp, sign);
    } else {
      if (last && !LAST_SMEM) fft_pass_r<C>(R, rd, dst, n, Ns, mg, twp, sign);
      else fft_pass_r<C>(R, rd, wr, n, Ns, mg, twp, sign);
    }
    __syncthreads();
    cur = wb;
    nxt = rb;
    Ns *= R;
  }
  return cur;
}

// ---- transforms of fixed length (n = 384, 768, 1536: the T127, T255 and T511 grids) ---------
// The same Stockham passes with the length known at compile time: radices, strides Ns, twiddle
// offsets and trip counts are constants, j / Ns is a constant division, and each padded index is
// formed once per butterfly and advanced by constant steps (fpad(x + 8k) = fpad(x) + 9k).  The
// factorisation is fft_factor's (radix 8 first, then 4, 2, 3); the plan checks that they agree.
// Used by the FP32 and double-float FFTs; the FP64 one is bound by the FP64 pipe.
constexpr int ct_nrad(int n) {
  int k = 0;
  while (n % 8 == 0) n /= 8, ++k;
  while (n % 4 == 0) n /= 4, ++k;
  while (n % 2 == 0) n /= 2, ++k;
  while (n % 3 == 0) n /= 3, ++k;
  return k;
}
constexpr int ct_rad(int n, int s) {
  const int rs[4] = {8, 4, 2, 3};
  int k = 0;
  for (int i = 0; i < 4; ++i)
    while (n % rs[i] == 0) {
      if (k++ == s) return rs[i];
      n /= rs[i];
    }
  return 0;
}
constexpr int ct_ns(int n, int s) {
  int p = 1;
  for (int i = 0; i < s; ++i) p *= ct_rad(n, i);
  return p;
}
constexpr int ct_twoff(int n, int s) {
  int off = 0;
  for (int i = 0; i < s; ++i) off += ct_ns(n, i) * tw_width(ct_rad(n, i));
  return off;
}

// padded index of element j + r nb (the pass's reads) and of base + r Ns (its writes)
template <int NB> __device__ __forceinline__ int ct_rd(int pj, int j, int r) {
  if constexpr (NB % 8 == 0) return pj + r * (NB + NB / 8);
  else return fpad(j + r * NB);
}
template <int NS, int R> __device__ __forceinline__ int ct_wr(int pb, int base, int r) {
  if constexpr (NS % 8 == 0) return pb + r * (NS + NS / 8);
  else if constexpr (NS == 1 && 8 % R == 0) return pb + r;  // base = q R, a multiple of R dividing 8
  else return fpad(base + r * NS);
}

// One pass: radix R, length N, stride NS; reads the padded shared buffer rb or, with SRC_G,
// global memory through src(k); writes the padded buffer wb or, with DST_G, dst(k, v).
template <typename C, int R, int N, int NS, int SIGN, bool SRC_G, bool DST_G, typename Src, typename Dst>
__device__ __forceinline__ void fft_pass_ct(const C* rb, Src src, C* wb, Dst dst, const C* twp) {
  using Rt = typename Cx<C>::R;
  constexpr int NB = N / R, W = tw_width(R), IT = (NB + FTH - 1) / FTH;
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = it * FTH + (int)threadIdx.x;
    if (NB % FTH != 0 && j >= NB) break;
    const int q = j / NS, jm = j - q * NS;
    C v[R];
    const int pj = fpad(j);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (SRC_G) v[r] = src(j + r * NB);
      else v[r] = rb[ct_rd<NB>(pj, j, r)];
    }
    if constexpr (NS > 1) {
      auto apply = [&](int r, C tr) {
        if (SIGN > 0) tr.y = -tr.y;
        v[r] = c_mul(v[r], tr);
      };
      if constexpr (std::is_same<C, float2>::value) {
        const float4* tp = reinterpret_cast<const float4*>(twp + jm * W);
#pragma unroll
        for (int h = 0; h < W / 2; ++h) {  // a 16-byte pair per load, applied as it arrives
          const float4 pr = __ldg(tp + h);
          if (h > 0) apply(2 * h, make_float2(pr.x, pr.y));
          if (2 * h + 1 < R) apply(2 * h + 1, make_float2(pr.z, pr.w));
        }
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) apply(r, ld_tw(twp + jm * W + r));
      }
    }
    if constexpr (R == 2) {
      dft2(v[0], v[1]);
    } else if constexpr (R == 4) {
      dft4(v[0], v[1], v[2], v[3], SIGN);
    } else if constexpr (R == 8) {
      dft8(v, SIGN);
    } else {
      static_assert(R == 3, "radix 2, 3, 4 or 8");
      const C s1 = c_add(v[1], v[2]);
      const C t2 = Cx<C>::make(v[0].x - Cx<C>::half() * s1.x, v[0].y - Cx<C>::half() * s1.y);
      const C d = c_sub(v[1], v[2]);
      const Rt sg = SIGN * Cx<C>::sqrt3_2();
      const C x0 = c_add(v[0], s1);
      v[1] = Cx<C>::make(t2.x - sg * d.y, t2.y + sg * d.x);
      v[2] = Cx<C>::make(t2.x + sg * d.y, t2.y - sg * d.x);
      v[0] = x0;
    }
    const int base = q * NS * R + jm;
    const int pb = fpad(base);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (DST_G) dst(base + r * NS, v[r]);
      else wb[ct_wr<NS, R>(pb, base, r)] = v[r];
    }
  }
}

// Passes S.. of the length-N transform: pass S reads cur (global memory through src when
// S = 0 and FIRST_G) and writes nxt (dst when it is the last pass and not LAST_SMEM); the next
// pass swaps the two buffers.  Returns the shared buffer holding the result (LAST_SMEM).
template <typename C, int N, int S, int SIGN, bool FIRST_G, bool LAST_SMEM, typename Src, typename Dst>
__device__ __forceinline__ C* fft_run_ct(Src src, Dst dst, C* cur, C* nxt, const C* tw) {
  constexpr int R = ct_rad(N, S), NS = ct_ns(N, S);
  constexpr bool last = S == ct_nrad(N) - 1;
  fft_pass_ct<C, R, N, NS, SIGN, FIRST_G && S == 0, last && !LAST_SMEM>(cur, src, nxt, dst, tw + ct_twoff(N, S));
  __syncthreads();
  if constexpr (last) return nxt;
  else return fft_run_ct<C, N, S + 1, SIGN, FIRST_G, LAST_SMEM>(src, dst, nxt, cur, tw);
}

// the lengths with fixed-length kernels
constexpr bool fft_fixed_len(int n) { return n == 384 || n == 768 || n == 1536; }


__device__ __forceinline__ int fft_seg(const FftSegs& sg, int y) {
  return (y >= sg.start[1]) + (y >= sg.start[2]);
}

// synthesis: F[field][m][nlat] (m <= T) -> grid[field][nlat][nlon], two latitude rows per block
// (row j0 in the real part, j0 + 1 in the imaginary part of one complex sequence)
template <typename C, int N = 0>  // N > 0: the fixed-length passes of that length
__device__ __forceinline__ void fft_synth_block(const FftSegs& sg, const FftPlan& fp, const C* __restrict__ tw, int T,
                                                int nlat) {
  extern __shared__ __align__(16) unsigned char fsm[];
  using R = typename Cx<C>::R;
  const int n = N ? N : fp.n, np = fft_padded(n);
  C* a = reinterpret_cast<C*>(fsm);
  C* b = a + np;
  const int s = fft_seg(sg, blockIdx.y), f = blockIdx.y - sg.start[s];
  const int j0 = 2 * blockIdx.x;
  const double2* in = sg.F[s] + (size_t)f * (T + 1) * nlat;
  double* r0 = sg.g[s] + ((size_t)f * nlat + j0) * n;
  double* r1 = r0 + n;
  // input element k: A + i B of order m = k (k <= T), conj(A) + i conj(B) of m = n - k
  // (k >= n - T), else 0; A, B = latitudes j0, j0 + 1 of order m, one aligned 32-byte load per
  // m for both entries.  Filled into the padded buffer b, which the first pass reads.
  for (int m = threadIdx.x; m <= T; m += blockDim.x) {
    const D4 AB = *reinterpret_cast<const D4*>(in + (size_t)m * nlat + j0);
    // in the transform's own precision: FP32 plans convert first and combine in FP32
    const R ax = from_f64<R>(AB.x), ay = from_f64<R>(AB.y), bx = from_f64<R>(AB.z), by = from_f64<R>(AB.w);
    if (m == 0) {
      b[0] = Cx<C>::make(ax, bx);
    } else {
      b[fpad(m)] = Cx<C>::make(ax - by, ay + bx);
      b[fpad(n - m)] = Cx<C>::make(ax + by, bx - ay);
    }
  }
  for (int k = T + 1 + threadIdx.x; k < n - T; k += blockDim.x) b[fpad(k)] = Cx<C>::make(R(0), R(0));
  __syncthreads();
  const C* bin = b;
  auto src = [bin](int k) -> C { return bin[fpad(k)]; };
  auto dst = [r0, r1](int k, C v) {
    r0[k] = to_f64(v.x);
    r1[k] = to_f64(v.y);
  };
  if constexpr (N > 0) fft_run_ct<C, N, 0, +1, false, false>(src, dst, b, a, tw);  // reads b, writes a first
  else fft_run<C, false>(src, dst, b, a, fp, tw, +1);  // the first pass reads b and writes a
}

// analysis: grid[field][nlat][nlon] -> F[field][m][nlat] = (2 pi / n) sum_k f e^{-i m lambda_k}
template <typename C, int N = 0>  // N > 0: the fixed-length passes of that length
__device__ __forceinline__ void fft_anal_block(const FftSegs& sg, const FftPlan& fp, const C* __restrict__ tw, int T,
                                               int nlat) {
  extern __shared__ __align__(16) unsigned char fsm[];
  using R = typename Cx<C>::R;
  const int n = N ? N : fp.n, np = fft_padded(n);
  C* a = reinterpret_cast<C*>(fsm);
  C* b = a + np;
  const int s = fft_seg(sg, blockIdx.y), f = blockIdx.y - sg.start[s];
  const int j0 = 2 * blockIdx.x;
  const double* r0 = sg.g[s] + ((size_t)f * nlat + j0) * n;
  const double* r1 = r0 + n;
  auto src = [r0, r1](int k) -> C { return Cx<C>::make(from_f64<R>(__ldg(r0 + k)), from_f64<R>(__ldg(r1 + k))); };
  auto none = [](int, C) {};
  const C* z;
  if constexpr (N > 0) z = fft_run_ct<C, N, 0, -1, true, true>(src, none, a, b, tw);
  else z = fft_run<C, true>(src, none, a, b, fp, tw, -1);
  const R sc = R(3.14159265358979323846 / n);  // (2 pi / n) / 2, in the transform's precision
  double2* out = sg.F[s] + (size_t)f * (T + 1) * nlat;
  for (int m = threadIdx.x; m <= T; m += blockDim.x) {
    const C zm = z[fpad(m)], zn = z[fpad(m == 0 ? 0 : n - m)];
    // A = (Z_m + conj(Z_{n-m})) / 2,  B = (Z_m - conj(Z_{n-m})) / (2i); one aligned 32-byte store
    *reinterpret_cast<D4*>(out + (size_t)m * nlat + j0) =
        D4{to_f64(sc * (zm.x + zn.x)), to_f64(sc * (zm.y - zn.y)), to_f64(sc * (zm.y + zn.y)),
           to_f64(-sc * (zm.x - zn.x))};
  }
}

// FP32 transforms (tensor-core plans) keep six blocks per SM resident; FP64 ones are bound by
// the FP64 pipe and keep their registers
// (N > 0: the fixed-length passes; N = 0: the length from fp)
template <int N>
__global__ void __launch_bounds__(FTH, 6) k_fft_synth32(const __grid_constant__ FftSegs sg,
                                                        const __grid_constant__ FftPlan fp,
                                                        const float2* __restrict__ tw, int T, int nlat) {
  fft_synth_block<float2, N>(sg, fp, tw, T, nlat);
}
__global__ void __launch_bounds__(FTH) k_fft_synth64(const __grid_constant__ FftSegs sg,
                                                     const __grid_constant__ FftPlan fp,
                                                     const double2* __restrict__ tw, int T, int nlat) {
  fft_synth_block<double2>(sg, fp, tw, T, nlat);
}
template <int N>
__global__ void __launch_bounds__(FTH, 6) k_fft_anal32(const __grid_constant__ FftSegs sg,
                                                       const __grid_constant__ FftPlan fp,
                                                       const float2* __restrict__ tw, int T, int nlat) {
  fft_anal_block<float2, N>(sg, fp, tw, T, nlat);
}
__global__ void __launch_bounds__(FTH) k_fft_anal64(const __grid_constant__ FftSegs sg,
                                                    const __grid_constant__ FftPlan fp,
                                                    const double2* __restrict__ tw, int T, int nlat) {
  fft_anal_block<double2>(sg, fp, tw, T, nlat);
}

// double-float transforms (SH_DF plans): FP64 inputs and outputs, arithmetic on the FP32 pipe;
// four blocks per SM, which their shared memory allows (at 76 registers only three fit: the
// one-pass N(U) synthesis at T511 took 0.086 ms that way, 0.078 ms with four)
template <int N>
__global__ void __launch_bounds__(FTH, 4) k_fft_synth_df(const __grid_constant__ FftSegs sg,
                                                      const __grid_constant__ FftPlan fp,
                                                      const dfcx* __restrict__ tw, int T, int nlat) {
  fft_synth_block<dfcx, N>(sg, fp, tw, T, nlat);
}
template <int N>
__global__ void __launch_bounds__(FTH, 4) k_fft_anal_df(const __grid_constant__ FftSegs sg,
                                                     const __grid_constant__ FftPlan fp,
                                                     const dfcx* __restrict__ tw, int T, int nlat) {
  fft_anal_block<dfcx, N>(sg, fp, tw, T, nlat);
}

// the instantiation for length n: fixed-length kernels for 384, 768, 1536, else the general one
#define FFT_KERNEL_FAMILY(NAME, C)                                                        \
  struct NAME##_fam {                                                                     \
    using Fn = void (*)(FftSegs, FftPlan, const C*, int, int);                            \
    static Fn pick(int n, bool fixed) {                                                   \
      if (fixed && n == 1536) return NAME<1536>;                                          \
      if (fixed && n == 768) return NAME<768>;                                            \
      if (fixed && n == 384) return NAME<384>;                                            \
      return NAME<0>;                                                                     \
    }                                                                                     \
    static cudaError_t limits(size_t bytes) {                                             \
      cudaError_t e = raise_smem_limit(NAME<0>, bytes);                                   \
      if (!e) e = raise_smem_limit(NAME<384>, bytes);                                     \
      if (!e) e = raise_smem_limit(NAME<768>, bytes);                                     \
      if (!e) e = raise_smem_limit(NAME<1536>, bytes);                                    \
      return e;                                                                           \
    }                                                                                     \
  };
FFT_KERNEL_FAMILY(k_fft_synth32, float2)
FFT_KERNEL_FAMILY(k_fft_anal32, float2)
FFT_KERNEL_FAMILY(k_fft_synth_df, dfcx)
FFT_KERNEL_FAMILY(k_fft_anal_df, dfcx)
#undef FFT_KERNEL_FAMILY

// Gauss-Legendre nodes (north to south) and weights: Newton iteration on P_n
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = z;
    x[n - 1 - i] = -z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

bool fft_factor(int n, FftPlan& fp) {
  fp.n = n;
  fp.nrad = 0;
  int m = n;
  while (m % 8 == 0 && fp.nrad < 24) {
    fp.rad[fp.nrad++] = 8;
    m /= 8;
  }
  while (m % 4 == 0 && fp.nrad < 24) {
    fp.rad[fp.nrad++] = 4;
    m /= 4;
  }
  while (m % 2 == 0 && fp.nrad < 24) {
    fp.rad[fp.nrad++] = 2;
    m /= 2;
  }
  while (m % 3 == 0 && fp.nrad < 24) {
    fp.rad[fp.nrad++] = 3;
    m /= 3;
  }
  unsigned long long Ns = 1;
  int off = 0;
  for (int s = 0; s < fp.nrad; ++s) {
    fp.magic[s] = Ns == 1 ? 0u : (unsigned)(((1ULL << 32) + Ns - 1) / Ns);  // ceil(2^32 / Ns); unused for Ns = 1
    fp.twoff[s] = off;
    off += (int)Ns * tw_width(fp.rad[s]);
    Ns *= fp.rad[s];
  }
  return m == 1;
}

// Twiddle tables of all passes: pass s (radix R, Ns = product of the earlier radices, stride
// n / (Ns R)) holds, for jm < Ns, the row (e^{-2 pi i r jm stride / n}, r < R) padded to
// tw_width(R) entries; the total is fp.twoff[nrad - 1] + Ns_last * tw_width(R_last) entries.
static std::vector<std::complex<double>> fft_twiddle_tables(const FftPlan& fp) {
  std::vector<std::complex<double>> t;
  long long Ns = 1;
  for (int s = 0; s < fp.nrad; ++s) {
    const int R = fp.rad[s], W = tw_width(R);
    const long long stride = fp.n / (Ns * R);
    for (long long jm = 0; jm < Ns; ++jm)
      for (int r = 0; r < W; ++r) {
        const long long k = r < R ? (r * jm * stride) % fp.n : 0;
        const double a = -2.0 * M_PI * (double)k / fp.n;
        t.push_back(r < R ? std::complex<double>(std::cos(a), std::sin(a)) : 0.0);
      }
    Ns *= R;
  }
  return t;
}

}  // namespace

void launch_divcurl_from_p(const double2* raw, double2* dv, double2* cu, int nfv, int T, double inv_a, cudaStream_t s) {
  if (nfv < 1) return;
  const int nlm = (T + 1) * (T + 2) / 2, nlme = (T + 1) * (T + 4) / 2;
  k_divcurl_from_p<<<dim3(T + 1, nfv), 128, 0, s>>>(raw, dv, cu, T, nlm, nlme, inv_a);
}

}  // namespace rexi

using namespace rexi;

struct sh_plan {
  sh_plan_desc d{};
  int nh = 0, nlm = 0;
  cudaStream_t stream = nullptr;
  std::vector<double> mu, w;
  double* d_mu = nullptr;   // northern nodes [nh]
  double* d_w = nullptr;    // northern weights [nh]
  double* d_wq = nullptr;   // w / (1 - mu^2) [nh]
  double* d_P = nullptr;    // [nlm][nh]
  double* d_H = nullptr;
  double* d_Pn = nullptr;   // P_{T+1}^m [T+1][nh]
  double2* d_raw = nullptr; // P-sums of the FP64 vector analysis [max_fields][2][nlme]
  double2* d_uv = nullptr;  // u and v spectra of the FP64 vector synthesis [2 max_fields][nlme]
  double2* d_tw = nullptr;  // twiddle tables of the FFT passes (fft_twiddle_tables)
  float2* d_tw32 = nullptr; // the same in FP32, for the FFT of the tensor-core plans
  float4* d_twdf = nullptr; // the same as double-float pairs (re.hi, re.lo, im.hi, im.lo), SH_DF
  bool fft32 = false;
  bool fftdf = false;       // double-float FFT (SH_DF)
  bool fft_fixed = false;   // FP32 / double-float FFT by the fixed-length kernels
  double2* d_F = nullptr;   // Fourier workspace [2 * max_fields][T+1][nlat]
  FftPlan fp{};
  TcLegendre* tc = nullptr;  // tensor-core Legendre state (SH_TF32 / SH_BF16 / SH_TF32X3)
  DfLegendre* dfl = nullptr;  // double-float Legendre state (SH_DF)
  StageProf prof;            // per-stage event timing (sh_plan_set_profiling)
  // polar truncation: threshold (0 = off), start indices per (m, group) on host and device
  double polar_thr = 0.0;
  std::vector<int> ks, ja;
  int* d_ks = nullptr;
  int* d_ja = nullptr;
  PolarBounds pb;
  long long need_syn = 0, need_ana = 0;  // entries the method needs per table (sh_table_use)
};

// two padded work buffers
static size_t fft_smem(const sh_plan* p) {
  return (p->fft32 ? sizeof(float2) : sizeof(double2)) * 2 * (size_t)fft_padded(p->d.nlon);
}

extern "C" int sh_plan_create(const sh_plan_desc* desc, sh_plan** out) {
  if (!desc || !out) return fail(REXI_EINVAL, "sh_plan_create: null argument");
  *out = nullptr;
  const sh_plan_desc& d = *desc;
  if (d.T < 1 || d.T > 1023) return fail(REXI_EINVAL, "sh_plan_create: T = %d outside [1, 1023]", d.T);
  if (d.nlat < 2 || d.nlat % 2 || d.nlat <= d.T)
    return fail(REXI_EINVAL, "sh_plan_create: nlat must be even and > T (got %d)", d.nlat);
  if (d.nlon <= 2 * d.T) return fail(REXI_EINVAL, "sh_plan_create: nlon must exceed 2T");
  if (!(d.radius > 0) || d.max_fields < 1) return fail(REXI_EINVAL, "sh_plan_create: radius > 0, max_fields >= 1");
  if (d.epilogue_wait_polls < 0) return fail(REXI_EINVAL, "sh_plan_create: epilogue_wait_polls < 0");
  if (!(d.polar_threshold == d.polar_threshold) || d.polar_threshold >= 1e-3)
    return fail(REXI_EINVAL, "sh_plan_create: polar_threshold must be below 1e-3 (or <= 0)");
  if (d.precision != SH_FP64 && d.precision != SH_TF32 && d.precision != SH_BF16 && d.precision != SH_TF32X3 &&
      d.precision != SH_DF)
    return fail(REXI_EINVAL, "sh_plan_create: unknown precision %d", d.precision);
  sh_plan* p = new sh_plan();
  p->d = d;
  p->nh = d.nlat / 2;
  p->nlm = (d.T + 1) * (d.T + 2) / 2;
  p->stream = (cudaStream_t)d.stream;
  p->prof.stream = p->stream;
  p->fft32 = d.precision != SH_FP64 && d.precision != SH_DF;
  p->fftdf = d.precision == SH_DF;
  auto bail = [&](int code) {
    sh_plan_destroy(p);
    return code;
  };
  if (!fft_factor(d.nlon, p->fp)) return bail(fail(REXI_EINVAL, "nlon = %d is not 2^p 3^q", d.nlon));
  if (fft_smem(p) > 200 * 1024) return bail(fail(REXI_EINVAL, "nlon = %d too large", d.nlon));
  if ((p->fft32 || p->fftdf) && fft_fixed_len(d.nlon)) {  // their passes and twiddle offsets are fft_factor's
    bool same = p->fp.nrad == ct_nrad(d.nlon);
    for (int s = 0; same && s < p->fp.nrad; ++s)
      same = p->fp.rad[s] == ct_rad(d.nlon, s) && p->fp.twoff[s] == ct_twoff(d.nlon, s);
    p->fft_fixed = same;
  }
  gauss_legendre(d.nlat, p->mu, p->w);
  std::vector<double> wq(p->nh);
  for (int j = 0; j < p->nh; ++j) wq[j] = p->w[j] / ((1.0 - p->mu[j]) * (1.0 + p->mu[j]));
  const std::vector<std::complex<double>> twt = fft_twiddle_tables(p->fp);
  const size_t ntw = twt.size();
  std::vector<double2> tw(ntw);
  std::vector<float2> tw32(ntw);
  std::vector<float4> twdf(ntw);
  auto lo_of = [](double x) { return (float)(x - (double)(float)x); };
  for (size_t k = 0; k < ntw; ++k) {
    const double re = twt[k].real(), im = twt[k].imag();
    tw[k] = make_double2(re, im);
    tw32[k] = make_float2((float)re, (float)im);
    twdf[k] = make_float4((float)re, lo_of(re), (float)im, lo_of(im));
  }
  const size_t tab = (size_t)p->nlm * p->nh;
  cudaError_t e;
  if ((e = cudaMalloc(&p->d_mu, sizeof(double) * p->nh)) || (e = cudaMalloc(&p->d_w, sizeof(double) * p->nh)) ||
      (e = cudaMalloc(&p->d_wq, sizeof(double) * p->nh)) || (e = cudaMalloc(&p->d_P, sizeof(double) * tab)) ||
      (e = cudaMalloc(&p->d_H, sizeof(double) * tab)) ||
      (e = cudaMalloc(&p->d_Pn, sizeof(double) * (size_t)(d.T + 1) * p->nh)) ||
      (d.precision == SH_FP64 &&
       ((e = cudaMalloc(&p->d_raw, sizeof(double2) * 2 * (size_t)d.max_fields * nlm_ext(d.T))) ||
        (e = cudaMalloc(&p->d_uv, sizeof(double2) * 2 * (size_t)d.max_fields * nlm_ext(d.T))))) ||
      (e = cudaMalloc(&p->d_tw, sizeof(double2) * ntw)) ||
      (e = cudaMalloc(&p->d_tw32, sizeof(float2) * ntw)) || (e = cudaMalloc(&p->d_twdf, sizeof(float4) * ntw)) ||
      (e = cudaMalloc(&p->d_F, sizeof(double2) * 2 * (size_t)d.max_fields * (d.T + 1) * d.nlat))) {
    cudaGetLastError();
    return bail(fail(REXI_ENOMEM, "sh_plan_create: cudaMalloc failed: %s", cudaGetErrorString(e)));
  }
  if ((e = cudaMemcpy(p->d_mu, p->mu.data(), sizeof(double) * p->nh, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(p->d_w, p->w.data(), sizeof(double) * p->nh, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(p->d_wq, wq.data(), sizeof(double) * p->nh, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(p->d_tw, tw.data(), sizeof(double2) * ntw, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(p->d_tw32, tw32.data(), sizeof(float2) * ntw, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(p->d_twdf, twdf.data(), sizeof(float4) * ntw, cudaMemcpyHostToDevice)))
    return bail(cuda_fail(e, "sh_plan_create: cudaMemcpy"));
  k_legendre_table<<<dim3((p->nh + 127) / 128, d.T + 1), 128, 0, p->stream>>>(p->d_mu, p->d_P, p->d_H, p->d_Pn, d.T,
                                                                                p->nh);
  if ((e = cudaGetLastError())) return bail(cuda_fail(e, "k_legendre_table"));
  // polar bounds
  p->polar_thr = d.polar_threshold == 0.0 ? SH_POLAR_THRESHOLD_DEFAULT : d.polar_threshold > 0 ? d.polar_threshold : 0.0;
  {
    const int ngl = (p->nh + 31) / 32, ngd = (d.T + 2 + 31) / 32;  // degrees to n = T + 1
    const size_t nks = (size_t)(d.T + 1) * ngl, nja = (size_t)(d.T + 1) * ngd;
    p->ks.assign(nks, 0);
    p->ja.assign(nja, 0);
    std::vector<int> nds(nks, 0), nda(nja, 0);
    int *d_nds = nullptr, *d_nda = nullptr;
    if ((e = cudaMalloc(&p->d_ks, sizeof(int) * nks)) || (e = cudaMalloc(&p->d_ja, sizeof(int) * nja))) {
      cudaGetLastError();
      return bail(fail(REXI_ENOMEM, "sh_plan_create: cudaMalloc failed: %s", cudaGetErrorString(e)));
    }
    if (p->polar_thr > 0) {
      if ((e = cudaMalloc(&d_nds, sizeof(int) * nks)) || (e = cudaMalloc(&d_nda, sizeof(int) * nja))) {
        cudaFree(d_nds);
        cudaGetLastError();
        return bail(fail(REXI_ENOMEM, "sh_plan_create: cudaMalloc failed: %s", cudaGetErrorString(e)));
      }
      k_polar_synth<<<dim3(ngl, d.T + 1), 32, 0, p->stream>>>(p->d_P, p->d_H, d.T, p->nh, p->polar_thr, ngl, p->d_ks,
                                                               d_nds);
      k_polar_anal<<<dim3(ngd, d.T + 1), 32, 0, p->stream>>>(p->d_P, p->d_H, p->d_Pn, d.T, p->nh, p->polar_thr, ngd,
                                                              p->d_ja, d_nda);
      if (!(e = cudaGetLastError()) && !(e = cudaStreamSynchronize(p->stream)) &&
          !(e = cudaMemcpy(p->ks.data(), p->d_ks, sizeof(int) * nks, cudaMemcpyDeviceToHost)) &&
          !(e = cudaMemcpy(p->ja.data(), p->d_ja, sizeof(int) * nja, cudaMemcpyDeviceToHost)) &&
          !(e = cudaMemcpy(nds.data(), d_nds, sizeof(int) * nks, cudaMemcpyDeviceToHost)))
        e = cudaMemcpy(nda.data(), d_nda, sizeof(int) * nja, cudaMemcpyDeviceToHost);
      cudaFree(d_nds);
      cudaFree(d_nda);
      if (e) return bail(cuda_fail(e, "sh_plan_create: polar bounds"));
      for (int v : nds) p->need_syn += v;
      for (int v : nda) p->need_ana += v;
    } else {
      if ((e = cudaMemset(p->d_ks, 0, sizeof(int) * nks)) || (e = cudaMemset(p->d_ja, 0, sizeof(int) * nja)))
        return bail(cuda_fail(e, "sh_plan_create: polar bounds"));
      p->need_syn = p->need_ana = (long long)p->nlm * p->nh;
    }
    p->pb.ngl = ngl;
    p->pb.ngd = ngd;
    p->pb.d_ks = p->d_ks;
    p->pb.d_ja = p->d_ja;
    p->pb.ks = p->ks.data();
    p->pb.ja = p->ja.data();
  }
  if (p->fft32) {
    e = k_fft_synth32_fam::limits(fft_smem(p));
    if (!e) e = k_fft_anal32_fam::limits(fft_smem(p));
  } else if (p->fftdf) {
    e = k_fft_synth_df_fam::limits(fft_smem(p));
    if (!e) e = k_fft_anal_df_fam::limits(fft_smem(p));
  } else {
    e = raise_smem_limit(k_fft_synth64, fft_smem(p));
    if (!e) e = raise_smem_limit(k_fft_anal64, fft_smem(p));
  }
  if (e) return bail(cuda_fail(e, "cudaFuncSetAttribute(fft)"));
  if (d.precision == SH_DF) {
    int rc = df_legendre_create(&p->dfl, p->d_P, p->d_Pn, p->d_w, p->d_wq, d.T, d.nlat, d.max_fields, p->pb,
                                p->stream);
    if (rc) return bail(rc);
    df_legendre_set_prof(p->dfl, &p->prof);
  } else if (d.precision != SH_FP64) {
    int rc = tc_legendre_create(&p->tc, p->d_P, p->d_H, p->d_w, p->d_wq, d.T, d.nlat, d.max_fields,
                                d.precision, p->pb, p->stream);
    if (rc) return bail(rc);
    tc_legendre_set_prof(p->tc, &p->prof);
    tc_legendre_set_epilogue_polls(p->tc, d.epilogue_wait_polls);
  }
  if ((e = cudaStreamSynchronize(p->stream))) return bail(cuda_fail(e, "sh_plan_create: table kernel"));
  *out = p;
  return REXI_OK;
}

extern "C" int sh_plan_destroy(sh_plan* p) {
  if (!p) return REXI_OK;
  cudaStreamSynchronize(p->stream);
  cudaFree(p->d_mu);
  cudaFree(p->d_w);
  cudaFree(p->d_wq);
  cudaFree(p->d_P);
  cudaFree(p->d_H);
  cudaFree(p->d_Pn);
  cudaFree(p->d_raw);
  cudaFree(p->d_uv);
  cudaFree(p->d_tw);
  cudaFree(p->d_tw32);
  cudaFree(p->d_twdf);
  cudaFree(p->d_F);
  tc_legendre_destroy(p->tc);
  df_legendre_destroy(p->dfl);
  cudaFree(p->d_ks);
  cudaFree(p->d_ja);
  p->prof.release();
  delete p;
  return REXI_OK;
}

extern "C" int sh_plan_get_grid(const sh_plan* p, double* mu, double* w) {
  if (!p) return fail(REXI_EINVAL, "sh_plan_get_grid: null plan");
  for (int j = 0; j < p->d.nlat; ++j) {
    if (mu) mu[j] = p->mu[j];
    if (w) w[j] = p->w[j];
  }
  return REXI_OK;
}

static int check_call(sh_plan* p, const void* a, const void* b, int nf, const char* who) {
  if (!p || !a || !b) return fail(REXI_EINVAL, "%s: null argument", who);
  if (nf < 1 || nf > p->d.max_fields) return fail(REXI_EINVAL, "%s: nfields %d outside [1, %d]", who, nf, p->d.max_fields);
  return REXI_OK;
}


// FFT segments: up to three (Fourier, grid) array pairs of nf_s fields each
static FftSegs make_segs(std::initializer_list<std::tuple<double2*, double*, int>> list) {
  FftSegs sg{};
  int k = 0, tot = 0;
  sg.start[0] = 0;
  for (const auto& e : list) {
    sg.F[k] = std::get<0>(e);
    sg.g[k] = std::get<1>(e);
    tot += std::get<2>(e);
    sg.start[++k] = tot;
  }
  for (; k < 3; ++k) sg.start[k + 1] = tot;
  return sg;
}

static void launch_fft_synth(sh_plan* p, const FftSegs& sg) {
  const int ph = p->prof.begin(4);
  const dim3 grid(p->d.nlat / 2, sg.start[3]);
  const int n = p->d.nlon;
  if (p->fft32)
    k_fft_synth32_fam::pick(n, p->fft_fixed)<<<grid, FTH, fft_smem(p), p->stream>>>(sg, p->fp, p->d_tw32, p->d.T,
                                                                                   p->d.nlat);
  else if (p->fftdf)
    k_fft_synth_df_fam::pick(n, p->fft_fixed)<<<grid, FTH, fft_smem(p), p->stream>>>(
        sg, p->fp, reinterpret_cast<const dfcx*>(p->d_twdf), p->d.T, p->d.nlat);
  else
    k_fft_synth64<<<grid, FTH, fft_smem(p), p->stream>>>(sg, p->fp, p->d_tw, p->d.T, p->d.nlat);
  p->prof.end(ph);
}
static void launch_fft_anal(sh_plan* p, const FftSegs& sg) {
  const int ph = p->prof.begin(4);
  const dim3 grid(p->d.nlat / 2, sg.start[3]);
  const int n = p->d.nlon;
  if (p->fft32)
    k_fft_anal32_fam::pick(n, p->fft_fixed)<<<grid, FTH, fft_smem(p), p->stream>>>(sg, p->fp, p->d_tw32, p->d.T,
                                                                                  p->d.nlat);
  else if (p->fftdf)
    k_fft_anal_df_fam::pick(n, p->fft_fixed)<<<grid, FTH, fft_smem(p), p->stream>>>(
        sg, p->fp, reinterpret_cast<const dfcx*>(p->d_twdf), p->d.T, p->d.nlat);
  else
    k_fft_anal64<<<grid, FTH, fft_smem(p), p->stream>>>(sg, p->fp, p->d_tw, p->d.T, p->d.nlat);
  p->prof.end(ph);
}

// Legendre stages (FP64 kernels or the tensor-core path) between spectra and Fourier arrays
static int leg_synth(sh_plan* p, const double2* spec, double2* F, int nf) {
  if (p->tc) return tc_leg_synth(p->tc, spec, F, nf, p->stream);
  if (p->dfl) return df_leg_synth(p->dfl, spec, F, nf, nullptr, nullptr, nullptr, nullptr, 0, 0.0, p->stream);
  const int ph = p->prof.begin(0);
  k_leg_synth<<<dim3(p->d.T + 1, nf, (p->nh + LTH - 1) / LTH), LTH, 0, p->stream>>>(
      p->d_P, nullptr, spec, F, nullptr, nf, p->d.T, p->d.nlat, p->nlm, p->d_ks, p->pb.ngl);
  p->prof.end(ph);
  return REXI_OK;
}
static int leg_synth_uv(sh_plan* p, const double2* psi, const double2* chi, double2* FU, double2* FV, int nf) {
  if (p->tc) return tc_leg_synth_uv(p->tc, psi, chi, FU, FV, nf, 1.0 / p->d.radius, p->stream);
  if (p->dfl) return df_leg_synth(p->dfl, nullptr, nullptr, 0, psi, chi, FU, FV, nf, 1.0 / p->d.radius, p->stream);
  const int ph = p->prof.begin(0);
  // u and v spectra (k_uv_coeffs), then one scalar synthesis of the 2 nf fields: u to FU, v to FV
  const int nlme = nlm_ext(p->d.T);
  k_uv_coeffs<<<dim3(p->d.T + 1, nf), 128, 0, p->stream>>>(psi, chi, p->d_uv, p->d_uv + (size_t)nf * nlme, p->d.T,
                                                            p->nlm, nlme, 1.0 / p->d.radius);
  k_leg_synth<<<dim3(p->d.T + 1, 2 * nf, (p->nh + LTH - 1) / LTH), LTH, 0, p->stream>>>(
      p->d_P, p->d_Pn, p->d_uv, FU, FV, nf, p->d.T, p->d.nlat, nlme, p->d_ks, p->pb.ngl);
  p->prof.end(ph);
  return REXI_OK;
}
static int leg_anal(sh_plan* p, const double2* F, double2* spec, int nf) {
  if (p->tc) return tc_leg_anal(p->tc, F, spec, nf, p->stream);
  if (p->dfl) return df_leg_anal(p->dfl, nullptr, nullptr, nullptr, nullptr, 0, F, spec, nf, 0.0, p->stream);
  const int ph = p->prof.begin(0);
  k_leg_anal<<<dim3(p->d.T + 1, nf), ATH, sizeof(double2) * 2 * p->nh, p->stream>>>(
      p->d_P, p->d_w, F, spec, p->d.T, p->d.nlat, p->nlm, p->d_ja, p->pb.ngd);
  p->prof.end(ph);
  return REXI_OK;
}
static int leg_anal_divcurl(sh_plan* p, const double2* FA, const double2* FB, double2* dv, double2* cu, int nf) {
  if (p->tc) return tc_leg_anal_divcurl(p->tc, FA, FB, dv, cu, nf, 1.0 / p->d.radius, p->stream);
  if (p->dfl) return df_leg_anal(p->dfl, FA, FB, dv, cu, nf, nullptr, nullptr, 0, 1.0 / p->d.radius, p->stream);
  const int ph = p->prof.begin(0);
  k_leg_anal_divcurl<<<dim3(p->d.T + 1, nf, (p->d.T + 1 + ATH) / ATH), ATH, sizeof(double2) * 4 * p->nh,
                       p->stream>>>(
      p->d_P, p->d_Pn, p->d_wq, FA, FB, p->d_raw, p->d.T, p->d.nlat, nlm_ext(p->d.T), p->d_ja, p->pb.ngd);
  launch_divcurl_from_p(p->d_raw, dv, cu, nf, p->d.T, 1.0 / p->d.radius, p->stream);
  p->prof.end(ph);
  return REXI_OK;
}

// Fourier work slot k (one field) of the plan's buffer of 2 max_fields slots
static double2* fslot(sh_plan* p, int k) { return p->d_F + (size_t)k * (p->d.T + 1) * p->d.nlat; }

static int launched(const char* who) {
  cudaError_t e = cudaGetLastError();
  return e ? cuda_fail(e, who) : REXI_OK;
}

extern "C" int sh_synthesis(sh_plan* p, const void* spec, void* grid, int nf) {
  int rc = check_call(p, spec, grid, nf, "sh_synthesis");
  if (rc) return rc;
  double2* F = fslot(p, 0);
  if ((rc = leg_synth(p, (const double2*)spec, F, nf))) return rc;
  launch_fft_synth(p, make_segs({{F, (double*)grid, nf}}));
  return launched("sh_synthesis");
}

extern "C" int sh_analysis(sh_plan* p, const void* grid, void* spec, int nf) {
  int rc = check_call(p, grid, spec, nf, "sh_analysis");
  if (rc) return rc;
  double2* F = fslot(p, 0);
  launch_fft_anal(p, make_segs({{F, (double*)grid, nf}}));
  if ((rc = leg_anal(p, F, (double2*)spec, nf))) return rc;
  return launched("sh_analysis");
}

extern "C" int sh_synthesis_uv(sh_plan* p, const void* psi, const void* chi, void* U, void* V, int nf) {
  int rc = check_call(p, psi, chi, nf, "sh_synthesis_uv");
  if (rc) return rc;
  if (!U || !V) return fail(REXI_EINVAL, "sh_synthesis_uv: null output");
  double2* FU = fslot(p, 0);
  double2* FV = fslot(p, p->d.max_fields);
  if ((rc = leg_synth_uv(p, (const double2*)psi, (const double2*)chi, FU, FV, nf))) return rc;
  launch_fft_synth(p, make_segs({{FU, (double*)U, nf}, {FV, (double*)V, nf}}));
  return launched("sh_synthesis_uv");
}

extern "C" int sh_analysis_divcurl(sh_plan* p, const void* A, const void* B, void* dv, void* cu, int nf) {
  int rc = check_call(p, A, B, nf, "sh_analysis_divcurl");
  if (rc) return rc;
  if (!dv || !cu) return fail(REXI_EINVAL, "sh_analysis_divcurl: null output");
  double2* FA = fslot(p, 0);
  double2* FB = fslot(p, p->d.max_fields);
  launch_fft_anal(p, make_segs({{FA, (double*)A, nf}, {FB, (double*)B, nf}}));
  if ((rc = leg_anal_divcurl(p, FA, FB, (double2*)dv, (double2*)cu, nf))) return rc;
  return launched("sh_analysis_divcurl");
}

static int check_mixed(sh_plan* p, int nf, int nfv, const char* who) {
  if (!p) return fail(REXI_EINVAL, "%s: null plan", who);
  if (nf < 1 || nfv < 1 || nf > p->d.max_fields || nfv > p->d.max_fields || nf + 2 * nfv > 2 * p->d.max_fields)
    return fail(REXI_EINVAL, "%s: %d scalar + 2 x %d vector fields exceed the plan's %d work slots", who, nf, nfv,
                2 * p->d.max_fields);
  return REXI_OK;
}

extern "C" int sh_synthesis_mixed(sh_plan* p, const void* spec, void* grid, int nf, const void* psi, const void* chi,
                                  void* U, void* V, int nfv) {
  int rc = check_mixed(p, nf, nfv, "sh_synthesis_mixed");
  if (rc) return rc;
  if (!spec || !grid || !psi || !chi || !U || !V) return fail(REXI_EINVAL, "sh_synthesis_mixed: null argument");
  double2* F = fslot(p, 0);
  double2* FU = fslot(p, nf);
  double2* FV = fslot(p, nf + nfv);
  if (p->tc) {
    if ((rc = tc_leg_synth_mixed(p->tc, (const double2*)psi, (const double2*)chi, FU, FV, nfv, (const double2*)spec, F,
                                 nf, 1.0 / p->d.radius, p->stream)))
      return rc;
  } else if (p->dfl) {
    if ((rc = df_leg_synth(p->dfl, (const double2*)spec, F, nf, (const double2*)psi, (const double2*)chi, FU, FV, nfv,
                           1.0 / p->d.radius, p->stream)))
      return rc;
  } else {
    if ((rc = leg_synth(p, (const double2*)spec, F, nf))) return rc;
    if ((rc = leg_synth_uv(p, (const double2*)psi, (const double2*)chi, FU, FV, nfv))) return rc;
  }
  launch_fft_synth(p, make_segs({{F, (double*)grid, nf}, {FU, (double*)U, nfv}, {FV, (double*)V, nfv}}));
  return launched("sh_synthesis_mixed");
}

extern "C" int sh_analysis_mixed(sh_plan* p, const void* A, const void* B, void* dv, void* cu, int nfv,
                                 const void* grid, void* spec, int nf) {
  int rc = check_mixed(p, nf, nfv, "sh_analysis_mixed");
  if (rc) return rc;
  if (!A || !B || !dv || !cu || !grid || !spec) return fail(REXI_EINVAL, "sh_analysis_mixed: null argument");
  double2* FA = fslot(p, 0);
  double2* FB = fslot(p, nfv);
  double2* FG = fslot(p, 2 * nfv);
  launch_fft_anal(p, make_segs({{FA, (double*)A, nfv}, {FB, (double*)B, nfv}, {FG, (double*)grid, nf}}));
  if (p->tc) {
    if ((rc = tc_leg_anal_mixed(p->tc, FA, FB, (double2*)dv, (double2*)cu, nfv, FG, (double2*)spec, nf,
                                1.0 / p->d.radius, p->stream)))
      return rc;
  } else if (p->dfl) {
    if ((rc = df_leg_anal(p->dfl, FA, FB, (double2*)dv, (double2*)cu, nfv, FG, (double2*)spec, nf, 1.0 / p->d.radius,
                          p->stream)))
      return rc;
  } else {
    if ((rc = leg_anal_divcurl(p, FA, FB, (double2*)dv, (double2*)cu, nfv))) return rc;
    if ((rc = leg_anal(p, FG, (double2*)spec, nf))) return rc;
  }
  return launched("sh_analysis_mixed");
}

extern "C" int sh_plan_get_table_use(const sh_plan* p, sh_table_use* u) {
  if (!p || !u) return fail(REXI_EINVAL, "sh_plan_get_table_use: null argument");
  const int T = p->d.T, nh = p->nh, ngl = p->pb.ngl, ngd = p->pb.ngd;
  u->total = (long long)p->nlm * nh;
  u->needed_synth = p->need_syn;
  u->needed_anal = p->need_ana;
  u->threshold = p->polar_thr;
  if (p->tc) {
    tc_legendre_streamed(p->tc, &u->streamed_synth, &u->streamed_anal);
  } else if (p->dfl) {
    df_legendre_streamed(p->dfl, &u->streamed_synth, &u->streamed_anal);
  } else {  // the FP64 kernels: whole warps from their group's start (rounded as they round it)
    long long s = 0, a = 0;
    for (int m = 0; m <= T; ++m) {
      const int K = T + 1 - m;
      for (int g = 0; g < ngl; ++g)
        s += (long long)std::min(32, nh - 32 * g) * (K - (p->ks[m * ngl + g] & ~1));
      for (int g = 0; g < ngd && 32 * g < K; ++g) {
        const int jb = p->ja[m * ngd + g];
        a += (long long)std::min(32, K - 32 * g) * (nh - ((nh & 3) == 0 ? jb & ~3 : jb));
      }
    }
    u->streamed_synth = s;
    u->streamed_anal = a;
  }
  return REXI_OK;
}

extern "C" int sh_plan_check(sh_plan* p) {
  if (!p) return fail(REXI_EINVAL, "sh_plan_check: null plan");
  REXI_CUDA_TRY(cudaStreamSynchronize(p->stream));
  REXI_CUDA_TRY(cudaGetLastError());
  int flag = 0;
  int rc = tc_legendre_error(p->tc, &flag);
  if (rc) return rc;
  if (flag) return fail(REXI_ETIMEOUT, "sh_plan_check: a tensor-core wait timed out (code %d)", flag);
  return REXI_OK;
}

extern "C" int sh_plan_set_profiling(sh_plan* p, int enable) {
  if (!p) return fail(REXI_EINVAL, "sh_plan_set_profiling: null plan");
  p->prof.on = enable != 0;
  return REXI_OK;
}

extern "C" int sh_plan_get_profile(sh_plan* p, double* ms, int* launches, int reset) {
  if (!p) return fail(REXI_EINVAL, "sh_plan_get_profile: null plan");
  REXI_CUDA_TRY(p->prof.collect());
  for (int k = 0; k < StageProf::NSTAGE; ++k) {
    if (ms) ms[k] = p->prof.ms[k];
    if (launches) launches[k] = p->prof.n[k];
    if (reset) {
      p->prof.ms[k] = 0.0;
      p->prof.n[k] = 0;
    }
  }
  return REXI_OK;
}
