// Allocation-free FP64 REXI step for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a host framework which owns
// all device memory through its own pool (a plugin must not grow the footprint behind the
// pool's back), real-time loops where a device allocation would synchronise the device, or
// embedded deployments that fix every byte at load time.  rexi_step_fp64_static serves
// them: the same FP64 solve and finalize kernels as rexi_step, with every table, the
// elimination scratch and the partial sums carved out of one file-scope __device__ array of
// fixed size, so the call allocates nothing.
#include <algorithm>
#include <cmath>
#include <complex>

#include "common.cuh"
#include "rexi_fp64.cuh"

namespace rexi {
namespace {

constexpr int ST_TMAX = 63;
constexpr int ST_NMAX = 1024;
constexpr int ST_KMAX = ST_TMAX + 1;
constexpr int ST_NLM = (ST_TMAX + 1) * (ST_TMAX + 2) / 2;
constexpr int ST_BLOCKS = 64;
constexpr int ST_WARPS = ST_BLOCKS * FP64_WARPS;
constexpr int ST_QMAX = 8;
constexpr int ST_TILES = ST_QMAX * 2 * (ST_TMAX + 1);

// layout of the static array (byte offsets, each 256-byte aligned)
constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_SCR = 0;
constexpr size_t SZ_SCR = sizeof(D4) * (size_t)ST_WARPS * ST_KMAX * 32;
constexpr size_t OFF_PART = al(OFF_SCR + SZ_SCR);
constexpr size_t SZ_PART = sizeof(double2) * (size_t)ST_QMAX * 3 * ST_NLM;
constexpr size_t OFF_TAB = al(OFF_PART + SZ_PART);
constexpr size_t SZ_TAB = sizeof(D4) * (size_t)ST_NLM;
constexpr size_t OFF_POLE = al(OFF_TAB + SZ_TAB);
constexpr size_t SZ_POLE = sizeof(PoleD) * (size_t)ST_NMAX;
constexpr size_t OFF_TILE = al(OFF_POLE + SZ_POLE);
constexpr size_t SZ_TILE = sizeof(Tile) * (size_t)ST_TILES;
constexpr size_t OFF_INST = al(OFF_TILE + SZ_TILE);
constexpr size_t OFF_ECUM = al(OFF_INST + sizeof(Inst));
constexpr size_t ST_BYTES = al(OFF_ECUM + 2 * sizeof(long long));

// The scratch.  In host code this name is only a stand-in for the symbol: the device
// address comes from cudaGetSymbolAddress, with the caller's device current.
static __device__ __align__(256) unsigned char g_rexi_static[ST_BYTES];

// Looks the array's address up and sets the solve kernel's shared-memory limit on every call.
// Both are cheap host calls that allocate nothing; doing them per call (instead of caching
// the address per device index) keeps the address valid after cudaDeviceReset or a new
// primary context, which reload the module.
int static_setup(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_rexi_static);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_rexi_static)");
  e = cudaFuncSetAttribute(k_rexi_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fp64_smem_bytes());
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_rexi_fp64)");
  *out = static_cast<unsigned char*>(p);
  return REXI_OK;
}

__device__ __forceinline__ double eps_dev(int n, int m) {
  if (n <= m) return 0.0;
  return sqrt((double(n) * n - double(m) * m) / (4.0 * n * n - 1.0));
}

// dt-free tables (w_n, cm_n, cp_n, q_n), poles scaled by 1/dt (z/dt, w/dt, w/z, dt/z,
// Phibar dt/z), tiles in decreasing-cost order, the instance descriptor
__global__ void k_static_setup(D4* tab, PoleD* poles, Tile* tiles, Inst* inst, long long* ecum, int T,
                               int N, int Npad, double dt, double omega, double radius, double phibar,
                               double p0, double Xc, int Q, int per, int G, double2 S0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nlm = (T + 1) * (T + 2) / 2;
  if (i < nlm) {
    int m = 0;
    while (moff(T, m + 1) <= i && m < T) ++m;
    const int n = m + (i - moff(T, m));
    const double nn1 = double(n) * (n + 1);
    const double wn = n > 0 ? 2.0 * omega * m / nn1 : 0.0;
    const double cm = (n > m && n - 1 > 0) ? 2.0 * omega * (n + 1.0) / n * eps_dev(n, m) : 0.0;
    const double cp = 2.0 * omega * n / (n + 1.0) * eps_dev(n + 1, m);
    tab[i] = D4{wn, cm, cp, nn1 / (radius * radius)};
  }
  if (i < Npad) {
    const double hpb = dt * phibar;
    if (i < N) {
      const double R = (p0 * p0 + Xc * Xc) / (2.0 * p0), mu = p0 - R;
      double s, c;
      sincospi(2.0 * (i + 0.5) / N, &s, &c);
      const double2 ring = make_double2(R * c, R * s);
      const double2 z = make_double2(ring.x + mu, ring.y);
      double es, ec;
      sincos(z.y, &es, &ec);
      const double ex = exp(z.x) / N;
      const double2 w = cmul(ring, make_double2(ex * ec, ex * es));
      const double zz = z.x * z.x + z.y * z.y;
      const double2 iz = make_double2(z.x / zz, -z.y / zz);
      poles[i] = PoleD{make_double2(z.x / dt, z.y / dt), make_double2(w.x / dt, w.y / dt), cmul(w, iz),
                       make_double2(dt * iz.x, dt * iz.y), make_double2(hpb * iz.x, hpb * iz.y)};
    } else {
      poles[i] = PoleD{make_double2(1.0 / dt, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                       make_double2(dt, 0.0), make_double2(hpb, 0.0)};
    }
  }
  if (i == 0) {
    Inst I;
    I.soff = 0;
    I.poff = 0;
    I.roff = 0;
    I.T = T;
    I.nlm = nlm;
    I.Q = Q;
    I.pole0 = 0;
    I.S0 = S0;
    *inst = I;
    ecum[0] = 0;
    ecum[1] = nlm;
  }
  if (i < 2 * (T + 1) * Q) {
    const int m = i / (2 * Q), r = i % (2 * Q);
    Tile t{};
    t.m = m;
    t.chain = r / Q;
    t.q = r % Q;
    t.g0 = t.q * per;
    t.ng = min(per, G - t.g0);
    t.heavy = 1;
    t.cost = (T + 1 - m) * t.ng;
    t.inst = 0;
    t.inst2 = t.inst3 = t.inst4 = -1;
    tiles[i] = t;
  }
}

}  // namespace
}  // namespace rexi

using namespace rexi;

extern "C" int rexi_step_fp64_static(int T, int N, double dt, double omega, double radius,
                                     double phibar, double p0, double Xc, const void* U0,
                                     void* U1, void* stream) {
  if (T < 1 || T > ST_TMAX)
    return fail(REXI_EINVAL, "rexi_step_fp64_static: T = %d outside [1, %d]", T, ST_TMAX);
  if (N < 1 || N > ST_NMAX)
    return fail(REXI_EINVAL, "rexi_step_fp64_static: N = %d outside [1, %d]", N, ST_NMAX);
  if (!(dt > 0) || !(radius > 0) || !(phibar > 0) || !(omega >= 0) || !(p0 > 0) || !(Xc > 0))
    return fail(REXI_EINVAL, "rexi_step_fp64_static: need dt, radius, phibar, p0, Xc > 0, omega >= 0");
  if (!U0 || !U1) return fail(REXI_EINVAL, "rexi_step_fp64_static: null state pointer");
  const int nlm = (T + 1) * (T + 2) / 2;
  const size_t bytes = sizeof(double2) * 3 * (size_t)nlm;
  const char* a0 = (const char*)U0;
  const char* a1 = (const char*)U1;
  if (a0 < a1 + bytes && a1 < a0 + bytes)
    return fail(REXI_EINVAL, "rexi_step_fp64_static: U0 and U1 overlap");
  unsigned char* base = nullptr;
  int rc = static_setup(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  const int Npad = (N + 31) / 32 * 32, G = Npad / 32;
  int Q = (2 * ST_WARPS + 2 * (T + 1) - 1) / (2 * (T + 1));
  Q = std::max(1, std::min(Q, std::min(G, ST_QMAX)));
  const int per = (G + Q - 1) / Q;
  Q = (G + per - 1) / per;
  const int ntiles = 2 * (T + 1) * Q;

  // S0 = sum_n w_n / z_n = sum_n (R e^{i theta_n} / N) e^{z_n} / z_n, host FP64
  std::complex<double> S0 = 0.0;
  {
    const double R = (p0 * p0 + Xc * Xc) / (2.0 * p0), mu = p0 - R;
    for (int n = 0; n < N; ++n) {
      const double th = 2.0 * M_PI * (n + 0.5) / N;
      const std::complex<double> ring = R * std::complex<double>(std::cos(th), std::sin(th));
      const std::complex<double> z = ring + mu;
      S0 += ring * std::exp(z) / double(N) / z;
    }
  }
  D4* tab = reinterpret_cast<D4*>(base + OFF_TAB);
  PoleD* poles = reinterpret_cast<PoleD*>(base + OFF_POLE);
  Tile* tiles = reinterpret_cast<Tile*>(base + OFF_TILE);
  Inst* inst = reinterpret_cast<Inst*>(base + OFF_INST);
  long long* ecum = reinterpret_cast<long long*>(base + OFF_ECUM);
  double2* part = reinterpret_cast<double2*>(base + OFF_PART);
  const int nset = std::max(std::max(nlm, Npad), ntiles);
  k_static_setup<<<(nset + 127) / 128, 128, 0, s>>>(tab, poles, tiles, inst, ecum, T, N, Npad, dt, omega,
                                                   radius, phibar, p0, Xc, Q, per, G,
                                                   make_double2(S0.real(), S0.imag()));
  Fp64Args a;
  a.U0 = (const double2*)U0;
  a.partial = part;
  a.tab = tab;
  a.poles = poles;
  a.tiles = tiles;
  a.insts = inst;
  a.scratch = reinterpret_cast<D4*>(base + OFF_SCR);
  a.ntiles = ntiles;
  a.Ttab = T;
  a.kmax = ST_KMAX;
  k_rexi_fp64<<<ST_BLOCKS, FP64_WARPS * 32, fp64_smem_bytes(), s>>>(a);
  k_rexi_finalize<false><<<(nlm + 255) / 256, 256, 0, s>>>((const double2*)U0, part, (double2*)U1, inst, ecum, 1,
                                                    (long long)nlm, phibar, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rexi_step_fp64_static launch");
  return REXI_OK;
}

extern "C" long long rexi_static_scratch_bytes(void) { return (long long)ST_BYTES; }
