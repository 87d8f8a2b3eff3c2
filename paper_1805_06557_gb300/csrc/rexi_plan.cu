// REXI plans (paper Sec. 4.2, Eq. rexi): tables, pole sets, tiles and launches.
//
// An engine owns the dt-free tables of one largest truncation, an arena of scaled pole sets
// (one per (T, N, dt, contour)), the workspace and the launch descriptors.  A launch is a
// list of instances (states), each with its own truncation and pole set, cut into tiles
// (instance, m, chain, pole range) sorted by cost; the kernels are the same for a uniform
// batch (rexi_plan) and a ragged one (rexi_ragged).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <array>
#include <map>
#include <numeric>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "rexi_fp64.cuh"
#include "rexi_mixed.cuh"

using namespace rexi;
using cplx = std::complex<double>;

namespace {

double eps_nm(int n, int m) {
  if (n <= m) return 0.0;
  return std::sqrt((double(n) * n - double(m) * m) / (4.0 * n * n - 1.0));
}

template <class P>
int dev_alloc(P** p, size_t bytes, long long* acc) {
  cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(REXI_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  *acc += (long long)bytes;
  return REXI_OK;
}

// ---- pole sets (host) -----------------------------------------------------------------
struct PoleSet {
  int T = 0, N = 0, Npad = 0, ngroups = 0, n_heavy = 0, g_light = 0, g_heavy = 0;
  int g_heavy16 = 0;        // heavy poles in 16-pole groups (tiles of state pairs); g_heavy counts 32-pole groups
  int n_pruned = 0;         // poles left out (their summed gain is <= the pruning threshold)
  double pruned_gain = 0;   // sum of the gains of the poles left out
  double dt = 0, X = 0;
  cplx S0 = 0;
  std::vector<cplx> z, w;   // internal order, padded, unscaled
  std::vector<int> heavy;
  std::vector<cplx> zp, wp; // poles left out (reported by rexi_plan_get_poles)
  std::vector<int> cls;     // per input pole: 1 heavy, 0 light, -1 pruned
  int pole0 = -1;           // position in the device arena (-1: not uploaded)
  int n_fp64 = 0, g_fp64 = 0;  // mixed plans: poles solved in FP64 (whole 32-pole groups, after heavy)
  int mrank = 0, msize = 0; // zonal-order partition (msize > 1): only the owned orders get tiles
  bool owns(int m) const { return msize <= 1 || m_pair(T, m) % msize == mrank; }
};

// Default pruning threshold of mixed plans: the summed gain of the poles left out is at most
// 1e-10, the change of the result in the energy norm relative to the state: 1/100 of the 1e-8
// relative error the mixed path is held to.  The far poles that pruning removes act on U0
// nearly as the scalar w/z, so each field changes by about the same relative amount.
constexpr double PRUNE_TAU_MIXED = 1e-10;

// Default gain above which a mixed plan solves a pole in FP64 (the FP64 kernel, FP64 partial
// sums).  The refined FP32 solve and the double-float partial slots keep about 2^-48 of the
// magnitude of a 32-pole partial sum, up to the gain sum of the group times the state: at
// gains <= 5e4 that stays within 2e-9 of the state.  Contours with a larger cancellation (T511
// at dt = 7200 s: gains up to 2e7) move their largest poles to FP64; the T255 contour at
// dt = 3600 s (largest gain 2.6e4) has none.
constexpr double FP64_TAU_MIXED = 5e4;

// Orders (and pads) the poles.  Every pole n has the gain g_n = |w_n| / dist(z_n, [-iX, iX]),
// a bound on the energy-norm size of its term w_n (z_n - dt L)^-1 U0 relative to U0 (dt L is
// skew-adjoint in the energy inner product with its spectrum in [-iX, iX]).  Pruning: the
// poles of smallest gain are left out while their summed gain stays <= prune_tau (conjugate
// pairs, which have equal gains, stay together); prune_tau = 0 selects the default (mixed:
// 1e-10, FP64: no pruning), prune_tau < 0 no pruning; mixed plans then refill the last light
// group's idle lanes with the largest pruned poles.  FP64: the kept poles in the given
// order, padding at the end.
// MIXED: light poles first, heavy ones (gain > heavy_tau, padded to whole groups) last.
int make_poleset(PoleSet& ps, int precision, int T, int N, double dt, double X, const cplx* z,
                 const cplx* w, double heavy_tau, double prune_tau, int heavy_align, double fp64_tau = 0.0) {
  ps.T = T;
  ps.N = N;
  ps.dt = dt;
  ps.X = X;
  for (int n = 0; n < N; ++n)
    if (std::abs(z[n]) < 1e-12) return fail(REXI_EINVAL, "pole %d is zero", n);
  std::vector<double> gain(N);
  for (int n = 0; n < N; ++n) {
    const double yi = std::min(std::max(z[n].imag(), -X), X);
    gain[n] = std::abs(w[n]) / std::max(std::abs(z[n] - cplx(0.0, yi)), 1e-300);
  }
  std::vector<int> by_gain(N);
  std::iota(by_gain.begin(), by_gain.end(), 0);
  std::stable_sort(by_gain.begin(), by_gain.end(), [&](int a, int b) { return gain[a] > gain[b]; });
  const double ptau = prune_tau > 0 ? prune_tau : (prune_tau == 0 && precision == REXI_MIXED ? PRUNE_TAU_MIXED : -1.0);
  int nkeep = N;
  ps.pruned_gain = 0.0;
  if (ptau >= 0) {
    double tail = 0.0;  // summed gain of by_gain[nkeep..N)
    while (nkeep > 1 && tail + gain[by_gain[nkeep - 1]] <= ptau) tail += gain[by_gain[--nkeep]];
    while (nkeep < N && nkeep > 0 && gain[by_gain[nkeep]] == gain[by_gain[nkeep - 1]])  // keep pairs whole
      tail -= gain[by_gain[nkeep++]];
    if (precision == REXI_MIXED) {
      // light poles are solved 32 to a warp: the largest pruned poles fill the last light
      // group's idle lanes (conjugate pairs whole), at no cost and with a smaller pruned gain
      const double tau = heavy_tau < 0 ? 1e-3 : heavy_tau;
      int nh = 0;
      for (int i = 0; i < nkeep; ++i) nh += gain[by_gain[i]] > tau;
      const int nh16 = std::min((nh + heavy_align - 1) / heavy_align * heavy_align, nkeep);
      int room = nh16 < nkeep ? (nkeep - nh16 + 31) / 32 * 32 - (nkeep - nh16) : 0;
      while (room > 0 && nkeep < N) {
        const int take = nkeep + 1 < N && gain[by_gain[nkeep + 1]] == gain[by_gain[nkeep]] ? 2 : 1;
        if (take > room) break;
        nkeep += take;
        room -= take;
      }
    }
    for (int i = N - 1; i >= nkeep; --i) ps.pruned_gain += gain[by_gain[i]];  // smallest first
  }
  std::vector<char> keep(N, 0);
  for (int i = 0; i < nkeep; ++i) keep[by_gain[i]] = 1;
  ps.n_pruned = N - nkeep;
  ps.zp.clear();
  ps.wp.clear();
  for (int n = 0; n < N; ++n)
    if (!keep[n]) {
      ps.zp.push_back(z[n]);
      ps.wp.push_back(w[n]);
    }
  cplx s = 0, comp = 0;  // S0 = sum w/z over the kept poles, compensated
  for (int n = 0; n < N; ++n) {
    if (!keep[n]) continue;
    const cplx yv = w[n] / z[n] - comp;
    const cplx t = s + yv;
    comp = (t - s) - yv;
    s = t;
  }
  ps.S0 = s;
  ps.Npad = (nkeep + 31) / 32 * 32;
  ps.ngroups = ps.Npad / 32;
  const int npad = ps.Npad - nkeep;
  ps.z.clear();
  ps.w.clear();
  ps.heavy.clear();
  auto push = [&](cplx zz, cplx ww, int h) {
    ps.z.push_back(zz);
    ps.w.push_back(ww);
    ps.heavy.push_back(h);
  };
  auto all_heavy = [&]() {
    for (int n = 0; n < N; ++n)
      if (keep[n]) push(z[n], w[n], 1);
    for (int i = 0; i < npad; ++i) push(1.0, 0.0, 1);
    ps.n_heavy = nkeep;
    ps.cls.assign(N, -1);
    for (int n = 0; n < N; ++n)
      if (keep[n]) ps.cls[n] = 1;
    ps.g_light = 0;
    ps.g_heavy = ps.ngroups;
    ps.g_heavy16 = 2 * ps.ngroups;
    return REXI_OK;
  };
  if (precision == REXI_FP64) return all_heavy();
  const double tau = heavy_tau < 0 ? 1e-3 : heavy_tau;
  // FP64 class: the poles of largest gain above fp64_tau, rounded up to whole 32-pole groups
  // with the next-largest gains (conjugate pairs, of equal gain, stay together)
  const double t64 = fp64_tau > 0 ? fp64_tau : FP64_TAU_MIXED;
  int n64 = 0;
  for (int i = 0; i < nkeep; ++i)
    if (gain[by_gain[i]] > t64) ++n64;
  if (n64 > 0) n64 = std::min((n64 + 31) / 32 * 32, nkeep);
  int nh = 0;
  for (int i = n64; i < nkeep; ++i)
    if (gain[by_gain[i]] > tau) ++nh;
  // heavy class: the next poles of largest gain, rounded up to heavy_align (16 where tiles of
  // state pairs take 16 poles per half-warp, 32 where most tiles carry one state) with the
  // next-largest gains; the pole array pads it to 32 for tiles of one state
  const int nh16 = std::min((nh + heavy_align - 1) / heavy_align * heavy_align, nkeep - n64);
  if (n64 == 0 && nh16 == nkeep && nkeep % 16 != 0) return all_heavy();  // everything heavy, padding at the end
  const int nl = nkeep - n64 - nh16, lpad = (nl + 31) / 32 * 32, hpad = (nh16 + 31) / 32 * 32;
  ps.Npad = lpad + hpad + n64;
  ps.ngroups = ps.Npad / 32;
  ps.z.clear();
  ps.w.clear();
  ps.heavy.clear();
  std::vector<int> hv(N, 0);  // 1 heavy, 2 FP64
  for (int i = 0; i < n64; ++i) hv[by_gain[i]] = 2;
  for (int i = n64; i < n64 + nh16; ++i) hv[by_gain[i]] = 1;
  for (int n = 0; n < N; ++n)
    if (keep[n] && !hv[n]) push(z[n], w[n], 0);
  for (int i = nl; i < lpad; ++i) push(1.0, 0.0, 0);
  for (int n = 0; n < N; ++n)
    if (hv[n] == 1) push(z[n], w[n], 1);
  for (int i = nh16; i < hpad; ++i) push(1.0, 0.0, 1);
  for (int n = 0; n < N; ++n)
    if (hv[n] == 2) push(z[n], w[n], 2);
  ps.n_heavy = nh16;
  ps.n_fp64 = n64;
  ps.g_fp64 = n64 / 32;
  ps.cls.assign(N, -1);
  for (int n = 0; n < N; ++n)
    if (keep[n]) ps.cls[n] = hv[n];
  ps.g_light = lpad / 32;
  ps.g_heavy = hpad / 32;
  ps.g_heavy16 = nh16 / 16;
  return REXI_OK;
}

int make_poleset_from_contour(PoleSet& ps, int precision, int T, int N, double dt, double X, double p0,
                              double Xc, double heavy_tau, double prune_tau, int heavy_align,
                              double fp64_tau = 0.0) {
  std::vector<double> zz(2 * N), ww(2 * N);
  int rc = rexi_coeffs(N, p0, Xc, 0, zz.data(), ww.data());
  if (rc) return rc;
  std::vector<cplx> z(N), w(N);
  for (int n = 0; n < N; ++n) {
    z[n] = cplx(zz[2 * n], zz[2 * n + 1]);
    w[n] = cplx(ww[2 * n], ww[2 * n + 1]);
  }
  return make_poleset(ps, precision, T, N, dt, X, z.data(), w.data(), heavy_tau, prune_tau, heavy_align, fp64_tau);
}

int ranges_used(int G, int Q) {
  if (G == 0) return 0;
  const int per = (G + Q - 1) / Q;
  return (G + per - 1) / per;
}

}  // namespace

// ---- engine -----------------------------------------------------------------------------
struct Engine {
  int precision = 0, Ttab = 0, device = 0, nsm = 0, kmax = 0, nseg_max = 0;
  double omega = 0, radius = 0, phibar = 0;
  cudaStream_t stream = nullptr;
  // mixed plans: the light kernel runs on `side`, forked after the right-hand-side pre-pass and
  // joined before the finalize, beside the heavy kernels on `stream` (the two write disjoint
  // partial slots and scratch regions)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  D4* tab64 = nullptr;
  float4* tab32 = nullptr;
  TabDF* tabdf = nullptr;
  PoleD* p64 = nullptr;
  PoleF* p32 = nullptr;
  PoleDF* pdf = nullptr;
  int pole_cap = 0, pole_used = 0;
  double2* partial = nullptr;
  size_t partial_cap = 0;
  // mixed plans with poles solved in FP64: their partial sums and the FP64 kernel's scratch,
  // allocated when a pole set first needs them
  double2* partial64 = nullptr;
  size_t partial64_cap = 0;
  D4* scratch64 = nullptr;
  void* rhs = nullptr;
  size_t rhs_cap = 0;  // elements
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  int grid_fp64 = 0, grid_light = 0, grid_heavy = 0, grid_heavy2 = 0;  // heavy: tiles of one state, of state pairs
  int max_q = 0;  // cap on pole ranges per class and instance (0: none)
  long long workspace = 0;
  // profiling
  int profiling = 0;
  struct Pend {
    cudaEvent_t a, b;
    int kid;
    cudaStream_t st;  // the stream the pair is recorded on
  };
  std::vector<Pend> pending;
  std::vector<cudaEvent_t> event_pool;
  double prof_ms[REXI_NKERNELS] = {0};
  int prof_n[REXI_NKERNELS] = {0};
};

// Device copy of one launch: instances, tiles (light then heavy), element prefix sums.
struct LaunchSet {
  Inst* insts = nullptr;
  Tile* tiles = nullptr;
  long long* ecum = nullptr;
  int ninst = 0, ntiles = 0, ntiles_light = 0, ntiles_quad = 0, ntiles_pair = 0;
  long long total = 0, partial_elems = 0;
  int ntiles_fp64 = 0;           // the last tiles: FP64 class of mixed plans
  long long partial64_elems = 0;
};

namespace {

void free_launch(LaunchSet& L) {
  cudaFree(L.insts);
  cudaFree(L.tiles);
  cudaFree(L.ecum);
  L = LaunchSet();
}

void engine_free(Engine& e) {
  if (e.stream || e.tab64) cudaStreamSynchronize(e.stream);
  for (void* p : {(void*)e.tab64, (void*)e.tab32, (void*)e.tabdf, (void*)e.p64, (void*)e.p32, (void*)e.pdf,
                  (void*)e.partial, (void*)e.rhs, (void*)e.scratch, (void*)e.partial64, (void*)e.scratch64})
    cudaFree(p);
  for (auto& q : e.pending) {
    cudaEventDestroy(q.a);
    cudaEventDestroy(q.b);
  }
  for (auto ev : e.event_pool) cudaEventDestroy(ev);
  e.pending.clear();
  e.event_pool.clear();
  if (e.side) {
    cudaStreamSynchronize(e.side);
    cudaStreamDestroy(e.side);
  }
  if (e.fork) cudaEventDestroy(e.fork);
  if (e.join) cudaEventDestroy(e.join);
  e.side = nullptr;
  e.fork = e.join = nullptr;
}

size_t rhs32_bytes(size_t elems) { return (sizeof(Rhs32) * elems + 255) / 256 * 256; }

// tables for truncation Ttab (dt-free), persistent grids, scratch, pole arena, workspace
int engine_init(Engine& e, int precision, int Ttab, double omega, double radius, double phibar,
                cudaStream_t stream, int pole_cap, size_t partial_cap, size_t rhs_cap) {
  e.precision = precision;
  e.Ttab = Ttab;
  e.omega = omega;
  e.radius = radius;
  e.phibar = phibar;
  e.stream = stream;
  if (precision == REXI_MIXED) {
    cudaError_t es;
    if ((es = cudaStreamCreateWithFlags(&e.side, cudaStreamNonBlocking)) ||
        (es = cudaEventCreateWithFlags(&e.fork, cudaEventDisableTiming)) ||
        (es = cudaEventCreateWithFlags(&e.join, cudaEventDisableTiming)))
      return cuda_fail(es, "engine side stream");
  }
  e.kmax = Ttab + 1;
  e.nseg_max = (e.kmax + LSEG - 1) / LSEG;
  if (cudaGetDevice(&e.device) != cudaSuccess) return fail(REXI_ECUDA, "no CUDA device");
  cudaDeviceGetAttribute(&e.nsm, cudaDevAttrMultiProcessorCount, e.device);
  const int nlm = (Ttab + 1) * (Ttab + 2) / 2;
  std::vector<D4> t64(nlm);
  std::vector<float4> t32(nlm);
  std::vector<TabDF> tdf(nlm);
  for (int m = 0; m <= Ttab; ++m)
    for (int n = m; n <= Ttab; ++n) {
      const int idx = moff(Ttab, m) + (n - m);
      const double nn1 = double(n) * (n + 1);
      const double wn = n > 0 ? 2.0 * omega * m / nn1 : 0.0;
      const double cm = (n > m && n - 1 > 0) ? 2.0 * omega * (n + 1.0) / n * eps_nm(n, m) : 0.0;
      const double cp = 2.0 * omega * n / (n + 1.0) * eps_nm(n + 1, m);
      const double q = nn1 / (radius * radius);
      t64[idx] = D4{wn, cm, cp, q};
      t32[idx] = make_float4((float)wn, (float)cm, (float)cp, (float)q);
      tdf[idx] = TabDF{split4(wn, cm), split4(cp, q)};
    }
  long long& ws = e.workspace;
  int rc;
  cudaError_t ce;
  if ((rc = dev_alloc(&e.tab64, sizeof(D4) * nlm, &ws))) return rc;
  if ((ce = cudaMemcpy(e.tab64, t64.data(), sizeof(D4) * nlm, cudaMemcpyHostToDevice)))
    return cuda_fail(ce, "cudaMemcpy(tables)");
  e.pole_cap = pole_cap;
  if ((rc = dev_alloc(&e.p64, sizeof(PoleD) * pole_cap, &ws))) return rc;
  if (precision == REXI_FP64) {
    const size_t smem = fp64_smem_bytes();
    if ((ce = cudaFuncSetAttribute(k_rexi_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return cuda_fail(ce, "cudaFuncSetAttribute(k_rexi_fp64)");
    int per_sm = 0;
    if ((ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rexi_fp64, FP64_WARPS * 32, smem)))
      return cuda_fail(ce, "occupancy(k_rexi_fp64)");
    e.grid_fp64 = e.nsm * std::max(1, std::min(per_sm, 2));
    e.scratch_bytes = sizeof(D4) * (size_t)e.grid_fp64 * FP64_WARPS * e.kmax * 32;
  } else {
    if ((rc = dev_alloc(&e.tab32, sizeof(float4) * nlm, &ws))) return rc;
    if ((rc = dev_alloc(&e.tabdf, sizeof(TabDF) * nlm, &ws))) return rc;
    if ((ce = cudaMemcpy(e.tab32, t32.data(), sizeof(float4) * nlm, cudaMemcpyHostToDevice)) ||
        (ce = cudaMemcpy(e.tabdf, tdf.data(), sizeof(TabDF) * nlm, cudaMemcpyHostToDevice)))
      return cuda_fail(ce, "cudaMemcpy(tables)");
    if ((rc = dev_alloc(&e.p32, sizeof(PoleF) * pole_cap, &ws))) return rc;
    if ((rc = dev_alloc(&e.pdf, sizeof(PoleDF) * pole_cap, &ws))) return rc;
    const size_t hsm = heavy_smem_bytes<1>(), hsm2 = heavy_smem_bytes<2>();
    if ((ce = cudaFuncSetAttribute(k_rexi_heavy<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm)) ||
        (ce = cudaFuncSetAttribute(k_rexi_heavy<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm2)) ||
        (ce = cudaFuncSetAttribute(k_rexi_heavy<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm2)))
      return cuda_fail(ce, "cudaFuncSetAttribute(k_rexi_heavy)");
    int per_l = 0, per_h = 0;
    if ((ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_l, k_rexi_light, MIX_WARPS * 32, 0)))
      return cuda_fail(ce, "occupancy(k_rexi_light)");
    int per_h2 = 0;
    int per_h2b = 0;
    if ((ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_h, k_rexi_heavy<1, false>, MIX_WARPS * 32, hsm)) ||
        (ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_h2, k_rexi_heavy<2, false>, MIX_WARPS * 32, hsm2)) ||
        (ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_h2b, k_rexi_heavy<2, true>, MIX_WARPS * 32, hsm2)))
      return cuda_fail(ce, "occupancy(k_rexi_heavy)");
    per_h2 = std::min(per_h2, per_h2b);  // one grid size serves both tile forms of state pairs
    {  // the FP64 class of a mixed plan runs on the FP64 kernel
      const size_t smem = fp64_smem_bytes();
      int per64 = 0;
      if ((ce = cudaFuncSetAttribute(k_rexi_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ||
          (ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per64, k_rexi_fp64, FP64_WARPS * 32, smem)))
        return cuda_fail(ce, "k_rexi_fp64 (FP64 class)");
      e.grid_fp64 = e.nsm * std::max(1, std::min(per64, 2));
    }
    e.grid_light = e.nsm * std::max(1, std::min(per_l, 4));
    e.grid_heavy = e.nsm * std::max(1, std::min(per_h, 6));
    e.grid_heavy2 = e.nsm * std::max(1, std::min(per_h2, 4));
    e.scratch_bytes = sizeof(float4) * (size_t)e.grid_light * MIX_WARPS * light_ckpt_f4_per_warp(e.nseg_max) +
                      sizeof(float2) * (size_t)std::max(e.grid_heavy, e.grid_heavy2) * MIX_WARPS *
                          heavy_scratch_f2_per_warp(e.kmax);
    e.rhs_cap = rhs_cap;
    if ((rc = dev_alloc((char**)&e.rhs, rhs32_bytes(rhs_cap) + sizeof(RhsDF) * rhs_cap, &ws))) return rc;
  }
  if ((rc = dev_alloc((char**)&e.scratch, e.scratch_bytes, &ws))) return rc;
  e.partial_cap = partial_cap;
  if ((rc = dev_alloc(&e.partial, sizeof(double2) * partial_cap, &ws))) return rc;
  return REXI_OK;
}

// Appends a pole set to the arena (scaled by 1/dt: z' = z/dt, w' = w/dt, w/z, 1/z', Phibar/z').
// The FP64-class buffers of a mixed engine, grown to `p64_elems` partial-sum entries (after the
// stream's queued work, which may still use the old ones); the scratch is made once.
int engine_ensure_fp64(Engine& e, size_t p64_elems) {
  cudaError_t ce;
  if (p64_elems > e.partial64_cap) {
    if ((ce = cudaStreamSynchronize(e.stream))) return cuda_fail(ce, "FP64 class: stream");
    cudaFree(e.partial64);
    e.partial64 = nullptr;
    e.partial64_cap = 0;
    if ((ce = cudaMalloc(&e.partial64, sizeof(double2) * p64_elems))) {
      cudaGetLastError();
      return fail(REXI_ENOMEM, "FP64 class: partial sums (%zu entries)", p64_elems);
    }
    e.partial64_cap = p64_elems;
    e.workspace += (long long)(sizeof(double2) * p64_elems);
  }
  if (p64_elems > 0 && !e.scratch64) {
    const size_t bytes = sizeof(D4) * (size_t)e.grid_fp64 * FP64_WARPS * e.kmax * 32;
    if ((ce = cudaMalloc(&e.scratch64, bytes))) {
      cudaGetLastError();
      return fail(REXI_ENOMEM, "FP64 class: elimination scratch");
    }
    e.workspace += (long long)bytes;
  }
  return REXI_OK;
}

// the device forms of a pole set: FP64, FP32 and double-float constants of every (padded) pole
void pack_poles(const Engine& e, const PoleSet& ps, PoleD* pd, PoleF* pf, PoleDF* pq) {
  for (int i = 0; i < ps.Npad; ++i) {
    const cplx z = ps.z[i], w = ps.w[i];
    const cplx zs = z / ps.dt, ws = w / ps.dt, wz = w / z, iz = 1.0 / zs, gz = e.phibar / zs;
    auto D = [](cplx c) { return make_double2(c.real(), c.imag()); };
    auto F = [](cplx c) { return make_float2((float)c.real(), (float)c.imag()); };
    pd[i] = PoleD{D(zs), D(ws), D(wz), D(iz), D(gz)};
    pf[i] = PoleF{F(zs), F(ws), F(wz), F(iz), F(gz)};
    pq[i] = PoleDF{split4(zs.real(), zs.imag()), split4(iz.real(), iz.imag()), split4(gz.real(), gz.imag()),
                   split4(ws.real(), ws.imag()), split4(wz.real(), wz.imag())};
  }
}

int engine_upload_poles(Engine& e, PoleSet& ps) {
  if (e.pole_used + ps.Npad > e.pole_cap)
    return fail(REXI_EBUSY, "pole arena full (%d + %d > %d)", e.pole_used, ps.Npad, e.pole_cap);
  std::vector<PoleD> pd(ps.Npad);
  std::vector<PoleF> pf(ps.Npad);
  std::vector<PoleDF> pq(ps.Npad);
  pack_poles(e, ps, pd.data(), pf.data(), pq.data());
  cudaError_t ce = cudaMemcpy(e.p64 + e.pole_used, pd.data(), sizeof(PoleD) * ps.Npad, cudaMemcpyHostToDevice);
  if (!ce && e.p32) ce = cudaMemcpy(e.p32 + e.pole_used, pf.data(), sizeof(PoleF) * ps.Npad, cudaMemcpyHostToDevice);
  if (!ce && e.pdf) ce = cudaMemcpy(e.pdf + e.pole_used, pq.data(), sizeof(PoleDF) * ps.Npad, cudaMemcpyHostToDevice);
  if (ce) return cuda_fail(ce, "cudaMemcpy(poles)");
  ps.pole0 = e.pole_used;
  e.pole_used += ps.Npad;
  return REXI_OK;
}

struct InstReq {
  const PoleSet* ps;
  long long soff;
};

// Builds the host launch description: per-instance descriptors (partial / rhs offsets),
// tiles sorted by cost (light first, then heavy), element prefix sums.  Pole groups are cut
// into ranges so that the launch has about qmul tiles per resident warp.
struct LaunchExtra {  // the FP64 class of mixed plans
  int ntiles_fp64 = 0;
  long long partial64_elems = 0;
};

void build_launch(const Engine& e, const std::vector<InstReq>& req, std::vector<Inst>& insts,
                  std::vector<Tile>& tiles, std::vector<long long>& ecum, int& ntiles_light,
                  long long& partial_elems, int& ntiles_quad, int& ntiles_pair, int qmul = 4,
                  LaunchExtra* extra = nullptr) {
  insts.clear();
  tiles.clear();
  ecum.clear();
  // Heavy tiles of instances with the same pole set (same truncation, same poles): instances are
  // paired, and pairs grouped by two into one tile (one pair per half-warp).  group[i] lists the
  // (up to four) instances led by i; led[i] = 1 when i leads a group, 2 when i joined one.
  std::vector<std::array<int, 4>> group(req.size(), std::array<int, 4>{-1, -1, -1, -1});
  std::vector<char> led(req.size(), 0), in_quad(req.size(), 0);
  if (e.precision == REXI_MIXED) {
    std::map<const PoleSet*, std::vector<int>> by_set;  // instances of each pole set, in order
    for (size_t i = 0; i < req.size(); ++i) by_set[req[i].ps].push_back((int)i);
    for (auto& kv : by_set) {
      const std::vector<int>& v = kv.second;
      size_t k = 0;
      while (k + 1 < v.size()) {  // a pair is left: four together if there are four, else a lone pair
        const size_t take = v.size() - k >= 4 ? 4 : 2;
        std::array<int, 4> gr{-1, -1, -1, -1};
        for (size_t j = 0; j < take; ++j) gr[j] = v[k + j];
        group[v[k]] = gr;
        led[v[k]] = 1;
        for (size_t j = 1; j < take; ++j) led[v[k + j]] = 2;
        for (size_t j = 0; j < take; ++j) in_quad[v[k + j]] = take == 4;
        k += take;
      }
      // a last odd instance keeps tiles of one state
    }
  }
  // units = tiles per pole range: (m, chain) pairs; a light tile holds both chains of its m
  long long units = 0, units_h = 0;
  for (size_t i = 0; i < req.size(); ++i) {
    units += 2LL * (req[i].ps->T + 1);
    if (led[i] != 2) units_h += 2LL * (req[i].ps->T + 1);
  }
  units = std::max<long long>(units, 1);
  units_h = std::max<long long>(units_h, 1);
  const long long units_l = std::max<long long>(units / 2, 1);
  int Ql_glob = 1, Qh_glob = 1;
  if (e.precision == REXI_FP64) {
    Qh_glob = (int)std::max<long long>(1, (qmul * (long long)e.grid_fp64 * FP64_WARPS + units - 1) / units);
  } else {
    Ql_glob = (int)std::max<long long>(1, (qmul * (long long)e.grid_light * MIX_WARPS + units_l - 1) / units_l);
    Qh_glob = (int)std::max<long long>(1, (qmul * (long long)e.grid_heavy * MIX_WARPS + units_h - 1) / units_h);
  }
  if (e.max_q > 0) {
    Ql_glob = std::min(Ql_glob, e.max_q);
    Qh_glob = std::min(Qh_glob, e.max_q);
  }
  long long poff = 0, roff = 0, ec = 0, poff64 = 0;
  std::vector<Tile> light, heavy, heavyQ, heavyP, fp64t;
  for (size_t i = 0; i < req.size(); ++i) {
    const PoleSet& ps = *req[i].ps;
    const int T = ps.T, nlm = (T + 1) * (T + 2) / 2;
    // heavy work of an instance grouped by four runs on 16-pole groups (tiles of two pairs); a
    // lone pair and a single instance run on 32-pole groups
    const int lead = led[i] == 1 ? (int)i : -1;
    const bool quad = in_quad[i];
    const int Gh = quad ? ps.g_heavy16 : ps.g_heavy;
    const int Ql = ps.g_light ? std::min(Ql_glob, ps.g_light) : 1;
    const int Qh = Gh ? std::min(Qh_glob, Gh) : 1;
    const int ql = ranges_used(ps.g_light, Ql), qh = ranges_used(Gh, Qh);
    Inst I;
    I.soff = req[i].soff;
    I.poff = poff;
    I.roff = roff;
    I.T = T;
    I.nlm = nlm;
    I.Q = ql + qh;
    I.pole0 = ps.pole0;
    I.S0 = make_double2(ps.S0.real(), ps.S0.imag());
    I.mrank = ps.mrank;
    I.msize = ps.msize;
    // FP64 class: one 32-pole group per range (its own FP64 partial slots)
    const int q64 = e.precision == REXI_MIXED ? ps.g_fp64 : 0;
    I.poff64 = poff64;
    I.Q64 = q64;
    for (int g = 0; g < q64; ++g)
      for (int m = 0; m <= T; ++m)
        for (int c = 0; c < 2 && ps.owns(m); ++c)
          fp64t.push_back(Tile{m, c, ps.g_light + ps.g_heavy + g, 1, g, 2, (T + 1 - m) * 8, (int)i, -1, -1, -1});
    poff64 += (long long)q64 * 3 * nlm;
    insts.push_back(I);
    ecum.push_back(ec);
    auto add = [&](int gbase, int G, int Q, int qbase, int hv, std::vector<Tile>& out) {
      if (G == 0) return;
      const int per = (G + Q - 1) / Q;
      int q = qbase;
      for (int g = 0; g < G; g += per, ++q) {
        const int ng = std::min(per, G - g);
        for (int m = 0; m <= T; ++m) {
          if (!ps.owns(m)) continue;
          if (!hv && e.precision != REXI_FP64) {  // light: both chains in one tile (chain = 2)
            out.push_back(Tile{m, 2, gbase + g, ng, q, 0, 2 * (T + 1 - m) * ng, (int)i, -1, -1, -1});
            continue;
          }
          for (int c = 0; c < 2; ++c) {
            const int w = (hv && e.precision != REXI_FP64) ? 3 : 1;
            out.push_back(Tile{m, c, gbase + g, ng, q, hv, (T + 1 - m) * ng * w, (int)i, -1, -1, -1});
          }
        }
      }
    };
    add(0, ps.g_light, Ql, 0, 0, light);
    if (!led[i]) {
      add(ps.g_light, ps.g_heavy, Qh, ql, 1, heavy);
    } else if (lead >= 0) {  // tiles of the group led by i
      const std::array<int, 4>& gr = group[i];
      const int per = (Gh + Qh - 1) / Qh;
      int q = ql;
      for (int g = 0; g < Gh; g += per, ++q) {
        const int ng = std::min(per, Gh - g);
        for (int m = 0; m <= T; ++m)
          for (int c = 0; c < 2 && ps.owns(m); ++c) {
            if (quad)  // g0 = pole offset, ng = 16-pole groups
              heavyQ.push_back(Tile{m, c, 32 * ps.g_light + 16 * g, ng, q, 1, (T + 1 - m) * ng * 6, gr[0], gr[1],
                                    gr[2], gr[3]});
            else  // lone pair: g0, ng in 32-pole groups
              heavyP.push_back(Tile{m, c, ps.g_light + g, ng, q, 1, (T + 1 - m) * ng * 6, gr[0], gr[1], -1, -1});
          }
      }
    }
    poff += (long long)I.Q * 3 * nlm;
    roff += nlm;
    ec += nlm;
  }
  ecum.push_back(ec);
  auto bycost = [](const Tile& a, const Tile& b) { return a.cost > b.cost; };
  std::stable_sort(light.begin(), light.end(), bycost);
  std::stable_sort(heavyQ.begin(), heavyQ.end(), bycost);
  std::stable_sort(heavyP.begin(), heavyP.end(), bycost);
  std::stable_sort(heavy.begin(), heavy.end(), bycost);
  std::stable_sort(fp64t.begin(), fp64t.end(), bycost);
  ntiles_light = (int)light.size();
  ntiles_quad = (int)heavyQ.size();
  ntiles_pair = (int)heavyP.size();
  tiles = light;  // light, then heavy tiles of two pairs, of one pair, of one state
  tiles.insert(tiles.end(), heavyQ.begin(), heavyQ.end());
  tiles.insert(tiles.end(), heavyP.begin(), heavyP.end());
  tiles.insert(tiles.end(), heavy.begin(), heavy.end());
  tiles.insert(tiles.end(), fp64t.begin(), fp64t.end());  // last: the FP64 class
  partial_elems = poff;
  if (extra) {
    extra->ntiles_fp64 = (int)fp64t.size();
    extra->partial64_elems = poff64;
  }
}

int upload_launch(LaunchSet& L, const std::vector<Inst>& insts, const std::vector<Tile>& tiles,
                  const std::vector<long long>& ecum, int ntiles_light, int ntiles_quad, int ntiles_pair,
                  long long partial_elems, const LaunchExtra& extra = LaunchExtra()) {
  free_launch(L);
  cudaError_t ce;
  if ((ce = cudaMalloc(&L.insts, sizeof(Inst) * std::max<size_t>(insts.size(), 1))) ||
      (ce = cudaMalloc(&L.tiles, sizeof(Tile) * std::max<size_t>(tiles.size(), 1))) ||
      (ce = cudaMalloc(&L.ecum, sizeof(long long) * ecum.size()))) {
    cudaGetLastError();
    return fail(REXI_ENOMEM, "launch descriptors: cudaMalloc failed");
  }
  if ((ce = cudaMemcpy(L.insts, insts.data(), sizeof(Inst) * insts.size(), cudaMemcpyHostToDevice)) ||
      (ce = cudaMemcpy(L.tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice)) ||
      (ce = cudaMemcpy(L.ecum, ecum.data(), sizeof(long long) * ecum.size(), cudaMemcpyHostToDevice)))
    return cuda_fail(ce, "cudaMemcpy(launch descriptors)");
  L.ninst = (int)insts.size();
  L.ntiles = (int)tiles.size();
  L.ntiles_light = ntiles_light;
  L.ntiles_quad = ntiles_quad;
  L.ntiles_pair = ntiles_pair;
  L.total = ecum.back();
  L.partial_elems = partial_elems;
  L.ntiles_fp64 = extra.ntiles_fp64;
  L.partial64_elems = extra.partial64_elems;
  return REXI_OK;
}

cudaEvent_t take_event(Engine& e) {
  if (!e.event_pool.empty()) {
    cudaEvent_t ev = e.event_pool.back();
    e.event_pool.pop_back();
    return ev;
  }
  cudaEvent_t ev;
  cudaEventCreate(&ev);
  return ev;
}
int prof_begin(Engine& e, int kid, cudaStream_t st = nullptr) {
  if (!e.profiling) return -1;
  Engine::Pend q{take_event(e), take_event(e), kid};
  q.st = st ? st : e.stream;
  cudaEventRecord(q.a, q.st);
  e.pending.push_back(q);
  return (int)e.pending.size() - 1;
}
void prof_end(Engine& e, int h) {
  if (h >= 0) cudaEventRecord(e.pending[h].b, e.pending[h].st);
}

// Launches one REXI step of the launch set.  No allocation.
int engine_launch(Engine& e, const LaunchSet& L, const double2* U0, double2* U1) {
  if (L.partial_elems > (long long)e.partial_cap) return fail(REXI_EINVAL, "internal: partial buffer too small");
  if (e.precision == REXI_FP64) {
    Fp64Args a;
    a.U0 = U0;
    a.partial = e.partial;
    a.tab = e.tab64;
    a.poles = e.p64;
    a.tiles = L.tiles;
    a.insts = L.insts;
    a.scratch = (D4*)e.scratch;
    a.ntiles = L.ntiles;
    a.Ttab = e.Ttab;
    a.kmax = e.kmax;
    const int h = prof_begin(e, 1);
    k_rexi_fp64<<<e.grid_fp64, FP64_WARPS * 32, fp64_smem_bytes(), e.stream>>>(a);
    prof_end(e, h);
  } else {
    if (L.total > (long long)e.rhs_cap) return fail(REXI_EINVAL, "internal: rhs buffer too small");
    Rhs32* r32 = (Rhs32*)e.rhs;
    RhsDF* rdf = (RhsDF*)((char*)e.rhs + rhs32_bytes(e.rhs_cap));
    int h = prof_begin(e, 0);
    k_mixed_rhs<<<(unsigned)((L.total + 255) / 256), 256, 0, e.stream>>>(U0, e.tab64, e.Ttab, r32, rdf, L.insts,
                                                                         L.ecum, L.ninst, L.total);
    prof_end(e, h);
    MixedArgs a;
    a.U0 = U0;
    a.partial = e.partial;
    a.tab32 = e.tab32;
    a.tabdf = e.tabdf;
    a.p32 = e.p32;
    a.p64 = e.p64;
    a.pdf = e.pdf;
    a.tiles = L.tiles;
    a.insts = L.insts;
    a.rhs32 = r32;
    a.rhsdf = rdf;
    a.scratch = e.scratch;
    a.ntiles_light = L.ntiles_light;
    a.ntiles_heavy = L.ntiles - L.ntiles_light - L.ntiles_fp64;
    a.Ttab = e.Ttab;
    a.kmax = e.kmax;
    a.nseg_max = e.nseg_max;
    a.warps_light = e.grid_light * MIX_WARPS;
    const int nq = L.ntiles_quad, np = L.ntiles_pair, n1 = a.ntiles_heavy - nq - np;
    // light beside heavy, when the heavy tiles do not fill the heavy grid's resident warps (a
    // latency-bound launch, e.g. one state): the light blocks then run in the room the idle
    // heavy warps leave.  A batched launch fills every SM with heavy warps, so light would only
    // share the tail, and the order in which the two become resident is not fixed: it stays
    // after heavy on the plan stream.
    const bool both = a.ntiles_light && a.ntiles_heavy && e.side &&
                      a.ntiles_heavy < (long long)std::max(e.grid_heavy, e.grid_heavy2) * MIX_WARPS;
    cudaStream_t ls = both ? e.side : e.stream;
    if (both) {
      cudaEventRecord(e.fork, e.stream);
      cudaStreamWaitEvent(e.side, e.fork, 0);
    }
    int t0 = L.ntiles_light;
    if (nq) {  // tiles of two state pairs (half-warps, 16-pole groups)
      h = prof_begin(e, 3);
      k_rexi_heavy<2, true><<<e.grid_heavy2, MIX_WARPS * 32, heavy_smem_bytes<2>(), e.stream>>>(a, t0, nq);
      prof_end(e, h);
      t0 += nq;
    }
    if (np) {  // tiles of one state pair (32-pole groups)
      h = prof_begin(e, 3);
      k_rexi_heavy<2, false><<<e.grid_heavy2, MIX_WARPS * 32, heavy_smem_bytes<2>(), e.stream>>>(a, t0, np);
      prof_end(e, h);
      t0 += np;
    }
    if (n1) {
      h = prof_begin(e, 3);
      k_rexi_heavy<1, false><<<e.grid_heavy, MIX_WARPS * 32, heavy_smem_bytes<1>(), e.stream>>>(a, t0, n1);
      prof_end(e, h);
    }
    if (L.ntiles_fp64) {  // the FP64 class: the FP64 kernel on its tiles, FP64 partial slots
      if ((long long)e.partial64_cap < L.partial64_elems || !e.scratch64)
        return fail(REXI_EINVAL, "internal: FP64-class buffers too small");
      Fp64Args f;
      f.U0 = U0;
      f.partial = e.partial64;
      f.tab = e.tab64;
      f.poles = e.p64;
      f.tiles = L.tiles + (L.ntiles - L.ntiles_fp64);
      f.insts = L.insts;
      f.scratch = e.scratch64;
      f.ntiles = L.ntiles_fp64;
      f.Ttab = e.Ttab;
      f.kmax = e.kmax;
      f.alt = 1;
      h = prof_begin(e, 1);
      k_rexi_fp64<<<e.grid_fp64, FP64_WARPS * 32, fp64_smem_bytes(), e.stream>>>(f);
      prof_end(e, h);
    }
    if (a.ntiles_light) {
      h = prof_begin(e, 2, ls);
      k_rexi_light<<<e.grid_light, MIX_WARPS * 32, 0, ls>>>(a);
      prof_end(e, h);
    }
    if (both) {
      cudaEventRecord(e.join, e.side);
      cudaStreamWaitEvent(e.stream, e.join, 0);
    }
  }
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return cuda_fail(ce, "solve kernel launch");
  const int hf = prof_begin(e, 4);
  if (e.precision == REXI_FP64)
    k_rexi_finalize<false><<<(unsigned)((L.total + 255) / 256), 256, 0, e.stream>>>(U0, e.partial, U1, L.insts,
                                                                                   L.ecum, L.ninst, L.total, e.phibar,
                                                                                   nullptr);
  else
    k_rexi_finalize<true><<<(unsigned)((L.total + 255) / 256), 256, 0, e.stream>>>(U0, e.partial, U1, L.insts,
                                                                                  L.ecum, L.ninst, L.total, e.phibar,
                                                                                  e.partial64);
  prof_end(e, hf);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return cuda_fail(ce, "finalize kernel launch");
  return REXI_OK;
}

int engine_profile(Engine& e, double* ms, int* launches, int reset) {
  REXI_CUDA_TRY(cudaStreamSynchronize(e.stream));
  for (auto& q : e.pending) {
    float t = 0.f;
    REXI_CUDA_TRY(cudaEventElapsedTime(&t, q.a, q.b));
    e.prof_ms[q.kid] += t;
    e.prof_n[q.kid] += 1;
    e.event_pool.push_back(q.a);
    e.event_pool.push_back(q.b);
  }
  e.pending.clear();
  for (int i = 0; i < REXI_NKERNELS; ++i) {
    if (ms) ms[i] = e.prof_ms[i];
    if (launches) launches[i] = e.prof_n[i];
    if (reset) {
      e.prof_ms[i] = 0;
      e.prof_n[i] = 0;
    }
  }
  return REXI_OK;
}

bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + bytes && y < x + bytes;
}

}  // namespace

// =========================================================================================
// Uniform plans: one pole set, batches of states with the same truncation
// =========================================================================================
struct rexi_plan {
  rexi_plan_desc d{};
  Engine e;
  PoleSet ps;
  int nlm = 0;
  std::map<int, LaunchSet> launches;  // by batch size
  double2* stage_in = nullptr;
  double2* stage_out = nullptr;
  // rexi_step_host_async (set up on its first call): two device staging slots, a copy-in and a
  // copy-out stream, and per slot the events that order the copies and the step
  struct Async {
    bool ready = false;
    double2* in[2] = {};
    double2* out[2] = {};
    cudaStream_t cin = nullptr, cout = nullptr;
    cudaEvent_t ev_in[2] = {}, ev_comp[2] = {}, ev_out[2] = {};
    long long calls = 0;
  } as;
};

// Creates the asynchronous host-step resources; every event is recorded once on the plan
// stream so that the first waits on them are satisfied.
static int async_setup(rexi_plan* p) {
  rexi_plan::Async& a = p->as;
  if (a.ready) return REXI_OK;
  const size_t sb = sizeof(double2) * 3 * (size_t)p->nlm * p->d.max_batch;
  int rc;
  for (int s = 0; s < 2; ++s) {
    if ((rc = dev_alloc(&a.in[s], sb, &p->e.workspace)) || (rc = dev_alloc(&a.out[s], sb, &p->e.workspace)))
      return rc;
  }
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&a.cin, cudaStreamNonBlocking)) ||
      (e = cudaStreamCreateWithFlags(&a.cout, cudaStreamNonBlocking)))
    return cuda_fail(e, "rexi_step_host_async: stream creation");
  for (int s = 0; s < 2; ++s) {
    for (cudaEvent_t* ev : {&a.ev_in[s], &a.ev_comp[s], &a.ev_out[s]}) {
      if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)))
        return cuda_fail(e, "rexi_step_host_async: event creation");
      if ((e = cudaEventRecord(*ev, p->e.stream))) return cuda_fail(e, "rexi_step_host_async: event record");
    }
  }
  a.ready = true;
  return REXI_OK;
}

static void async_free(rexi_plan* p) {
  rexi_plan::Async& a = p->as;
  if (a.ready) cudaStreamSynchronize(p->e.stream);  // a step may still write a slot
  if (a.cin) cudaStreamSynchronize(a.cin);
  if (a.cout) cudaStreamSynchronize(a.cout);
  for (int s = 0; s < 2; ++s) {
    cudaFree(a.in[s]);
    cudaFree(a.out[s]);
    for (cudaEvent_t ev : {a.ev_in[s], a.ev_comp[s], a.ev_out[s]})
      if (ev) cudaEventDestroy(ev);
  }
  if (a.cin) cudaStreamDestroy(a.cin);
  if (a.cout) cudaStreamDestroy(a.cout);
  a = rexi_plan::Async();
}

extern "C" int rexi_plan_create(const rexi_plan_desc* desc, rexi_plan** out) {
  if (!desc || !out) return fail(REXI_EINVAL, "rexi_plan_create: null argument");
  *out = nullptr;
  const rexi_plan_desc& d = *desc;
  if (d.T < 1 || d.T > 1023) return fail(REXI_EINVAL, "T must be in [1, 1023] (got %d)", d.T);
  if (d.N < 1 || d.N > 8192) return fail(REXI_EINVAL, "N must be in [1, 8192] (got %d)", d.N);
  if (!(d.dt > 0) || !(d.radius > 0) || !(d.phibar > 0) || !(d.omega >= 0))
    return fail(REXI_EINVAL, "need dt > 0, radius > 0, phibar > 0, omega >= 0");
  if (d.precision != REXI_FP64 && d.precision != REXI_MIXED)
    return fail(REXI_EINVAL, "precision must be REXI_FP64 or REXI_MIXED");
  if (d.max_batch < 1) return fail(REXI_EINVAL, "max_batch must be >= 1");
  if ((d.z == nullptr) != (d.w == nullptr)) return fail(REXI_EINVAL, "give both z and w or neither");
  if (!d.z && (!(d.p0 > 0) || !(d.Xc > 0))) return fail(REXI_EINVAL, "need p0 > 0 and Xc > 0");
  if (d.part_mode != REXI_PART_NONE && d.part_mode != REXI_PART_POLES && d.part_mode != REXI_PART_M)
    return fail(REXI_EINVAL, "part_mode must be REXI_PART_NONE, REXI_PART_POLES or REXI_PART_M");
  if (d.part_mode != REXI_PART_NONE && (d.part_size < 1 || d.part_rank < 0 || d.part_rank >= d.part_size))
    return fail(REXI_EINVAL, "partition rank %d of %d", d.part_rank, d.part_size);
  rexi_plan* p = new rexi_plan();
  p->d = d;
  p->d.z = p->d.w = nullptr;
  p->nlm = (d.T + 1) * (d.T + 2) / 2;
  auto bail = [&](int code) {
    rexi_plan_destroy(p);
    return code;
  };
  const double X = rexi_spectrum_bound(d.T, d.dt, d.omega, d.radius, d.phibar);
  // batches of four or more run heavy tiles of two state pairs on 16-pole groups
  const int halign = d.max_batch >= 4 ? 16 : 32;
  int rc;
  std::vector<cplx> z(d.N), w(d.N);
  if (d.z) {
    for (int n = 0; n < d.N; ++n) {
      z[n] = cplx(d.z[2 * n], d.z[2 * n + 1]);
      w[n] = cplx(d.w[2 * n], d.w[2 * n + 1]);
    }
  } else {
    std::vector<double> zz(2 * (size_t)d.N), ww(2 * (size_t)d.N);
    if ((rc = rexi_coeffs(d.N, d.p0, d.Xc, 0, zz.data(), ww.data()))) return bail(rc);
    for (int n = 0; n < d.N; ++n) {
      z[n] = cplx(zz[2 * n], zz[2 * n + 1]);
      w[n] = cplx(ww[2 * n], ww[2 * n + 1]);
    }
  }
  double prune_tau = d.prune_tau;
  if (d.part_mode == REXI_PART_POLES && d.part_size > 1) {
    // this rank's conjugate pairs; each rank prunes within 1/part_size of the pruning budget, so
    // the poles left out over all ranks still sum to at most the plan's threshold
    std::vector<int> own(d.N);
    rexi_partition(REXI_PART_POLES, d.T, d.N, d.part_rank, d.part_size, own.data());
    std::vector<cplx> zs, ws;
    for (int n = 0; n < d.N; ++n)
      if (own[n]) {
        zs.push_back(z[n]);
        ws.push_back(w[n]);
      }
    if (zs.empty()) return bail(fail(REXI_EINVAL, "partition rank %d of %d owns no pole of %d", d.part_rank,
                                     d.part_size, d.N));
    z.swap(zs);
    w.swap(ws);
    p->d.N = (int)z.size();
    const double base = prune_tau > 0 ? prune_tau : (prune_tau == 0 && d.precision == REXI_MIXED ? 1e-10 : -1.0);
    prune_tau = base > 0 ? base / d.part_size : base;
  }
  rc = make_poleset(p->ps, d.precision, d.T, p->d.N, d.dt, X, z.data(), w.data(), d.heavy_tau, prune_tau, halign,
                    d.fp64_tau);
  if (rc) return bail(rc);
  if (d.part_mode == REXI_PART_M && d.part_size > 1) {
    p->ps.mrank = d.part_rank;
    p->ps.msize = d.part_size;
  }
  rc = engine_init(p->e, d.precision, d.T, d.omega, d.radius, d.phibar, (cudaStream_t)d.stream, p->ps.Npad, 0,
                   (size_t)p->nlm * d.max_batch);
  if (rc) return bail(rc);
  // largest partial-sum footprint over the batch sizes a call may use
  size_t maxp = 0, maxp64 = 0;
  for (int B = 1; B <= d.max_batch; ++B) {
    std::vector<InstReq> req;
    for (int b = 0; b < B; ++b) req.push_back(InstReq{&p->ps, (long long)b * 3 * p->nlm});
    std::vector<Inst> I;
    std::vector<Tile> Tl;
    std::vector<long long> ec;
    int ntl, ntq, ntp;
    long long pe;
    LaunchExtra x;
    build_launch(p->e, req, I, Tl, ec, ntl, pe, ntq, ntp, 4, &x);
    maxp = std::max(maxp, (size_t)pe);
    maxp64 = std::max(maxp64, (size_t)x.partial64_elems);
  }
  if (maxp64 > 0 && (rc = engine_ensure_fp64(p->e, maxp64))) return bail(rc);
  cudaFree(p->e.partial);
  p->e.partial = nullptr;
  p->e.partial_cap = maxp;
  if ((rc = dev_alloc(&p->e.partial, sizeof(double2) * maxp, &p->e.workspace))) return bail(rc);
  if ((rc = engine_upload_poles(p->e, p->ps))) return bail(rc);
  const size_t sb = sizeof(double2) * 3 * (size_t)p->nlm * d.max_batch;
  if ((rc = dev_alloc(&p->stage_in, sb, &p->e.workspace))) return bail(rc);
  if ((rc = dev_alloc(&p->stage_out, sb, &p->e.workspace))) return bail(rc);
  *out = p;
  return REXI_OK;
}

extern "C" int rexi_plan_destroy(rexi_plan* p) {
  if (!p) return REXI_OK;
  async_free(p);
  engine_free(p->e);
  for (auto& kv : p->launches) free_launch(kv.second);
  cudaFree(p->stage_in);
  cudaFree(p->stage_out);
  delete p;
  return REXI_OK;
}

static int plan_launchset(rexi_plan* p, int B, LaunchSet** out) {
  auto it = p->launches.find(B);
  if (it == p->launches.end()) {
    std::vector<InstReq> req;
    for (int b = 0; b < B; ++b) req.push_back(InstReq{&p->ps, (long long)b * 3 * p->nlm});
    std::vector<Inst> I;
    std::vector<Tile> Tl;
    std::vector<long long> ec;
    int ntl, ntq, ntp;
    long long pe;
    LaunchExtra x;
    build_launch(p->e, req, I, Tl, ec, ntl, pe, ntq, ntp, 4, &x);
    LaunchSet L;
    int rc = upload_launch(L, I, Tl, ec, ntl, ntq, ntp, pe, x);
    if (rc) {
      free_launch(L);
      return rc;
    }
    it = p->launches.emplace(B, L).first;
  }
  *out = &it->second;
  return REXI_OK;
}

extern "C" int rexi_step(rexi_plan* p, const void* U0, void* U1, int batch) {
  if (!p || !U0 || !U1) return fail(REXI_EINVAL, "rexi_step: null argument");
  if (batch < 1 || batch > p->d.max_batch)
    return fail(REXI_EINVAL, "rexi_step: batch %d outside [1, %d]", batch, p->d.max_batch);
  if (overlaps(U0, U1, sizeof(double2) * 3 * (size_t)p->nlm * batch))
    return fail(REXI_EINVAL, "rexi_step: U0 and U1 overlap");
  LaunchSet* L = nullptr;
  int rc = plan_launchset(p, batch, &L);
  if (rc) return rc;
  return engine_launch(p->e, *L, (const double2*)U0, (double2*)U1);
}

// Device address of page-locked host memory mapped into the device's address space (pinned
// allocations are, with unified addressing), else null.
static void* mapped_host(const void* h) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

extern "C" int rexi_step_host(rexi_plan* p, const double* U0, double* U1, int batch) {
  if (!p || !U0 || !U1) return fail(REXI_EINVAL, "rexi_step_host: null argument");
  if (batch < 1 || batch > p->d.max_batch)
    return fail(REXI_EINVAL, "rexi_step_host: batch %d outside [1, %d]", batch, p->d.max_batch);
  const size_t bytes = sizeof(double2) * 3 * (size_t)p->nlm * batch;
  if (p->d.precision == REXI_MIXED) {
    // a mixed step reads U0 once (the right-hand-side pre-pass, and Phi in the finalize) and
    // writes U1 once (the finalize): with mapped pinned buffers those kernels use the host
    // memory in place over the host link, without the staging copies
    const void* d0 = mapped_host(U0);
    void* d1 = mapped_host(U1);
    if (d0 && d1) {
      int rc = rexi_step(p, d0, d1, batch);
      if (rc) return rc;
      REXI_CUDA_TRY(cudaStreamSynchronize(p->e.stream));
      return REXI_OK;
    }
  }
  REXI_CUDA_TRY(cudaMemcpyAsync(p->stage_in, U0, bytes, cudaMemcpyHostToDevice, p->e.stream));
  int rc = rexi_step(p, p->stage_in, p->stage_out, batch);
  if (rc) return rc;
  REXI_CUDA_TRY(cudaMemcpyAsync(U1, p->stage_out, bytes, cudaMemcpyDeviceToHost, p->e.stream));
  REXI_CUDA_TRY(cudaStreamSynchronize(p->e.stream));
  return REXI_OK;
}

// Pipelined host steps: call i uses staging slot s = i mod 2.  Its input copy (copy-in stream)
// waits until the step of call i - 2 has read slot s; its step (plan stream) waits for that
// copy and for the output copy of call i - 2 to have read slot s; its output copy (copy-out
// stream) waits for its step.  So the copies of calls i + 1 and i - 1 run on the copy engines
// while the kernels of call i run.
extern "C" int rexi_step_host_async(rexi_plan* p, const double* U0, double* U1, int batch) {
  if (!p || !U0 || !U1) return fail(REXI_EINVAL, "rexi_step_host_async: null argument");
  if (batch < 1 || batch > p->d.max_batch)
    return fail(REXI_EINVAL, "rexi_step_host_async: batch %d outside [1, %d]", batch, p->d.max_batch);
  const size_t bytes = sizeof(double2) * 3 * (size_t)p->nlm * batch;
  if (overlaps(U0, U1, bytes)) return fail(REXI_EINVAL, "rexi_step_host_async: U0 and U1 overlap");
  int rc = async_setup(p);
  if (rc) return rc;
  rexi_plan::Async& a = p->as;
  const int s = (int)(a.calls & 1);
  cudaStream_t st = p->e.stream;
  REXI_CUDA_TRY(cudaStreamWaitEvent(a.cin, a.ev_comp[s], 0));
  REXI_CUDA_TRY(cudaMemcpyAsync(a.in[s], U0, bytes, cudaMemcpyHostToDevice, a.cin));
  REXI_CUDA_TRY(cudaEventRecord(a.ev_in[s], a.cin));
  REXI_CUDA_TRY(cudaStreamWaitEvent(st, a.ev_in[s], 0));
  REXI_CUDA_TRY(cudaStreamWaitEvent(st, a.ev_out[s], 0));
  if ((rc = rexi_step(p, a.in[s], a.out[s], batch))) return rc;
  REXI_CUDA_TRY(cudaEventRecord(a.ev_comp[s], st));
  REXI_CUDA_TRY(cudaStreamWaitEvent(a.cout, a.ev_comp[s], 0));
  REXI_CUDA_TRY(cudaMemcpyAsync(U1, a.out[s], bytes, cudaMemcpyDeviceToHost, a.cout));
  REXI_CUDA_TRY(cudaEventRecord(a.ev_out[s], a.cout));
  ++a.calls;
  return REXI_OK;
}

extern "C" int rexi_sync(rexi_plan* p) {
  if (!p) return fail(REXI_EINVAL, "rexi_sync: null plan");
  if (p->as.ready) {
    REXI_CUDA_TRY(cudaStreamSynchronize(p->as.cin));
    REXI_CUDA_TRY(cudaStreamSynchronize(p->as.cout));
  }
  REXI_CUDA_TRY(cudaStreamSynchronize(p->e.stream));
  REXI_CUDA_TRY(cudaGetLastError());
  return REXI_OK;
}

extern "C" int rexi_plan_get_info(const rexi_plan* p, rexi_plan_info* info) {
  if (!p || !info) return fail(REXI_EINVAL, "rexi_plan_get_info: null argument");
  std::memset(info, 0, sizeof(*info));
  info->T = p->ps.T;
  info->N = p->ps.N;
  info->nlm = p->nlm;
  info->precision = p->e.precision;
  info->n_heavy = p->ps.n_heavy;
  info->n_groups = p->ps.ngroups;
  if (!p->launches.empty()) {
    info->n_tiles = p->launches.begin()->second.ntiles;
    info->q_slots = (int)(p->launches.begin()->second.partial_elems / (3 * (long long)p->nlm));
  }
  info->grid_fp64 = p->e.grid_fp64;
  info->grid_light = p->e.grid_light;
  info->grid_heavy = p->e.grid_heavy;
  info->workspace_bytes = p->e.workspace;
  info->s0_re = p->ps.S0.real();
  info->s0_im = p->ps.S0.imag();
  info->X = p->ps.X;
  info->n_pruned = p->ps.n_pruned;
  info->pruned_gain = p->ps.pruned_gain;
  info->n_fp64 = p->ps.n_fp64;
  return REXI_OK;
}

extern "C" int rexi_plan_get_poles(const rexi_plan* p, double* z, double* w, int* heavy) {
  if (!p) return fail(REXI_EINVAL, "rexi_plan_get_poles: null plan");
  int k = 0;
  for (int i = 0; i < p->ps.Npad && k < p->ps.N; ++i) {
    if (std::abs(p->ps.w[i]) == 0.0 && p->ps.z[i] == cplx(1.0, 0.0)) continue;  // padding
    if (z) {
      z[2 * k] = p->ps.z[i].real();
      z[2 * k + 1] = p->ps.z[i].imag();
    }
    if (w) {
      w[2 * k] = p->ps.w[i].real();
      w[2 * k + 1] = p->ps.w[i].imag();
    }
    if (heavy) heavy[k] = p->ps.heavy[i];
    ++k;
  }
  for (size_t i = 0; i < p->ps.zp.size() && k < p->ps.N; ++i, ++k) {  // poles left out
    if (z) {
      z[2 * k] = p->ps.zp[i].real();
      z[2 * k + 1] = p->ps.zp[i].imag();
    }
    if (w) {
      w[2 * k] = p->ps.wp[i].real();
      w[2 * k + 1] = p->ps.wp[i].imag();
    }
    if (heavy) heavy[k] = -1;
  }
  return REXI_OK;
}

extern "C" int rexi_partition(int mode, int T, int N, int rank, int size, int* owned) {
  if (!owned || size < 1 || rank < 0 || rank >= size || T < 1 || N < 1)
    return fail(REXI_EINVAL, "rexi_partition: bad arguments");
  if (mode == REXI_PART_POLES) {
    // conjugate pair k = {k, N - 1 - k} (the middle pole of an odd N alone), dealt round robin
    for (int n = 0; n < N; ++n) owned[n] = std::min(n, N - 1 - n) % size == rank;
  } else if (mode == REXI_PART_M) {
    for (int m = 0; m <= T; ++m) owned[m] = m_pair(T, m) % size == rank;
  } else {
    return fail(REXI_EINVAL, "rexi_partition: mode must be REXI_PART_POLES or REXI_PART_M");
  }
  return REXI_OK;
}

extern "C" int rexi_select_poles(int precision, int N, const double* z, const double* w, double X,
                                 double heavy_tau, double prune_tau, int heavy_align, int* cls,
                                 double* pruned_gain) {
  if (N < 1 || !z || !w || !cls) return fail(REXI_EINVAL, "rexi_select_poles: need N >= 1 and z, w, cls");
  if (precision != REXI_FP64 && precision != REXI_MIXED)
    return fail(REXI_EINVAL, "rexi_select_poles: unknown precision %d", precision);
  if (heavy_align != 16 && heavy_align != 32)
    return fail(REXI_EINVAL, "rexi_select_poles: heavy_align must be 16 or 32");
  if (!(X >= 0.0) || !std::isfinite(X)) return fail(REXI_EINVAL, "rexi_select_poles: need finite X >= 0");
  std::vector<cplx> zz(N), ww(N);
  for (int n = 0; n < N; ++n) {
    zz[n] = cplx(z[2 * n], z[2 * n + 1]);
    ww[n] = cplx(w[2 * n], w[2 * n + 1]);
  }
  PoleSet ps;
  const int rc = make_poleset(ps, precision, 0, N, 0.0, X, zz.data(), ww.data(), heavy_tau, prune_tau, heavy_align);
  if (rc) return rc;
  std::copy(ps.cls.begin(), ps.cls.end(), cls);
  if (pruned_gain) *pruned_gain = ps.pruned_gain;
  return REXI_OK;
}

extern "C" int rexi_plan_set_profiling(rexi_plan* p, int enable) {
  if (!p) return fail(REXI_EINVAL, "rexi_plan_set_profiling: null plan");
  p->e.profiling = enable ? 1 : 0;
  return REXI_OK;
}

extern "C" int rexi_plan_get_profile(rexi_plan* p, double* ms, int* launches, int reset) {
  if (!p) return fail(REXI_EINVAL, "rexi_plan_get_profile: null plan");
  return engine_profile(p->e, ms, launches, reset);
}

// =========================================================================================
// Ragged plans: instances of different truncation, time step and pole count in one launch
// =========================================================================================
struct rexi_ragged {
  rexi_ragged_desc d{};
  Engine e;
  std::map<std::tuple<int, int, double, double, double>, PoleSet> cache;
  std::vector<const PoleSet*> cur;
  std::vector<long long> soff;
  long long extent = 0;  // complex elements spanned by the states in U0 / U1
  LaunchSet L;  // device descriptors, kept between sets and grown when a set needs more
  size_t cap_inst = 0, cap_tiles = 0, cap_ecum = 0;
  int qmul = 4;
  // captured graph of one step for fixed (U0, U1)
  cudaGraphExec_t gexec = nullptr;
  const void* g_u0 = nullptr;
  void* g_u1 = nullptr;
  // pinned host packets for the asynchronous uploads of a set (new poles and descriptors),
  // used alternately; a packet is rewritten once the copies from its previous use have run
  struct Packet {
    unsigned char* h = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
  } pk[2];
  int pk_i = 0;
  std::vector<PoleSet*> fresh;  // pole sets of the current set call not yet uploaded
  std::vector<std::tuple<int, int, double, double, double>> fresh_keys;
};

// A set call that fails after reserving new pole sets drops them from the cache (they were
// never uploaded, so a later call must not find them).
static void drop_fresh(rexi_ragged* r) {
  for (auto& k : r->fresh_keys) r->cache.erase(k);
  r->fresh.clear();
  r->fresh_keys.clear();
}

extern "C" int rexi_ragged_create(const rexi_ragged_desc* desc, rexi_ragged** out) {
  if (!desc || !out) return fail(REXI_EINVAL, "rexi_ragged_create: null argument");
  *out = nullptr;
  const rexi_ragged_desc& d = *desc;
  if (d.Tmax < 1 || d.Tmax > 1023) return fail(REXI_EINVAL, "rexi_ragged_create: Tmax must be in [1, 1023]");
  if (d.max_inst < 1 || d.max_poles < 32 || d.max_elems < 3)
    return fail(REXI_EINVAL, "rexi_ragged_create: need max_inst >= 1, max_poles >= 32, max_elems >= 3");
  if (d.precision != REXI_FP64 && d.precision != REXI_MIXED)
    return fail(REXI_EINVAL, "rexi_ragged_create: bad precision");
  if (!(d.radius > 0) || !(d.phibar > 0) || !(d.omega >= 0))
    return fail(REXI_EINVAL, "rexi_ragged_create: bad physical constants");
  rexi_ragged* r = new rexi_ragged();
  r->d = d;
  // partial sums: at most RAGGED_MAXQ pole ranges per class and instance
  const int RAGGED_MAXQ = 2;
  const size_t partial_cap = (size_t)3 * d.max_elems * 2 * RAGGED_MAXQ;
  r->e.max_q = RAGGED_MAXQ;
  int rc = engine_init(r->e, d.precision, d.Tmax, d.omega, d.radius, d.phibar, (cudaStream_t)d.stream, d.max_poles,
                       partial_cap, (size_t)d.max_elems);
  if (rc) {
    rexi_ragged_destroy(r);
    return rc;
  }
  *out = r;
  return REXI_OK;
}

extern "C" int rexi_ragged_destroy(rexi_ragged* r) {
  if (!r) return REXI_OK;
  cudaStreamSynchronize(r->e.stream);
  if (r->gexec) cudaGraphExecDestroy(r->gexec);
  engine_free(r->e);
  free_launch(r->L);
  for (auto& q : r->pk) {
    cudaFreeHost(q.h);
    if (q.ev) cudaEventDestroy(q.ev);
  }
  delete r;
  return REXI_OK;
}

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Rebuilds the tiles of the current instances and uploads them, with the pole sets in r->fresh,
// asynchronously on the plan stream: everything is packed into a pinned host packet and copied
// by cudaMemcpyAsync, so the copies run in stream order after the work already queued (a tick
// in flight keeps its descriptors and poles until it has finished) and the host does not wait
// for the device.  Only growing a device buffer synchronises the stream.
static int ragged_rebuild(rexi_ragged* r) {
  std::vector<InstReq> req;
  for (size_t i = 0; i < r->cur.size(); ++i) req.push_back(InstReq{r->cur[i], r->soff[i]});
  std::vector<Inst> I;
  std::vector<Tile> Tl;
  std::vector<long long> ec;
  int ntl, ntq, ntp;
  long long pe;
  LaunchExtra x;
  build_launch(r->e, req, I, Tl, ec, ntl, pe, ntq, ntp, r->qmul, &x);
  if (pe > (long long)r->e.partial_cap) return fail(REXI_EBUSY, "rexi_ragged: partial-sum workspace exceeded");
  Engine& e = r->e;
  int rce = x.partial64_elems > 0 ? engine_ensure_fp64(e, (size_t)x.partial64_elems) : REXI_OK;
  if (rce) return rce;
  cudaError_t ce;
  // device descriptors: grow (after the stream's queued work) when this set needs more room
  if (I.size() > r->cap_inst || Tl.size() > r->cap_tiles || ec.size() > r->cap_ecum) {
    if ((ce = cudaStreamSynchronize(e.stream))) return cuda_fail(ce, "rexi_ragged: stream");
    free_launch(r->L);
    r->cap_inst = std::max(I.size(), r->cap_inst) * 3 / 2 + 16;
    r->cap_tiles = std::max(Tl.size(), r->cap_tiles) * 3 / 2 + 64;
    r->cap_ecum = std::max(ec.size(), r->cap_ecum) * 3 / 2 + 16;
    if ((ce = cudaMalloc(&r->L.insts, sizeof(Inst) * r->cap_inst)) ||
        (ce = cudaMalloc(&r->L.tiles, sizeof(Tile) * r->cap_tiles)) ||
        (ce = cudaMalloc(&r->L.ecum, sizeof(long long) * r->cap_ecum))) {
      cudaGetLastError();
      r->cap_inst = r->cap_tiles = r->cap_ecum = 0;
      return fail(REXI_ENOMEM, "rexi_ragged: launch descriptors: cudaMalloc failed");
    }
  }
  // the packet: [poles of each fresh set: PoleD, PoleF, PoleDF][insts][tiles][ecum]
  size_t bytes = 0;
  for (const PoleSet* ps : r->fresh)
    bytes += al256(sizeof(PoleD) * ps->Npad) + al256(sizeof(PoleF) * ps->Npad) + al256(sizeof(PoleDF) * ps->Npad);
  const size_t o_inst = bytes, o_tile = o_inst + al256(sizeof(Inst) * I.size()),
               o_ecum = o_tile + al256(sizeof(Tile) * Tl.size());
  bytes = o_ecum + al256(sizeof(long long) * ec.size());
  rexi_ragged::Packet& q = r->pk[r->pk_i];
  r->pk_i ^= 1;
  if (q.ev && (ce = cudaEventSynchronize(q.ev))) return cuda_fail(ce, "rexi_ragged: packet event");
  if (!q.ev && (ce = cudaEventCreateWithFlags(&q.ev, cudaEventDisableTiming)))
    return cuda_fail(ce, "rexi_ragged: cudaEventCreate");
  if (bytes > q.cap) {
    cudaFreeHost(q.h);
    q.h = nullptr;
    q.cap = 0;
    if ((ce = cudaMallocHost((void**)&q.h, bytes * 3 / 2))) {
      cudaGetLastError();
      return fail(REXI_ENOMEM, "rexi_ragged: pinned upload buffer");
    }
    q.cap = bytes * 3 / 2;
  }
  size_t o = 0;
  for (const PoleSet* ps : r->fresh) {
    PoleD* pd = reinterpret_cast<PoleD*>(q.h + o);
    o += al256(sizeof(PoleD) * ps->Npad);
    PoleF* pf = reinterpret_cast<PoleF*>(q.h + o);
    o += al256(sizeof(PoleF) * ps->Npad);
    PoleDF* pq = reinterpret_cast<PoleDF*>(q.h + o);
    o += al256(sizeof(PoleDF) * ps->Npad);
    pack_poles(e, *ps, pd, pf, pq);
    const int p0 = ps->pole0;
    ce = cudaMemcpyAsync(e.p64 + p0, pd, sizeof(PoleD) * ps->Npad, cudaMemcpyHostToDevice, e.stream);
    if (!ce && e.p32) ce = cudaMemcpyAsync(e.p32 + p0, pf, sizeof(PoleF) * ps->Npad, cudaMemcpyHostToDevice, e.stream);
    if (!ce && e.pdf) ce = cudaMemcpyAsync(e.pdf + p0, pq, sizeof(PoleDF) * ps->Npad, cudaMemcpyHostToDevice, e.stream);
    if (ce) return cuda_fail(ce, "rexi_ragged: cudaMemcpyAsync(poles)");
  }
  r->fresh.clear();
  memcpy(q.h + o_inst, I.data(), sizeof(Inst) * I.size());
  memcpy(q.h + o_tile, Tl.data(), sizeof(Tile) * Tl.size());
  memcpy(q.h + o_ecum, ec.data(), sizeof(long long) * ec.size());
  if ((ce = cudaMemcpyAsync(r->L.insts, q.h + o_inst, sizeof(Inst) * I.size(), cudaMemcpyHostToDevice, e.stream)) ||
      (ce = cudaMemcpyAsync(r->L.tiles, q.h + o_tile, sizeof(Tile) * Tl.size(), cudaMemcpyHostToDevice, e.stream)) ||
      (ce = cudaMemcpyAsync(r->L.ecum, q.h + o_ecum, sizeof(long long) * ec.size(), cudaMemcpyHostToDevice,
                            e.stream)) ||
      (ce = cudaEventRecord(q.ev, e.stream)))
    return cuda_fail(ce, "rexi_ragged: cudaMemcpyAsync(launch descriptors)");
  r->L.ninst = (int)I.size();
  r->L.ntiles = (int)Tl.size();
  r->L.ntiles_light = ntl;
  r->L.ntiles_quad = ntq;
  r->L.ntiles_pair = ntp;
  r->L.total = ec.back();
  r->L.partial_elems = pe;
  r->L.ntiles_fp64 = x.ntiles_fp64;
  r->L.partial64_elems = x.partial64_elems;
  return REXI_OK;
}

extern "C" int rexi_ragged_set(rexi_ragged* r, int ninst, const rexi_instance* inst) {
  if (!r || !inst || ninst < 1) return fail(REXI_EINVAL, "rexi_ragged_set: bad arguments");
  if (ninst > r->d.max_inst)
    return fail(REXI_EBUSY, "rexi_ragged_set: %d instances > max_inst %d", ninst, r->d.max_inst);
  long long elems = 0;
  for (int i = 0; i < ninst; ++i) {
    const rexi_instance& q = inst[i];
    if (q.T < 1 || q.T > r->d.Tmax)
      return fail(REXI_EINVAL, "rexi_ragged_set: instance %d: T = %d outside [1, %d]", i, q.T, r->d.Tmax);
    if (q.N < 1 || q.N > 8192 || !(q.dt > 0) || !(q.p0 > 0) || !(q.Xc > 0))
      return fail(REXI_EINVAL, "rexi_ragged_set: instance %d: need 1 <= N <= 8192, dt, p0, Xc > 0", i);
    elems += (long long)(q.T + 1) * (q.T + 2) / 2;
  }
  if (elems > r->d.max_elems)
    return fail(REXI_EBUSY, "rexi_ragged_set: %lld coefficients > max_elems %lld", elems, r->d.max_elems);
  if (r->gexec) {
    cudaGraphExecDestroy(r->gexec);
    r->gexec = nullptr;
  }
  const bool given = inst[0].soff >= 0;
  for (int i = 0; i < ninst; ++i)
    if ((inst[i].soff >= 0) != given)
      return fail(REXI_EINVAL, "rexi_ragged_set: either every instance gives soff or none");
  std::vector<long long> so(ninst);
  long long off = 0, ext = 0;
  for (int i = 0; i < ninst; ++i) {
    const long long sz = 3LL * (inst[i].T + 1) * (inst[i].T + 2) / 2;
    so[i] = given ? inst[i].soff : off;
    off += sz;
    ext = std::max(ext, so[i] + sz);
  }
  if (given) {  // states must not overlap
    std::vector<int> ord(ninst);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return so[a] < so[b]; });
    for (int k = 1; k < ninst; ++k) {
      const int a = ord[k - 1], b = ord[k];
      if (so[a] + 3LL * (inst[a].T + 1) * (inst[a].T + 2) / 2 > so[b])
        return fail(REXI_EINVAL, "rexi_ragged_set: states %d and %d overlap", a, b);
    }
  }
  // pole sets are cached by (T, N, dt, p0, Xc); the arena starts over when it overflows
  auto ensure = [&](const rexi_instance& q, const PoleSet** out) -> int {
    auto key = std::make_tuple(q.T, q.N, q.dt, q.p0, q.Xc);
    auto it = r->cache.find(key);
    if (it != r->cache.end()) {
      *out = &it->second;
      return REXI_OK;
    }
    PoleSet ps;
    const double X = rexi_spectrum_bound(q.T, q.dt, r->d.omega, r->d.radius, r->d.phibar);
    // ragged sets: most instances have a pole set of their own and run tiles of one state
    int rc = make_poleset_from_contour(ps, r->d.precision, q.T, q.N, q.dt, X, q.p0, q.Xc, r->d.heavy_tau,
                                       r->d.prune_tau, 32, r->d.fp64_tau);
    if (rc) return rc;
    if (r->e.pole_used + ps.Npad > r->e.pole_cap) return REXI_EBUSY;
    // a place in the pole arena now; the upload goes with this set's descriptors (stream order:
    // after the work already queued, which may still read the arena's earlier contents)
    ps.pole0 = r->e.pole_used;
    r->e.pole_used += ps.Npad;
    it = r->cache.emplace(key, std::move(ps)).first;
    r->fresh.push_back(&it->second);
    r->fresh_keys.push_back(key);
    *out = &it->second;
    return REXI_OK;
  };
  std::vector<const PoleSet*> cur(ninst);
  int rc = REXI_OK;
  r->fresh.clear();
  r->fresh_keys.clear();
  for (int i = 0; i < ninst && !rc; ++i) rc = ensure(inst[i], &cur[i]);
  if (rc == REXI_EBUSY) {  // arena full: start over with the current pole sets only
    r->cache.clear();
    r->fresh.clear();
    r->fresh_keys.clear();
    r->e.pole_used = 0;
    rc = REXI_OK;
    for (int i = 0; i < ninst && !rc; ++i) rc = ensure(inst[i], &cur[i]);
    if (rc == REXI_EBUSY) {
      drop_fresh(r);
      return fail(REXI_EBUSY, "rexi_ragged_set: pole sets exceed max_poles");
    }
  }
  if (rc) {
    drop_fresh(r);
    return rc;
  }
  r->cur = cur;
  r->soff = so;
  r->extent = ext;
  rc = ragged_rebuild(r);
  if (rc) {  // nothing of this set is usable: no step until a set succeeds
    drop_fresh(r);
    r->cur.clear();
    r->soff.clear();
    r->extent = 0;
  }
  r->fresh_keys.clear();
  return rc;
}

extern "C" int rexi_ragged_offsets(const rexi_ragged* r, long long* soff) {
  if (!r || !soff) return fail(REXI_EINVAL, "rexi_ragged_offsets: null argument");
  for (size_t i = 0; i < r->soff.size(); ++i) soff[i] = r->soff[i];
  soff[r->soff.size()] = r->extent;
  return REXI_OK;
}

extern "C" int rexi_ragged_step(rexi_ragged* r, const void* U0, void* U1) {
  if (!r || !U0 || !U1) return fail(REXI_EINVAL, "rexi_ragged_step: null argument");
  if (r->cur.empty()) return fail(REXI_EINVAL, "rexi_ragged_step: no instances set");
  if (overlaps(U0, U1, sizeof(double2) * (size_t)r->extent))
    return fail(REXI_EINVAL, "rexi_ragged_step: U0 and U1 overlap");
  if (r->gexec && U0 == r->g_u0 && U1 == r->g_u1) {
    REXI_CUDA_TRY(cudaGraphLaunch(r->gexec, r->e.stream));
    return REXI_OK;
  }
  return engine_launch(r->e, r->L, (const double2*)U0, (double2*)U1);
}

extern "C" int rexi_ragged_capture(rexi_ragged* r, const void* U0, void* U1) {
  if (!r || !U0 || !U1) return fail(REXI_EINVAL, "rexi_ragged_capture: null argument");
  if (r->cur.empty()) return fail(REXI_EINVAL, "rexi_ragged_capture: no instances set");
  if (r->e.stream == nullptr) return fail(REXI_EINVAL, "rexi_ragged_capture: needs a non-default stream");
  if (r->gexec) {
    cudaGraphExecDestroy(r->gexec);
    r->gexec = nullptr;
  }
  const int prof = r->e.profiling;
  r->e.profiling = 0;
  REXI_CUDA_TRY(cudaStreamBeginCapture(r->e.stream, cudaStreamCaptureModeThreadLocal));
  int rc = engine_launch(r->e, r->L, (const double2*)U0, (double2*)U1);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(r->e.stream, &g);
  r->e.profiling = prof;
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
  ce = cudaGraphInstantiate(&r->gexec, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
  r->g_u0 = U0;
  r->g_u1 = U1;
  return REXI_OK;
}

// Autotuner: times the candidate tile densities (pole ranges per (m, chain), expressed as
// tiles per resident warp) on the current instance set and keeps the fastest.
extern "C" int rexi_ragged_tune(rexi_ragged* r, const void* U0, void* U1, int reps, int* best_qmul,
                                double* best_ms) {
  if (!r || !U0 || !U1) return fail(REXI_EINVAL, "rexi_ragged_tune: null argument");
  if (r->cur.empty()) return fail(REXI_EINVAL, "rexi_ragged_tune: no instances set");
  if (reps < 1) reps = 3;
  const int cand[] = {1, 2, 4, 8};
  double best = 1e300;
  int bq = r->qmul;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int rc = REXI_OK;
  for (int qm : cand) {
    r->qmul = qm;
    rc = ragged_rebuild(r);
    if (rc == REXI_EBUSY) {
      rc = REXI_OK;
      continue;
    }
    if (rc) break;
    if ((rc = engine_launch(r->e, r->L, (const double2*)U0, (double2*)U1))) break;  // warm-up
    cudaEventRecord(a, r->e.stream);
    for (int i = 0; i < reps && !rc; ++i) rc = engine_launch(r->e, r->L, (const double2*)U0, (double2*)U1);
    cudaEventRecord(b, r->e.stream);
    cudaError_t ce = cudaEventSynchronize(b);
    if (ce != cudaSuccess) {
      rc = cuda_fail(ce, "rexi_ragged_tune");
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (ms / reps < best) {
      best = ms / reps;
      bq = qm;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  r->qmul = bq;
  if (r->gexec) {
    cudaGraphExecDestroy(r->gexec);
    r->gexec = nullptr;
  }
  rc = ragged_rebuild(r);
  if (rc) return rc;
  if (best_qmul) *best_qmul = bq;
  if (best_ms) *best_ms = best;
  return REXI_OK;
}

extern "C" int rexi_ragged_sync(rexi_ragged* r) {
  if (!r) return fail(REXI_EINVAL, "rexi_ragged_sync: null plan");
  REXI_CUDA_TRY(cudaStreamSynchronize(r->e.stream));
  REXI_CUDA_TRY(cudaGetLastError());
  return REXI_OK;
}

extern "C" int rexi_ragged_set_profiling(rexi_ragged* r, int enable) {
  if (!r) return fail(REXI_EINVAL, "rexi_ragged_set_profiling: null plan");
  r->e.profiling = enable ? 1 : 0;
  return REXI_OK;
}

extern "C" int rexi_ragged_get_profile(rexi_ragged* r, double* ms, int* launches, int reset) {
  if (!r) return fail(REXI_EINVAL, "rexi_ragged_get_profile: null plan");
  return engine_profile(r->e, ms, launches, reset);
}
