// REXI plan: tables, pole ordering, tiles and launches (paper Sec. 4.2, Eq. rexi).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "rexi_fp64.cuh"
#include "rexi_mixed.cuh"

using namespace rexi;
using cplx = std::complex<double>;

struct rexi_plan {
  rexi_plan_desc d{};
  int T = 0, N = 0, nlm = 0, Npad = 0, ngroups = 0, precision = 0, device = 0, nsm = 0;
  int n_heavy = 0, g_light = 0, g_heavy = 0;
  double X = 0;
  cplx S0 = 0;
  std::vector<cplx> z_sorted, w_sorted;  // internal order (padded)
  std::vector<int> heavy_sorted;
  cudaStream_t stream = nullptr;
  // device
  D4* d_tab64 = nullptr;
  float4* d_tab32 = nullptr;
  PoleD* d_p64 = nullptr;
  PoleF* d_p32 = nullptr;
  double2* d_partial = nullptr;
  size_t partial_elems = 0;
  void* d_scratch = nullptr;
  size_t scratch_bytes = 0;
  void* d_rhs = nullptr;  // mixed pre-pass output: Rhs32[max_batch][nlm] then RhsDF[max_batch][nlm]
  TabDF* d_tabdf = nullptr;
  PoleDF* d_pdf = nullptr;
  double2* d_stage_in = nullptr;
  double2* d_stage_out = nullptr;
  // persistent grids
  int grid_fp64 = 0, grid_light = 0, grid_heavy = 0;
  // tiles per Q choice: Q -> (device tiles, count)
  struct TileSet {
    Tile* d = nullptr;
    int n = 0, n_light = 0, Q = 0;
  };
  std::map<int, TileSet> tilesets;
  long long workspace = 0;
  // per-kernel event timing
  int profiling = 0;
  struct Pend {
    cudaEvent_t a, b;
    int kid;
  };
  std::vector<Pend> pending;
  std::vector<cudaEvent_t> event_pool;
  double prof_ms[REXI_NKERNELS] = {0};
  int prof_n[REXI_NKERNELS] = {0};
};

namespace {
cudaEvent_t take_event(rexi_plan* p) {
  if (!p->event_pool.empty()) {
    cudaEvent_t e = p->event_pool.back();
    p->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
// Records the start event of kernel `kid` (profiling only); returns the pending index.
int prof_begin(rexi_plan* p, int kid) {
  if (!p->profiling) return -1;
  rexi_plan::Pend q{take_event(p), take_event(p), kid};
  cudaEventRecord(q.a, p->stream);
  p->pending.push_back(q);
  return (int)p->pending.size() - 1;
}
void prof_end(rexi_plan* p, int h) {
  if (h >= 0) cudaEventRecord(p->pending[h].b, p->stream);
}
}  // namespace

namespace {

double eps_nm(int n, int m) {
  if (n <= m) return 0.0;
  return std::sqrt((double(n) * n - double(m) * m) / (4.0 * n * n - 1.0));
}

template <class P>
int dev_alloc(P** p, size_t bytes, long long* acc) {
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(REXI_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  *acc += (long long)bytes;
  return REXI_OK;
}

int ranges_used(int G, int Q) {
  if (G == 0) return 0;
  const int per = (G + Q - 1) / Q;
  return (G + per - 1) / per;
}

// Tiles for one state: light groups [0, gl) split into Ql ranges, heavy groups [gl, gl+gh)
// into Qh ranges; every range gets one tile per (m, chain).  Sorted by decreasing cost.
std::vector<Tile> build_tiles(int T, int gl, int Ql, int gh, int Qh, int heavy_cost) {
  std::vector<Tile> v;
  auto add_ranges = [&](int gbase, int G, int Q, int qbase, int heavy) {
    if (G == 0) return;
    const int per = (G + Q - 1) / Q;
    int q = qbase;
    for (int g = 0; g < G; g += per, ++q) {
      const int ng = std::min(per, G - g);
      for (int m = 0; m <= T; ++m)
        for (int c = 0; c < 2; ++c) {
          Tile t{};
          t.m = m;
          t.chain = c;
          t.g0 = gbase + g;
          t.ng = ng;
          t.q = q;
          t.heavy = heavy;
          t.cost = (T + 1 - m) * ng * (heavy ? heavy_cost : 1);
          v.push_back(t);
        }
    }
  };
  add_ranges(0, gl, Ql, 0, 0);
  add_ranges(gl, gh, Qh, ranges_used(gl, Ql), 1);
  // light tiles first, then heavy tiles; each part sorted by decreasing cost
  std::stable_sort(v.begin(), v.end(), [](const Tile& a, const Tile& b) {
    if (a.heavy != b.heavy) return a.heavy < b.heavy;
    return a.cost > b.cost;
  });
  return v;
}

// Number of pole ranges so that a batch of B states gives about `target` warp tiles.
int choose_Q(int groups, int B, int T, int target) {
  const long long per_q = (long long)B * 2 * (T + 1);
  int Q = (int)std::max<long long>(1, (target + per_q - 1) / per_q);
  return std::min(Q, std::max(groups, 1));
}

int get_tiles(rexi_plan* p, int B, rexi_plan::TileSet** out) {
  int Ql = 0, Qh = 0;
  const int hc = 3;
  if (p->precision == REXI_FP64) {
    Qh = choose_Q(p->ngroups, B, p->T, 4 * p->grid_fp64 * FP64_WARPS);
  } else {
    const int target_l = 4 * p->grid_light * MIX_WARPS;
    const int target_h = 4 * p->grid_heavy * MIX_WARPS;
    Ql = p->g_light ? choose_Q(p->g_light, B, p->T, target_l) : 0;
    Qh = p->g_heavy ? choose_Q(p->g_heavy, B, p->T, target_h) : 0;
  }
  const int key = Ql * 100000 + Qh;
  auto it = p->tilesets.find(key);
  if (it == p->tilesets.end()) {
    std::vector<Tile> v = (p->precision == REXI_FP64)
                              ? build_tiles(p->T, 0, 1, p->ngroups, Qh, 1)
                              : build_tiles(p->T, p->g_light, std::max(Ql, 1), p->g_heavy,
                                            std::max(Qh, 1), hc);
    rexi_plan::TileSet ts;
    ts.n = (int)v.size();
    ts.n_light = 0;
    for (const Tile& t : v) ts.n_light += t.heavy ? 0 : 1;
    ts.Q = ranges_used(p->precision == REXI_FP64 ? 0 : p->g_light, std::max(Ql, 1)) +
           ranges_used(p->precision == REXI_FP64 ? p->ngroups : p->g_heavy, std::max(Qh, 1));
    cudaError_t e = cudaMalloc(&ts.d, sizeof(Tile) * v.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(tiles)");
    e = cudaMemcpy(ts.d, v.data(), sizeof(Tile) * v.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(tiles)");
    p->workspace += (long long)(sizeof(Tile) * v.size());
    it = p->tilesets.emplace(key, ts).first;
  }
  if ((size_t)B * it->second.Q * 3 * p->nlm > p->partial_elems)
    return fail(REXI_EINVAL, "internal: partial buffer too small (B=%d Q=%d)", B, it->second.Q);
  *out = &it->second;
  return REXI_OK;
}

}  // namespace

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

  rexi_plan* p = new rexi_plan();
  p->d = d;
  p->d.z = p->d.w = nullptr;
  p->T = d.T;
  p->N = d.N;
  p->nlm = (d.T + 1) * (d.T + 2) / 2;
  p->precision = d.precision;
  p->stream = (cudaStream_t)d.stream;
  auto bail = [&](int code) {
    rexi_plan_destroy(p);
    return code;
  };
  if (cudaGetDevice(&p->device) != cudaSuccess) return bail(fail(REXI_ECUDA, "no CUDA device"));
  cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device);

  // ---- poles and weights --------------------------------------------------------------
  std::vector<cplx> z(d.N), w(d.N);
  if (d.z) {
    for (int n = 0; n < d.N; ++n) {
      z[n] = cplx(d.z[2 * n], d.z[2 * n + 1]);
      w[n] = cplx(d.w[2 * n], d.w[2 * n + 1]);
    }
  } else {
    std::vector<double> zz(2 * d.N), ww(2 * d.N);
    int rc = rexi_coeffs(d.N, d.p0, d.Xc, 0, zz.data(), ww.data());
    if (rc) return bail(rc);
    for (int n = 0; n < d.N; ++n) {
      z[n] = cplx(zz[2 * n], zz[2 * n + 1]);
      w[n] = cplx(ww[2 * n], ww[2 * n + 1]);
    }
  }
  for (int n = 0; n < d.N; ++n)
    if (std::abs(z[n]) < 1e-12) return bail(fail(REXI_EINVAL, "pole %d is zero", n));
  // S0 = sum w/z with compensated summation
  {
    cplx s = 0, comp = 0;
    for (int n = 0; n < d.N; ++n) {
      cplx yv = w[n] / z[n] - comp;
      cplx t = s + yv;
      comp = (t - s) - yv;
      s = t;
    }
    p->S0 = s;
  }
  p->X = rexi_spectrum_bound(d.T, d.dt, d.omega, d.radius, d.phibar);
  p->Npad = (d.N + 31) / 32 * 32;
  p->ngroups = p->Npad / 32;

  // internal order: FP64 keeps the given order; MIXED puts the light poles first and the
  // heavy ones (largest gain |w| / dist(z, [-iX, iX]), padded to whole groups) last.
  std::vector<int> order(d.N);
  std::iota(order.begin(), order.end(), 0);
  std::vector<int> heavy(d.N, p->precision == REXI_FP64 ? 1 : 0);
  if (p->precision == REXI_MIXED) {
    const double tau = d.heavy_tau < 0 ? 1e-3 : d.heavy_tau;
    std::vector<double> gain(d.N);
    int nh = 0;
    for (int n = 0; n < d.N; ++n) {
      const double yi = std::min(std::max(z[n].imag(), -p->X), p->X);
      const double dist = std::abs(z[n] - cplx(0.0, yi));
      gain[n] = std::abs(w[n]) / std::max(dist, 1e-300);
      if (gain[n] > tau) ++nh;
    }
    const int nh_pad = std::min((nh + 31) / 32 * 32, d.N);
    std::vector<int> by_gain(d.N);
    std::iota(by_gain.begin(), by_gain.end(), 0);
    std::stable_sort(by_gain.begin(), by_gain.end(), [&](int a, int b) { return gain[a] > gain[b]; });
    for (int i = 0; i < nh_pad; ++i) heavy[by_gain[i]] = 1;
    p->n_heavy = nh_pad;
    std::stable_partition(order.begin(), order.end(), [&](int n) { return !heavy[n]; });
  } else {
    p->n_heavy = d.N;
  }
  // padding: dummy poles (w = 0) fill the light part (mixed) or the tail (FP64)
  const int npad = p->Npad - d.N;
  p->z_sorted.clear();
  p->w_sorted.clear();
  p->heavy_sorted.clear();
  const int nlight = d.N - (p->precision == REXI_MIXED ? p->n_heavy : d.N);
  for (int i = 0; i < (p->precision == REXI_MIXED ? nlight : d.N); ++i) {
    p->z_sorted.push_back(z[order[i]]);
    p->w_sorted.push_back(w[order[i]]);
    p->heavy_sorted.push_back(heavy[order[i]]);
  }
  if (p->precision == REXI_MIXED) {
    // light part padded to whole groups, then the heavy groups
    for (int i = 0; i < npad; ++i) {
      p->z_sorted.push_back(cplx(1.0, 0.0));
      p->w_sorted.push_back(0.0);
      p->heavy_sorted.push_back(0);
    }
    for (int i = nlight; i < d.N; ++i) {
      p->z_sorted.push_back(z[order[i]]);
      p->w_sorted.push_back(w[order[i]]);
      p->heavy_sorted.push_back(1);
    }
    p->g_light = (nlight + npad) / 32;
    p->g_heavy = p->n_heavy / 32;
    if ((nlight + npad) % 32 != 0 || p->n_heavy % 32 != 0) {
      // nh_pad == N with N not a multiple of 32: everything heavy, padding at the end
      p->z_sorted.clear();
      p->w_sorted.clear();
      p->heavy_sorted.clear();
      for (int n = 0; n < d.N; ++n) {
        p->z_sorted.push_back(z[n]);
        p->w_sorted.push_back(w[n]);
        p->heavy_sorted.push_back(1);
      }
      for (int i = 0; i < npad; ++i) {
        p->z_sorted.push_back(cplx(1.0, 0.0));
        p->w_sorted.push_back(0.0);
        p->heavy_sorted.push_back(1);
      }
      p->g_light = 0;
      p->g_heavy = p->ngroups;
      p->n_heavy = d.N;
    }
  } else {
    for (int i = 0; i < npad; ++i) {
      p->z_sorted.push_back(cplx(1.0, 0.0));
      p->w_sorted.push_back(0.0);
      p->heavy_sorted.push_back(1);
    }
  }

  // ---- device tables ------------------------------------------------------------------
  const int T = d.T;
  std::vector<D4> tab64(p->nlm);
  std::vector<float4> tab32(p->nlm);
  for (int m = 0; m <= T; ++m)
    for (int n = m; n <= T; ++n) {
      const int idx = moff(T, m) + (n - m);
      const double nn1 = double(n) * (n + 1);
      const double wn = n > 0 ? 2.0 * d.omega * m / nn1 : 0.0;
      const double cm = (n > m && n - 1 > 0) ? d.dt * 2.0 * d.omega * (n + 1.0) / n * eps_nm(n, m) : 0.0;
      const double cp = (n < T) ? d.dt * 2.0 * d.omega * n / (n + 1.0) * eps_nm(n + 1, m) : 0.0;
      const double q = d.dt * nn1 / (d.radius * d.radius);
      tab64[idx] = D4{d.dt * wn, cm, cp, q};
      tab32[idx] = make_float4((float)(d.dt * wn), (float)cm, (float)cp, (float)q);
    }
  std::vector<PoleD> p64(p->Npad);
  std::vector<PoleF> p32(p->Npad);
  const double hpb = d.dt * d.phibar;
  for (int i = 0; i < p->Npad; ++i) {
    const cplx zz = p->z_sorted[i], ww = p->w_sorted[i];
    const cplx iz = 1.0 / zz, wz = ww / zz, gz = hpb / zz;
    auto D = [](cplx c) { return make_double2(c.real(), c.imag()); };
    auto F = [](cplx c) { return make_float2((float)c.real(), (float)c.imag()); };
    p64[i] = PoleD{D(zz), D(ww), D(wz), D(iz), D(gz)};
    p32[i] = PoleF{F(zz), F(ww), F(wz), F(iz), F(gz)};
  }
  long long& ws = p->workspace;
  int rc;
  if ((rc = dev_alloc(&p->d_tab64, sizeof(D4) * p->nlm, &ws))) return bail(rc);
  if ((rc = dev_alloc(&p->d_tab32, sizeof(float4) * p->nlm, &ws))) return bail(rc);
  if ((rc = dev_alloc(&p->d_p64, sizeof(PoleD) * p->Npad, &ws))) return bail(rc);
  if ((rc = dev_alloc(&p->d_p32, sizeof(PoleF) * p->Npad, &ws))) return bail(rc);
  cudaError_t e;
  if ((e = cudaMemcpy(p->d_tab64, tab64.data(), sizeof(D4) * p->nlm, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(p->d_tab32, tab32.data(), sizeof(float4) * p->nlm, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(p->d_p64, p64.data(), sizeof(PoleD) * p->Npad, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(p->d_p32, p32.data(), sizeof(PoleF) * p->Npad, cudaMemcpyHostToDevice)))
    return bail(cuda_fail(e, "cudaMemcpy(tables)"));

  // ---- persistent grids and scratch ----------------------------------------------------
  const int kmax = T + 1;
  if (p->precision == REXI_FP64) {
    const size_t smem = fp64_smem_bytes();
    if ((e = cudaFuncSetAttribute(k_rexi_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return bail(cuda_fail(e, "cudaFuncSetAttribute(k_rexi_fp64)"));
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rexi_fp64, FP64_WARPS * 32, smem)))
      return bail(cuda_fail(e, "occupancy(k_rexi_fp64)"));
    per_sm = std::max(1, std::min(per_sm, 2));
    p->grid_fp64 = p->nsm * per_sm;
    p->scratch_bytes = sizeof(D4) * (size_t)p->grid_fp64 * FP64_WARPS * kmax * 32;
  } else {
    const size_t hsm = heavy_smem_bytes();
    if ((e = cudaFuncSetAttribute(k_rexi_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm)))
      return bail(cuda_fail(e, "cudaFuncSetAttribute(k_rexi_heavy)"));
    int per_l = 0, per_h = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_l, k_rexi_light, MIX_WARPS * 32, 0)))
      return bail(cuda_fail(e, "occupancy(k_rexi_light)"));
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_h, k_rexi_heavy, MIX_WARPS * 32, hsm)))
      return bail(cuda_fail(e, "occupancy(k_rexi_heavy)"));
    p->grid_light = p->nsm * std::max(1, std::min(per_l, 4));
    p->grid_heavy = p->nsm * std::max(1, std::min(per_h, 2));
    const int nseg_max = (kmax + SEG - 1) / SEG;
    p->scratch_bytes = sizeof(float4) * (size_t)p->grid_light * MIX_WARPS * nseg_max * 32 +
                       (sizeof(float4) + sizeof(float2)) * (size_t)p->grid_heavy * MIX_WARPS * kmax * 32;
    if ((rc = dev_alloc((char**)&p->d_rhs, mixed_rhs_bytes(p->nlm, d.max_batch), &ws))) return bail(rc);
    std::vector<TabDF> tdf(p->nlm);
    for (int i = 0; i < p->nlm; ++i)
      tdf[i] = TabDF{split4(tab64[i].x, tab64[i].y), split4(tab64[i].z, tab64[i].w)};
    std::vector<PoleDF> pdf(p->Npad);
    for (int i = 0; i < p->Npad; ++i)
      pdf[i] = PoleDF{split4(p64[i].z.x, p64[i].z.y), split4(p64[i].iz.x, p64[i].iz.y),
                      split4(p64[i].gz.x, p64[i].gz.y)};
    if ((rc = dev_alloc(&p->d_tabdf, sizeof(TabDF) * p->nlm, &ws))) return bail(rc);
    if ((rc = dev_alloc(&p->d_pdf, sizeof(PoleDF) * p->Npad, &ws))) return bail(rc);
    if ((e = cudaMemcpy(p->d_tabdf, tdf.data(), sizeof(TabDF) * p->nlm, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(p->d_pdf, pdf.data(), sizeof(PoleDF) * p->Npad, cudaMemcpyHostToDevice)))
      return bail(cuda_fail(e, "cudaMemcpy(double-float tables)"));
  }
  if ((rc = dev_alloc((char**)&p->d_scratch, p->scratch_bytes, &ws))) return bail(rc);

  // partial sums: the largest B * Q over the batch sizes a call may use
  size_t maxBQ = 0;
  for (int B = 1; B <= d.max_batch; ++B) {
    int Ql = 0, Qh = 0;
    if (p->precision == REXI_FP64) {
      Qh = ranges_used(p->ngroups, choose_Q(p->ngroups, B, T, 4 * p->grid_fp64 * FP64_WARPS));
    } else {
      if (p->g_light) Ql = ranges_used(p->g_light, choose_Q(p->g_light, B, T, 4 * p->grid_light * MIX_WARPS));
      if (p->g_heavy) Qh = ranges_used(p->g_heavy, choose_Q(p->g_heavy, B, T, 4 * p->grid_heavy * MIX_WARPS));
    }
    maxBQ = std::max(maxBQ, (size_t)B * (Ql + Qh));
  }
  p->partial_elems = maxBQ * 3 * p->nlm;
  if ((rc = dev_alloc(&p->d_partial, sizeof(double2) * p->partial_elems, &ws))) return bail(rc);
  const size_t state_bytes = sizeof(double2) * 3 * (size_t)p->nlm * d.max_batch;
  if ((rc = dev_alloc(&p->d_stage_in, state_bytes, &ws))) return bail(rc);
  if ((rc = dev_alloc(&p->d_stage_out, state_bytes, &ws))) return bail(rc);
  *out = p;
  return REXI_OK;
}

extern "C" int rexi_plan_destroy(rexi_plan* p) {
  if (!p) return REXI_OK;
  if (p->stream || p->d_tab64) cudaStreamSynchronize(p->stream);
  cudaFree(p->d_tab64);
  cudaFree(p->d_tab32);
  cudaFree(p->d_p64);
  cudaFree(p->d_p32);
  cudaFree(p->d_partial);
  cudaFree(p->d_scratch);
  cudaFree(p->d_rhs);
  cudaFree(p->d_tabdf);
  cudaFree(p->d_pdf);
  cudaFree(p->d_stage_in);
  cudaFree(p->d_stage_out);
  for (auto& kv : p->tilesets) cudaFree(kv.second.d);
  for (auto& q : p->pending) {
    cudaEventDestroy(q.a);
    cudaEventDestroy(q.b);
  }
  for (auto ev : p->event_pool) cudaEventDestroy(ev);
  delete p;
  return REXI_OK;
}

extern "C" int rexi_step(rexi_plan* p, const void* U0v, void* U1v, int batch) {
  if (!p || !U0v || !U1v) return fail(REXI_EINVAL, "rexi_step: null argument");
  if (batch < 1 || batch > p->d.max_batch)
    return fail(REXI_EINVAL, "rexi_step: batch %d outside [1, %d]", batch, p->d.max_batch);
  const size_t bytes = sizeof(double2) * 3 * (size_t)p->nlm * batch;
  const char* a0 = (const char*)U0v;
  const char* a1 = (const char*)U1v;
  if (a0 < a1 + bytes && a1 < a0 + bytes) return fail(REXI_EINVAL, "rexi_step: U0 and U1 overlap");
  const double2* U0 = (const double2*)U0v;
  double2* U1 = (double2*)U1v;
  rexi_plan::TileSet* ts = nullptr;
  int rc = get_tiles(p, batch, &ts);
  if (rc) return rc;
  if (p->precision == REXI_FP64) {
    Fp64Args a;
    a.U0 = U0;
    a.partial = p->d_partial;
    a.tab = p->d_tab64;
    a.poles = p->d_p64;
    a.tiles = ts->d;
    a.scratch = (D4*)p->d_scratch;
    a.ntiles = ts->n;
    a.B = batch;
    a.T = p->T;
    a.nlm = p->nlm;
    a.Q = ts->Q;
    a.kmax = p->T + 1;
    const int h = prof_begin(p, 1);
    k_rexi_fp64<<<p->grid_fp64, FP64_WARPS * 32, fp64_smem_bytes(), p->stream>>>(a);
    prof_end(p, h);
  } else {
    const long long tot = (long long)batch * p->nlm;
    Rhs32* r32 = (Rhs32*)p->d_rhs;
    RhsDF* rdf = (RhsDF*)((char*)p->d_rhs + mixed_rhs32_bytes(p->nlm, p->d.max_batch));
    int h = prof_begin(p, 0);
    k_mixed_rhs<<<(unsigned)((tot + 255) / 256), 256, 0, p->stream>>>(U0, p->d_tab64, r32, rdf,
                                                                       batch, p->nlm);
    prof_end(p, h);
    MixedArgs a;
    a.U0 = U0;
    a.partial = p->d_partial;
    a.tab32 = p->d_tab32;
    a.tabdf = p->d_tabdf;
    a.p32 = p->d_p32;
    a.p64 = p->d_p64;
    a.pdf = p->d_pdf;
    a.tiles = ts->d;
    a.rhs32 = r32;
    a.rhsdf = rdf;
    a.scratch = p->d_scratch;
    a.ntiles_light = ts->n_light;
    a.ntiles_heavy = ts->n - ts->n_light;
    a.B = batch;
    a.T = p->T;
    a.nlm = p->nlm;
    a.Q = ts->Q;
    a.kmax = p->T + 1;
    a.nseg_max = (p->T + 1 + SEG - 1) / SEG;
    a.warps_light = p->grid_light * MIX_WARPS;
    if (p->g_light) {
      h = prof_begin(p, 2);
      k_rexi_light<<<p->grid_light, MIX_WARPS * 32, 0, p->stream>>>(a);
      prof_end(p, h);
    }
    if (p->g_heavy) {
      h = prof_begin(p, 3);
      k_rexi_heavy<<<p->grid_heavy, MIX_WARPS * 32, heavy_smem_bytes(), p->stream>>>(a);
      prof_end(p, h);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "solve kernel launch");
  const long long tot = (long long)batch * p->nlm;
  const int hf = prof_begin(p, 4);
  k_rexi_finalize<<<(unsigned)((tot + 255) / 256), 256, 0, p->stream>>>(
      U0, p->d_partial, U1, batch, p->nlm, ts->Q, make_double2(p->S0.real(), p->S0.imag()),
      p->d.dt * p->d.phibar);
  prof_end(p, hf);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "finalize kernel launch");
  return REXI_OK;
}

extern "C" int rexi_step_host(rexi_plan* p, const double* U0, double* U1, int batch) {
  if (!p || !U0 || !U1) return fail(REXI_EINVAL, "rexi_step_host: null argument");
  if (batch < 1 || batch > p->d.max_batch)
    return fail(REXI_EINVAL, "rexi_step_host: batch %d outside [1, %d]", batch, p->d.max_batch);
  const size_t bytes = sizeof(double2) * 3 * (size_t)p->nlm * batch;
  REXI_CUDA_TRY(cudaMemcpyAsync(p->d_stage_in, U0, bytes, cudaMemcpyHostToDevice, p->stream));
  int rc = rexi_step(p, p->d_stage_in, p->d_stage_out, batch);
  if (rc) return rc;
  REXI_CUDA_TRY(cudaMemcpyAsync(U1, p->d_stage_out, bytes, cudaMemcpyDeviceToHost, p->stream));
  REXI_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return REXI_OK;
}

extern "C" int rexi_sync(rexi_plan* p) {
  if (!p) return fail(REXI_EINVAL, "rexi_sync: null plan");
  REXI_CUDA_TRY(cudaStreamSynchronize(p->stream));
  REXI_CUDA_TRY(cudaGetLastError());
  return REXI_OK;
}

extern "C" int rexi_plan_get_info(const rexi_plan* p, rexi_plan_info* info) {
  if (!p || !info) return fail(REXI_EINVAL, "rexi_plan_get_info: null argument");
  std::memset(info, 0, sizeof(*info));
  info->T = p->T;
  info->N = p->N;
  info->nlm = p->nlm;
  info->precision = p->precision;
  info->n_heavy = p->n_heavy;
  info->n_groups = p->ngroups;
  info->n_tiles = p->tilesets.empty() ? 0 : p->tilesets.begin()->second.n;
  info->q_slots = p->tilesets.empty() ? 0 : p->tilesets.begin()->second.Q;
  info->grid_fp64 = p->grid_fp64;
  info->grid_light = p->grid_light;
  info->grid_heavy = p->grid_heavy;
  info->workspace_bytes = p->workspace;
  info->s0_re = p->S0.real();
  info->s0_im = p->S0.imag();
  info->X = p->X;
  return REXI_OK;
}

extern "C" int rexi_plan_get_poles(const rexi_plan* p, double* z, double* w, int* heavy) {
  if (!p) return fail(REXI_EINVAL, "rexi_plan_get_poles: null plan");
  int k = 0;
  for (int i = 0; i < p->Npad; ++i) {
    if (std::abs(p->w_sorted[i]) == 0.0 && p->z_sorted[i] == cplx(1.0, 0.0)) continue;  // padding
    if (k >= p->N) break;
    if (z) {
      z[2 * k] = p->z_sorted[i].real();
      z[2 * k + 1] = p->z_sorted[i].imag();
    }
    if (w) {
      w[2 * k] = p->w_sorted[i].real();
      w[2 * k + 1] = p->w_sorted[i].imag();
    }
    if (heavy) heavy[k] = p->heavy_sorted[i];
    ++k;
  }
  return REXI_OK;
}

extern "C" int rexi_plan_set_profiling(rexi_plan* p, int enable) {
  if (!p) return fail(REXI_EINVAL, "rexi_plan_set_profiling: null plan");
  p->profiling = enable ? 1 : 0;
  return REXI_OK;
}

extern "C" int rexi_plan_get_profile(rexi_plan* p, double* ms, int* launches, int reset) {
  if (!p) return fail(REXI_EINVAL, "rexi_plan_get_profile: null plan");
  REXI_CUDA_TRY(cudaStreamSynchronize(p->stream));
  for (auto& q : p->pending) {
    float t = 0.f;
    REXI_CUDA_TRY(cudaEventElapsedTime(&t, q.a, q.b));
    p->prof_ms[q.kid] += t;
    p->prof_n[q.kid] += 1;
    p->event_pool.push_back(q.a);
    p->event_pool.push_back(q.b);
  }
  p->pending.clear();
  for (int i = 0; i < REXI_NKERNELS; ++i) {
    if (ms) ms[i] = p->prof_ms[i];
    if (launches) launches[i] = p->prof_n[i];
    if (reset) {
      p->prof_ms[i] = 0;
      p->prof_n[i] = 0;
    }
  }
  return REXI_OK;
}
