// Mixed-precision REXI solve kernels.
//
// The poles split into two classes at plan time by their gain
//     g_n = |w_n| / dist(z_n, [-iX, iX]),
// the largest factor by which an error in the solve of pole n reaches the REXI sum.  Only a
// few poles near the positive real end of the contour have large weights e^{Re z}; for the
// rest an FP32 solve already contributes less than the target error.
//
//  * light poles (k_rexi_light): FP32 Thomas elimination, weighted sums in FP32 over the 32
//    poles of a warp, added into the FP64 partial sums.  The forward coefficients are not
//    stored: the sweep keeps a checkpoint of the recurrence state every LSEG = 8 elements and
//    the backward pass recomputes each 8-element segment in registers, so the kernel needs no
//    per-element scratch traffic.
//  * heavy poles (k_rexi_heavy): FP32 solve (checkpoints every heavy_seg() elements: 8 for one
//    state, 4 for state pairs), one step of iterative refinement whose residual r - A x is
//    evaluated in double-float arithmetic (pairs of FP32 numbers, error-free products by FMA,
//    Knuth's two-sum), FP32 solve of the correction by bottom-up (UL) elimination, and
//    weighted sums over poles in double-float arithmetic (16 poles at a time), added in FP64
//    across the pole halves and tiles.
// Both kernels share the tile scheme and chain equations of the FP64 kernel.
#pragma once
#include "common.cuh"
#include "df.cuh"
#include "rexi_fp64.cuh"

namespace rexi {

constexpr int MIX_WARPS = 4;
constexpr int LTROW = 33;      // padded row (float2) of the light transposition tile

struct dfc {
  df re, im;
};
__device__ __forceinline__ dfc dfc_mul(dfc a, dfc b) {
  return dfc{df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))),
             df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
// Double-float partial slot (re.hi, re.lo, im.hi, im.lo): set, or add a complex value given as
// a double-float pair per component; the error of each two-sum is kept in the low word.
__device__ __forceinline__ void dfp_add(float4* dst, float4 v, bool first) {
  if (first) {
    *dst = v;
    return;
  }
  float4 o = *dst;
  const df a = df_two_sum(o.x, v.x), b = df_two_sum(o.z, v.z);
  *dst = make_float4(a.hi, (o.y + v.y) + a.lo, b.hi, (o.w + v.w) + b.lo);
}
__host__ __device__ inline float4 split4(double a, double b) {
  float ah = (float)a, bh = (float)b;
  return make_float4(ah, (float)(a - (double)ah), bh, (float)(b - (double)bh));
}
__device__ __forceinline__ dfc dfc_of(float4 v) { return dfc{df{v.x, v.y}, df{v.z, v.w}}; }

// ---- packed (FP32x2) double-float accumulation ------------------------------------------
// Blackwell issues two FP32 operations per thread with one FADD2 / FMUL2 / FFMA2 instruction;
// each component is rounded exactly as by the scalar instruction.
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
// (AH, AL) += W * X per component, W = Wh + Wl in double-float, X in FP32: the product's rounding
// error is recovered by FMA and the sum's by two-sum; AL is left unnormalised.
__device__ __forceinline__ void df2_acc(float2& AH, float2& AL, float2 Wh, float2 Wl, float2 X) {
  const float2 P = __fmul2_rn(Wh, X);
  float2 E = __ffma2_rn(Wh, X, f2neg(P));
  E = __ffma2_rn(Wl, X, E);
  const float2 S = __fadd2_rn(AH, P);
  const float2 BB = __fadd2_rn(S, f2neg(AH));
  const float2 err = __fadd2_rn(__fadd2_rn(AH, f2neg(__fadd2_rn(S, f2neg(BB)))), __fadd2_rn(P, f2neg(BB)));
  AL = __fadd2_rn(AL, __fadd2_rn(err, E));
  AH = S;
}
// Weight in the packed shared-memory layout (re.hi, im.hi, re.lo, im.lo) from a double-float
// complex (re.hi, re.lo, im.hi, im.lo).
__device__ __forceinline__ float4 w_packed(float4 w) { return make_float4(w.x, w.z, w.y, w.w); }

// per-(m,n) table in double-float: (dt w, cm), (cp, q) as (hi, lo) pairs
struct TabDF {
  float4 a, b;  // a = (hw.hi, hw.lo, cm.hi, cm.lo), b = (cp.hi, cp.lo, q.hi, q.lo)
};
// per-pole constants in double-float
struct PoleDF {
  float4 z, iz, gz, w, wz;
};
// right-hand-side pieces produced by the pre-pass for every (state, m, n)
struct Rhs32 {
  float2 bz, bd, qbp;  // bzeta, bdelta, q * bPhi
};
struct RhsDF {
  float4 bz, bd, qbp;
};

// Rhs32[batch][nlm] followed (256-byte aligned) by RhsDF[batch][nlm]
inline size_t mixed_rhs32_bytes(int nlm, int batch) {
  return (sizeof(Rhs32) * (size_t)nlm * batch + 255) / 256 * 256;
}
inline size_t mixed_rhs_bytes(int nlm, int batch) {
  return mixed_rhs32_bytes(nlm, batch) + sizeof(RhsDF) * (size_t)nlm * batch;
}


struct MixedArgs {
  const double2* U0;    // state base
  double2* partial;
  const float4* tab32;
  const TabDF* tabdf;
  const PoleF* p32;
  const PoleD* p64;
  const PoleDF* pdf;
  const Tile* tiles;
  const Inst* insts;
  const Rhs32* rhs32;   // [sum nlm]
  const RhsDF* rhsdf;   // [sum nlm]
  void* scratch;
  int ntiles_light, ntiles_heavy;  // light tiles first, then heavy tiles, in `tiles`
  int Ttab, kmax, nseg_max;
  int warps_light;      // warps of the light grid (the heavy scratch starts after theirs)
};

// ---- pre-pass: FP32 and double-float right-hand-side pieces ----------------------------
static __global__ void k_mixed_rhs(const double2* __restrict__ U0, const D4* __restrict__ tab, int Ttab,
                                   Rhs32* __restrict__ r32, RhsDF* __restrict__ rdf,
                                   const Inst* __restrict__ insts, const long long* __restrict__ ecum,
                                   int ninst, long long total) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int i = inst_of(ecum, ninst, e);
  const Inst I = insts[i];
  const int nlm = I.nlm, idx = (int)(e - ecum[i]);
  const int m = m_of(I.T, idx);
  const double q = tab[moff(Ttab, m) + (idx - moff(I.T, m))].w;
  const double2* u = U0 + I.soff;
  const double2 bp = u[idx], bz = u[nlm + idx], bd = u[2 * nlm + idx];
  const double2 qbp = make_double2(q * bp.x, q * bp.y);
  const size_t o = I.roff + idx;
  r32[o] = Rhs32{make_float2((float)bz.x, (float)bz.y), make_float2((float)bd.x, (float)bd.y),
                 make_float2((float)qbp.x, (float)qbp.y)};
  rdf[o] = RhsDF{split4(bz.x, bz.y), split4(bd.x, bd.y), split4(qbp.x, qbp.y)};
}

// Cache hint: bring the line holding p from DRAM into L2 ahead of its load (the heavy
// kernel's per-warp scratch, which does not fit in L2).  Only addresses inside buffers the
// kernel reads anyway are passed.
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// ---- light kernel ------------------------------------------------------------------
// One lane solves BOTH parity chains of its (pole, m): at element k (n = m + k) chain k & 1
// holds the zeta row and the other chain the delta row, so the two recurrences share every
// table and right-hand-side load and give each lane two independent dependency chains.
constexpr int LSEG = 8;        // checkpoint interval and transposition block of the light path

struct LightSmem {
  float2 tz[LSEG][LTROW], td[LSEG][LTROW];  // zeta_n and delta_n of the block's rows, per pole
  float2 w[32], wz[32];
};

// Light checkpoints per warp: [segment][chain][lane] float4 (ct, y).
__host__ __device__ inline size_t light_ckpt_f4_per_warp(int nseg_max) { return (size_t)nseg_max * 2 * 32; }

// One forward step of both chains at element k: (ctz, yz) is the chain whose row k is a zeta
// row (diagonal z - i hw, off-diagonals +cm, +cp, right-hand side bzeta), (ctd, yd) the chain
// whose row k is a delta row (diagonal z - i hw + q Phibar/z, off-diagonals -cm, -cp,
// right-hand side bdelta + q bPhi / z).
__device__ __forceinline__ void light_fwd2(const MixedArgs& a, const PoleF& pf, const Rhs32* rb,
                                           int off, int toff, int k, float2& ctz, float2& yz,
                                           float2& ctd, float2& yd) {
  const float4 tb = __ldg(a.tab32 + toff + k);
  const Rhs32 rr = rb[off + k];
  const float2 dz = make_float2(pf.z.x, pf.z.y - tb.x);
  {
    const float2 den = make_float2(fmaf(-tb.y, ctz.x, dz.x), fmaf(-tb.y, ctz.y, dz.y));
    const float2 inv = crcpf(den);
    ctz = make_float2(tb.z * inv.x, tb.z * inv.y);
    yz = cmulf(make_float2(fmaf(-tb.y, yz.x, rr.bz.x), fmaf(-tb.y, yz.y, rr.bz.y)), inv);
  }
  {
    const float2 dd = make_float2(fmaf(tb.w, pf.gz.x, dz.x), fmaf(tb.w, pf.gz.y, dz.y));
    const float2 r = cfmaf(pf.iz, rr.qbp, rr.bd);
    const float2 den = make_float2(fmaf(tb.y, ctd.x, dd.x), fmaf(tb.y, ctd.y, dd.y));
    const float2 inv = crcpf(den);
    ctd = make_float2(-tb.z * inv.x, -tb.z * inv.y);
    yd = cmulf(make_float2(fmaf(tb.y, yd.x, r.x), fmaf(tb.y, yd.y, r.y)), inv);
  }
}

static __global__ void __launch_bounds__(MIX_WARPS * 32, 4)
k_rexi_light(MixedArgs a) {
  __shared__ LightSmem sm[MIX_WARPS];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  LightSmem& S = sm[wib];
  const int gw = blockIdx.x * MIX_WARPS + wib;
  const int W = gridDim.x * MIX_WARPS;
  float4* ckpt = reinterpret_cast<float4*>(a.scratch) + (size_t)gw * light_ckpt_f4_per_warp(a.nseg_max);
  const int total = a.ntiles_light;
  for (int round = 0; round * W < total; ++round) {
    const int t = round * W + ((round & 1) ? (W - 1 - gw) : gw);
    if (t >= total) continue;
    const Tile tl = a.tiles[t];
    const Inst I = a.insts[tl.inst];
    const int T = I.T, nlm = I.nlm;
    const int m = tl.m, K = T + 1 - m, off = moff(T, m), toff = moff(a.Ttab, m);
    const int nseg = (K + LSEG - 1) / LSEG;
    const Rhs32* rb = a.rhs32 + I.roff;
    double2* part = a.partial + I.poff + (size_t)tl.q * 3 * nlm;

    for (int gi = 0; gi < tl.ng; ++gi) {
      const PoleF pf = a.p32[I.pole0 + (tl.g0 + gi) * 32 + lane];
      __syncwarp();
      S.w[lane] = pf.w;
      S.wz[lane] = pf.wz;
      // ca[c][i], ya[c][i]: forward state of chain c after element i of the current segment
      float2 ca[2][LSEG], ya[2][LSEG];
      float2 ct[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      float2 y[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      // ---- pass 1: forward sweep of both chains with checkpoints ---------------------------
      for (int s = 0; s < nseg; ++s) {
#pragma unroll
        for (int i = 0; i < LSEG; ++i) {
          const int k = s * LSEG + i;
          const int P = i & 1;  // k & 1, the segment start being even
          if (k < K) light_fwd2(a, pf, rb, off, toff, k, ct[P], y[P], ct[1 - P], y[1 - P]);
          ca[0][i] = ct[0];
          ya[0][i] = y[0];
          ca[1][i] = ct[1];
          ya[1][i] = y[1];
        }
        if (s + 1 < nseg) {
          ckpt[((size_t)s * 2 + 0) * 32 + lane] = make_float4(ct[0].x, ct[0].y, y[0].x, y[0].y);
          ckpt[((size_t)s * 2 + 1) * 32 + lane] = make_float4(ct[1].x, ct[1].y, y[1].x, y[1].y);
        }
      }
      // ---- pass 2: backward over segments, recomputing each from its checkpoint -----------
      float2 xn[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      for (int s = nseg - 1; s >= 0; --s) {
        if (s != nseg - 1) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            if (s > 0) {
              const float4 st = ckpt[((size_t)(s - 1) * 2 + c) * 32 + lane];
              ct[c] = make_float2(st.x, st.y);
              y[c] = make_float2(st.z, st.w);
            } else {
              ct[c] = make_float2(0.f, 0.f);
              y[c] = make_float2(0.f, 0.f);
            }
          }
#pragma unroll
          for (int i = 0; i < LSEG; ++i) {
            const int P = i & 1;
            light_fwd2(a, pf, rb, off, toff, s * LSEG + i, ct[P], y[P], ct[1 - P], y[1 - P]);  // k < K
            ca[0][i] = ct[0];
            ya[0][i] = y[0];
            ca[1][i] = ct[1];
            ya[1][i] = y[1];
          }
        }
#pragma unroll
        for (int i = LSEG - 1; i >= 0; --i) {
          const int k = s * LSEG + i;
          if (k < K) {
            float2 x[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              x[c] = make_float2(ya[c][i].x - fmaf(ca[c][i].x, xn[c].x, -ca[c][i].y * xn[c].y),
                                 ya[c][i].y - fmaf(ca[c][i].x, xn[c].y, ca[c][i].y * xn[c].x));
              xn[c] = x[c];
            }
            S.tz[i][lane] = x[i & 1];        // zeta_{m+k}
            S.td[i][lane] = x[1 - (i & 1)];  // delta_{m+k}
          }
        }
        __syncwarp();
        // block reduction: lane (r, h) sums row r over the 8 poles [8h, 8h + 8); the four
        // quarters are combined by shuffles
        {
          const int r = lane & (LSEG - 1), h = lane >> 3;
          const int k = s * LSEG + r;
          const bool valid = k < K;
          float2 az = make_float2(0.f, 0.f), ad = az, af = az;
          if (valid) {
#pragma unroll
            for (int p = 8 * h; p < 8 * h + 8; ++p) {
              const float2 xz = S.tz[r][p], xd = S.td[r][p];
              const float2 wp = S.w[p];
              az = cfmaf(wp, xz, az);
              ad = cfmaf(wp, xd, ad);
              af = cfmaf(S.wz[p], xd, af);
            }
          }
#pragma unroll
          for (int sh = 8; sh <= 16; sh <<= 1) {
            az.x += __shfl_xor_sync(0xffffffffu, az.x, sh);
            az.y += __shfl_xor_sync(0xffffffffu, az.y, sh);
            ad.x += __shfl_xor_sync(0xffffffffu, ad.x, sh);
            ad.y += __shfl_xor_sync(0xffffffffu, ad.y, sh);
            af.x += __shfl_xor_sync(0xffffffffu, af.x, sh);
            af.y += __shfl_xor_sync(0xffffffffu, af.y, sh);
          }
          if (h == 0 && valid) {  // double-float partial slots (no FP64 arithmetic here)
            float4* d0 = reinterpret_cast<float4*>(part + off + k);
            dfp_add(d0, make_float4(az.x, 0.f, az.y, 0.f), gi == 0);
            dfp_add(d0 + nlm, make_float4(ad.x, 0.f, ad.y, 0.f), gi == 0);
            dfp_add(d0 + 2 * nlm, make_float4(af.x, 0.f, af.y, 0.f), gi == 0);
          }
        }
        __syncwarp();
      }
    }
  }
}

// ---- heavy kernel ------------------------------------------------------------------
// Row k of a heavy chain in double-float: the diagonal d_k and the off-diagonals lo_k, up_k.
// They depend on the pole and the matrix only, so a tile that carries two states forms them once.
struct HeavyRow {
  dfc d;
  df lo, up;
};
__device__ __forceinline__ HeavyRow heavy_row(const MixedArgs& a, const PoleDF& pq, int toff, int k, bool isZ) {
  const TabDF tb = a.tabdf[toff + k];
  const df hw{tb.a.x, tb.a.y}, cm{tb.a.z, tb.a.w}, cp{tb.b.x, tb.b.y}, q{tb.b.z, tb.b.w};
  const dfc z = dfc_of(pq.z);
  HeavyRow R;
  if (isZ) {
    R.d = dfc{z.re, df_add(z.im, df_neg(hw))};
  } else {
    const dfc gz = dfc_of(pq.gz);
    R.d = dfc{df_add(z.re, df_mul(q, gz.re)), df_add(df_add(z.im, df_neg(hw)), df_mul(q, gz.im))};
  }
  R.lo = isZ ? cm : df_neg(cm);
  R.up = isZ ? cp : df_neg(cp);
  return R;
}

// residual of one state's chain row k:  r_k - d_k x_k - lo_k x_{k-1} - up_k x_{k+1}, each
// component one compensated dot product of the double-float row and right-hand side with the
// FP32 solution; delta rows add q bPhi / z (double-float times double-float) to the right-hand
// side inside the same sum
__device__ __forceinline__ float2 heavy_residual(const HeavyRow& R, const PoleDF& pq, const RhsDF& rr, bool isZ,
                                                 bool has_m, bool has_p, float2 xm, float2 x0, float2 xp) {
  dot2 re, im;
  if (isZ) {
    re = dot2{rr.bz.x, rr.bz.y};
    im = dot2{rr.bz.z, rr.bz.w};
  } else {
    re = dot2{rr.bd.x, rr.bd.y};
    im = dot2{rr.bd.z, rr.bd.w};
    const df izr{pq.iz.x, pq.iz.y}, izi{pq.iz.z, pq.iz.w}, qr{rr.qbp.x, rr.qbp.y}, qi{rr.qbp.z, rr.qbp.w};
    dot2_add2(re, izr, qr);
    dot2_add2(re, df_neg(izi), qi);
    dot2_add2(im, izr, qi);
    dot2_add2(im, izi, qr);
  }
  // - d x0 = -(d.re x0.re - d.im x0.im) - i (d.re x0.im + d.im x0.re)
  dot2_add(re, R.d.re, -x0.x);
  dot2_add(re, R.d.im, x0.y);
  dot2_add(im, R.d.re, -x0.y);
  dot2_add(im, R.d.im, -x0.x);
  if (has_m) {
    dot2_add(re, R.lo, -xm.x);
    dot2_add(im, R.lo, -xm.y);
  }
  if (has_p) {
    dot2_add(re, R.up, -xp.x);
    dot2_add(im, R.up, -xp.y);
  }
  return make_float2(re.s + re.err, im.s + im.err);
}

// FP32 pivot recurrence of a chain at element k: returns the inverse pivot 1/(d_k - lo_k ct_{k-1})
// and advances ct to ct_k = up_k / pivot (the LU form of Thomas elimination).
__device__ __forceinline__ float2 heavy_pivot(const float4 tb, const PoleF& pf, bool isZ, float2& ct) {
  const float lo = isZ ? tb.y : -tb.y;
  const float up = isZ ? tb.z : -tb.z;
  float2 d;
  if (isZ) d = make_float2(pf.z.x, pf.z.y - tb.x);
  else d = make_float2(fmaf(tb.w, pf.gz.x, pf.z.x), fmaf(tb.w, pf.gz.y, pf.z.y - tb.x));
  const float2 den = make_float2(fmaf(-lo, ct.x, d.x), fmaf(-lo, ct.y, d.y));
  const float2 inv = crcpf(den);
  ct = make_float2(up * inv.x, up * inv.y);
  return inv;
}

// One state's forward value at element k: y_k = (r_k - lo_k y_{k-1}) / pivot_k.
__device__ __forceinline__ float2 heavy_y(const PoleF& pf, const Rhs32& rr, bool isZ, float lo, float2 inv, float2 y) {
  const float2 r = isZ ? rr.bz : cfmaf(pf.iz, rr.qbp, rr.bd);
  return cmulf(make_float2(fmaf(-lo, y.x, r.x), fmaf(-lo, y.y, r.y)), inv);
}

constexpr int HBLK = 16;     // heavy: rows per transposition block of the pole sums
constexpr int HSEG_MIN = 4;  // heavy: shortest checkpoint interval (sizes the checkpoint scratch)
// checkpoint interval of a heavy tile carrying G states (segments recomputed into shared memory)
template <int G>
__host__ __device__ constexpr int heavy_seg() { return G == 2 ? 4 : 8; }
static_assert((HBLK & (HBLK - 1)) == 0, "power of two: block positions use masks");
__device__ __forceinline__ int hblk_pos(int k) { return k & (HBLK - 1); }

// Heavy per-warp scratch in float2 units, sized for the shortest interval and two states:
// forward checkpoints [ceil(kmax / HSEG_MIN)][32][3] (ct, y of each state), the correction's
// factor g[kmax][32] (shared by the states of a tile), and h[2][kmax][32].
__host__ __device__ inline int heavy_nseg(int kmax) { return (kmax + HSEG_MIN - 1) / HSEG_MIN; }
__host__ __device__ inline size_t heavy_scratch_f2_per_warp(int kmax) {
  return (size_t)heavy_nseg(kmax) * 32 * 3 + (size_t)kmax * 32 * 3;
}

// sum over 16 poles of w_p x_p in double-float (w in the packed layout, x in FP32), returned
// as (re.hi, re.lo, im.hi, im.lo): two packed accumulators, sum_p (w.re x.re, w.im x.re) and
// sum_p (w.re x.im, w.im x.im), combined once: re = first.re - second.im, im = second.re + first.im
__device__ __forceinline__ float4 heavy_dfsum16(const float2* x, const float4* w) {
  const float2 z2 = make_float2(0.f, 0.f);
  float2 a1h = z2, a1l = z2, a2h = z2, a2l = z2;
#pragma unroll 4
  for (int p = 0; p < 16; ++p) {
    const float2 v = x[p];
    const float4 wp = w[p];
    df2_acc(a1h, a1l, make_float2(wp.x, wp.y), make_float2(wp.z, wp.w), make_float2(v.x, v.x));
    df2_acc(a2h, a2l, make_float2(wp.x, wp.y), make_float2(wp.z, wp.w), make_float2(v.y, v.y));
  }
  const df re = df_add(df{a1h.x, a1l.x}, df{-a2h.y, -a2l.y}), im = df_add(df{a2h.x, a2l.x}, df{a1h.y, a1l.y});
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}

// Pole sums of one transposition block: lane (r, h) sums row kb + r over the 16 poles of half
// h; dfsum: double-float products with the double-float weights (the solution x), else FP32
// (the small correction); the halves are combined by a shuffle and added into the tile's
// double-float partial slots (written when first = true).  Weights are in the packed layout
// (re.hi, im.hi, re.lo, im.lo).
// HALVES (tiles of state pairs): the two half-warps hold different states on the same 16 poles,
// so each half writes its own row sums (when wr) and nothing is combined across halves.
template <bool HALVES>
__device__ __forceinline__ void heavy_block_sum(const float2* tile, const float4* s_w, const float4* s_wz, int kb,
                                                int K, int c, int lane, bool dfsum, bool first, double2* part,
                                                int off, int nlm, bool wr = true) {
  const int r = lane & 15, h = lane >> 4;
  const int kk = kb + r;
  const bool valid = kk < K;
  const bool isD = ((kk & 1) != c);
  float4 f1 = make_float4(0.f, 0.f, 0.f, 0.f), f2 = f1;  // double-float (re.hi, re.lo, im.hi, im.lo)
  if (valid) {
    if (dfsum) {
      f1 = heavy_dfsum16(tile + r * LTROW + 16 * h, s_w + 16 * h);
      if (isD) f2 = heavy_dfsum16(tile + r * LTROW + 16 * h, s_wz + 16 * h);
    } else {
      float2 g1 = make_float2(0.f, 0.f), g2 = g1;
#pragma unroll 4
      for (int p = 16 * h; p < 16 * h + 16; ++p) {
        const float2 v = tile[r * LTROW + p];
        const float4 w = s_w[p];
        g1 = cfmaf(make_float2(w.x, w.y), v, g1);
        if (isD) {
          const float4 wz = s_wz[p];
          g2 = cfmaf(make_float2(wz.x, wz.y), v, g2);
        }
      }
      f1 = make_float4(g1.x, 0.f, g1.y, 0.f);
      f2 = make_float4(g2.x, 0.f, g2.y, 0.f);
    }
  }
  if (HALVES) {
    if (valid && wr) {
      dfp_add(reinterpret_cast<float4*>(part + (isD ? nlm : 0) + off + kk), f1, first);
      if (isD) dfp_add(reinterpret_cast<float4*>(part + 2 * nlm + off + kk), f2, first);
    }
    return;
  }
  // combine the two halves: two-sum of the high words, low words added
  float4 o1, o2;
  o1.x = __shfl_xor_sync(0xffffffffu, f1.x, 16);
  o1.y = __shfl_xor_sync(0xffffffffu, f1.y, 16);
  o1.z = __shfl_xor_sync(0xffffffffu, f1.z, 16);
  o1.w = __shfl_xor_sync(0xffffffffu, f1.w, 16);
  o2.x = __shfl_xor_sync(0xffffffffu, f2.x, 16);
  o2.y = __shfl_xor_sync(0xffffffffu, f2.y, 16);
  o2.z = __shfl_xor_sync(0xffffffffu, f2.z, 16);
  o2.w = __shfl_xor_sync(0xffffffffu, f2.w, 16);
  if (h == 0 && valid) {
    float4 s1, s2;
    {
      const df a = df_two_sum(f1.x, o1.x), b = df_two_sum(f1.z, o1.z);
      s1 = make_float4(a.hi, (f1.y + o1.y) + a.lo, b.hi, (f1.w + o1.w) + b.lo);
      const df c2 = df_two_sum(f2.x, o2.x), d2 = df_two_sum(f2.z, o2.z);
      s2 = make_float4(c2.hi, (f2.y + o2.y) + c2.lo, d2.hi, (f2.w + o2.w) + d2.lo);
    }
    float4* dst = reinterpret_cast<float4*>(part + (isD ? nlm : 0) + off + kk);
    dfp_add(dst, s1, first);
    if (isD) dfp_add(reinterpret_cast<float4*>(part + 2 * nlm + off + kk), s2, first);
  }
}

// Heavy poles: FP32 LU solve with checkpoints (pass A, upward); pass B (downward) recomputes
// each segment into a per-warp shared buffer, back-substitutes x, forms the residual r - A x of
// element k + 1 in double-float once x_k is known, and eliminates the correction system
// bottom-up (UL form of Thomas: p_k = d_k - up_k g_{k+1}, g_k = lo_k / p_k,
// h_k = (res_k - up_k h_{k+1}) / p_k), storing g and h; pass C (upward) completes the
// correction dx_k = h_k - g_k dx_{k-1}.  Pole sums: x in double-float in pass B, dx in FP32
// in pass C (|dx| ~ 1e-6 |x|).  A tile carries G states of the same truncation and pole set
// (G = 2 pairs the states of a batch): the pivots, the correction's factor g, the double-float
// diagonal and every table load are formed once for both; right-hand sides, x, residuals, h
// and the pole sums are per state.  All loops stay rolled so that the residual's code exists
// once per state.
template <int G, bool HALVES>
static __global__ void __launch_bounds__(MIX_WARPS * 32, G == 2 ? 4 : 6)
k_rexi_heavy(MixedArgs a, int t0, int nt) {
  static_assert(G == 2 || !HALVES, "half-warp tiles carry state pairs");
  constexpr int SEG = heavy_seg<G>();
  constexpr int SW = 1 + G;  // float2 per lane and element in the segment buffer: inv, y of each state
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // per warp: transposition tiles [G][HBLK][LTROW] float2, the double-float weights w, w/z,
  // and the recomputed segment [SEG][32][SW] float2
  float2* s_tile = reinterpret_cast<float2*>(smem_raw) + wib * (G * HBLK * LTROW);
  float4* s_w = reinterpret_cast<float4*>(smem_raw + (size_t)MIX_WARPS * G * HBLK * LTROW * sizeof(float2)) + wib * 64;
  float4* s_wz = s_w + 32;
  float2* s_seg = reinterpret_cast<float2*>(smem_raw + (size_t)MIX_WARPS * G * HBLK * LTROW * sizeof(float2) +
                                            (size_t)MIX_WARPS * 64 * sizeof(float4)) + wib * (SEG * 32 * SW);
  const int gw = blockIdx.x * MIX_WARPS + wib;
  const int W = gridDim.x * MIX_WARPS;
  float2* hs = reinterpret_cast<float2*>(reinterpret_cast<char*>(a.scratch) +
                                         (size_t)a.warps_light * light_ckpt_f4_per_warp(a.nseg_max) * sizeof(float4)) +
               (size_t)gw * heavy_scratch_f2_per_warp(a.kmax);
  float2* ck = hs;                                              // [nseg][32][SW]
  float2* Gs = hs + (size_t)heavy_nseg(a.kmax) * 32 * 3;        // [kmax][32]
  float2* Hs = Gs + (size_t)a.kmax * 32;                        // [G][kmax][32]

  for (int round = 0; round * W < nt; ++round) {
    const int t = round * W + ((round & 1) ? (W - 1 - gw) : gw);
    if (t >= nt) continue;
    const Tile tl = a.tiles[t0 + t];
    // HALVES: half-warp h solves pair h on the same 16 poles; a missing second pair (inst3 < 0)
    // is replaced by the first, whose results that half then does not write
    const int half = lane >> 4;
    const bool second = HALVES && half && tl.inst3 >= 0;
    const bool wr = !HALVES || !half || second;
    Inst I[G];
    I[0] = a.insts[second ? tl.inst3 : tl.inst];
    if (G == 2) I[G - 1] = a.insts[second ? tl.inst4 : tl.inst2];
    const int T = I[0].T, nlm = I[0].nlm;
    const int m = tl.m, c = tl.chain, K = T + 1 - m, off = moff(T, m), toff = moff(a.Ttab, m);
    const Rhs32* rb[G];
    const RhsDF* rbd[G];
    double2* part[G];
#pragma unroll
    for (int s = 0; s < G; ++s) {
      rb[s] = a.rhs32 + I[s].roff + off;
      rbd[s] = a.rhsdf + I[s].roff + off;
      part[s] = a.partial + I[s].poff + (size_t)tl.q * 3 * nlm;
    }

    for (int gi = 0; gi < tl.ng; ++gi) {
      // 32 poles of the 32-pole group g0 + gi; HALVES: 16 poles from the pole offset g0 + 16 gi
      const int pidx = HALVES ? I[0].pole0 + tl.g0 + 16 * gi + (lane & 15) : I[0].pole0 + (tl.g0 + gi) * 32 + lane;
      const PoleF pf = a.p32[pidx];
      const PoleDF pq = a.pdf[pidx];
      __syncwarp();
      s_w[lane] = w_packed(pq.w);
      s_wz[lane] = w_packed(pq.wz);
      // ---- A: FP32 forward sweep, checkpoint (ct, y) after every full segment ---------------
      {
        float2 ct = make_float2(0.f, 0.f), y[G];
#pragma unroll
        for (int s = 0; s < G; ++s) y[s] = make_float2(0.f, 0.f);
#pragma unroll 4  // loads of four elements in flight
        for (int k = 0; k < K; ++k) {
          const float4 tb = __ldg(a.tab32 + toff + k);
          const bool isZ = ((k & 1) == c);
          const float lo = isZ ? tb.y : -tb.y;
          const float2 inv = heavy_pivot(tb, pf, isZ, ct);
#pragma unroll
          for (int s = 0; s < G; ++s) y[s] = heavy_y(pf, rb[s][k], isZ, lo, inv, y[s]);
          if ((k & (SEG - 1)) == SEG - 1 && k + 1 < K) {
            float2* cp = ck + ((size_t)(k / SEG) * 32 + lane) * SW;
            cp[0] = ct;
#pragma unroll
            for (int s = 0; s < G; ++s) cp[1 + s] = y[s];
          }
        }
      }
      // ---- B: downward; e = -1 only finalises element 0 ----------------------------------
      float2 x0[G], x1[G], x2[G], hU[G];  // x_e, x_{e+1}, x_{e+2}; h of element e + 2
#pragma unroll
      for (int s = 0; s < G; ++s) x1[s] = x2[s] = hU[s] = make_float2(0.f, 0.f);
      float2 gU = make_float2(0.f, 0.f);  // g of element e + 2
#pragma unroll 1
      for (int e = K - 1; e >= -1; --e) {
#pragma unroll
        for (int s = 0; s < G; ++s) x0[s] = make_float2(0.f, 0.f);
        if (e >= 0) {
          const int i = e & (SEG - 1);
          if (e == K - 1 || i == SEG - 1) {  // entering a segment from above: recompute it
            const int sg = e / SEG;
            float2 cs = make_float2(0.f, 0.f), ys[G];
#pragma unroll
            for (int s = 0; s < G; ++s) ys[s] = make_float2(0.f, 0.f);
            if (sg > 0) {
              const float2* cp = ck + ((size_t)(sg - 1) * 32 + lane) * SW;
              cs = cp[0];
#pragma unroll
              for (int s = 0; s < G; ++s) ys[s] = cp[1 + s];
              // checkpoints of the segments below (DRAM) into L2 while this one is worked on: two
              // segments ahead, both on entering the top segment
              if (sg > 2) prefetch_l2(ck + ((size_t)(sg - 3) * 32 + lane) * SW);
              if (e == K - 1 && sg > 1) prefetch_l2(ck + ((size_t)(sg - 2) * 32 + lane) * SW);
            }
#pragma unroll
            for (int k = sg * SEG; k <= e; ++k) {
              const float4 tb = __ldg(a.tab32 + toff + k);
              const bool isZ = ((k & 1) == c);
              const float lo = isZ ? tb.y : -tb.y;
              const float2 inv = heavy_pivot(tb, pf, isZ, cs);
              float2* sp = s_seg + ((k & (SEG - 1)) * 32 + lane) * SW;
              sp[0] = inv;
#pragma unroll
              for (int s = 0; s < G; ++s) {
                ys[s] = heavy_y(pf, rb[s][k], isZ, lo, inv, ys[s]);
                sp[1 + s] = ys[s];
              }
            }
          }
          const float2* sp = s_seg + (i * 32 + lane) * SW;
          const float4 tb = __ldg(a.tab32 + toff + e);
          const float up = ((e & 1) == c) ? tb.z : -tb.z;
          const float2 cc = make_float2(up * sp[0].x, up * sp[0].y);
#pragma unroll
          for (int s = 0; s < G; ++s) {
            const float2 yv = sp[1 + s];
            x0[s] = make_float2(yv.x - fmaf(cc.x, x1[s].x, -cc.y * x1[s].y),
                                yv.y - fmaf(cc.x, x1[s].y, cc.y * x1[s].x));
            s_tile[(s * HBLK + hblk_pos(e)) * LTROW + lane] = x0[s];
          }
        }
        if (e + 1 < K) {  // element k = e + 1: residual with x_{k-1} = x0, x_k = x1, x_{k+1} = x2
          const int k = e + 1;
          const float4 tb = __ldg(a.tab32 + toff + k);
          const bool isZ = ((k & 1) == c);
          const float lo = isZ ? tb.y : -tb.y;
          const float up = isZ ? tb.z : -tb.z;
          float2 d;
          if (isZ) d = make_float2(pf.z.x, pf.z.y - tb.x);
          else d = make_float2(fmaf(tb.w, pf.gz.x, pf.z.x), fmaf(tb.w, pf.gz.y, pf.z.y - tb.x));
          const float2 den = make_float2(fmaf(-up, gU.x, d.x), fmaf(-up, gU.y, d.y));
          const float2 inv = crcpf(den);
          gU = make_float2(lo * inv.x, lo * inv.y);
          // g depends on the pole only: with half-warps, lanes r and r + 16 hold the same pole, so
          // the lower half stores it and both halves read that copy
          if (!HALVES || half == 0) Gs[(size_t)k * 32 + lane] = gU;
          const HeavyRow R = heavy_row(a, pq, toff, k, isZ);
#pragma unroll
          for (int s = 0; s < G; ++s) {
            const float2 res = heavy_residual(R, pq, rbd[s][k], isZ, k > 0, k + 1 < K, x0[s], x1[s], x2[s]);
            hU[s] = cmulf(make_float2(fmaf(-up, hU[s].x, res.x), fmaf(-up, hU[s].y, res.y)), inv);
            Hs[((size_t)s * a.kmax + k) * 32 + lane] = hU[s];
          }
        }
        if (e >= 0) {
          if (hblk_pos(e) == 0) {
            __syncwarp();
#pragma unroll
            for (int s = 0; s < G; ++s)
              heavy_block_sum<HALVES>(s_tile + s * HBLK * LTROW, s_w, s_wz, e, K, c, lane, true, gi == 0, part[s], off,
                                      nlm, wr);
            __syncwarp();
          }
#pragma unroll
          for (int s = 0; s < G; ++s) {
            x2[s] = x1[s];
            x1[s] = x0[s];
          }
        }
      }
      // ---- C: upward: dx_k = h_k - g_k dx_{k-1}, FP32 pole sums of dx ----------------------
      if (HALVES) __syncwarp();  // orders the lower half's g stores before the upper half's loads
      float2 dxm[G];
#pragma unroll
      for (int s = 0; s < G; ++s) dxm[s] = make_float2(0.f, 0.f);
      constexpr int PFD = 4;  // pass C: g and h rows brought into L2 this many elements ahead
#pragma unroll 4  // loads of four elements in flight
      for (int k = 0; k < K; ++k) {
        // four rows (1 KB per array) per hint, lane l at byte 32 l; rows below kmax are in the buffer
        if ((k & 3) == 0 && k + PFD + 4 <= a.kmax) {
          // half-warps: only the first 128 bytes of each g row are used (8 lanes per row)
          prefetch_l2(HALVES ? Gs + (size_t)(k + PFD + (lane >> 3)) * 32 + 2 * (lane & 7)
                             : Gs + (size_t)(k + PFD) * 32 + 4 * lane);
#pragma unroll
          for (int s = 0; s < G; ++s) prefetch_l2(Hs + ((size_t)s * a.kmax + k + PFD) * 32 + 4 * lane);
        }
        const float2 g = Gs[(size_t)k * 32 + (HALVES ? (lane & 15) : lane)];
#pragma unroll
        for (int s = 0; s < G; ++s) {
          const float2 h = Hs[((size_t)s * a.kmax + k) * 32 + lane];
          const float2 dx = make_float2(h.x - fmaf(g.x, dxm[s].x, -g.y * dxm[s].y),
                                        h.y - fmaf(g.x, dxm[s].y, g.y * dxm[s].x));
          dxm[s] = dx;
          s_tile[(s * HBLK + hblk_pos(k)) * LTROW + lane] = dx;
        }
        if (hblk_pos(k) == HBLK - 1 || k == K - 1) {
          __syncwarp();
#pragma unroll
          for (int s = 0; s < G; ++s)
            heavy_block_sum<HALVES>(s_tile + s * HBLK * LTROW, s_w, s_wz, k - hblk_pos(k), K, c, lane, false, false,
                                    part[s], off, nlm, wr);
          __syncwarp();
        }
      }
    }
  }
}

template <int G>
inline size_t heavy_smem_bytes() {
  return sizeof(float2) * MIX_WARPS * G * HBLK * LTROW + sizeof(float4) * MIX_WARPS * 64 +
         sizeof(float2) * MIX_WARPS * heavy_seg<G>() * 32 * (1 + G);
}

}  // namespace rexi
