// FP64 REXI solve kernel (the plain FP64 path).
//
// Work decomposition: a tile is (instance, zonal order m, parity chain c, range of 32-pole
// groups of the instance's pole set).  One warp owns a tile; lane l solves the chain for
// pole g*32 + l, so the 32 systems of a warp share m, the chain and every table /
// right-hand-side element (warp broadcast loads), and differ only in the pole.  Instances
// may differ in truncation, time step and pole set (ragged launches).
//
// The system (z - dt L_m) u = U0_m is solved in the equivalent scaled form
// (z' - L_m) v = U0_m with z' = z / dt and v = dt u, so the tables are independent of dt and
// every instance brings its own scaled poles (z', w' = w / dt, w/z, 1/z', Phibar / z').
// Eliminating Phi_n = (bPhi_n - Phibar delta_n) / z' leaves two tridiagonal chains in
// (zeta, delta) by parity of n - m.  Row n reads
//   zeta row : (z' - i w_n) zeta_n + cm_n x_{n-1} + cp_n x_{n+1} = bzeta_n
//   delta row: (z' - i w_n + q_n Phibar / z') delta_n - cm_n x_{n-1} - cp_n x_{n+1}
//              = bdelta_n + q_n bPhi_n / z'
// with w_n = 2 Omega m / (n(n+1)), cm_n = 2 Omega (n+1)/n eps_n, cp_n = 2 Omega n/(n+1) eps_{n+1},
// q_n = n(n+1)/a^2 (one table for the largest truncation of the launch serves all: the
// coupling beyond an instance's last degree never enters its elimination).
// The chain is solved by the Thomas algorithm without pivoting: for the REXI poles the
// shifted operator is a scaled identity plus a skew-adjoint part in the energy norm, so the
// elimination is stable.  The forward coefficients are kept in a per-warp global scratch
// slot ([k][lane], coalesced); FP64 arithmetic is slow enough on this part that the scratch
// traffic is far below the HBM roofline.
//
// The weighted sums over poles are formed by transposing 32 solution rows through shared
// memory, so that lane r sums row r over the 32 poles of the group:
//   S_zeta / S_delta = sum_p w_p x_p,   S_wz = sum_p (w_p / z_p) delta_p,
// (S over the scaled solutions with the scaled weights), and
// Phi = bPhi * sum_p w_p/z_p - Phibar * S_wz is formed in the finalize kernel.
#pragma once
#include "common.cuh"

namespace rexi {

struct Fp64Args {
  const double2* U0;   // state base
  double2* partial;    // partial-sum base
  const D4* tab;       // [moff(Ttab, m) + n - m] (w_n, cm_n, cp_n, q_n)
  const PoleD* poles;  // scaled poles of every pole set of the launch
  const Tile* tiles;   // [ntiles]
  const Inst* insts;
  D4* scratch;         // [warps][kmax][32]
  int ntiles, Ttab, kmax;
  int alt = 0;         // 1: the FP64 class of a mixed plan (partial slots at Inst::poff64)
};

constexpr int FP64_WARPS = 4;
constexpr int FP64_TROW = 33;  // padded row (in double2) of the transposition tile

static __global__ void __launch_bounds__(FP64_WARPS * 32)
k_rexi_fp64(Fp64Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double2* s_tile = reinterpret_cast<double2*>(smem_raw) + wib * (32 * FP64_TROW);
  double2* s_w = reinterpret_cast<double2*>(smem_raw) + FP64_WARPS * 32 * FP64_TROW + wib * 64;
  double2* s_wz = s_w + 32;

  const int gw = blockIdx.x * FP64_WARPS + wib;
  const int W = gridDim.x * FP64_WARPS;
  D4* scr = a.scratch + (size_t)gw * a.kmax * 32;
  const int total = a.ntiles;

  for (int round = 0; round * W < total; ++round) {
    const int t = round * W + ((round & 1) ? (W - 1 - gw) : gw);  // snake over LPT order
    if (t >= total) continue;
    const Tile tl = a.tiles[t];
    const Inst I = a.insts[tl.inst];
    const int T = I.T, nlm = I.nlm;
    const int m = tl.m, c = tl.chain, K = T + 1 - m, off = moff(T, m), toff = moff(a.Ttab, m);
    const double2* bP = a.U0 + I.soff;
    const double2* bZ = bP + nlm;
    const double2* bD = bP + 2 * nlm;
    double2* part = a.partial + (a.alt ? I.poff64 : I.poff) + (size_t)tl.q * 3 * nlm;

    for (int gi = 0; gi < tl.ng; ++gi) {
      const PoleD pd = a.poles[I.pole0 + (tl.g0 + gi) * 32 + lane];
      __syncwarp();
      s_w[lane] = pd.w;
      s_wz[lane] = pd.wz;

      // ---- forward elimination --------------------------------------------------
      double2 ct = make_double2(0.0, 0.0), y = make_double2(0.0, 0.0);
      for (int k = 0; k < K; ++k) {
        const int idx = off + k;
        const D4 tb = a.tab[toff + k];  // x: w_n, y: cm, z: cp, w: q
        const bool isZ = ((k & 1) == c);
        const double lo = isZ ? tb.y : -tb.y;
        const double up = isZ ? tb.z : -tb.z;
        double2 d, r;
        if (isZ) {
          d = make_double2(pd.z.x, pd.z.y - tb.x);
          r = bZ[idx];
        } else {
          d = make_double2(fma(tb.w, pd.gz.x, pd.z.x), fma(tb.w, pd.gz.y, pd.z.y - tb.x));
          const double2 t2 = cmul(pd.iz, bP[idx]);
          const double2 bd = bD[idx];
          r = make_double2(fma(tb.w, t2.x, bd.x), fma(tb.w, t2.y, bd.y));
        }
        const double2 den = make_double2(fma(-lo, ct.x, d.x), fma(-lo, ct.y, d.y));
        const double2 inv = crcp64(den);
        ct = make_double2(up * inv.x, up * inv.y);
        y = cmul(make_double2(fma(-lo, y.x, r.x), fma(-lo, y.y, r.y)), inv);
        scr[(size_t)k * 32 + lane] = D4{ct.x, ct.y, y.x, y.y};
      }

      // ---- back substitution with transposed weighted sums ------------------------
      double2 xn = make_double2(0.0, 0.0);
      for (int k = K - 1; k >= 0; --k) {
        const D4 s = scr[(size_t)k * 32 + lane];
        const double2 x = make_double2(s.z - fma(s.x, xn.x, -s.y * xn.y),
                                       s.w - fma(s.x, xn.y, s.y * xn.x));
        s_tile[(k & 31) * FP64_TROW + lane] = x;
        xn = x;
        if ((k & 31) == 0) {
          __syncwarp();
          // lane r: row r, sum over the 32 poles with w
          const int kk = k + lane;
          if (kk < K) {
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll 8
            for (int p = 0; p < 32; ++p) acc = cfma(s_w[p], s_tile[lane * FP64_TROW + p], acc);
            double2* dst = part + (((kk & 1) == c) ? 0 : nlm) + off + kk;
            if (gi == 0) *dst = acc;
            else *dst = cadd(*dst, acc);
          }
          // delta rows (parity != c): sum with w/z, two half-warps over 16 poles each
          const int j = lane & 15, h = lane >> 4;
          const int rowd = 2 * j + (1 - c);
          const int kd = k + rowd;
          double2 acc2 = make_double2(0.0, 0.0);
          if (kd < K) {
#pragma unroll 8
            for (int p = 16 * h; p < 16 * h + 16; ++p)
              acc2 = cfma(s_wz[p], s_tile[rowd * FP64_TROW + p], acc2);
          }
          acc2.x += __shfl_xor_sync(0xffffffffu, acc2.x, 16);
          acc2.y += __shfl_xor_sync(0xffffffffu, acc2.y, 16);
          if (h == 0 && kd < K) {
            double2* dst = part + 2 * nlm + off + kd;
            if (gi == 0) *dst = acc2;
            else *dst = cadd(*dst, acc2);
          }
          __syncwarp();
        }
      }
    }
  }
}

inline size_t fp64_smem_bytes() {
  return sizeof(double2) * (FP64_WARPS * 32 * FP64_TROW + FP64_WARPS * 64);
}

// U1 = (bPhi S0 - Phibar S_wz, S_zeta, S_delta) for every coefficient of every instance,
// summing the instance's Q partial slots in order, then (mixed plans with poles solved in FP64)
// its Q64 FP64 slots in partial64, in FP64.
// Partial slots hold FP64 complex sums (DF = false, FP64 plans) or double-float pairs
// (DF = true, mixed plans: float4 = re.hi, re.lo, im.hi, im.lo, the same 16 bytes per entry).
template <bool DF>
static __global__ void k_rexi_finalize(const double2* __restrict__ U0, const double2* __restrict__ partial,
                                       double2* __restrict__ U1, const Inst* __restrict__ insts,
                                       const long long* __restrict__ ecum, int ninst, long long total,
                                       double phibar, const double2* __restrict__ partial64) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int i = inst_of(ecum, ninst, e);
  const Inst I = insts[i];
  const int nlm = I.nlm, idx = (int)(e - ecum[i]);
  double2 sz = make_double2(0, 0), sd = sz, sw = sz;
  if (I.msize > 1 && m_pair(I.T, m_of(I.T, idx)) % I.msize != I.mrank) {  // another rank's order
    double2* o = U1 + I.soff + idx;
    o[0] = sz;
    o[nlm] = sz;
    o[2 * nlm] = sz;
    return;
  }
  const double2* p = partial + I.poff + idx;
  if (DF) {
    // double-float slots summed in double-float (two-sum of the high words, low words added),
    // in the same fixed order; one conversion to FP64 at the end
    float4 az = make_float4(0.f, 0.f, 0.f, 0.f), ad = az, aw = az;
    auto add = [](float4& acc, const double2* q) {
      const float4 v = *reinterpret_cast<const float4*>(q);
      float s = acc.x + v.x, bb = s - acc.x;
      const float ex = (acc.x - (s - bb)) + (v.x - bb);
      acc.x = s;
      acc.y += v.y + ex;
      s = acc.z + v.z;
      bb = s - acc.z;
      const float ez = (acc.z - (s - bb)) + (v.z - bb);
      acc.z = s;
      acc.w += v.w + ez;
    };
#pragma unroll 4  // loads of several slots in flight; the order of the sums is unchanged
    for (int q = 0; q < I.Q; ++q) {
      add(az, p);
      add(ad, p + nlm);
      add(aw, p + 2 * nlm);
      p += 3 * nlm;
    }
    sz = make_double2((double)az.x + (double)az.y, (double)az.z + (double)az.w);
    sd = make_double2((double)ad.x + (double)ad.y, (double)ad.z + (double)ad.w);
    sw = make_double2((double)aw.x + (double)aw.y, (double)aw.z + (double)aw.w);
  } else {
    for (int q = 0; q < I.Q; ++q) {
      sz = cadd(sz, p[0]);
      sd = cadd(sd, p[nlm]);
      sw = cadd(sw, p[2 * nlm]);
      p += 3 * nlm;
    }
  }
  if (I.Q64 > 0) {  // the FP64 class: sums whose cancellation double-float slots cannot carry
    const double2* p64 = partial64 + I.poff64 + idx;
    for (int q = 0; q < I.Q64; ++q) {
      sz = cadd(sz, p64[0]);
      sd = cadd(sd, p64[nlm]);
      sw = cadd(sw, p64[2 * nlm]);
      p64 += 3 * nlm;
    }
  }
  const double2 bp = U0[I.soff + idx];
  double2 phi = cmul(I.S0, bp);
  if (idx != 0) phi = make_double2(fma(-phibar, sw.x, phi.x), fma(-phibar, sw.y, phi.y));
  double2* o = U1 + I.soff + idx;
  o[0] = phi;
  o[nlm] = sz;
  o[2 * nlm] = sd;
}

}  // namespace rexi
