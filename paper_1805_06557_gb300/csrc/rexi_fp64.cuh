// FP64 REXI solve kernel (the plain FP64 path).
//
// Work decomposition: a tile is (state b, zonal order m, parity chain c, range of 32-pole
// groups).  One warp owns a tile; lane l solves the chain for pole g*32 + l, so the 32
// systems of a warp share m, the chain and every table / right-hand-side element (warp
// broadcast loads), and differ only in the pole z.
//
// Per (pole, m) the banded system (z - dt L_m) u = U0_m is reduced exactly as follows:
//   Phi_n = (bPhi_n - dt Phibar delta_n) / z                       (Phi row)
// which leaves two tridiagonal chains in (zeta, delta) by parity of n - m.  Row n reads
//   zeta row : (z - i dt w_n) zeta_n + cm_n x_{n-1} + cp_n x_{n+1} = bzeta_n
//   delta row: (z - i dt w_n + q_n dt Phibar / z) delta_n - cm_n x_{n-1} - cp_n x_{n+1}
//              = bdelta_n + q_n bPhi_n / z
// with cm_n = dt 2 Omega (n+1)/n eps_n, cp_n = dt 2 Omega n/(n+1) eps_{n+1}, q_n = dt n(n+1)/a^2.
// The chain is solved by the Thomas algorithm without pivoting: for the REXI poles the
// shifted operator is a scaled identity plus a skew-adjoint part in the energy norm, so the
// elimination is stable.  The forward coefficients are kept in a per-warp global scratch
// slot ([k][lane], coalesced); FP64 arithmetic is slow enough on this part that the scratch
// traffic is far below the HBM roofline.
//
// The weighted sums over poles are formed by transposing 32 solution rows through shared
// memory, so that lane r sums row r over the 32 poles of the group:
//   S_zeta / S_delta = sum_p w_p x_p,   S_wz = sum_p (w_p / z_p) delta_p,
// and Phi = bPhi * sum_p w_p/z_p - dt Phibar * S_wz is formed in the finalize kernel.
#pragma once
#include "common.cuh"

namespace rexi {

struct Fp64Args {
  const double2* U0;   // [B][3][nlm]
  double2* partial;    // [B][Q][3][nlm]
  const D4* tab;  // [nlm] (dt w_n, cm_n, cp_n, q_n)
  const PoleD* poles;  // [Npad]
  const Tile* tiles;   // [ntiles] for one state
  D4* scratch;    // [warps][kmax][32]
  int ntiles, B, T, nlm, Q, kmax;
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
  const int total = a.ntiles * a.B;
  const int T = a.T, nlm = a.nlm;

  for (int round = 0; round * W < total; ++round) {
    const int t = round * W + ((round & 1) ? (W - 1 - gw) : gw);  // snake over LPT order
    if (t >= total) continue;
    const int it = t / a.B, b = t - it * a.B;
    const Tile tl = a.tiles[it];
    const int m = tl.m, c = tl.chain, K = T + 1 - m, off = moff(T, m);
    const double2* bP = a.U0 + (size_t)b * 3 * nlm;
    const double2* bZ = bP + nlm;
    const double2* bD = bP + 2 * nlm;
    double2* part = a.partial + ((size_t)b * a.Q + tl.q) * 3 * nlm;

    for (int gi = 0; gi < tl.ng; ++gi) {
      const PoleD pd = a.poles[(tl.g0 + gi) * 32 + lane];
      __syncwarp();
      s_w[lane] = pd.w;
      s_wz[lane] = pd.wz;

      // ---- forward elimination --------------------------------------------------
      double2 ct = make_double2(0.0, 0.0), y = make_double2(0.0, 0.0);
      for (int k = 0; k < K; ++k) {
        const int idx = off + k;
        const D4 tb = a.tab[idx];  // x: dt w, y: cm, z: cp, w: q
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

// U1 = (bPhi S0 - dt Phibar S_wz, S_zeta, S_delta), summing the Q partial slots in order.
static __global__ void k_rexi_finalize(const double2* __restrict__ U0, const double2* __restrict__ partial,
                                double2* __restrict__ U1, int B, int nlm, int Q, double2 S0,
                                double hphibar) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)B * nlm) return;
  const int b = (int)(i / nlm), idx = (int)(i - (long long)b * nlm);
  double2 sz = make_double2(0, 0), sd = sz, sw = sz;
  const double2* p = partial + (size_t)b * Q * 3 * nlm + idx;
  for (int q = 0; q < Q; ++q) {
    sz = cadd(sz, p[0]);
    sd = cadd(sd, p[nlm]);
    sw = cadd(sw, p[2 * nlm]);
    p += 3 * nlm;
  }
  const double2 bp = U0[(size_t)b * 3 * nlm + idx];
  double2 phi = cmul(S0, bp);
  if (idx != 0) phi = make_double2(fma(-hphibar, sw.x, phi.x), fma(-hphibar, sw.y, phi.y));
  double2* o = U1 + (size_t)b * 3 * nlm + idx;
  o[0] = phi;
  o[nlm] = sz;
  o[2 * nlm] = sd;
}

}  // namespace rexi
