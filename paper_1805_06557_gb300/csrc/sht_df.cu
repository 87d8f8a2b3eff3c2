// Double-float Legendre contractions (sh_plan precision SH_DF; paper Sec. 3.2: the Legendre
// contraction per zonal order m of the SH transforms).
//
// GB300 issues about two FP64 FMAs per clock and SM against 128 FP32 ones, so the FP64
// contraction is bound by its pipe while the tensor-core precisions stop near 1e-6.  Here every
// operand is a double-float pair (hi + lo, two FP32 words; about 48 significand bits) and every
// sum a compensated dot product (Ogita, Rump & Oishi's Dot2: TwoProduct by FMA, Knuth's TwoSum,
// the errors gathered in one FP32 word), all on the FP32 pipe.  Only the conversions touch FP64:
// the tables are split once at plan time, the inputs of a call by one pass kernel, and the
// results are formed in FP64 from the two words of each sum.  The longitude FFT of these plans
// runs in double-float arithmetic as well (sht.cu).
//
// Tables (split from the FP64 table of P, over the degrees n = m .. T + 1): synthesis
// [moff(T+1, m) + k][nh] (latitude fastest: threads that own latitudes read coalesced);
// analysis, per m [nh][K + 1] with the even degree indices k first and the odd ones after them,
// so that the warps of one parity, which own consecutive degrees, read coalesced.  No table of
// H: with Ht_n = (n+1) eps_n Pt_{n-1} - n eps_{n+1} Pt_{n+1}, a vector synthesis is the scalar
// synthesis of the spectra u, v of its velocity components (k_df_synth_coeffs), and a vector
// analysis takes P-sums only, whose neighbouring degrees give the H-sums (k_divcurl_from_p).
//
// One launch contracts up to four fields (synthesis: scalar spectra and the u, v spectra of
// vector pairs) or NS scalar fields and NV vector pairs (analysis, NS, NV <= 2) against the
// same table reads.  The real and imaginary parts of every sum run together on the packed
// FP32x2 instructions.
#include <algorithm>
#include <cuda_runtime.h>
#include <vector>

#include "../../include/sht.h"
#include "common.cuh"
#include "df.cuh"
#include "sht_df.cuh"

namespace rexi {

namespace {

constexpr int DF_STH = 128;  // synthesis: threads per block (one northern latitude each)
constexpr int DF_ATH = 128;  // analysis: threads per block (64 even and 64 odd degrees)

__device__ __forceinline__ float2 split_df(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}
// A split complex value is held as (re.hi, im.hi, re.lo, im.lo): its high words and its low
// words are each a pair for the packed FP32x2 instructions.  The inputs of a call are split by
// the bit patterns (integer pipe), not by FP64 arithmetic.
__device__ __forceinline__ float4 split_dfc(double2 v) {
  const dfr a = dfr_from_bits(v.x), b = dfr_from_bits(v.y);
  return make_float4(a.hi, b.hi, a.lo, b.lo);
}
__device__ __forceinline__ df df_of(float2 v) { return df{v.x, v.y}; }
__device__ __forceinline__ df dfre(float4 v) { return df{v.x, v.z}; }
__device__ __forceinline__ df dfim(float4 v) { return df{v.y, v.w}; }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.z, v.w); }
// acc += p * c for a double-float real p and a split complex c, both components packed
__device__ __forceinline__ void madd(dot2c& acc, df p, float4 c) { dot2c_add(acc, p, hi2(c), lo2(c)); }

// the value of a + sg b (sg = +-1) of two compensated sums, rounded once to FP64; BITS widens
// the two words from their bit patterns (integer pipe) instead of by FP64 conversions -- the
// two forms give the same value and differ only in the registers the synthesis kernel takes
template <bool BITS>
__device__ __forceinline__ double dsum(const dot2& a, const dot2& b, float sg) {
  const df t = df_two_sum(a.s, sg * b.s);
  const float lo = t.lo + (a.err + sg * b.err);
  return BITS ? df_widen(t.hi) + df_widen(lo) : (double)t.hi + (double)lo;
}
__device__ __forceinline__ double dval(const dot2& a) { return (double)a.s + (double)a.err; }

// ---- plan-time splits --------------------------------------------------------------------
// FP64 table of P [moff(m)+k][nh] and the next degree's row next [m][nh] -> synthesis table
// [moff(T+1, m) + k][nh] and analysis table (per m at moff(T+1, m) nh: [nh][K + 1], even k
// first), k = 0 .. K; one thread per (m, latitude)
__global__ void k_df_split_table(const double* __restrict__ src, const double* __restrict__ next,
                                 float2* __restrict__ syn, float2* __restrict__ ana, int T, int nh) {
  const int m = blockIdx.x, j = blockIdx.y * blockDim.x + threadIdx.x;
  if (j >= nh) return;
  const int K = T + 1 - m, Kx = K + 1, Ke = (Kx + 1) / 2;
  const size_t base = (size_t)moff(T, m) * nh, xbase = (size_t)moff(T + 1, m) * nh;
  for (int k = 0; k < Kx; ++k) {
    const float2 v = split_df(k < K ? src[base + (size_t)k * nh + j] : next[(size_t)m * nh + j]);
    syn[xbase + (size_t)k * nh + j] = v;
    ana[xbase + (size_t)j * Kx + ((k & 1) ? Ke + (k >> 1) : (k >> 1))] = v;
  }
}

__device__ __forceinline__ double eps_nm(int n, int m) {  // eps_n^m, 0 for n <= m
  return n <= m ? 0.0 : sqrt((double(n) * n - double(m) * m) / (4.0 * n * n - 1.0));
}

// Split spectra of one synthesis in the layout of n = m .. T + 1 ([q][nlme] at moff(T+1, m)):
// fields q < nfs the scalar spectra (0 at n = T + 1); then the u and v spectra of the nfv
// (psi, chi) pairs, u_p = (-psi'_p + i m chi_p) / a and v_p = (i m psi_p + chi'_p) / a with
// x'_p = (p + 2) eps_{p+1} x_{p+1} - (p - 1) eps_p x_{p-1} (formed in FP64, then split), whose
// scalar syntheses are the velocity components U, V (Ht_n = (n+1) eps_n Pt_{n-1} -
// n eps_{n+1} Pt_{n+1}).  Grid (T + 1, nfs + 2 nfv).
__global__ void k_df_synth_coeffs(const double2* __restrict__ spec, const double2* __restrict__ psi,
                                  const double2* __restrict__ chi, int nfs, int nfv, double inv_a,
                                  float4* __restrict__ dst, int T, int nlm, int nlme) {
  const int m = blockIdx.x, q = blockIdx.y, K = T + 1 - m;
  float4* o = dst + (size_t)q * nlme + moff(T + 1, m);
  const double2 z = make_double2(0.0, 0.0);
  if (q < nfs) {
    const double2* c = spec + (size_t)q * nlm + moff(T, m);
    for (int k = threadIdx.x; k <= K; k += blockDim.x) o[k] = split_dfc(k < K ? c[k] : z);
    return;
  }
  const int r = q - nfs, v = r < nfv ? r : r - nfv;
  const bool uu = r < nfv;  // u of pair v, else v of pair v
  const double2* ps = psi + (size_t)v * nlm + moff(T, m);
  const double2* ch = chi + (size_t)v * nlm + moff(T, m);
  const double fm = (double)m;
  for (int k = threadIdx.x; k <= K; k += blockDim.x) {
    const int p = m + k;
    const double a1 = (p + 2.0) * eps_nm(p + 1, m), a0 = (p - 1.0) * eps_nm(p, m);
    const double2 x0 = uu ? (k < K ? ch[k] : z) : (k < K ? ps[k] : z);   // the i m term's spectrum
    const double2* d = uu ? ps : ch;                                      // the primed one's
    const double2 dp = k + 1 < K ? d[k + 1] : z, dm = k > 0 ? d[k - 1] : z;
    const double dx = a1 * dp.x - a0 * dm.x, dy = a1 * dp.y - a0 * dm.y;
    // u = (-psi' + i m chi) / a;  v = (i m psi + chi') / a
    const double2 val = uu ? make_double2(inv_a * (-dx - fm * x0.y), inv_a * (-dy + fm * x0.x))
                           : make_double2(inv_a * (-fm * x0.y + dx), inv_a * (fm * x0.x + dy));
    o[k] = split_dfc(val);
  }
}
__global__ void k_df_split_weights(const double* __restrict__ w, const double* __restrict__ wq,
                                   float4* __restrict__ out, int nh) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nh) return;
  const float2 a = split_df(w[j]), b = split_df(wq[j]);
  out[j] = make_float4(a.x, a.y, b.x, b.y);
}

// ---- per-call split of the complex FP64 inputs (up to three arrays) into one float4 buffer ---
struct SplitSegs {
  const double2* src[3];
  long long end[3];  // cumulative element counts
};
__global__ void k_df_split_inputs(const __grid_constant__ SplitSegs sg, float4* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sg.end[2]) return;
  const int s = (i >= sg.end[0]) + (i >= sg.end[1]);
  const long long o = s ? i - sg.end[s - 1] : i;
  dst[i] = split_dfc(sg.src[s][o]);
}

// ---- synthesis ----------------------------------------------------------------------------
struct DfSynthArgs {
  const float2* P;      // synthesis table [moff(T+1, m) + k][nh], k = 0 .. K
  const float4* c;      // split spectra of the launch's fields [NF][nlme] at moff(T+1, m) + k
  double2* out[4];      // Fourier coefficients of each field [T+1][nlat]
  const int* ks;        // polar bounds: first degree index per (m, 32-latitude group) [T+1][ngl]
  int T, nlat, nh, nlme, ngl;
};

// k-step of parity PAR: the table entry p of degree k against every field's coefficient
// (split coefficients of the block's zonal order staged in shared memory, field f at
// cf + f L, L = T + 2)
template <int NF, int PAR>
__device__ __forceinline__ void df_synth_step(float2 pv, const float4* cf, int L, int k, dot2c (&S)[NF][2]) {
  const df p = df_of(pv);
#pragma unroll
  for (int f = 0; f < NF; ++f) madd(S[f][PAR], p, cf[f * L + k]);
}

constexpr int DF_PF = 4;  // table entries loaded this many degrees (synthesis) or latitudes (analysis) ahead

// One thread per northern latitude jh of zonal order m: even and odd partial sums of NF fields
// over the degrees n = m .. T + 1, combined for the latitude and its mirror
// (P_n(-mu) = (-1)^(n-m) P_n(mu)).  The block (four warps over 128 consecutive latitudes)
// stages its zonal order's split coefficients in shared memory; each warp starts at the first
// degree its 32 latitudes need (polar bounds, rounded down to even).
// MINB: blocks per SM the registers must allow (5 for launches of several waves, where
// occupancy hides the table loads; 1 for small ones, where each block's own overlap counts)
template <int NF, int MINB>
__global__ void __launch_bounds__(DF_STH, MINB) k_df_synth(const __grid_constant__ DfSynthArgs a) {
  constexpr bool BITS = MINB > 1;  // the result form that fits the tighter register budget
  extern __shared__ float4 cf[];
  const int m = blockIdx.x;
  const int T = a.T, K = T + 1 - m, Kx = K + 1, L = T + 2, nlat = a.nlat, nh = a.nh;
  // latitude tiles run equator first: the last tile has the most work left after the polar
  // truncation, and the first blocks launched finish last
  const int jh = (gridDim.y - 1 - blockIdx.y) * DF_STH + threadIdx.x;
  // from the warp's first degree kb (even: the parity of k - kb is that of k) on; requested
  // before the staging, whose time hides its latency
  const int kb = jh < nh ? __ldg(a.ks + m * a.ngl + (jh >> 5)) & ~1 : 0;  // warp-uniform, <= K
  const float4* src = a.c + moff(T + 1, m);
  for (int i = threadIdx.x; i < NF * Kx; i += DF_STH) {
    const int q = i / Kx, k = i - q * Kx;
    cf[q * L + k] = __ldg(src + (size_t)q * a.nlme + k);
  }
  __syncthreads();
  if (jh >= nh) return;  // no barrier below
  const float2* Pm = a.P + (size_t)(moff(T + 1, m) + kb) * nh + jh;
  const int Kr = Kx - kb;
  const float2 z2 = make_float2(0.f, 0.f);
  dot2c S[NF][2];  // field, parity of k
#pragma unroll
  for (int f = 0; f < NF; ++f) S[f][0] = S[f][1] = dot2c{z2, z2};
  // Table rows in flight.  Under the tight register budget (MINB > 1) with three or four fields
  // a rolling prefetch: slot u holds row k0 + u and, once consumed, is refilled with row
  // k0 + PF + u, so every row is requested PF rows before its use with one register set (six
  // rows: what five blocks per SM leave registers for; the one-pass N(U) synthesis at T511
  // took 0.277 ms with four, 0.258 ms with six).  Otherwise a double buffer of eight rows: the
  // next PF rows are requested together before the current ones are used.
  constexpr bool ROLL = MINB > 1 && NF > 2;
  constexpr int PF = ROLL ? DF_PF + 2 : 2 * DF_PF;
  float2 pb[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) pb[u] = u < Kr ? __ldg(Pm + (size_t)u * nh) : z2;
  for (int k0 = 0; k0 < Kr; k0 += PF) {
    float2 pn[ROLL ? 1 : PF];
    if (!ROLL) {
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int kk = k0 + PF + u;
        pn[ROLL ? 0 : u] = kk < Kr ? __ldg(Pm + (size_t)kk * nh) : z2;
      }
    }
#pragma unroll
    for (int u = 0; u < PF; u += 2) {  // k0 is even: the parity of k0 + u is that of u
      if (k0 + u < Kr) df_synth_step<NF, 0>(pb[u], cf, L, kb + k0 + u, S);
      if (k0 + u + 1 < Kr) df_synth_step<NF, 1>(pb[u + 1], cf, L, kb + k0 + u + 1, S);
      if (ROLL) {
#pragma unroll
        for (int v = u; v < u + 2; ++v) {
          const int kk = k0 + PF + v;
          pb[v] = kk < Kr ? __ldg(Pm + (size_t)kk * nh) : z2;
        }
      }
    }
    if (!ROLL) {
#pragma unroll
      for (int u = 0; u < PF; ++u) pb[u] = pn[ROLL ? 0 : u];
    }
  }
  const int lat = jh, lats = nlat - 1 - jh;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    double2* o = a.out[f] + (size_t)m * nlat;
    const dot2 er = dot2c_re(S[f][0]), ei = dot2c_im(S[f][0]), od = dot2c_re(S[f][1]), oi = dot2c_im(S[f][1]);
    o[lat] = make_double2(dsum<BITS>(er, od, 1.f), dsum<BITS>(ei, oi, 1.f));
    o[lats] = make_double2(dsum<BITS>(er, od, -1.f), dsum<BITS>(ei, oi, -1.f));
  }
}

// ---- analysis -----------------------------------------------------------------------------
struct DfAnalArgs {
  const float2* P;      // analysis table: per m [nh][K + 1], even k first
  const float4* wdf;    // (w.hi, w.lo, wq.hi, wq.lo) [nh]
  const float4* fa;     // split Fourier coefficients: A [NV][T+1][nlat]
  const float4* fb;     // B [NV][T+1][nlat]
  const float4* fg;     // scalar [NS][T+1][nlat]
  double2* raw;         // P-sums of A and B: [NV][2][nlme], degree index k at moff(T+1, m) + k
  double2* spec;        // [NS][nlm]
  const int* ja;        // polar bounds: first latitude per (m, 32-degree group) [T+1][ngd]
  int T, nlat, nh, nlm, nlme, ngd;
};

__device__ __forceinline__ float4 dfc_pack(df re, df im) { return make_float4(re.hi, im.hi, re.lo, im.lo); }
// w (F_N + s F_S) of one latitude pair, in double-float
__device__ __forceinline__ float4 df_wsum(df w, float4 n, float4 s, float sg) {
  const df sr = dfre(s), si = dfim(s);
  const df re = df_mul(w, df_add(dfre(n), df{sg * sr.hi, sg * sr.lo}));
  const df im = df_mul(w, df_add(dfim(n), df{sg * si.hi, sg * si.lo}));
  return dfc_pack(re, im);
}

// latitude j of one degree: the table entry p against the staged sums (sP selects the sum or
// the difference array of the degree's parity)
template <int NS, int NV>
__device__ __forceinline__ void df_anal_step(float2 pv, const float4* sm4, int nh, int j, int sP,
                                             dot2c (&S)[NS > 0 ? NS : 1], dot2c (&V)[NV > 0 ? NV : 1][2]) {
  const df p = df_of(pv);
#pragma unroll
  for (int f = 0; f < NS; ++f) madd(S[f], p, sm4[(4 * NV + 2 * f + sP) * nh + j]);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    madd(V[v][0], p, sm4[(4 * v + 0 + sP) * nh + j]);  // P.A
    madd(V[v][1], p, sm4[(4 * v + 2 + sP) * nh + j]);  // P.B
  }
}

// Block (m, tile): shared memory holds, per northern latitude j, the weighted hemispheric sums
// and differences of every field (vector pair v: A+, A-, B+, B- with w / (1 - mu^2); scalar f:
// G+, G- with w); warps 0-1 own the even degree indices k = 128 tile + 2 i, warps 2-3 the odd
// ones, and each thread streams its table column over the latitudes, DF_PF latitudes of table
// entries in flight, from the first latitude that the 64 degrees of its warp's span need
// (polar bounds).  P pairs with the sums for even k and the differences for odd k.  Scalar
// fields give their spectra (k < K); vector fields give the P-sums of A and B (k <= K, n up to
// T + 1), from which k_divcurl_from_p forms divergence and curl.
template <int NS, int NV>
__global__ void __launch_bounds__(DF_ATH, 4) k_df_anal(const __grid_constant__ DfAnalArgs a) {
  extern __shared__ float4 sm4[];
  const int m = blockIdx.x, tile = blockIdx.y;
  const int T = a.T, K = T + 1 - m, nh = a.nh, nlat = a.nlat;
  const int Kx = K + 1;                   // table rows of m (degrees to n = T + 1)
  const int Kl = NV > 0 ? Kx : K;         // degree indices this launch needs
  if (tile * DF_ATH >= Kl) return;  // uniform over the block
  const int par = threadIdx.x >= DF_ATH / 2;  // uniform over each warp
  const int idx = threadIdx.x & (DF_ATH / 2 - 1);
  const int k = tile * DF_ATH + 2 * idx + par;
  // first latitude: warp w spans the degree indices tile 128 + 64 (w & 1) .. + 63, bound groups
  // g0 and g0 + 1; requested before the staging, whose time hides its latency
  int jb = nh;
  if (k < Kl) {
    const int g0 = tile * (DF_ATH / 32) + 2 * ((threadIdx.x >> 5) & 1);
    const int* jam = a.ja + m * a.ngd;
    jb = min(__ldg(jam + g0), g0 + 1 < a.ngd ? __ldg(jam + g0 + 1) : nh);  // warp-uniform
  }
  // staging
  for (int j = threadIdx.x; j < nh; j += DF_ATH) {
    const float4 wv = __ldg(a.wdf + j);
    const df w{wv.x, wv.y}, wq{wv.z, wv.w};
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float4* A = a.fa + ((size_t)v * (T + 1) + m) * nlat;
      const float4* B = a.fb + ((size_t)v * (T + 1) + m) * nlat;
      const float4 an = __ldg(A + j), as = __ldg(A + nlat - 1 - j);
      const float4 bn = __ldg(B + j), bs = __ldg(B + nlat - 1 - j);
      sm4[(4 * v + 0) * nh + j] = df_wsum(wq, an, as, 1.f);
      sm4[(4 * v + 1) * nh + j] = df_wsum(wq, an, as, -1.f);
      sm4[(4 * v + 2) * nh + j] = df_wsum(wq, bn, bs, 1.f);
      sm4[(4 * v + 3) * nh + j] = df_wsum(wq, bn, bs, -1.f);
    }
#pragma unroll
    for (int f = 0; f < NS; ++f) {
      const float4* G = a.fg + ((size_t)f * (T + 1) + m) * nlat;
      const float4 gn = __ldg(G + j), gs = __ldg(G + nlat - 1 - j);
      sm4[(4 * NV + 2 * f + 0) * nh + j] = df_wsum(w, gn, gs, 1.f);
      sm4[(4 * NV + 2 * f + 1) * nh + j] = df_wsum(w, gn, gs, -1.f);
    }
  }
  __syncthreads();
  if (k >= Kl) return;  // no barrier below
  const int Ke = (Kx + 1) / 2;
  const size_t col = (size_t)moff(T + 1, m) * nh + (par ? Ke : 0) + tile * (DF_ATH / 2) + idx;
  const float2* Pc = a.P + col;
  const int sP = par;  // P meets (N + S) for even k, (N - S) for odd k
  const float2 z2 = make_float2(0.f, 0.f);
  dot2c S[NS > 0 ? NS : 1];
  dot2c V[NV > 0 ? NV : 1][2];  // [0] P.A, [1] P.B
#pragma unroll
  for (int f = 0; f < (NS > 0 ? NS : 1); ++f) S[f] = dot2c{z2, z2};
#pragma unroll
  for (int v = 0; v < (NV > 0 ? NV : 1); ++v) V[v][0] = V[v][1] = dot2c{z2, z2};
  float2 pb[DF_PF];
#pragma unroll
  for (int u = 0; u < DF_PF; ++u) pb[u] = jb + u < nh ? __ldg(Pc + (size_t)(jb + u) * Kx) : z2;
  for (int j0 = jb; j0 < nh; j0 += DF_PF) {
    float2 pn[DF_PF];
#pragma unroll
    for (int u = 0; u < DF_PF; ++u) {
      const int jj = j0 + DF_PF + u;
      pn[u] = jj < nh ? __ldg(Pc + (size_t)jj * Kx) : z2;
    }
#pragma unroll
    for (int u = 0; u < DF_PF; ++u) {
      const int j = j0 + u;
      if (j >= nh) break;
      df_anal_step<NS, NV>(pb[u], sm4, nh, j, sP, S, V);
    }
#pragma unroll
    for (int u = 0; u < DF_PF; ++u) pb[u] = pn[u];
  }
  if (k < K) {
    const size_t i = (size_t)moff(T, m) + k;
#pragma unroll
    for (int f = 0; f < NS; ++f)
      a.spec[(size_t)f * a.nlm + i] = make_double2(dval(dot2c_re(S[f])), dval(dot2c_im(S[f])));
  }
  const size_t ie = (size_t)moff(T + 1, m) + k;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    a.raw[(size_t)(2 * v) * a.nlme + ie] = make_double2(dval(dot2c_re(V[v][0])), dval(dot2c_im(V[v][0])));
    a.raw[(size_t)(2 * v + 1) * a.nlme + ie] = make_double2(dval(dot2c_re(V[v][1])), dval(dot2c_im(V[v][1])));
  }
}

template <int NF>
size_t df_synth_smem(int T) {
  return sizeof(float4) * (size_t)NF * (T + 2);
}
template <int NS, int NV>
size_t df_anal_smem(int nh) {
  return sizeof(float4) * (size_t)(4 * NV + 2 * NS) * nh;
}

}  // namespace

struct DfLegendre {
  int T = 0, nlat = 0, nh = 0, nlm = 0, max_fields = 0, nsm = 0;
  PolarBounds pb;
  float2 *Ps = nullptr, *Pa = nullptr;  // synthesis and analysis tables of P (to n = T + 1)
  float4* wdf = nullptr;
  float4* in = nullptr;  // split inputs of one call: [2 max_fields][max(nlm, (T+1) nlat)]
  double2* raw = nullptr;  // P-sums of the vector fields of one call: [2 max_fields][2][nlme]
  StageProf* prof = nullptr;
};

static int df_smem_attr(int nh, int T) {
  cudaError_t e = cudaSuccess;
#define DF_ATTR(NS, NV)                                                                                    \
  if (!e)                                                                                                 \
    e = raise_smem_limit(k_df_anal<NS, NV>, df_anal_smem<NS, NV>(nh));
  DF_ATTR(1, 0) DF_ATTR(2, 0) DF_ATTR(0, 1) DF_ATTR(1, 1) DF_ATTR(2, 1) DF_ATTR(0, 2) DF_ATTR(1, 2) DF_ATTR(2, 2)
#undef DF_ATTR
#define DF_SATTR(NF)                                                                                       \
  if (!e)                                                                                                 \
    e = raise_smem_limit(k_df_synth<NF, 1>, df_synth_smem<NF>(T));                                       \
  if (!e)                                                                                                 \
    e = raise_smem_limit(k_df_synth<NF, 5>, df_synth_smem<NF>(T));
  DF_SATTR(1) DF_SATTR(2) DF_SATTR(3) DF_SATTR(4)
#undef DF_SATTR
  return e ? cuda_fail(e, "cudaFuncSetAttribute(k_df_*)") : REXI_OK;
}

int df_legendre_create(DfLegendre** out, const double* P, const double* Pn, const double* w, const double* wq, int T,
                       int nlat, int max_fields, const PolarBounds& pb, cudaStream_t stream) {
  *out = nullptr;
  const int nh = nlat / 2;
  if (df_anal_smem<2, 2>(nh) > 200 * 1024)  // 12 staged arrays of nh float4
    return fail(REXI_EINVAL, "sh_plan_create: SH_DF supports nlat <= 2132 (got %d)", nlat);
  DfLegendre* t = new DfLegendre();
  t->T = T;
  t->nlat = nlat;
  t->nh = nh;
  t->nlm = (T + 1) * (T + 2) / 2;
  t->max_fields = max_fields;
  t->pb = pb;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&t->nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  const size_t tab = (size_t)t->nlm * nh;
  const size_t per = std::max<size_t>(t->nlm, (size_t)(T + 1) * nlat);
  cudaError_t e;
  const size_t tabx = (size_t)nlm_ext(T) * nh;
  if ((e = cudaMalloc(&t->Ps, sizeof(float2) * tabx)) || (e = cudaMalloc(&t->Pa, sizeof(float2) * tabx)) ||
      (e = cudaMalloc(&t->raw, sizeof(double2) * 2 * 2 * (size_t)max_fields * nlm_ext(T))) ||
      (e = cudaMalloc(&t->wdf, sizeof(float4) * nh)) ||
      (e = cudaMalloc(&t->in, sizeof(float4) * per * 2 * (size_t)max_fields))) {
    cudaGetLastError();
    df_legendre_destroy(t);
    return fail(REXI_ENOMEM, "double-float Legendre tables: cudaMalloc failed: %s", cudaGetErrorString(e));
  }
  k_df_split_table<<<dim3(T + 1, (nh + 127) / 128), 128, 0, stream>>>(P, Pn, t->Ps, t->Pa, T, nh);
  k_df_split_weights<<<(nh + 127) / 128, 128, 0, stream>>>(w, wq, t->wdf, nh);
  int rc = REXI_OK;
  if ((e = cudaGetLastError())) rc = cuda_fail(e, "double-float table kernels");
  if (!rc) rc = df_smem_attr(nh, T);
  if (rc) {
    df_legendre_destroy(t);
    return rc;
  }
  *out = t;
  return REXI_OK;
}

void df_legendre_destroy(DfLegendre* t) {
  if (!t) return;
  for (void* p : {(void*)t->Ps, (void*)t->Pa, (void*)t->wdf, (void*)t->in, (void*)t->raw}) cudaFree(p);
  delete t;
}

void df_legendre_streamed(const DfLegendre* t, long long* syn, long long* ana) {
  const int T = t->T, nh = t->nh, ngl = t->pb.ngl, ngd = t->pb.ngd;
  long long s = 0, a = 0;
  for (int m = 0; m <= T; ++m) {
    const int K = T + 1 - m;
    for (int g = 0; g < ngl; ++g) s += (long long)std::min(32, nh - 32 * g) * (K - (t->pb.ks[m * ngl + g] & ~1));
    for (int g = 0; 32 * g < K; g += 2) {  // one warp pair per 64-degree span (entries of n <= T)
      const int jb = std::min(t->pb.ja[m * ngd + g], g + 1 < ngd ? t->pb.ja[m * ngd + g + 1] : nh);
      a += (long long)std::min(64, K - 32 * g) * (nh - jb);
    }
  }
  *syn = s;
  *ana = a;
}

void df_legendre_set_prof(DfLegendre* t, StageProf* prof) {
  if (t) t->prof = prof;
}

static void split_inputs(DfLegendre* t, const double2* s0, long long n0, const double2* s1, long long n1,
                         const double2* s2, long long n2, cudaStream_t s) {
  SplitSegs sg{};
  sg.src[0] = s0;
  sg.src[1] = s1;
  sg.src[2] = s2;
  sg.end[0] = n0;
  sg.end[1] = n0 + n1;
  sg.end[2] = n0 + n1 + n2;
  if (sg.end[2] == 0) return;
  k_df_split_inputs<<<(unsigned)((sg.end[2] + 255) / 256), 256, 0, s>>>(sg, t->in);
}

template <int NF>
static void launch_synth(DfLegendre* t, const DfSynthArgs& a, cudaStream_t s) {
  const dim3 grid(t->T + 1, (t->nh + DF_STH - 1) / DF_STH);
  const size_t smem = df_synth_smem<NF>(t->T);
  if ((long long)grid.x * grid.y >= 4LL * t->nsm)
    k_df_synth<NF, 5><<<grid, DF_STH, smem, s>>>(a);
  else
    k_df_synth<NF, 1><<<grid, DF_STH, smem, s>>>(a);
}

// Scalar spectra and (psi, chi) pairs as the scalar syntheses of nfs + 2 nfv spectra (the
// scalars, the u's, the v's; k_df_synth_coeffs), up to four per launch, one table read each.
int df_leg_synth(DfLegendre* t, const double2* spec, double2* F, int nfs, const double2* psi, const double2* chi,
                 double2* FU, double2* FV, int nfv, double inv_a, cudaStream_t s) {
  if (nfs < 0 || nfv < 0 || nfs + 2 * nfv > 2 * t->max_fields) return fail(REXI_EINVAL, "df synthesis: too many fields");
  const int ph = t->prof ? t->prof->begin(1) : -1;
  const int nft = nfs + 2 * nfv, nlme = nlm_ext(t->T);
  if (nft > 0)
    k_df_synth_coeffs<<<dim3(t->T + 1, nft), 128, 0, s>>>(spec, psi, chi, nfs, nfv, inv_a, t->in, t->T, t->nlm, nlme);
  const size_t fo = (size_t)(t->T + 1) * t->nlat;
  DfSynthArgs a{};
  a.P = t->Ps;
  a.T = t->T;
  a.nlat = t->nlat;
  a.nh = t->nh;
  a.nlme = nlme;
  a.ks = t->pb.d_ks;
  a.ngl = t->pb.ngl;
  for (int q0 = 0; q0 < nft; q0 += 4) {
    const int nf = std::min(4, nft - q0);
    a.c = t->in + (size_t)q0 * nlme;
    for (int i = 0; i < 4; ++i) {
      const int q = q0 + i;
      a.out[i] = i >= nf ? nullptr : q < nfs ? F + q * fo : q < nfs + nfv ? FU + (q - nfs) * fo : FV + (q - nfs - nfv) * fo;
    }
    if (nf == 4) launch_synth<4>(t, a, s);
    else if (nf == 3) launch_synth<3>(t, a, s);
    else if (nf == 2) launch_synth<2>(t, a, s);
    else launch_synth<1>(t, a, s);
  }
  if (t->prof) t->prof->end(ph);
  cudaError_t e = cudaGetLastError();
  return e ? cuda_fail(e, "k_df_synth launch") : REXI_OK;
}

template <int NS, int NV>
static void launch_anal(DfLegendre* t, DfAnalArgs a, cudaStream_t s) {
  // degree tiles over n = m .. T + 1 (vector fields need n = T + 1)
  k_df_anal<NS, NV><<<dim3(t->T + 1, (t->T + 1 + DF_ATH) / DF_ATH), DF_ATH, df_anal_smem<NS, NV>(t->nh), s>>>(a);
}

int df_leg_anal(DfLegendre* t, const double2* FA, const double2* FB, double2* dv, double2* cu, int nfv,
                const double2* F, double2* spec, int nfs, double inv_a, cudaStream_t s) {
  if (nfs < 0 || nfv < 0 || nfs + 2 * nfv > 2 * t->max_fields) return fail(REXI_EINVAL, "df analysis: too many fields");
  const int ph = t->prof ? t->prof->begin(1) : -1;
  const long long fo = (long long)(t->T + 1) * t->nlat;
  split_inputs(t, FA, nfv * fo, FB, nfv * fo, F, nfs * fo, s);
  DfAnalArgs a{};
  a.P = t->Pa;
  a.wdf = t->wdf;
  a.T = t->T;
  a.nlat = t->nlat;
  a.nh = t->nh;
  a.nlm = t->nlm;
  a.nlme = nlm_ext(t->T);
  a.ja = t->pb.d_ja;
  a.ngd = t->pb.ngd;
  const float4* fa = t->in;
  const float4* fb = fa + nfv * fo;
  const float4* fg = fb + nfv * fo;
  int fs = 0, fv = 0;
  while (fs < nfs || fv < nfv) {
    const int ns = std::min(2, nfs - fs), nv = std::min(2, nfv - fv);
    a.fa = fa + fv * fo;
    a.fb = fb + fv * fo;
    a.fg = fg + fs * fo;
    a.raw = t->raw + (size_t)(2 * fv) * a.nlme;
    a.spec = spec ? spec + (size_t)fs * t->nlm : nullptr;
#define DF_CASE(NS, NV) \
  else if (ns == NS && nv == NV) launch_anal<NS, NV>(t, a, s);
    if (false) {
    }
    DF_CASE(1, 0) DF_CASE(2, 0) DF_CASE(0, 1) DF_CASE(1, 1) DF_CASE(2, 1) DF_CASE(0, 2) DF_CASE(1, 2) DF_CASE(2, 2)
#undef DF_CASE
    fs += ns;
    fv += nv;
  }
  launch_divcurl_from_p(t->raw, dv, cu, nfv, t->T, inv_a, s);
  if (t->prof) t->prof->end(ph);
  cudaError_t e = cudaGetLastError();
  return e ? cuda_fail(e, "k_df_anal launch") : REXI_OK;
}

}  // namespace rexi
