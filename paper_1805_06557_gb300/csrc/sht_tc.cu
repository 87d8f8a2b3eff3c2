// Tensor-core (tcgen05) Legendre contractions for sh_plan precisions SH_TF32, SH_BF16 and
// SH_TF32X3 (paper Sec. 3.2: the dense Legendre contraction per zonal order m of the SH
// transforms).
//
// Every contraction is a set of GEMM jobs [128 x Ncols] = A[128 x K] B[K x Ncols]:
//   synthesis, per (m, 128-latitude tile, table P or H):
//       A = table^T (rows = northern latitudes, K = all degrees n = m + k),
//       B = spectral coefficients c_n beside (-1)^k c_n (columns: the northern and the
//           mirrored southern value of each field x re/im [x psi/chi])
//   analysis, per (m, 128-degree tile, table P or H):
//       A = table (rows = degrees, K = northern latitudes),
//       B = weighted hemispheric sums and differences of the Fourier coefficients.
// Operands are stored in the canonical no-swizzle K-major layout of the tensor cores
// (8-row x 16-byte core matrices; cores adjacent along K 128 B apart), the tables pre-tiled
// at plan time so that each K-chunk of A is one contiguous block moved by the bulk-copy
// engine (cp.async.bulk, completion on an mbarrier).  The GEMM is a persistent kernel, one
// CTA per SM, each with its own list of jobs (longest first, assigned to the least-loaded CTA
// at plan time): a copy warp streams A chunks through a ring of up to 8 stages; the B
// operands go through up to four shared-memory buffers that eight builder warps fill from the
// spectral or Fourier coefficients, an MMA warp accumulates in TMEM (FP32), and four
// epilogue warps read the accumulators with tcgen05.ld and write the FP64 results directly
// (hemisphere and parity combination, and for vector transforms the P and H sums of one
// (m, tile), which run as consecutive jobs of one CTA).  All mbarrier waits are bounded; on a
// timeout the kernel records an error flag.
//
// SH_TF32X3 (split TF32): every operand x is carried as x_hi + x_lo, x_hi = tf32(x) and
// x_lo = tf32(x - x_hi), and each k-step issues three MMAs into the same FP32 accumulator,
// a_hi b_lo + a_lo b_hi + a_hi b_hi; the dropped a_lo b_lo and the rounding of the lo parts
// leave a relative error of about 3 * 2^-22 per product instead of 2^-10.  A table chunk row
// holds 32 hi elements of K beside the same 32 lo elements (still 256 bytes), the B operand a
// hi and a lo copy.
#include <algorithm>
#include <map>
#include <cuda_bf16.h>
#include <vector>

#include "../../include/sht.h"
#include "sht_tc.cuh"
#include "tc_common.cuh"

namespace rexi {

namespace {

constexpr int TC_MAXSTAGES = 8;     // depth of the A-chunk ring
constexpr int TC_BUILD0 = 6;        // first of the warps that build the B operands
constexpr int TC_NBUILD = 8;        // builder warps
constexpr int TC_THREADS = 32 * (TC_BUILD0 + TC_NBUILD);  // warps 0-3 epilogue, 4 A copies, 5 MMA
                                                         // issue, 6-13 B operands
constexpr size_t TC_SMEM_BUDGET = 220 * 1024;

struct Job {
  long long a_off;  // byte offset of the job's first A chunk in its table
  int m, tile;      // zonal order and 128-row tile (latitudes or degrees k = n - m)
  int nchunk;       // K chunks
  int kpad;         // K extent of B (whole MMA k-steps; (nchunk - 1) * KC + kl)
  int tab;          // 0 = P, 1 = H
  int kl;           // K of the last chunk (a multiple of the MMA k-step, <= KC)
  int rows;         // A rows stored for the job (the valid rows rounded up to 8, <= 128): a
                    // chunk holds rows x KC elements; the MMA reads all 128 rows of a ring
                    // stage, and the accumulator rows past `rows` hold stale sums that the
                    // epilogue never stores
  int newb;         // 1: the job starts a B group (consecutive jobs of one m share a B operand)
  int c0;           // first K chunk streamed: the chunks before it hold only table entries below
                    // the polar threshold (never stored; a_off points at chunk c0; c0 < nchunk)
};

// precision modes of the GEMM (template parameter PM)
constexpr int PM_TF32 = 0, PM_BF16 = 1, PM_TF32X3 = 2;

// One call contracts nfv vector pairs and nfs scalar fields against the same table reads:
// columns [0, 8 nfv) hold the vector pairs (8 each), columns from 8 nfv the scalar fields (4
// each), so that every 8-column group is one vector pair or two scalar fields.
struct GemmArgs {
  const unsigned char* tabP;
  const unsigned char* tabH;
  // sources of the B operands: synthesis: spectra psi in0, chi in1 ([nfv][nlm]) and the scalar
  // spectra in2 ([nfs][nlm]); analysis: Fourier coefficients A in0, B in1 ([nfv][T+1][nlat])
  // and the scalar ones in2 ([nfs][T+1][nlat]), with the quadrature weights wts[nh]
  // (w / (1 - mu^2), vector) and wts2[nh] (w, scalar)
  const double2* in0;
  const double2* in1;
  const double2* in2;
  const double* wts;
  const double* wts2;
  const Job* jobs;      // per-CTA lists: CTA c runs jobs[cta_off[c] .. cta_off[c + 1])
  const int* cta_off;
  int ncols, bf16;
  int synth, pair;      // pair: (P, H) jobs of one (m, tile) follow each other (nfv > 0)
  double2* out0;        // synthesis: Fourier coefficients [nfv][T+1][nlat] of U; analysis: div
  double2* out1;        //   of V; analysis: curl ([nfv][nlm])
  double2* out2;        // scalar results: synthesis [nfs][T+1][nlat], analysis [nfs][nlm]
  int T, nlat, nlm, nfv, nfs;
  double inv_a;
  int stages;       // A ring depth (<= TC_MAXSTAGES)
  int nb;           // B buffers (1, 2 or 4): B operands are fetched up to nb - 1 jobs ahead
  int nj_max;       // jobs per CTA at most (their descriptors are staged in shared memory)
  uint32_t bslot;   // bytes of one B buffer
  uint32_t blo;     // PM_TF32X3: byte offset of the lo copy of B in its buffer (else 0)
  uint32_t epi_polls;  // 0: the epilogue waits for its accumulators with the normal bound; n > 0:
                       // it gives up after n non-blocking polls (a test of the timeout path)
  int* err;
};

// Persistent, warp-specialised GEMM over per-CTA job lists (longest first).  Warp 4 streams
// the A chunks of every job through the S-stage ring without pausing between jobs; warps 6-13
// build the B operands into NB buffers up to NB - 1 jobs ahead (so that a job's MMAs never
// wait for its operand); warp 5
// issues the MMAs of job i into TMEM job buffer i % njb and commits: the ring stage (empty),
// the B buffer (bempty) and the accumulator (tfull); warps 0-3 read the buffer (one TMEM lane
// quarter each), write the FP64 results, and release it (tempty), so that the MMAs of the next
// jobs overlap the epilogue.  Every wait is bounded; on a timeout the role records an error
// code and stops, and teardown drains the copies and MMAs in flight.
constexpr int TC_MAXNB = 4;
constexpr int TC_NACC = 4;          // independent accumulators per job (one per k-step of a chunk)
constexpr int TC_NJB = 3;           // job buffers of accumulators in TMEM (at most; 2 when N > 32)
constexpr uint32_t TC_TMEM_COLS = 512;  // TC_NJB x TC_NACC x 32 (N <= 32) or 2 x TC_NACC x 64 (N <= 64)

// 8 columns of this warp's 32 TMEM lanes: the sum of the first nacc of the TC_NACC
// accumulators (accumulator a at column offset a * cs), in order a = 0, 1, ...
__device__ __forceinline__ void tmem_sum8(uint32_t ta, uint32_t cs, int nacc, float* v) {
  uint32_t r[TC_NACC][8];
#pragma unroll
  for (int a = 0; a < TC_NACC; ++a) tc::tmem_ld8_nowait(ta + cs * a, r[a]);
  tc::tmem_wait_ld();
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float x = __uint_as_float(r[0][q]);
#pragma unroll
    for (int a = 1; a < TC_NACC; ++a)
      if (a < nacc) x += __uint_as_float(r[a][q]);
    v[q] = x;
  }
}

// Results of one row (synthesis: northern latitude `row`; analysis: k = n - m = row) from the
// 8-column group gq of the sums P (and H for vector pairs), combined in FP32 (the sums
// carry TF32 / BF16 operand rounding; FP64 arithmetic is a scarce pipe on this GPU) and stored
// as FP64.  Groups gq < nfv are vector pairs, the rest hold two scalar fields each:
//   synthesis scalar  (N re, N im, S re, S im): northern latitude and its mirror;
//   synthesis vector  (N: psi re, psi im, chi re, chi im; S: the same): U = (-H psi + i m P chi)/a,
//                     V = (i m P psi + H chi)/a, with the southern H sums negated
//                     (H_n(-mu) = -(-1)^(n-m) H_n(mu); the B operand carries (-1)^(n-m));
//   analysis scalar   (N+S re, N+S im, N-S re, N-S im): P pairs with N + S for even k, N - S odd;
//   analysis vector   (N+S: A re, A im, B re, B im; N-S: the same), H with the other block:
//                     div = (i m P.A - H.B)/a, curl = (i m P.B + H.A)/a.
__device__ __forceinline__ void epilogue8(const GemmArgs& g, int m, int row, int gq, const float* P,
                                          const float* H) {
  const float ia = (float)g.inv_a, fm = (float)m;
  if (g.synth) {
    if (row >= g.nlat / 2) return;
    const int lat = row, lats = g.nlat - 1 - row;
    if (gq >= g.nfv) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int f = 2 * (gq - g.nfv) + h;
        if (f >= g.nfs) break;
        double2* o = g.out2 + ((size_t)f * (g.T + 1) + m) * g.nlat;
        o[lat] = make_double2(P[4 * h], P[4 * h + 1]);
        o[lats] = make_double2(P[4 * h + 2], P[4 * h + 3]);
      }
    } else {
      const size_t o = ((size_t)gq * (g.T + 1) + m) * g.nlat;
#pragma unroll
      for (int hs = 0; hs < 2; ++hs) {
        const float* p = P + 4 * hs;
        const float* q = H + 4 * hs;
        const float sh = hs ? -1.f : 1.f;
        const int j = hs ? lats : lat;
        g.out0[o + j] = make_double2(ia * (-sh * q[0] - fm * p[3]), ia * (-sh * q[1] + fm * p[2]));
        g.out1[o + j] = make_double2(ia * (-fm * p[1] + sh * q[2]), ia * (fm * p[0] + sh * q[3]));
      }
    }
  } else {
    if (row >= g.T + 1 - m) return;
    const int par = row & 1;
    const size_t i = (size_t)moff(g.T, m) + row;
    if (gq >= g.nfv) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int f = 2 * (gq - g.nfv) + h;
        if (f >= g.nfs) break;
        g.out2[(size_t)f * g.nlm + i] = par ? make_double2(P[4 * h + 2], P[4 * h + 3])
                                            : make_double2(P[4 * h], P[4 * h + 1]);
      }
    } else {
      float p[4], q[4];  // register selects (no indexing by the parity)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        p[c] = par ? P[4 + c] : P[c];
        q[c] = par ? H[c] : H[4 + c];
      }
      const size_t o = (size_t)gq * g.nlm + i;
      g.out0[o] = make_double2(ia * (-fm * p[1] - q[2]), ia * (fm * p[0] - q[3]));
      g.out1[o] = make_double2(ia * (-fm * p[3] + q[0]), ia * (fm * p[2] + q[1]));
    }
  }
}

__device__ __forceinline__ uint32_t tf32_rna(float v) {
  uint32_t t;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
  return t;
}

// One 16-byte core-matrix row of a B operand: E consecutive K elements of column c of the
// K group whose first byte is `grp` (column c at (c >> 3) * sbo + (c & 7) * 16), rounded to
// TF32 (cvt.rna) or BF16 (round to nearest even); PM_TF32X3 also writes the lo parts
// tf32(v - tf32(v)) at grp + blo (v - tf32(v) is exact in FP32)
template <int PM>
__device__ __forceinline__ void store_row16(unsigned char* grp, int c, int sbo, uint32_t blo, const float* v) {
  uint4 u;
  uint32_t* w = reinterpret_cast<uint32_t*>(&u);
  const size_t off = (size_t)(c >> 3) * sbo + (c & 7) * 16;
  if (PM == PM_BF16) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
      w[e] = *reinterpret_cast<const uint32_t*>(&h);
    }
  } else if (PM == PM_TF32X3) {
    uint4 l;
    uint32_t* wl = reinterpret_cast<uint32_t*>(&l);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      w[e] = tf32_rna(v[e]);
      wl[e] = tf32_rna(v[e] - __uint_as_float(w[e]));
    }
    *reinterpret_cast<uint4*>(grp + blo + off) = l;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) w[e] = tf32_rna(v[e]);
  }
  *reinterpret_cast<uint4*>(grp + off) = u;
}

// B operand of job (m, kpad) written into shared memory at `base` by the threads of the
// builder warps (bt = thread index among them), in the tensor cores' canonical K-major layout
// (K group g of E elements at g * 128 B, column c at (c >> 3) * sbo + (c & 7) * 16).  A field
// (vector pair or scalar) with cpf values q per latitude owns 2 cpf columns from its first
// column c0: vector pair f from c0 = 8 f (cpf = 4), scalar field f from c0 = 8 nfv + 4 f
// (cpf = 2).  Columns past 8 nfv + 4 nfs are never written: each accumulator column depends
// on its own B column only, and the epilogue never reads them.
//   synthesis (K = degrees k = n - m): coefficient q of the field in column c0 + q (the
//     northern latitude's P_n(mu)), times (-1)^k in column c0 + cpf + q (the southern
//     one: P_n(-mu) = (-1)^(n-m) P_n(mu)); scalar q: re, im; vector q: psi re, im, chi re, im.
//   analysis (K = northern latitudes j): w_j (F_N + F_S) in column c0 + q, w_j (F_N - F_S)
//     in column c0 + cpf + q; scalar q: re, im; vector q: A re, im, B re, im.
// One item = (K group, column pair p < 2 nfv + nfs): E loads of its pair, four 16-byte rows;
// pairs 2 f and 2 f + 1 are the psi (A) and chi (B) columns of vector pair f, pair 2 nfv + f
// the columns of scalar field f.
template <int PM>
__device__ __forceinline__ void build_b(const GemmArgs& g, int m, int kpad, unsigned char* base, int bt) {
  constexpr int E = PM == PM_BF16 ? 8 : 4;
  const int nv = 2 * g.nfv, np = nv + g.nfs;
  const int sbo = (kpad / E) * 128;
  const int nitems = (kpad / E) * np;
  for (int it = bt; it < nitems; it += TC_NBUILD * 32) {
    const int gk = it / np, p = it - gk * np;
    const bool vec = p < nv;
    const int f = vec ? p >> 1 : p - nv;
    const int cpf = vec ? 4 : 2;
    const int cn = vec ? 8 * f + 2 * (p & 1) : 8 * g.nfv + 4 * f;  // the second block is cpf further
    const double2* in = vec ? ((p & 1) ? g.in1 : g.in0) : g.in2;
    unsigned char* grp = base + (size_t)gk * 128;
    float v0[E], v1[E], v2[E], v3[E];
    if (g.synth) {
      const int K = g.T + 1 - m;
      const double2* src = in + (size_t)f * g.nlm + moff(g.T, m);
      double2 c[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = gk * E + e;
        c[e] = k < K ? src[k] : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {  // gk * E is even: the parity of k is that of e
        v0[e] = (float)c[e].x;
        v1[e] = (float)c[e].y;
        v2[e] = (e & 1) ? -v0[e] : v0[e];
        v3[e] = (e & 1) ? -v1[e] : v1[e];
      }
    } else {
      const int nh = g.nlat / 2;
      const double2* Fq = in + ((size_t)f * (g.T + 1) + m) * g.nlat;
      const double* wt = vec ? g.wts : g.wts2;
      double2 a[E], b[E];
      double w[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int j = gk * E + e;
        const bool ok = j < nh;
        a[e] = ok ? Fq[j] : make_double2(0.0, 0.0);
        b[e] = ok ? Fq[g.nlat - 1 - j] : make_double2(0.0, 0.0);
        w[e] = ok ? wt[j] : 0.0;
      }
      // combinations in FP32 (the operand is rounded to TF32 / BF16 next; FP64 arithmetic is a
      // scarce pipe on this GPU): only the conversions of the inputs touch FP64 values
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const float ax = (float)a[e].x, ay = (float)a[e].y, bx = (float)b[e].x, by = (float)b[e].y;
        const float we = (float)w[e];
        v0[e] = we * (ax + bx);
        v1[e] = we * (ay + by);
        v2[e] = we * (ax - bx);
        v3[e] = we * (ay - by);
      }
    }
    store_row16<PM>(grp, cn, sbo, g.blo, v0);
    store_row16<PM>(grp, cn + 1, sbo, g.blo, v1);
    store_row16<PM>(grp, cn + cpf, sbo, g.blo, v2);
    store_row16<PM>(grp, cn + cpf + 1, sbo, g.blo, v3);
  }
}

// and-reduction of v over the threads of the builder warps (named barrier 1)
__device__ __forceinline__ bool builders_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(TC_NBUILD * 32)
      : "memory");
  return r != 0;
}

template <int PM>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_gemm(const __grid_constant__ GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // element type constants: 16-byte core-matrix rows hold E elements; a chunk (KC = 256 B of
  // K per row) is 8 MMA k-steps of 32 B; consecutive k-steps are 2 core matrices (256 B) apart.
  // PM_TF32X3: a chunk row holds KCK = 32 hi elements of K, then the same 32 lo elements
  constexpr bool BF = PM == PM_BF16, SPLIT = PM == PM_TF32X3;
  constexpr int E = BF ? 8 : 4, eb = BF ? 2 : 4, KC = BF ? 128 : 64, KSTEP = BF ? 16 : 8;
  constexpr int KCK = SPLIT ? KC / 2 : KC;  // K covered by one chunk
  constexpr uint32_t chunk_bytes = 128u * KC * eb;
  static_assert(KC * eb == 256, "a chunk row is 256 bytes of K");
  constexpr int KSTEPS = KCK / KSTEP;  // k-steps per full chunk (8; 4 split)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = g.stages, NB = g.nb;
  unsigned char* sA = smem;
  unsigned char* sB = smem + (size_t)S * chunk_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + (size_t)NB * g.bslot);
  // barriers: full[S], empty[S], bfull[NB], bempty[NB], tfull[NJB], tempty[NJB], fin
  const uint32_t full0 = tc::smem_u32(bars), empty0 = full0 + 8 * S;
  const uint32_t bfull0 = empty0 + 8 * S, bempty0 = bfull0 + 8 * NB, tfull0 = bempty0 + 8 * NB;
  const uint32_t tempty0 = tfull0 + 8 * TC_NJB, fin = tempty0 + 8 * TC_NJB;
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(bars + 2 * S + 2 * NB + 2 * TC_NJB + 1);
  Job* sjobs = reinterpret_cast<Job*>(bars + 2 * S + 2 * NB + 2 * TC_NJB + 2);
  // jobs of this CTA, descriptors staged in shared memory
  const int j0 = g.cta_off[blockIdx.x];
  const int nj = min(g.cta_off[blockIdx.x + 1] - j0, g.nj_max);
  for (int i = tid; i < nj; i += blockDim.x) sjobs[i] = g.jobs[j0 + i];
  if (tid == 0) {
    for (int i = 0; i < 2 * S + 2 * NB + TC_NJB; ++i) tc::mbar_init(full0 + 8 * i, 1);
    for (int i = 0; i < TC_NJB; ++i) tc::mbar_init(tempty0 + 8 * i, 4);
    tc::mbar_init(fin, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(taddr_s), TC_TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *taddr_s;
  // accumulator column stride (N rounded to 32) and the job buffers that fit in TMEM_COLS
  const uint32_t cs = (uint32_t)((g.ncols + 31) / 32 * 32);
  const int njb = min(TC_NJB, (int)(TC_TMEM_COLS / (cs * TC_NACC)));
  const uint32_t sa0 = tc::smem_u32(sA), sb0 = tc::smem_u32(sB);
  long long a_issued = 0;  // producer: A fills issued

  if (warp == 4) {
    if (lane == 0) {
      bool ok = true;
      int s = 0;
      uint32_t round = 0;  // number of completed passes over the ring
      for (int i = 0; i < nj && ok; ++i) {
        const Job jb = sjobs[i];
        const unsigned char* A = (jb.tab ? g.tabH : g.tabP) + jb.a_off;
        // rows / 8 core-matrix row groups: a prefix of the stage's canonical layout
        const uint32_t jchunk = (uint32_t)jb.rows * KC * eb;
        for (int c = jb.c0; c < jb.nchunk; ++c) {
          if (round > 0) ok = tc::mbar_wait(empty0 + 8 * s, (round - 1) & 1);
          if (!ok) break;
          const uint32_t cb = (c == jb.nchunk - 1) ? (uint32_t)jb.rows * jb.kl * eb * (SPLIT ? 2 : 1) : jchunk;
          tc::mbar_expect_tx(full0 + 8 * s, cb);
          tc::bulk_g2s(sa0 + s * chunk_bytes, A + (size_t)(c - jb.c0) * jchunk, cb, full0 + 8 * s);
          ++a_issued;
          if (++s == S) {
            s = 0;
            ++round;
          }
        }
      }
      if (!ok) atomicExch(g.err, 3);
    }
  } else if (warp >= TC_BUILD0) {
    // B operand of B group bg (first job q) into buffer bg % NB once its previous group has
    // released it
    // (its MMAs completed): written with ordinary shared-memory stores, made visible to the
    // tensor cores' (async) proxy by a proxy fence, then announced on bfull by one thread
    // (every thread of the builder warps takes the same path: the outcome of the bounded
    // wait is and-reduced over them, so that a timeout ends the loop for all at once)
    const int bt = tid - TC_BUILD0 * 32;
    int bg = -1;  // B group of the job: the jobs of one group (one m) share the buffer
    for (int q = 0; q < nj; ++q) {
      if (!sjobs[q].newb) continue;
      ++bg;
      const int b = bg % NB, u = bg / NB;
      const bool ok = builders_all(u == 0 || tc::mbar_wait(bempty0 + 8 * b, (u - 1) & 1));
      if (!ok) {
        if (bt == 0) atomicExch(g.err, 5);
        break;
      }
      const Job jq = sjobs[q];
      build_b<PM>(g, jq.m, jq.kpad, sB + (size_t)b * g.bslot, bt);
      tc::fence_proxy_async();
      builders_all(true);  // every row of the operand is written and fenced
      if (bt == 0) tc::mbar_arrive(bfull0 + 8 * b);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      bool ok = true;
      const uint32_t idesc = tc::instr_desc(128, g.ncols, BF ? 1 : 2);
      const uint32_t sboA = (uint32_t)(KC / E) * 128u;
      int s = 0;
      uint32_t round = 0;
      // B group bg (jobs from one with newb to the next) uses buffer bg % NB
      int bg = -1;
      for (int i = 0; i < nj && ok; ++i) {
        const Job jb = sjobs[i];
        if (jb.newb) ++bg;
        const int b = bg % NB, ub = bg / NB, acc = i % njb, ua = i / njb;
        const bool last_of_b = i + 1 == nj || sjobs[i + 1].newb;
        if (jb.newb) ok = tc::mbar_wait(bfull0 + 8 * b, ub & 1);
        if (ok && ua > 0) ok = tc::mbar_wait(tempty0 + 8 * acc, (ua - 1) & 1);
        if (!ok) break;
        tc::fence_after_sync();
        // k-step q of every chunk accumulates into accumulator q % TC_NACC of job buffer acc,
        // so that consecutive MMAs do not wait on each other's result
        const uint32_t dt = tmem + cs * TC_NACC * acc;
        const uint64_t bdesc0 = tc::smem_desc(sb0 + b * g.bslot, 128u, (uint32_t)(jb.kpad / E) * 128u);
        for (int c = jb.c0; c < jb.nchunk; ++c) {
          ok = tc::mbar_wait(full0 + 8 * s, round & 1);
          if (!ok) break;
          tc::fence_after_sync();
          // the last chunk may be short: its own core-matrix stride and fewer k-steps
          const int kc = (c == jb.nchunk - 1) ? jb.kl : KCK;
          const int kw = SPLIT ? 2 * kc : kc;  // K width of the stored chunk
          const uint64_t ad = tc::smem_desc(sa0 + s * chunk_bytes, 128u, kw == KC ? sboA : (uint32_t)(kw / E) * 128u);
          const uint64_t bd = bdesc0 + (uint64_t)(c * ((KCK / E) * 128 / 16));  // + c * KCK K elements
          const int nks = kc / KSTEP;
#pragma unroll
          for (int q = 0; q < KSTEPS; ++q) {  // + 256 B per k-step: +16 in the address field
            // k-step q goes to accumulator q % TC_NACC; its first use initialises it
            const uint32_t accum = (c > jb.c0 || q >= TC_NACC) ? 1u : 0u;
            const uint32_t da = dt + cs * (q % TC_NACC);
            if (q < nks) {
              if (BF) {
                tc::mma_f16(da, ad + 16u * q, bd + 16u * q, idesc, accum);
              } else if (SPLIT) {
                // the small products first: a_hi b_lo, a_lo b_hi (lo half of the chunk), a_hi b_hi
                const uint64_t alo = ad + (uint64_t)((kc / E) * 128 / 16);
                const uint64_t blo = bd + (uint64_t)(g.blo >> 4);
                tc::mma_tf32(da, ad + 16u * q, blo + 16u * q, idesc, accum);
                tc::mma_tf32(da, alo + 16u * q, bd + 16u * q, idesc, 1u);
                tc::mma_tf32(da, ad + 16u * q, bd + 16u * q, idesc, 1u);
              } else {
                tc::mma_tf32(da, ad + 16u * q, bd + 16u * q, idesc, accum);
              }
            }
          }
          tc::mma_commit(empty0 + 8 * s);
          if (++s == S) {
            s = 0;
            ++round;
          }
        }
        if (!ok) break;
        if (last_of_b) tc::mma_commit(bempty0 + 8 * b);
        tc::mma_commit(tfull0 + 8 * acc);
      }
      if (!ok) atomicExch(g.err, 4);
      tc::mma_commit(fin);  // arrives once every MMA issued above has completed
    }
  } else {
    // epilogue warps 0-3: warp w holds rows 32 w .. 32 w + 31 of every job (its TMEM lane
    // quarter); the jobs of a vector transform come in (P, H) pairs, released together
    const int step = g.pair ? 2 : 1;
    const int ngrp = g.nfv + (g.nfs + 1) / 2;  // 8-column groups holding results
    for (int i = 0; i + step <= nj; i += step) {
      const Job jb = sjobs[i];
      const int acc0 = i % njb, acc1 = (i + 1) % njb;
      auto wait_acc = [&](int acc, uint32_t parity) {
        if (!g.epi_polls) return tc::mbar_wait(tfull0 + 8 * acc, parity);
        for (uint32_t it = 0; it < g.epi_polls; ++it)
          if (tc::mbar_test(tfull0 + 8 * acc, parity)) return true;
        return false;
      };
      bool ok = wait_acc(acc0, (i / njb) & 1);
      if (ok && g.pair) ok = wait_acc(acc1, ((i + 1) / njb) & 1);
      if (!ok) {
        if (lane == 0) atomicExch(g.err, 2);
        break;
      }
      tc::fence_after_sync();
      if (32 * warp < jb.rows) {  // warp-uniform: tcgen05.ld is collective
        // accumulators a < nacc received k-steps (all four unless the job streams one short chunk)
        const int nacc = jb.nchunk - jb.c0 > 1 ? TC_NACC : min(TC_NACC, jb.kl / KSTEP);
        const uint32_t lq = (uint32_t)(32 * warp) << 16;
        const uint32_t ta0 = tmem + lq + cs * TC_NACC * acc0, ta1 = tmem + lq + cs * TC_NACC * acc1;
        const int row = jb.tile * 128 + 32 * warp + lane;
        for (int gq = 0; gq < ngrp; ++gq) {
          float P[8], H[8];
          tmem_sum8(ta0 + 8 * gq, cs, nacc, P);
          if (gq < g.nfv) tmem_sum8(ta1 + 8 * gq, cs, nacc, H);
          epilogue8(g, jb.m, row, gq, P, H);
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(tempty0 + 8 * acc0);
        if (g.pair) tc::mbar_arrive(tempty0 + 8 * acc1);
      }
    }
  }
  // ---- teardown: no copy may land in, and no MMA may read, a CTA that has exited ----------
  if (warp == 4 && lane == 0) {
    // the newest fill of each stage / B buffer: completed fills return at once
    for (long long q = a_issued - 1; q >= 0 && q >= a_issued - S; --q)
      tc::mbar_wait(full0 + 8 * (int)(q % S), (uint32_t)((q / S) & 1), 200000u);
  }
  if (warp == 5 && lane == 0) tc::mbar_wait(fin, 0, 4000000u);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, TC_TMEM_COLS);
}

// ---- canonical layout helpers ---------------------------------------------------------
__device__ __forceinline__ size_t canon_off(int row, int kk, int E, int eb, int sbo) {
  return (size_t)(row >> 3) * sbo + (size_t)(kk / E) * 128 + (row & 7) * 16 + (kk % E) * eb;
}
__device__ __forceinline__ void store_elem(unsigned char* base, size_t off, float v, int bf16) {
  if (bf16) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
  } else {
    *reinterpret_cast<uint32_t*>(base + off) = tf32_rna(v);
  }
}

// tables: one thread per (job, row), looping over K; src = FP64 table [moff+k][nh];
// pm = PM_TF32 / PM_BF16 / PM_TF32X3 (a chunk then holds kc hi elements, then kc lo elements)
struct TabJob {
  long long a_off;
  int m, rows, tile, nchunk, kl, c0;  // rows: stored rows (<= 128); kl: K of the last chunk;
                                      // chunks c0 .. nchunk - 1 are stored
};
__global__ void k_tc_table(const double* __restrict__ src, unsigned char* __restrict__ dst,
                           const TabJob* __restrict__ jobs, int njobs, int T, int nh, int synth,
                           int pm) {
  const int jid = blockIdx.x;
  if (jid >= njobs) return;
  const TabJob j = jobs[jid];
  const int r = threadIdx.x;  // 0..127
  if (r >= j.rows) return;
  const int bf16 = pm == PM_BF16, split = pm == PM_TF32X3;
  const int E = bf16 ? 8 : 4, eb = bf16 ? 2 : 4, KC = bf16 ? 128 : 64;  // as TcLegendre::KC
  const int KCK = split ? KC / 2 : KC;                                     // K per chunk
  const int K = T + 1 - j.m, base = moff(T, j.m);
  unsigned char* out = dst + j.a_off;
  for (int c = j.c0; c < j.nchunk; ++c) {
    // every chunk but the last covers KCK K-elements per row; the last covers j.kl
    const int kc = (c == j.nchunk - 1) ? j.kl : KCK;
    const int sbo = ((split ? 2 * kc : kc) / E) * 128;
    unsigned char* ch = out + (size_t)(c - j.c0) * j.rows * KC * eb;
    for (int kk = 0; kk < kc; ++kk) {
      double x = 0.0;
      if (synth) {  // rows = latitudes of the northern half, K = all degrees n = m + k
        const int lat = j.tile * 128 + r;
        const int k = c * KCK + kk;
        if (lat < nh && k < K) x = src[(size_t)(base + k) * nh + lat];
      } else {      // rows = degrees (both parities), K = latitudes
        const int k = j.tile * 128 + r;
        const int lat = c * KCK + kk;
        if (lat < nh && k < K) x = src[(size_t)(base + k) * nh + lat];
      }
      if (split) {
        const uint32_t hi = tf32_rna((float)x);
        const uint32_t lo = tf32_rna((float)(x - (double)__uint_as_float(hi)));
        *reinterpret_cast<uint32_t*>(ch + canon_off(r, kk, E, eb, sbo)) = hi;
        *reinterpret_cast<uint32_t*>(ch + canon_off(r, kc + kk, E, eb, sbo)) = lo;
      } else {
        store_elem(ch, canon_off(r, kk, E, eb, sbo), (float)x, bf16);
      }
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// A GEMM launch plan: per-CTA job lists, flattened (CTA c: jobs[off[c] .. off[c + 1])).
struct Sched {
  Job* jobs = nullptr;
  int* off = nullptr;
  int grid = 0, nj_max = 0;
};

struct TcLegendre {
  int T = 0, nlat = 0, nh = 0, nlm = 0, max_fields = 0, bf16 = 0, E = 4, eb = 4, KC = 32;
  int pm = PM_TF32, KCK = 64;  // precision mode; K covered by one chunk (KC, or KC / 2 split)
  uint32_t epi_polls = 0;      // see GemmArgs::epi_polls
  int ntile_s = 0, kpad_a = 0;
  unsigned char *tabPs = nullptr, *tabHs = nullptr, *tabPa = nullptr, *tabHa = nullptr;
  int* err = nullptr;
  const double *w = nullptr, *wq = nullptr;
  // launch plans: [synthesis, analysis][scalar (P jobs), vector ((P, H) pairs)]
  Sched sched[2][2];
  int kpad_smax = 0;  // largest K extent of a synthesis B operand
  int nsm = 0;
  long long streamed_s = 0, streamed_a = 0;  // table entries inside the streamed chunks (per table)
  StageProf* prof = nullptr;
};

static int tc_fail(const char* what, cudaError_t e) { return cuda_fail(e, what); }

// Per-CTA job lists.  A unit is all jobs of one zonal order m (the tiles of m; with H given,
// each tile's (P, H) pair), which then run back to back and share one B operand (the first job
// of a unit starts a B group, `newb`); a unit heavier than half the mean CTA load is split into
// its tiles, so that the heaviest zonal orders still balance.  Units go longest first (cost =
// A bytes, rows x the K streamed from chunk c0 on, kck K elements per chunk), each to the
// least-loaded CTA so far.
static cudaError_t make_sched(const std::vector<Job>& P, const std::vector<Job>* H, int nsm, int kck, Sched& sc) {
  auto cost = [&](int u) { return (long long)P[u].rows * (P[u].kpad - P[u].c0 * kck) * (H ? 2 : 1); };
  std::vector<std::vector<int>> units;
  {
    std::map<int, std::vector<int>> by_m;
    long long total = 0;
    for (int u = 0; u < (int)P.size(); ++u) {
      by_m[P[u].m].push_back(u);
      total += cost(u);
    }
    const long long cap = std::max<long long>(1, total / std::max(1, nsm) / 2);
    for (auto& kv : by_m) {
      long long c = 0;
      for (int u : kv.second) c += cost(u);
      if (c > cap && kv.second.size() > 1) {
        for (int u : kv.second) units.push_back({u});
      } else {
        units.push_back(kv.second);
      }
    }
  }
  const int nu = (int)units.size();
  const int grid = std::max(1, std::min(nu, nsm));
  auto ucost = [&](int k) {
    long long c = 0;
    for (int u : units[k]) c += cost(u);
    return c;
  };
  std::vector<int> order(nu);
  for (int k = 0; k < nu; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ucost(a) > ucost(b); });
  std::vector<long long> load(grid, 0);
  std::vector<std::vector<int>> per(grid);
  for (int k : order) {
    const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    per[c].push_back(k);
    load[c] += ucost(k);
  }
  std::vector<Job> jobs;
  std::vector<int> off(grid + 1);
  sc.nj_max = 0;
  for (int c = 0; c < grid; ++c) {
    off[c] = (int)jobs.size();
    for (int k : per[c]) {
      bool first = true;
      for (int u : units[k]) {
        Job jp = P[u];
        jp.newb = first ? 1 : 0;
        first = false;
        jobs.push_back(jp);
        if (H) {
          Job jh = (*H)[u];
          jh.newb = 0;
          jobs.push_back(jh);
        }
      }
    }
    sc.nj_max = std::max(sc.nj_max, (int)jobs.size() - off[c]);
  }
  off[grid] = (int)jobs.size();
  sc.grid = grid;
  cudaError_t e;
  if ((e = cudaMalloc(&sc.jobs, sizeof(Job) * std::max<size_t>(1, jobs.size()))) ||
      (e = cudaMalloc(&sc.off, sizeof(int) * off.size())))
    return e;
  if ((e = cudaMemcpy(sc.jobs, jobs.data(), sizeof(Job) * jobs.size(), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(sc.off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice)))
    return e;
  return cudaSuccess;
}

int tc_legendre_create(TcLegendre** out, const double* P, const double* H, const double* w, const double* wq,
                       int T, int nlat, int max_fields, int mode, const PolarBounds& pb, cudaStream_t stream) {
  *out = nullptr;
  if (max_fields > 8) return fail(REXI_EINVAL, "sh_plan_create: tensor-core precisions support max_fields <= 8");
  const bool bf16 = mode == SH_BF16, split = mode == SH_TF32X3;
  TcLegendre* t = new TcLegendre();
  t->T = T;
  t->nlat = nlat;
  t->nh = nlat / 2;
  t->nlm = (T + 1) * (T + 2) / 2;
  t->max_fields = max_fields;
  t->bf16 = bf16 ? 1 : 0;
  t->pm = bf16 ? PM_BF16 : split ? PM_TF32X3 : PM_TF32;
  t->E = bf16 ? 8 : 4;
  t->eb = bf16 ? 2 : 4;
  t->KC = bf16 ? 128 : 64;   // 256 bytes of K per chunk row
  t->KCK = split ? t->KC / 2 : t->KC;
  t->w = w;
  t->wq = wq;
  const int KC = t->KC, KCK = t->KCK, eb = t->eb, kw = split ? 2 : 1;
  const size_t chunk = 128ull * KC * eb;
  cudaError_t e;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    if ((e = cudaDeviceGetAttribute(&t->nsm, cudaDevAttrMultiProcessorCount, dev))) {
      tc_legendre_destroy(t);
      return tc_fail("cudaDeviceGetAttribute(SM count)", e);
    }
  }
  t->ntile_s = (t->nh + 127) / 128;
  const int kstep = bf16 ? 16 : 8;  // MMA K per instruction
  // ---- synthesis jobs: (m, tile, tab); rows = northern latitudes of the tile, K = all degrees
  // of m; B = [c | (-1)^(n-m) c] gives the northern and the southern values in one job -------
  std::vector<TabJob> tj;
  std::vector<Job> jsP, jsH;  // aligned: entry u of both is the same (m, tile)
  long long aoff = 0;
  for (int m = 0; m <= T; ++m) {
    const int K = T + 1 - m;
    const int kpad = (K + kstep - 1) / kstep * kstep;  // K padded to whole k-steps only
    const int nchunk = (kpad + KCK - 1) / KCK;
    const int kl = kpad - (nchunk - 1) * KCK;
    t->kpad_smax = std::max(t->kpad_smax, kpad);
    for (int tile = 0; tile < t->ntile_s; ++tile) {
      const int rows = std::min(128, (t->nh - 128 * tile + 7) / 8 * 8);
      // first chunk: the smallest polar start of the tile's four 32-latitude groups
      int kb = K;
      for (int g = 4 * tile; g < std::min(4 * tile + 4, pb.ngl); ++g) kb = std::min(kb, pb.ks[m * pb.ngl + g]);
      const int c0 = std::min(kb / KCK, nchunk - 1);
      tj.push_back(TabJob{aoff, m, rows, tile, nchunk, kl, c0});
      jsP.push_back(Job{aoff, m, tile, nchunk, kpad, 0, kl, rows, 0, c0});
      jsH.push_back(Job{aoff, m, tile, nchunk, kpad, 1, kl, rows, 0, c0});
      aoff += (long long)rows * ((nchunk - 1 - c0) * KC + kw * kl) * eb;
      t->streamed_s += (long long)std::min(128, t->nh - 128 * tile) * std::max(0, K - c0 * KCK);
    }
  }
  const long long tab_s_bytes = aoff;
  // ---- analysis jobs: (m, degree tile, tab), rows = degrees of both parities, K = northern
  // latitudes; B = [N + S | N - S] of each field of zonal order m --------------------------
  t->kpad_a = (t->nh + kstep - 1) / kstep * kstep;
  const int nchunk_a = (t->kpad_a + KCK - 1) / KCK;
  const int kl_a = t->kpad_a - (nchunk_a - 1) * KCK;
  std::vector<TabJob> ta;
  std::vector<Job> jaP, jaH;
  aoff = 0;
  for (int m = 0; m <= T; ++m) {
    const int K = T + 1 - m;
    const int ntiles = (K + 127) / 128;
    for (int tile = 0; tile < ntiles; ++tile) {
      const int rows = std::min(128, (K - 128 * tile + 7) / 8 * 8);
      // first chunk: the smallest polar start of the tile's 32-degree groups
      int jb = t->nh;
      for (int g = 4 * tile; g < std::min(4 * tile + 4, pb.ngd) && 32 * g < K; ++g)
        jb = std::min(jb, pb.ja[m * pb.ngd + g]);
      const int c0 = std::min(jb / KCK, nchunk_a - 1);
      ta.push_back(TabJob{aoff, m, rows, tile, nchunk_a, kl_a, c0});
      jaP.push_back(Job{aoff, m, tile, nchunk_a, t->kpad_a, 0, kl_a, rows, 0, c0});
      jaH.push_back(Job{aoff, m, tile, nchunk_a, t->kpad_a, 1, kl_a, rows, 0, c0});
      aoff += (long long)rows * ((nchunk_a - 1 - c0) * KC + kw * kl_a) * eb;
      t->streamed_a += (long long)std::min(128, K - 128 * tile) * std::max(0, t->nh - c0 * KCK);
    }
  }
  const long long tab_a_bytes = aoff;
  // the largest B operand of any call (a vector pair: 2 x 4 max_fields columns over all
  // latitudes or all degrees) must fit one B buffer and two ring stages in shared memory
  {
    auto ncols_of = [](int nf, int cpf) { return std::max(16, (nf * cpf + 15) / 16 * 16); };
    const size_t bmax = (size_t)kw * ncols_of(2 * max_fields, 4) * std::max(t->kpad_a, t->kpad_smax) * eb;
    if (bmax + 2 * chunk + 4096 > TC_SMEM_BUDGET) {
      tc_legendre_destroy(t);
      return fail(REXI_EINVAL,
                  "sh_plan_create: %d latitudes x %d fields exceed the tensor-core shared-memory budget; "
                  "use fewer fields per call", nlat, max_fields);
    }
  }
  // ---- device buffers and launch plans ------------------------------------------------------
  TabJob *d_tj = nullptr, *d_ta = nullptr;
  if ((e = cudaMalloc(&t->tabPs, tab_s_bytes)) || (e = cudaMalloc(&t->tabHs, tab_s_bytes)) ||
      (e = cudaMalloc(&t->tabPa, tab_a_bytes)) || (e = cudaMalloc(&t->tabHa, tab_a_bytes)) ||
      (e = cudaMalloc(&t->err, sizeof(int))) ||
      (e = cudaMalloc(&d_tj, sizeof(TabJob) * tj.size())) || (e = cudaMalloc(&d_ta, sizeof(TabJob) * ta.size())) ||
      (e = make_sched(jsP, nullptr, t->nsm, KCK, t->sched[0][0])) ||
      (e = make_sched(jsP, &jsH, t->nsm, KCK, t->sched[0][1])) ||
      (e = make_sched(jaP, nullptr, t->nsm, KCK, t->sched[1][0])) ||
      (e = make_sched(jaP, &jaH, t->nsm, KCK, t->sched[1][1]))) {
    cudaGetLastError();
    tc_legendre_destroy(t);
    cudaFree(d_tj);
    cudaFree(d_ta);
    return fail(REXI_ENOMEM, "tensor-core Legendre tables: cudaMalloc failed: %s", cudaGetErrorString(e));
  }
  cudaMemset(t->err, 0, sizeof(int));
  cudaMemcpy(d_tj, tj.data(), sizeof(TabJob) * tj.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(d_ta, ta.data(), sizeof(TabJob) * ta.size(), cudaMemcpyHostToDevice);
  k_tc_table<<<(int)tj.size(), 128, 0, stream>>>(P, t->tabPs, d_tj, (int)tj.size(), T, t->nh, 1, t->pm);
  k_tc_table<<<(int)tj.size(), 128, 0, stream>>>(H, t->tabHs, d_tj, (int)tj.size(), T, t->nh, 1, t->pm);
  k_tc_table<<<(int)ta.size(), 128, 0, stream>>>(P, t->tabPa, d_ta, (int)ta.size(), T, t->nh, 0, t->pm);
  k_tc_table<<<(int)ta.size(), 128, 0, stream>>>(H, t->tabHa, d_ta, (int)ta.size(), T, t->nh, 0, t->pm);
  e = cudaStreamSynchronize(stream);
  cudaFree(d_tj);
  cudaFree(d_ta);
  if (e != cudaSuccess) {
    tc_legendre_destroy(t);
    return tc_fail("tensor-core Legendre table kernels", e);
  }
  if ((e = cudaFuncSetAttribute(k_tc_gemm<PM_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_BUDGET)) ||
      (e = cudaFuncSetAttribute(k_tc_gemm<PM_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_BUDGET)) ||
      (e = cudaFuncSetAttribute(k_tc_gemm<PM_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_BUDGET))) {
    tc_legendre_destroy(t);
    return tc_fail("cudaFuncSetAttribute(k_tc_gemm)", e);
  }
  *out = t;
  return REXI_OK;
}

void tc_legendre_destroy(TcLegendre* t) {
  if (!t) return;
  for (void* p : {(void*)t->tabPs, (void*)t->tabHs, (void*)t->tabPa, (void*)t->tabHa, (void*)t->err})
    cudaFree(p);
  for (auto& row : t->sched)
    for (Sched& sc : row) {
      cudaFree(sc.jobs);
      cudaFree(sc.off);
    }
  delete t;
}

// One GEMM launch with the fused epilogue over nfv vector pairs and nfs scalar fields: ncols =
// MMA N (the real columns 8 nfv + 4 nfs, padded to a multiple of 16; the padding columns of B
// are never written and their sums never read).  With nfv > 0 the launch runs (P, H) job
// pairs, and the scalar fields ride on the P jobs' table reads.
static int gemm(TcLegendre* t, bool synth, int nfv, const double2* in0, const double2* in1, double2* out0,
                double2* out1, int nfs, const double2* in2, double2* out2, double inv_a, cudaStream_t s) {
  const int ncols = std::max(16, (8 * nfv + 4 * nfs + 15) / 16 * 16);
  const Sched& sc = t->sched[synth ? 0 : 1][nfv > 0 ? 1 : 0];
  GemmArgs g;
  g.tabP = synth ? t->tabPs : t->tabPa;
  g.tabH = synth ? t->tabHs : t->tabHa;
  g.in0 = in0;
  g.in1 = in1;
  g.in2 = in2;
  g.wts = synth ? nullptr : t->wq;
  g.wts2 = synth ? nullptr : t->w;
  g.jobs = sc.jobs;
  g.cta_off = sc.off;
  g.ncols = ncols;
  g.bf16 = t->bf16;
  g.synth = synth ? 1 : 0;
  g.pair = nfv > 0 ? 1 : 0;
  g.out0 = out0;
  g.out1 = out1;
  g.out2 = out2;
  g.T = t->T;
  g.nlat = t->nlat;
  g.nlm = t->nlm;
  g.nfv = nfv;
  g.nfs = nfs;
  g.inv_a = inv_a;
  g.err = t->err;
  g.nj_max = sc.nj_max;
  // B buffers of the largest B operand of the call, then as many A stages as fit
  const size_t chunk = 128ull * t->KC * t->eb;
  // one B copy, rounded to 128 bytes; PM_TF32X3 keeps the lo copy behind the hi copy
  const size_t bcopy = ((size_t)ncols * (synth ? t->kpad_smax : t->kpad_a) * t->eb + 127) / 128 * 128;
  const size_t bslot = t->pm == PM_TF32X3 ? 2 * bcopy : bcopy;
  const size_t jobs_bytes = sizeof(Job) * (size_t)g.nj_max;
  auto fixed = [&](int nb) { return nb * bslot + 8 * (2 * TC_MAXSTAGES + 2 * nb + 2 * TC_NJB + 2) + jobs_bytes; };
  // B buffers: 4 when that leaves >= 4 ring stages, else 2, else 1 (>= 2 ring stages always)
  g.nb = (fixed(TC_MAXNB) + 4 * chunk <= TC_SMEM_BUDGET) ? TC_MAXNB : (fixed(2) + 2 * chunk <= TC_SMEM_BUDGET) ? 2 : 1;
  if (fixed(g.nb) + 2 * chunk > TC_SMEM_BUDGET) return fail(REXI_EINVAL, "tensor-core Legendre: B operand too large");
  g.stages = (int)std::min<size_t>(TC_MAXSTAGES, (TC_SMEM_BUDGET - fixed(g.nb)) / chunk);
  g.bslot = (uint32_t)bslot;
  g.blo = t->pm == PM_TF32X3 ? (uint32_t)bcopy : 0u;
  g.epi_polls = t->epi_polls;
  const size_t smem =
      (size_t)g.stages * chunk + g.nb * bslot + 8 * (2 * g.stages + 2 * g.nb + 2 * TC_NJB + 2) + jobs_bytes;
  {
    const int ph = t->prof ? t->prof->begin(2) : -1;
    if (t->pm == PM_BF16) k_tc_gemm<PM_BF16><<<sc.grid, TC_THREADS, smem, s>>>(g);
    else if (t->pm == PM_TF32X3) k_tc_gemm<PM_TF32X3><<<sc.grid, TC_THREADS, smem, s>>>(g);
    else k_tc_gemm<PM_TF32><<<sc.grid, TC_THREADS, smem, s>>>(g);
    if (t->prof) t->prof->end(ph);
  }
  cudaError_t e = cudaGetLastError();
  return e ? cuda_fail(e, "k_tc_gemm launch") : REXI_OK;
}

int tc_leg_synth(TcLegendre* t, const double2* spec, double2* F, int nf, cudaStream_t s) {
  return gemm(t, true, 0, nullptr, nullptr, nullptr, nullptr, nf, spec, F, 0.0, s);
}

int tc_leg_synth_uv(TcLegendre* t, const double2* psi, const double2* chi, double2* FU, double2* FV, int nf,
                    double inv_a, cudaStream_t s) {
  return gemm(t, true, nf, psi, chi, FU, FV, 0, nullptr, nullptr, inv_a, s);
}

int tc_leg_anal(TcLegendre* t, const double2* F, double2* spec, int nf, cudaStream_t s) {
  return gemm(t, false, 0, nullptr, nullptr, nullptr, nullptr, nf, F, spec, 0.0, s);
}

int tc_leg_anal_divcurl(TcLegendre* t, const double2* FA, const double2* FB, double2* dv, double2* cu, int nf,
                        double inv_a, cudaStream_t s) {
  return gemm(t, false, nf, FA, FB, dv, cu, 0, nullptr, nullptr, inv_a, s);
}

int tc_leg_synth_mixed(TcLegendre* t, const double2* psi, const double2* chi, double2* FU, double2* FV, int nfv,
                       const double2* spec, double2* F, int nfs, double inv_a, cudaStream_t s) {
  return gemm(t, true, nfv, psi, chi, FU, FV, nfs, spec, F, inv_a, s);
}

int tc_leg_anal_mixed(TcLegendre* t, const double2* FA, const double2* FB, double2* dv, double2* cu, int nfv,
                      const double2* F, double2* spec, int nfs, double inv_a, cudaStream_t s) {
  return gemm(t, false, nfv, FA, FB, dv, cu, nfs, F, spec, inv_a, s);
}

void tc_legendre_streamed(const TcLegendre* t, long long* syn, long long* ana) {
  *syn = t->streamed_s;
  *ana = t->streamed_a;
}

void tc_legendre_set_prof(TcLegendre* t, StageProf* prof) {
  if (t) t->prof = prof;
}

void tc_legendre_set_epilogue_polls(TcLegendre* t, int polls) {
  if (t) t->epi_polls = polls > 0 ? (uint32_t)polls : 0u;
}

int tc_legendre_error(TcLegendre* t, int* flag) {
  if (!t) {
    *flag = 0;
    return REXI_OK;
  }
  cudaError_t e = cudaMemcpy(flag, t->err, sizeof(int), cudaMemcpyDeviceToHost);
  return e ? cuda_fail(e, "tc error flag") : REXI_OK;
}

}  // namespace rexi
