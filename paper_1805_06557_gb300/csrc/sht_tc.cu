// Tensor-core (tcgen05) Legendre contractions for sh_plan precisions SH_TF32 / SH_BF16
// (paper Sec. 3.2: the dense Legendre contraction per zonal order m of the SH transforms).
//
// Every contraction is a set of GEMM jobs D[128 x Ncols] = A[128 x K] B[K x Ncols]:
//   synthesis, per (m, parity of n - m, 128-latitude tile, table P or H):
//       A = table^T (rows = northern latitudes, K = degrees of that parity),
//       B = spectral coefficients (columns = fields x re/im [x psi/chi])
//   analysis, per (m, parity, 128-degree tile, table P or H):
//       A = table (rows = degrees of that parity, K = northern latitudes),
//       B = weighted hemispheric sums / differences of the Fourier coefficients.
// Operands are stored in the canonical no-swizzle K-major layout of the tensor cores
// (8-row x 16-byte core matrices; cores adjacent along K 128 B apart), the tables pre-tiled
// at plan time so that each K-chunk of A is one contiguous block moved by the bulk-copy
// engine (cp.async.bulk, completion on an mbarrier).  The GEMM is a persistent kernel, one
// CTA per SM, with a copy warp streaming A chunks through a ring of up to 8 stages and the
// B operands through two buffers, an MMA warp (accumulators in TMEM, FP32, two buffers) and
// four epilogue warps reading the accumulators with tcgen05.ld.  Epilogue kernels combine
// the parities (north = even + odd, south = even - odd for P; the opposite sign for H) in
// FP64.  All mbarrier waits are bounded; on a timeout the kernel records an error flag.
#include <algorithm>
#include <cuda_bf16.h>
#include <vector>

#include "sht_tc.cuh"
#include "tc_common.cuh"

namespace rexi {

namespace {

constexpr int TC_MAXSTAGES = 8;     // depth of the A-chunk ring
constexpr int TC_THREADS = 192;     // warps 0-3 epilogue, warp 4 bulk copies, warp 5 MMA issue
constexpr int TC_MAXCOL = 32;      // B columns of one half of a B operand (synthesis: north | south; analysis: N + S | N - S)
constexpr size_t TC_SMEM_BUDGET = 220 * 1024;

struct Job {
  long long a_off;  // byte offset of the job's first A chunk in its table
  int b_off;        // byte offset of the job's B operand in the B buffer
  int d_off;        // float offset of the job's D tile in the D buffer
  int nchunk;       // K chunks
  int kpad;         // K extent of B (whole MMA k-steps; (nchunk - 1) * KC + kl)
  int tab;          // 0 = P, 1 = H
  int kl;           // K of the last chunk (a multiple of the MMA k-step, <= KC)
};

struct GemmArgs {
  const unsigned char* tabP;
  const unsigned char* tabH;
  const unsigned char* B;
  float* D;
  const Job* jobs;
  int njobs, ncols, bf16;
  int stages;       // A ring depth (<= TC_MAXSTAGES)
  int nb;           // B buffers (1, 2 or 4): B operands are fetched up to nb - 1 jobs ahead
  int nj_max;       // jobs per CTA at most (their descriptors are staged in shared memory)
  uint32_t bslot;   // bytes of one B buffer
  int* err;
};

// Persistent, warp-specialised GEMM over the job list: CTA c takes jobs c, c + grid, ...
// (the list is sorted by decreasing length).  Warp 4 streams the A chunks of every job through
// the S-stage ring without pausing between jobs, and fetches B operands into NB buffers up to
// NB - 1 jobs ahead (so that a job's MMAs never wait for the latency of its B copy); warp 5
// issues the MMAs of job i into TMEM accumulator i & 1 and commits: the ring stage (empty),
// the B buffer (bempty) and the accumulator (tfull); warps 0-3 read accumulator i & 1 (one
// TMEM lane quarter each), store D, and release it (tempty), so that the MMAs of job i + 1
// overlap the epilogue of job i.  Every wait is bounded; on a timeout the role records an
// error code and stops, and teardown drains the copies and MMAs in flight.
constexpr int TC_MAXNB = 4;
constexpr int TC_NACC = 4;          // independent accumulators per job (one per k-step of a chunk)
constexpr int TC_NJB = 3;           // job buffers of accumulators in TMEM (at most; 2 when N > 32)
constexpr uint32_t TC_TMEM_COLS = 512;  // TC_NJB x TC_NACC x 32 (N <= 32) or 2 x TC_NACC x 64 (N <= 64)
template <bool BF>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_gemm(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // element type constants: 16-byte core-matrix rows hold E elements; a chunk (KC = 256 B of
  // K per row) is 8 MMA k-steps of 32 B; consecutive k-steps are 2 core matrices (256 B) apart
  constexpr int E = BF ? 8 : 4, eb = BF ? 2 : 4, KC = BF ? 128 : 64, KSTEP = BF ? 16 : 8;
  constexpr uint32_t chunk_bytes = 128u * KC * eb;
  static_assert(KC * eb == 256, "a chunk row is 256 bytes of K");
  constexpr int KSTEPS = KC / KSTEP;  // k-steps per full chunk (8)
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
  // jobs of this CTA: blockIdx.x + i * gridDim.x, i < nj; descriptors staged in shared memory
  const int nj = blockIdx.x < g.njobs ? (g.njobs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  for (int i = tid; i < nj && i < g.nj_max; i += blockDim.x) sjobs[i] = g.jobs[blockIdx.x + i * gridDim.x];
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
  int b_issued = 0;        // producer: B fills issued (jobs 0 .. b_issued - 1)

  if (warp == 4) {
    if (lane == 0) {
      bool ok = true;
      // B operand of job q into buffer q % NB once its previous user, job q - NB, is done:
      // between A chunks whenever that is already so (non-blocking test), and blocking only
      // when the next job would otherwise lack its operand
      int nb_next = 0;  // next job whose B operand is not issued
      auto issue_b = [&](int q) {
        const int b = q % NB;
        const Job jq = sjobs[q];
        const uint32_t bb = (uint32_t)g.ncols * jq.kpad * eb;
        tc::mbar_expect_tx(bfull0 + 8 * b, bb);
        tc::bulk_g2s(sb0 + b * g.bslot, g.B + jq.b_off, bb, bfull0 + 8 * b);
        ++b_issued;
        ++nb_next;
      };
      auto try_b = [&]() {
        while (nb_next < nj) {
          const int u = nb_next / NB;
          if (u > 0 && !tc::mbar_test(bempty0 + 8 * (nb_next % NB), (u - 1) & 1)) return;
          issue_b(nb_next);
        }
      };
      try_b();
      int s = 0;
      uint32_t round = 0;  // number of completed passes over the ring
      for (int i = 0; i < nj && ok; ++i) {
        if (nb_next <= i) {  // job i's operand must be on its way before its chunks
          const int u = i / NB;
          ok = u == 0 || tc::mbar_wait(bempty0 + 8 * (i % NB), (u - 1) & 1);
          if (!ok) break;
          issue_b(i);
        }
        const Job jb = sjobs[i];
        const unsigned char* A = (jb.tab ? g.tabH : g.tabP) + jb.a_off;
        for (int c = 0; c < jb.nchunk; ++c) {
          if (round > 0) ok = tc::mbar_wait(empty0 + 8 * s, (round - 1) & 1);
          if (!ok) break;
          const uint32_t cb = (c == jb.nchunk - 1) ? 128u * jb.kl * eb : chunk_bytes;
          tc::mbar_expect_tx(full0 + 8 * s, cb);
          tc::bulk_g2s(sa0 + s * chunk_bytes, A + (size_t)c * chunk_bytes, cb, full0 + 8 * s);
          ++a_issued;
          if (++s == S) {
            s = 0;
            ++round;
          }
          try_b();
        }
      }
      if (!ok) atomicExch(g.err, 3);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      bool ok = true;
      const uint32_t idesc = tc::instr_desc(128, g.ncols, BF ? 1 : 2);
      const uint32_t sboA = (uint32_t)(KC / E) * 128u;
      int s = 0;
      uint32_t round = 0;
      for (int i = 0; i < nj && ok; ++i) {
        const Job jb = sjobs[i];
        const int b = i % NB, ub = i / NB, acc = i % njb, ua = i / njb;
        ok = tc::mbar_wait(bfull0 + 8 * b, ub & 1);
        if (ok && ua > 0) ok = tc::mbar_wait(tempty0 + 8 * acc, (ua - 1) & 1);
        if (!ok) break;
        tc::fence_after_sync();
        // k-step q of every chunk accumulates into accumulator q % TC_NACC of job buffer acc,
        // so that consecutive MMAs do not wait on each other's result
        const uint32_t dt = tmem + cs * TC_NACC * acc;
        const uint64_t bdesc0 = tc::smem_desc(sb0 + b * g.bslot, 128u, (uint32_t)(jb.kpad / E) * 128u);
        for (int c = 0; c < jb.nchunk; ++c) {
          ok = tc::mbar_wait(full0 + 8 * s, round & 1);
          if (!ok) break;
          tc::fence_after_sync();
          // the last chunk may be short: its own core-matrix stride and fewer k-steps
          const int kc = (c == jb.nchunk - 1) ? jb.kl : KC;
          const uint64_t ad = tc::smem_desc(sa0 + s * chunk_bytes, 128u, kc == KC ? sboA : (uint32_t)(kc / E) * 128u);
          const uint64_t bd = bdesc0 + (uint64_t)(c * ((KC / E) * 128 / 16));  // + c * 2048 B
          const int nks = kc / KSTEP;
#pragma unroll
          for (int q = 0; q < KSTEPS; ++q) {  // + 256 B per k-step: +16 in the address field
            // k-step q goes to accumulator q % TC_NACC; its first use initialises it
            const uint32_t accum = (c > 0 || q >= TC_NACC) ? 1u : 0u;
            const uint32_t da = dt + cs * (q % TC_NACC);
            if (q < nks) {
              if (BF) tc::mma_f16(da, ad + 16u * q, bd + 16u * q, idesc, accum);
              else tc::mma_tf32(da, ad + 16u * q, bd + 16u * q, idesc, accum);
            }
          }
          tc::mma_commit(empty0 + 8 * s);
          if (++s == S) {
            s = 0;
            ++round;
          }
        }
        if (!ok) break;
        tc::mma_commit(bempty0 + 8 * b);
        tc::mma_commit(tfull0 + 8 * acc);
      }
      if (!ok) atomicExch(g.err, 4);
      tc::mma_commit(fin);  // arrives once every MMA issued above has completed
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 (rows of the job's D tile); all
    // loads of a 16-column group are issued before one wait
    for (int i = 0; i < nj; ++i) {
      const Job jb = sjobs[i];
      const int acc = i % njb, u = i / njb;
      if (!tc::mbar_wait(tfull0 + 8 * acc, u & 1)) {
        if (lane == 0) atomicExch(g.err, 2);
        break;
      }
      tc::fence_after_sync();
      float* Dj = g.D + jb.d_off + (size_t)(32 * warp + lane) * g.ncols;
      for (int c = 0; c < g.ncols; c += 16) {
        uint32_t r[TC_NACC][16];
        const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + cs * TC_NACC * acc + c;
#pragma unroll
        for (int a = 0; a < TC_NACC; ++a) {
          tc::tmem_ld8_nowait(ta + cs * a, r[a]);
          tc::tmem_ld8_nowait(ta + cs * a + 8, r[a] + 8);
        }
        tc::tmem_wait_ld();
        // accumulators a < nacc received k-steps (all four unless the job is one short chunk)
        const int nacc = jb.nchunk > 1 ? TC_NACC : min(TC_NACC, jb.kl / KSTEP);
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          v[q] = __uint_as_float(r[0][q]);
#pragma unroll
          for (int a = 1; a < TC_NACC; ++a)
            if (a < nacc) v[q] += __uint_as_float(r[a][q]);
        }
        float4* d4 = reinterpret_cast<float4*>(Dj + c);
#pragma unroll
        for (int q = 0; q < 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tempty0 + 8 * acc);
    }
  }
  // ---- teardown: no copy may land in, and no MMA may read, a CTA that has exited ----------
  if (warp == 4 && lane == 0) {
    // the newest fill of each stage / B buffer: completed fills return at once
    for (long long q = a_issued - 1; q >= 0 && q >= a_issued - S; --q)
      tc::mbar_wait(full0 + 8 * (int)(q % S), (uint32_t)((q / S) & 1), 200000u);
    for (int q = b_issued - 1; q >= 0 && q >= b_issued - NB; --q)
      tc::mbar_wait(bfull0 + 8 * (q % NB), (q / NB) & 1, 200000u);
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
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
    *reinterpret_cast<uint32_t*>(base + off) = t;
  }
}

// tables: one thread per (job, row), looping over K; src = FP64 table [moff+k][nh]
struct TabJob {
  long long a_off;
  int m, par, tile, nchunk, kl;  // kl: K of the last chunk
};
__global__ void k_tc_table(const double* __restrict__ src, unsigned char* __restrict__ dst,
                           const TabJob* __restrict__ jobs, int njobs, int T, int nh, int synth,
                           int bf16) {
  const int jid = blockIdx.x;
  if (jid >= njobs) return;
  const TabJob j = jobs[jid];
  const int r = threadIdx.x;  // 0..127
  const int E = bf16 ? 8 : 4, eb = bf16 ? 2 : 4, KC = bf16 ? 128 : 64;  // as TcLegendre::KC
  const int K = T + 1 - j.m, base = moff(T, j.m);
  unsigned char* out = dst + j.a_off;
  for (int c = 0; c < j.nchunk; ++c) {
    // every chunk but the last holds KC K-elements per row; the last holds j.kl
    const int kc = (c == j.nchunk - 1) ? j.kl : KC;
    const int sbo = (kc / E) * 128;
    unsigned char* ch = out + (size_t)c * 128 * KC * eb;
    for (int kk = 0; kk < kc; ++kk) {
      float v = 0.f;
      if (synth) {  // rows = latitudes of the northern half, K = all degrees n = m + k
        const int lat = j.tile * 128 + r;
        const int k = c * KC + kk;
        if (lat < nh && k < K) v = (float)src[(size_t)(base + k) * nh + lat];
      } else {      // rows = degrees (both parities), K = latitudes
        const int k = j.tile * 128 + r;
        const int lat = c * KC + kk;
        if (lat < nh && k < K) v = (float)src[(size_t)(base + k) * nh + lat];
      }
      store_elem(ch, canon_off(r, kk, E, eb, sbo), v, bf16);
    }
  }
}

// synthesis B operand of zonal order m: K index k = n - m over all degrees; columns
// [0, nr): coefficient (f, q) of column col = f * cpf + q (north: P_n(mu) of the northern
// latitude); [nr, 2 nr): the same times (-1)^k (south: P_n(-mu) = (-1)^(n-m) P_n(mu)); the rest 0;
// nr = nf * cpf.  q in [0, cpf): scalar (cpf = 2): re, im of spec f; vector (cpf = 4): psi re,
// psi im, chi re, chi im.
__global__ void k_tc_bsynth(const double2* __restrict__ s0, const double2* __restrict__ s1,
                            unsigned char* __restrict__ B, const int* __restrict__ boff,
                            const int* __restrict__ kpad, int T, int nlm, int nf, int cpf, int ncols,
                            int bf16) {
  const int m = blockIdx.x;
  const int kp = kpad[m];
  if (kp == 0) return;
  const int E = bf16 ? 8 : 4, eb = bf16 ? 2 : 4;
  const int sbo = (kp / E) * 128;
  const int K = T + 1 - m, base = moff(T, m), nr = nf * cpf;
  unsigned char* out = B + boff[m];
  for (int idx = threadIdx.x; idx < ncols * kp; idx += blockDim.x) {
    const int col = idx / kp, k = idx - col * kp;
    float v = 0.f;
    if (col < 2 * nr && k < K) {
      const int cc = col < nr ? col : col - nr;
      const int f = cc / cpf, q = cc - f * cpf;
      const double2 c = (q < 2 ? s0 : s1)[(size_t)f * nlm + base + k];
      const double x = (q & 1) ? c.y : c.x;
      v = (float)((col >= nr && (k & 1)) ? -x : x);
    }
    store_elem(out, canon_off(col, k, E, eb, sbo), v, bf16);
  }
}

// analysis B operand of (m, sign): K index = latitude j of the northern half,
//   scalar (cpf = 2):  w_j (F_N +- F_S)           columns (re, im) per field
//   vector (cpf = 4):  wq_j (A_N +- A_S), wq_j (B_N +- B_S)   columns (A re, A im, B re, B im)
__global__ void k_tc_banal(const double2* __restrict__ F0, const double2* __restrict__ F1,
                           const double* __restrict__ wts, unsigned char* __restrict__ B,
                           const int* __restrict__ boff, int kpad, int T, int nlat, int nf, int cpf,
                           int ncols, int bf16) {
  // B of zonal order m: 2 ncols rows (N + S combinations, then N - S), K = latitudes; one
  // thread per northern latitude j reads each Fourier coefficient pair (j and its mirror)
  // once and writes both combinations of every column
  const int m = blockIdx.x;
  const int E = bf16 ? 8 : 4, eb = bf16 ? 2 : 4;
  const int sbo = (kpad / E) * 128;
  const int nh = nlat / 2;
  unsigned char* out = B + boff[m];
  for (int j = threadIdx.x; j < kpad; j += blockDim.x) {
    const double wj = j < nh ? wts[j] : 0.0;
    for (int col = 0; col < ncols; col += 2) {  // columns come in (re, im) pairs
      float pr = 0.f, pi = 0.f, mr = 0.f, mi = 0.f;
      const int f = col / cpf, q = col - f * cpf;
      if (f < nf && j < nh) {
        const double2* Fq = (q < 2 ? F0 : F1) + ((size_t)f * (T + 1) + m) * nlat;
        const double2 a = Fq[j], b = Fq[nlat - 1 - j];
        pr = (float)(wj * (a.x + b.x));
        pi = (float)(wj * (a.y + b.y));
        mr = (float)(wj * (a.x - b.x));
        mi = (float)(wj * (a.y - b.y));
      }
      store_elem(out, canon_off(col, j, E, eb, sbo), pr, bf16);
      store_elem(out, canon_off(col + 1, j, E, eb, sbo), pi, bf16);
      store_elem(out, canon_off(ncols + col, j, E, eb, sbo), mr, bf16);
      store_elem(out, canon_off(ncols + col + 1, j, E, eb, sbo), mi, bf16);
    }
  }
}

__device__ __forceinline__ double2 imul_d(int m, double2 v) { return make_double2(-m * v.y, m * v.x); }

// synthesis epilogue: thread per (m, northern latitude); D rows of job (m, tile, tab) hold the
// northern values in columns [0, nr) and the southern ones in [nr, 2 nr) (H: minus the sum, since
// H_n(-mu) = -(-1)^(n-m) H_n(mu)); row stride ncols
__global__ void k_tc_esynth(const float* __restrict__ D, const int* __restrict__ dmap, double2* __restrict__ F0,
                            double2* __restrict__ F1, int T, int nlat, int nf, int cpf, int ncols, int ntile,
                            int vector, double inv_a) {
  const int m = blockIdx.y;
  const int nh = nlat / 2;
  const int lat = blockIdx.x * blockDim.x + threadIdx.x;
  if (lat >= nh) return;
  const int tile = lat / 128, r = lat % 128, nr = nf * cpf;
  auto val = [&](int tab, int hemi, int col) -> double {
    const int o = dmap[(m * ntile + tile) * 2 + tab];
    return o < 0 ? 0.0 : (double)D[o + (size_t)r * ncols + hemi * nr + col];
  };
  for (int f = 0; f < nf; ++f) {
    const int c0 = f * cpf;
    double2* o0 = F0 + ((size_t)f * (T + 1) + m) * nlat;
    if (!vector) {
      o0[lat] = make_double2(val(0, 0, c0), val(0, 0, c0 + 1));
      o0[nlat - 1 - lat] = make_double2(val(0, 1, c0), val(0, 1, c0 + 1));
    } else {
      double2* o1 = F1 + ((size_t)f * (T + 1) + m) * nlat;
      for (int hemi = 0; hemi < 2; ++hemi) {
        const double sh = hemi ? -1.0 : 1.0;  // H of the southern latitude
        const double2 pps = make_double2(val(0, hemi, c0), val(0, hemi, c0 + 1));
        const double2 pch = make_double2(val(0, hemi, c0 + 2), val(0, hemi, c0 + 3));
        const double2 hps = make_double2(sh * val(1, hemi, c0), sh * val(1, hemi, c0 + 1));
        const double2 hch = make_double2(sh * val(1, hemi, c0 + 2), sh * val(1, hemi, c0 + 3));
        const double2 ich = imul_d(m, pch), ips = imul_d(m, pps);
        const int jj = hemi ? nlat - 1 - lat : lat;
        o0[jj] = make_double2(inv_a * (-hps.x + ich.x), inv_a * (-hps.y + ich.y));
        o1[jj] = make_double2(inv_a * (ips.x + hch.x), inv_a * (ips.y + hch.y));
      }
    }
  }
}

// analysis epilogue: thread per (m, k)
__global__ void k_tc_eanal(const float* __restrict__ D, const int* __restrict__ dmap, double2* __restrict__ s0,
                           double2* __restrict__ s1, int T, int nlm, int nf, int cpf, int ncols, int ntile,
                           int vector, double inv_a) {
  const int m = blockIdx.y;
  const int K = T + 1 - m;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  // D rows: degree k of tile k / 128; columns: the N + S block, then the N - S block (ncols
  // each).  P pairs with N + S for even k - m and N - S for odd; H the other way round.
  const int par = k & 1, tile = k / 128, r = k % 128;
  auto val = [&](int tab, int col) -> float {
    const int o = dmap[(m * ntile + tile) * 2 + tab];
    const int coloff = ((tab == 0) != (par == 1)) ? 0 : ncols;
    return o < 0 ? 0.f : D[o + (size_t)r * (2 * ncols) + coloff + col];
  };
  const size_t i = moff(T, m) + k;
  for (int f = 0; f < nf; ++f) {
    const int c0 = f * cpf;
    if (!vector) {
      s0[(size_t)f * nlm + i] = make_double2(val(0, c0), val(0, c0 + 1));
    } else {
      const double2 PA = make_double2(val(0, c0), val(0, c0 + 1)), PB = make_double2(val(0, c0 + 2), val(0, c0 + 3));
      const double2 HA = make_double2(val(1, c0), val(1, c0 + 1)), HB = make_double2(val(1, c0 + 2), val(1, c0 + 3));
      const double2 iPA = imul_d(m, PA), iPB = imul_d(m, PB);
      s0[(size_t)f * nlm + i] = make_double2(inv_a * (iPA.x - HB.x), inv_a * (iPA.y - HB.y));
      s1[(size_t)f * nlm + i] = make_double2(inv_a * (iPB.x + HA.x), inv_a * (iPB.y + HA.y));
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
struct TcLegendre {
  int T = 0, nlat = 0, nh = 0, nlm = 0, max_fields = 0, bf16 = 0, E = 4, eb = 4, KC = 32;
  int ntile_s = 0, ntile_a = 0, kpad_a = 0;
  unsigned char *tabPs = nullptr, *tabHs = nullptr, *tabPa = nullptr, *tabHa = nullptr;
  unsigned char* B = nullptr;
  float* D = nullptr;
  int* err = nullptr;
  const double *w = nullptr, *wq = nullptr;
  // synthesis jobs (scalar uses the P half), analysis jobs; job lists and D maps per variant
  Job *jobs_s = nullptr, *jobs_a = nullptr;
  int njobs_s = 0, njobs_a = 0, njobs_sP = 0, njobs_aP = 0;
  int *dmap_s = nullptr, *dmap_a = nullptr;   // [m*ntile+tile][tab] -> D offset or -1 (synthesis, analysis)
  int *boff_s = nullptr, *kpad_s = nullptr, *boff_a = nullptr;
  int kpad_smax = 0;  // largest K extent of a synthesis B operand
  int nsm = 0;
  StageProf* prof = nullptr;
};

static int tc_fail(const char* what, cudaError_t e) { return cuda_fail(e, what); }

int tc_legendre_create(TcLegendre** out, const double* P, const double* H, const double* w, const double* wq,
                       int T, int nlat, int max_fields, bool bf16, cudaStream_t stream) {
  *out = nullptr;
  if (max_fields > 8) return fail(REXI_EINVAL, "sh_plan_create: tensor-core precisions support max_fields <= 8");
  TcLegendre* t = new TcLegendre();
  t->T = T;
  t->nlat = nlat;
  t->nh = nlat / 2;
  t->nlm = (T + 1) * (T + 2) / 2;
  t->max_fields = max_fields;
  t->bf16 = bf16 ? 1 : 0;
  t->E = bf16 ? 8 : 4;
  t->eb = bf16 ? 2 : 4;
  t->KC = bf16 ? 128 : 64;   // 256 bytes of K per chunk row
  t->w = w;
  t->wq = wq;
  const int KC = t->KC, eb = t->eb;
  const size_t chunk = 128ull * KC * eb;
  t->ntile_s = (t->nh + 127) / 128;
  // ---- synthesis jobs: (m, tile, tab); rows = northern latitudes of the tile, K = all degrees
  // of m; B = [c | (-1)^(n-m) c] gives the northern and the southern values in one job -------
  std::vector<TabJob> tj;
  std::vector<Job> js;
  std::vector<int> dmap_s((T + 1) * t->ntile_s * 2, -1), boff_s(T + 1), kpad_s(T + 1);
  long long aoff = 0;
  int boff = 0, doff = 0;
  const int ncols_max = TC_MAXCOL;
  std::vector<Job> jsP, jsH;
  const int kstep = bf16 ? 16 : 8;  // MMA K per instruction
  for (int m = 0; m <= T; ++m) {
    const int K = T + 1 - m;
    const int kpad = (K + kstep - 1) / kstep * kstep;  // K padded to whole k-steps only
    const int nchunk = (kpad + KC - 1) / KC;
    const int kl = kpad - (nchunk - 1) * KC;
    boff_s[m] = boff;
    kpad_s[m] = kpad;
    boff += 2 * ncols_max * kpad * eb;
    for (int tile = 0; tile < t->ntile_s; ++tile) {
      tj.push_back(TabJob{aoff, m, 0, tile, nchunk, kl});
      for (int tab = 0; tab < 2; ++tab) {
        Job j{aoff, boff_s[m], doff, nchunk, kpad, tab, kl};
        (tab ? jsH : jsP).push_back(j);
        dmap_s[(m * t->ntile_s + tile) * 2 + tab] = doff;
        doff += 128 * 2 * ncols_max;
      }
      aoff += (long long)(nchunk - 1) * chunk + 128LL * kl * eb;
    }
  }
  const long long tab_s_bytes = aoff;
  const int bsz_s = boff;
  const int dsz_s = doff;
  auto bylen = [](const Job& a, const Job& b) { return a.nchunk > b.nchunk; };
  std::stable_sort(jsP.begin(), jsP.end(), bylen);
  std::stable_sort(jsH.begin(), jsH.end(), bylen);
  t->njobs_sP = (int)jsP.size();
  js = jsP;
  js.insert(js.end(), jsH.begin(), jsH.end());
  t->njobs_s = (int)js.size();
  // ---- analysis jobs: (m, degree tile, tab), rows = degrees of both parities, K = northern
  // latitudes; B = [N + S | N - S] of zonal order m (2 ncols columns) ----------------------
  t->kpad_a = (t->nh + kstep - 1) / kstep * kstep;
  const int nchunk_a = (t->kpad_a + KC - 1) / KC;
  const int kl_a = t->kpad_a - (nchunk_a - 1) * KC;
  const int ntile_a = (T + 1 + 127) / 128;
  t->ntile_a = ntile_a;
  std::vector<TabJob> ta;
  std::vector<Job> jaP, jaH;
  std::vector<int> dmap_a((T + 1) * ntile_a * 2, -1), boff_a(T + 1);
  aoff = 0;
  boff = 0;
  doff = 0;
  for (int m = 0; m <= T; ++m) {
    boff_a[m] = boff;
    boff += 2 * ncols_max * t->kpad_a * eb;
  }
  for (int m = 0; m <= T; ++m) {
    const int K = T + 1 - m;
    const int ntiles = (K + 127) / 128;
    for (int tile = 0; tile < ntiles; ++tile) {
      ta.push_back(TabJob{aoff, m, 0, tile, nchunk_a, kl_a});
      for (int tab = 0; tab < 2; ++tab) {
        Job j{aoff, boff_a[m], doff, nchunk_a, t->kpad_a, tab, kl_a};
        (tab ? jaH : jaP).push_back(j);
        dmap_a[(m * ntile_a + tile) * 2 + tab] = doff;
        doff += 128 * 2 * ncols_max;
      }
      aoff += (long long)(nchunk_a - 1) * chunk + 128LL * kl_a * eb;
    }
  }
  const long long tab_a_bytes = aoff;
  const int bsz_a = boff;
  const int dsz = std::max(dsz_s, doff);
  t->njobs_aP = (int)jaP.size();
  std::vector<Job> ja = jaP;
  ja.insert(ja.end(), jaH.begin(), jaH.end());
  t->njobs_a = (int)ja.size();
  // the largest B operand of any call (analysis of a vector pair: 2 x 4 max_fields columns
  // over all latitudes) must fit one B buffer and two ring stages in shared memory
  {
    auto ncols_of = [](int nf, int cpf) { return std::max(16, (nf * cpf + 15) / 16 * 16); };
    int kpad_smax = 0;
    for (int v : kpad_s) kpad_smax = std::max(kpad_smax, v);
    const size_t bmax = std::max((size_t)ncols_of(max_fields, 4) * t->kpad_a * 2 * eb,
                                 (size_t)ncols_of(2 * max_fields, 4) * kpad_smax * eb);
    if (bmax + 2 * chunk + 4096 > TC_SMEM_BUDGET) {
      tc_legendre_destroy(t);
      return fail(REXI_EINVAL,
                  "sh_plan_create: %d latitudes x %d fields exceed the tensor-core shared-memory budget; "
                  "use fewer fields per call", nlat, max_fields);
    }
  }
  // ---- device buffers ---------------------------------------------------------------------
  TabJob *d_tj = nullptr, *d_ta = nullptr;
  cudaError_t e;
  if ((e = cudaMalloc(&t->tabPs, tab_s_bytes)) || (e = cudaMalloc(&t->tabHs, tab_s_bytes)) ||
      (e = cudaMalloc(&t->tabPa, tab_a_bytes)) || (e = cudaMalloc(&t->tabHa, tab_a_bytes)) ||
      (e = cudaMalloc(&t->B, std::max(bsz_s, bsz_a))) || (e = cudaMalloc(&t->D, sizeof(float) * (size_t)dsz)) ||
      (e = cudaMalloc(&t->err, sizeof(int))) || (e = cudaMalloc(&t->jobs_s, sizeof(Job) * js.size())) ||
      (e = cudaMalloc(&t->jobs_a, sizeof(Job) * ja.size())) ||
      (e = cudaMalloc(&t->dmap_s, sizeof(int) * dmap_s.size())) ||
      (e = cudaMalloc(&t->dmap_a, sizeof(int) * dmap_a.size())) ||
      (e = cudaMalloc(&t->boff_s, sizeof(int) * boff_s.size())) ||
      (e = cudaMalloc(&t->kpad_s, sizeof(int) * kpad_s.size())) ||
      (e = cudaMalloc(&t->boff_a, sizeof(int) * boff_a.size())) ||
      (e = cudaMalloc(&d_tj, sizeof(TabJob) * tj.size())) || (e = cudaMalloc(&d_ta, sizeof(TabJob) * ta.size()))) {
    cudaGetLastError();
    tc_legendre_destroy(t);
    cudaFree(d_tj);
    cudaFree(d_ta);
    return fail(REXI_ENOMEM, "tensor-core Legendre tables: cudaMalloc failed: %s", cudaGetErrorString(e));
  }
  cudaMemset(t->err, 0, sizeof(int));
  cudaMemcpy(t->jobs_s, js.data(), sizeof(Job) * js.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(t->jobs_a, ja.data(), sizeof(Job) * ja.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(t->dmap_s, dmap_s.data(), sizeof(int) * dmap_s.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(t->dmap_a, dmap_a.data(), sizeof(int) * dmap_a.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(t->boff_s, boff_s.data(), sizeof(int) * boff_s.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(t->kpad_s, kpad_s.data(), sizeof(int) * kpad_s.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(t->boff_a, boff_a.data(), sizeof(int) * boff_a.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(d_tj, tj.data(), sizeof(TabJob) * tj.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(d_ta, ta.data(), sizeof(TabJob) * ta.size(), cudaMemcpyHostToDevice);
  k_tc_table<<<(int)tj.size(), 128, 0, stream>>>(P, t->tabPs, d_tj, (int)tj.size(), T, t->nh, 1, t->bf16);
  k_tc_table<<<(int)tj.size(), 128, 0, stream>>>(H, t->tabHs, d_tj, (int)tj.size(), T, t->nh, 1, t->bf16);
  k_tc_table<<<(int)ta.size(), 128, 0, stream>>>(P, t->tabPa, d_ta, (int)ta.size(), T, t->nh, 0, t->bf16);
  k_tc_table<<<(int)ta.size(), 128, 0, stream>>>(H, t->tabHa, d_ta, (int)ta.size(), T, t->nh, 0, t->bf16);
  e = cudaStreamSynchronize(stream);
  cudaFree(d_tj);
  cudaFree(d_ta);
  if (e != cudaSuccess) {
    tc_legendre_destroy(t);
    return tc_fail("tensor-core Legendre table kernels", e);
  }
  for (int v : kpad_s) t->kpad_smax = std::max(t->kpad_smax, v);
  int dev = 0;
  cudaGetDevice(&dev);
  if ((e = cudaDeviceGetAttribute(&t->nsm, cudaDevAttrMultiProcessorCount, dev))) {
    tc_legendre_destroy(t);
    return tc_fail("cudaDeviceGetAttribute(SM count)", e);
  }
  if ((e = cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_BUDGET)) ||
      (e = cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_BUDGET))) {
    tc_legendre_destroy(t);
    return tc_fail("cudaFuncSetAttribute(k_tc_gemm)", e);
  }
  *out = t;
  return REXI_OK;
}

void tc_legendre_destroy(TcLegendre* t) {
  if (!t) return;
  for (void* p : {(void*)t->tabPs, (void*)t->tabHs, (void*)t->tabPa, (void*)t->tabHa, (void*)t->B, (void*)t->D,
                  (void*)t->err, (void*)t->jobs_s, (void*)t->jobs_a, (void*)t->dmap_s, (void*)t->dmap_a,
                  (void*)t->boff_s, (void*)t->kpad_s, (void*)t->boff_a})
    cudaFree(p);
  delete t;
}

static int gemm(TcLegendre* t, bool synth, bool both_tabs, int ncols, cudaStream_t s) {
  GemmArgs g;
  g.tabP = synth ? t->tabPs : t->tabPa;
  g.tabH = synth ? t->tabHs : t->tabHa;
  g.B = t->B;
  g.D = t->D;
  g.jobs = synth ? t->jobs_s : t->jobs_a;
  g.njobs = both_tabs ? (synth ? t->njobs_s : t->njobs_a) : (synth ? t->njobs_sP : t->njobs_aP);
  g.ncols = ncols;
  g.bf16 = t->bf16;
  g.err = t->err;
  // two B buffers of the largest B operand of the call, then as many A stages as fit
  const size_t chunk = 128ull * t->KC * t->eb;
  const size_t bslot = ((size_t)ncols * (synth ? t->kpad_smax : t->kpad_a) * t->eb + 127) / 128 * 128;
  const int grid = std::max(1, std::min(g.njobs, t->nsm));
  g.nj_max = (g.njobs + grid - 1) / grid;
  const size_t jobs_bytes = sizeof(Job) * (size_t)g.nj_max;
  auto fixed = [&](int nb) { return nb * bslot + 8 * (2 * TC_MAXSTAGES + 2 * nb + 2 * TC_NJB + 2) + jobs_bytes; };
  // B buffers: 4 when that leaves >= 4 ring stages, else 2, else 1 (>= 2 ring stages always)
  g.nb = (fixed(TC_MAXNB) + 4 * chunk <= TC_SMEM_BUDGET) ? TC_MAXNB : (fixed(2) + 2 * chunk <= TC_SMEM_BUDGET) ? 2 : 1;
  if (fixed(g.nb) + 2 * chunk > TC_SMEM_BUDGET) return fail(REXI_EINVAL, "tensor-core Legendre: B operand too large");
  g.stages = (int)std::min<size_t>(TC_MAXSTAGES, (TC_SMEM_BUDGET - fixed(g.nb)) / chunk);
  g.bslot = (uint32_t)bslot;
  const size_t smem =
      (size_t)g.stages * chunk + g.nb * bslot + 8 * (2 * g.stages + 2 * g.nb + 2 * TC_NJB + 2) + jobs_bytes;
  {
    const int ph = t->prof ? t->prof->begin(2) : -1;
    if (t->bf16) k_tc_gemm<true><<<grid, TC_THREADS, smem, s>>>(g);
    else k_tc_gemm<false><<<grid, TC_THREADS, smem, s>>>(g);
    if (t->prof) t->prof->end(ph);
  }
  cudaError_t e = cudaGetLastError();
  return e ? cuda_fail(e, "k_tc_gemm launch") : REXI_OK;
}

static int ncols_for(int nf, int cpf) {
  const int c = nf * cpf;
  return std::max(16, (c + 15) / 16 * 16);
}

int tc_leg_synth(TcLegendre* t, const double2* spec, double2* F, int nf, cudaStream_t s) {
  const int nc = ncols_for(2 * nf, 2);  // northern and southern columns
  {
    const int ph = t->prof ? t->prof->begin(1) : -1;
    k_tc_bsynth<<<t->T + 1, 256, 0, s>>>(spec, spec, t->B, t->boff_s, t->kpad_s, t->T, t->nlm, nf, 2, nc, t->bf16);
    if (t->prof) t->prof->end(ph);
  }
  int rc = gemm(t, true, false, nc, s);
  if (rc) return rc;
  {
    const int ph = t->prof ? t->prof->begin(3) : -1;
    k_tc_esynth<<<dim3((t->nh + 127) / 128, t->T + 1), 128, 0, s>>>(t->D, t->dmap_s, F, F, t->T, t->nlat, nf, 2, nc,
                                                                     t->ntile_s, 0, 0.0);
    if (t->prof) t->prof->end(ph);
  }
  return REXI_OK;
}

int tc_leg_synth_uv(TcLegendre* t, const double2* psi, const double2* chi, double2* FU, double2* FV, int nf,
                    double inv_a, cudaStream_t s) {
  const int nc = ncols_for(2 * nf, 4);  // northern and southern columns
  {
    const int ph = t->prof ? t->prof->begin(1) : -1;
    k_tc_bsynth<<<t->T + 1, 256, 0, s>>>(psi, chi, t->B, t->boff_s, t->kpad_s, t->T, t->nlm, nf, 4, nc, t->bf16);
    if (t->prof) t->prof->end(ph);
  }
  int rc = gemm(t, true, true, nc, s);
  if (rc) return rc;
  {
    const int ph = t->prof ? t->prof->begin(3) : -1;
    k_tc_esynth<<<dim3((t->nh + 127) / 128, t->T + 1), 128, 0, s>>>(t->D, t->dmap_s, FU, FV, t->T, t->nlat, nf, 4, nc,
                                                                     t->ntile_s, 1, inv_a);
    if (t->prof) t->prof->end(ph);
  }
  return REXI_OK;
}

int tc_leg_anal(TcLegendre* t, const double2* F, double2* spec, int nf, cudaStream_t s) {
  const int nc = ncols_for(nf, 2);
  {
    const int ph = t->prof ? t->prof->begin(1) : -1;
    k_tc_banal<<<t->T + 1, 128, 0, s>>>(F, F, t->w, t->B, t->boff_a, t->kpad_a, t->T, t->nlat, nf, 2, nc,
                                                 t->bf16);
    if (t->prof) t->prof->end(ph);
  }
  int rc = gemm(t, false, false, 2 * nc, s);  // columns: N + S block, N - S block
  if (rc) return rc;
  {
    const int ph = t->prof ? t->prof->begin(3) : -1;
    k_tc_eanal<<<dim3((t->T + 1 + 127) / 128, t->T + 1), 128, 0, s>>>(t->D, t->dmap_a, spec, spec, t->T, t->nlm, nf,
                                                                       2, nc, t->ntile_a, 0, 0.0);
    if (t->prof) t->prof->end(ph);
  }
  return REXI_OK;
}

int tc_leg_anal_divcurl(TcLegendre* t, const double2* FA, const double2* FB, double2* dv, double2* cu, int nf,
                        double inv_a, cudaStream_t s) {
  const int nc = ncols_for(nf, 4);
  {
    const int ph = t->prof ? t->prof->begin(1) : -1;
    k_tc_banal<<<t->T + 1, 128, 0, s>>>(FA, FB, t->wq, t->B, t->boff_a, t->kpad_a, t->T, t->nlat, nf, 4, nc,
                                                 t->bf16);
    if (t->prof) t->prof->end(ph);
  }
  int rc = gemm(t, false, true, 2 * nc, s);  // columns: N + S block, N - S block
  if (rc) return rc;
  {
    const int ph = t->prof ? t->prof->begin(3) : -1;
    k_tc_eanal<<<dim3((t->T + 1 + 127) / 128, t->T + 1), 128, 0, s>>>(t->D, t->dmap_a, dv, cu, t->T, t->nlm, nf, 4,
                                                                       nc, t->ntile_a, 1, inv_a);
    if (t->prof) t->prof->end(ph);
  }
  return REXI_OK;
}

void tc_legendre_set_prof(TcLegendre* t, StageProf* prof) {
  if (t) t->prof = prof;
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
