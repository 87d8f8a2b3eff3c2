// Tensor-core (tcgen05) Legendre contractions for sh_plan precisions SH_TF32, SH_BF16 and
// SH_TF32X3.
#pragma once
#include <vector>

#include "common.cuh"

namespace rexi {

// Per-stage CUDA-event timing of the SH transforms (off unless enabled): a pair of events on
// the plan stream around every kernel launch, accumulated when collected.
struct StageProf {
  static constexpr int NSTAGE = 5;  // FP64 Legendre, double-float Legendre, tcgen05 GEMM, TC epilogue, FFT
  bool on = false;
  cudaStream_t stream = nullptr;
  struct Pend {
    cudaEvent_t a, b;
    int k;
  };
  std::vector<Pend> pending;
  std::vector<cudaEvent_t> pool;
  double ms[NSTAGE] = {};
  int n[NSTAGE] = {};
  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  int begin(int k) {
    if (!on) return -1;
    Pend q{take(), take(), k};
    cudaEventRecord(q.a, stream);
    pending.push_back(q);
    return (int)pending.size() - 1;
  }
  void end(int h) {
    if (h >= 0) cudaEventRecord(pending[h].b, stream);
  }
  // synchronises the stream, adds the pending intervals
  cudaError_t collect() {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e) return e;
    for (auto& q : pending) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, q.a, q.b);
      if (e) return e;
      ms[q.k] += t;
      n[q.k] += 1;
      pool.push_back(q.a);
      pool.push_back(q.b);
    }
    pending.clear();
    return cudaSuccess;
  }
  void release() {
    cudaStreamSynchronize(stream);
    for (auto& q : pending) {
      pool.push_back(q.a);
      pool.push_back(q.b);
    }
    pending.clear();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

// Polar truncation of the Legendre contractions (the "polar optimisation" of SHTns, the
// transform library the paper uses): Pt_n^m and Ht_n^m carry the factor (1 - mu^2)^{m/2} and
// are negligible where sin(theta) is small against m / n, so near the poles the leading
// terms of every sum can be skipped.  Per zonal order m, from the FP64 tables:
//   ks[m * ngl + g]: first degree index k = n - m at which P or H exceeds the threshold in
//     magnitude at one of the northern latitudes 32 g .. 32 g + 31 (T + 1 - m if nowhere):
//     the synthesis of those latitudes starts there;
//   ja[m * ngd + g]: first northern latitude at which P or H of one of the degree indices
//     k = 32 g .. 32 g + 31 exceeds it (nh if nowhere): their analysis starts there.  The
//     groups reach degree index K = T + 1 - m (n = T + 1, judged by P alone), whose P-sums the
//     vector analysis uses (ngd = ceil((T + 2) / 32)).
// Every skipped entry is below the threshold.  With the truncation off, every start is 0.
struct PolarBounds {
  int ngl = 0, ngd = 0;        // groups of 32 latitudes, of 32 degrees
  const int* d_ks = nullptr;   // device [T+1][ngl]
  const int* d_ja = nullptr;   // device [T+1][ngd]
  const int* ks = nullptr;     // host copies
  const int* ja = nullptr;
};

// Divergence and curl of nfv vector fields [nfv][nlm] from the raw P-sums of their analysis,
// raw[(2 v + {0: A, 1: B}) nlme + moff(T+1, m) + k] for n = m + k = m .. T + 1,
// nlme = (T+1)(T+4)/2 (sht.cu, k_divcurl_from_p)
void launch_divcurl_from_p(const double2* raw, double2* dv, double2* cu, int nfv, int T, double inv_a, cudaStream_t s);
inline int nlm_ext(int T) { return (T + 1) * (T + 4) / 2; }

struct TcLegendre;
// stage timer of the owning plan (may be null)
void tc_legendre_set_prof(TcLegendre* t, StageProf* prof);
// test of the timeout path: the epilogue gives up after `polls` non-blocking polls (0: normal)
void tc_legendre_set_epilogue_polls(TcLegendre* t, int polls);

// mode: SH_TF32, SH_BF16 or SH_TF32X3
// pb: the plan's polar bounds (host copies read here; the tables skip what they exclude)
int tc_legendre_create(TcLegendre** out, const double* P, const double* H, const double* w,
                       const double* wq, int T, int nlat, int max_fields, int mode,
                       const PolarBounds& pb, cudaStream_t stream);
// table entries (k < T + 1 - m, j < nh) inside the chunks the GEMM streams, per table:
// synthesis, analysis
void tc_legendre_streamed(const TcLegendre* t, long long* syn, long long* ana);
void tc_legendre_destroy(TcLegendre* t);
int tc_leg_synth(TcLegendre* t, const double2* spec, double2* F, int nf, cudaStream_t s);
int tc_leg_anal(TcLegendre* t, const double2* F, double2* spec, int nf, cudaStream_t s);
int tc_leg_synth_uv(TcLegendre* t, const double2* psi, const double2* chi, double2* FU, double2* FV,
                    int nf, double inv_a, cudaStream_t s);
// nfv vector pairs and nfs scalar fields in one launch that reads each table once
int tc_leg_synth_mixed(TcLegendre* t, const double2* psi, const double2* chi, double2* FU, double2* FV, int nfv,
                       const double2* spec, double2* F, int nfs, double inv_a, cudaStream_t s);
int tc_leg_anal_mixed(TcLegendre* t, const double2* FA, const double2* FB, double2* dv, double2* cu, int nfv,
                      const double2* F, double2* spec, int nfs, double inv_a, cudaStream_t s);
// reads the device flag set by a tensor-core kernel whose bounded wait gave up (0 = none)
int tc_legendre_error(TcLegendre* t, int* flag);
int tc_leg_anal_divcurl(TcLegendre* t, const double2* FA, const double2* FB, double2* dv,
                        double2* cu, int nf, double inv_a, cudaStream_t s);

}  // namespace rexi
