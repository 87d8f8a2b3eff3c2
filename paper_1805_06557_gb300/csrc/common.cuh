// Shared device/host helpers of librexi: complex arithmetic, the FP64 reciprocal, error
// reporting.  Nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rexi.h"

namespace rexi {

// ---- error reporting (thread-local message, returned by rexi_last_error) ------------
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// Raises the dynamic shared-memory limit of kernel fn to at least `bytes`.  The limit is per
// kernel and process-wide, so it only grows: a plan created later with a smaller need must not
// lower it below what a live plan launches with.  Serialised across threads.
cudaError_t raise_smem_limit(const void* fn, size_t bytes);
template <typename F> cudaError_t raise_smem_limit(F* fn, size_t bytes) {
  return raise_smem_limit(reinterpret_cast<const void*>(fn), bytes);
}

#define REXI_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return ::rexi::cuda_fail(_e, #expr); \
  } while (0)

// ---- complex helpers ---------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + a * b
__host__ __device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  return make_double2(fma(-a.y, b.y, fma(a.x, b.x, acc.x)), fma(a.y, b.x, fma(a.x, b.y, acc.y)));
}
__host__ __device__ __forceinline__ float2 caddf(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ float2 cfmaf(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(-a.y, b.y, fmaf(a.x, b.x, acc.x)), fmaf(a.y, b.x, fmaf(a.x, b.y, acc.y)));
}

#ifdef __CUDACC__
// Reciprocal approximation of the SFU (about 1 ulp in FP32).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// FP64 reciprocal by Newton-Raphson from the FP32 seed, using the cubic form of the
// iteration  r <- r + r (e + e^2),  e = 1 - n r, which takes a 2^-23 seed past 2^-53 in one
// step.  Valid for 1e-30 < n < 1e30 (the seed must be a normal float).
__device__ __forceinline__ double rcp64(double n) {
  double r = (double)rcp_approx(__double2float_rn(n));
  double e = fma(-n, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// 1 / (a + i b) = (a - i b) / (a^2 + b^2)
__device__ __forceinline__ double2 crcp64(double2 d) {
  double s = rcp64(fma(d.x, d.x, d.y * d.y));
  return make_double2(d.x * s, -d.y * s);
}
__device__ __forceinline__ float2 crcpf(float2 d) {
  float s = rcp_approx(fmaf(d.x, d.x, d.y * d.y));
  return make_float2(d.x * s, -d.y * s);
}
#endif

// ---- plan-side data shared by host and device ----------------------------------------
// Per-pole constants in FP64 (z, w, w/z, 1/z, dt Phibar / z).
struct PoleD {
  double2 z, w, wz, iz, gz;
};
struct PoleF {
  float2 z, w, wz, iz, gz;
};

// One unit of work: instance, zonal order m, parity chain (2 = both chains, light tiles), a range of 32-pole groups of the
// instance's pole set, and the slot of the partial sums it owns.  Sorted by decreasing cost.  Heavy tiles may carry a
// pair of instances of the same truncation and pole set (inst, inst2) on 32-pole groups, or two such pairs, (inst,
// inst2) on lanes 0-15 and (inst3, inst4) on lanes 16-31, on 16-pole groups (g0 is then a pole offset and ng counts
// 16-pole groups).  Unused instance fields are -1.
struct Tile {
  int m, chain, g0, ng, q, heavy, cost, inst, inst2, inst3, inst4;
};

// One state of a launch.  Offsets are relative to the launch's base pointers.
struct Inst {
  long long soff;  // complex offset of the state [3][nlm] in U0 / U1
  long long poff;  // complex offset of its partial sums [Q][3][nlm]
  long long roff;  // element offset of its right-hand-side pieces [nlm]
  int T, nlm, Q, pole0;  // truncation, coefficients per field, pole ranges, first pole
  double2 S0;      // sum_n w_n / z_n of its pole set
  int mrank = 0, msize = 0;  // zonal-order partition: with msize > 1 the state owns the orders m
                             // with m_pair(T, m) % msize == mrank; the others are written as 0
  long long poff64 = 0;      // mixed plans: complex offset of the FP64 partial sums [Q64][3][nlm]
  int Q64 = 0;               // of the poles solved in FP64 (0: none)
};

// pair index of zonal order m when the orders are dealt in pairs (m, T - m), which have equal
// total chain length T + 2
__host__ __device__ __forceinline__ int m_pair(int T, int m) { return m < T - m ? m : T - m; }

// index of the instance owning global element e: largest i with ecum[i] <= e
__host__ __device__ __forceinline__ int inst_of(const long long* ecum, int ninst, long long e) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (ecum[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
// zonal order of coefficient idx for truncation T (m-major layout)
__host__ __device__ __forceinline__ int m_of(int T, int idx) {
  int lo = 0, hi = T;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (mid * (2 * T + 3 - mid) / 2 <= idx) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__host__ __device__ __forceinline__ int moff(int T, int m) { return m * (2 * T + 3 - m) / 2; }

// 32-byte aligned quadruple of doubles (one 256-bit access)
struct __align__(32) D4 {
  double x, y, z, w;
};

}  // namespace rexi
