// ALU throughput probes (FP64 and FP32 FMA) used as the roofline denominators of the
// ALU-bound solve kernels.  Each thread runs 8 independent FMA chains; the grid covers
// every SM several times; the result is timed with CUDA events.
#include "common.cuh"

namespace {

template <class F>
__global__ void k_fma_probe(F* out, int iters, F a, F b) {
  F x0 = threadIdx.x * F(1e-3), x1 = x0 + F(1), x2 = x0 + F(2), x3 = x0 + F(3);
  F x4 = x0 + F(4), x5 = x0 + F(5), x6 = x0 + F(6), x7 = x0 + F(7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  F s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == F(-12345.678)) out[blockIdx.x] = s;  // keeps the chains alive
}

template <class F>
int probe(double* tflops, int nsm) {
  F* out = nullptr;
  cudaError_t ae = cudaMalloc(&out, sizeof(F) * 65536);
  if (ae != cudaSuccess) return rexi::cuda_fail(ae, "cudaMalloc(probe)");
  const int blocks = nsm * 16, threads = 256;
  const int iters = sizeof(F) == 8 ? 64 : 2048;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_probe<F><<<blocks, threads>>>(out, iters / 8, F(0.999999), F(1e-7));  // warm-up
  cudaEventRecord(e0);
  k_fma_probe<F><<<blocks, threads>>>(out, iters, F(0.999999), F(1e-7));
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return rexi::cuda_fail(err, "alu probe");
  const double fmas = (double)blocks * threads * iters * 16 * 8;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return REXI_OK;
}

}  // namespace

extern "C" int rexi_alu_peaks(double* fp64_tflops, double* fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) return rexi::fail(REXI_EINVAL, "rexi_alu_peaks: null output");
  int dev = 0, nsm = 0;
  REXI_CUDA_TRY(cudaGetDevice(&dev));
  REXI_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int rc = probe<double>(fp64_tflops, nsm);
  if (rc) return rc;
  return probe<float>(fp32_tflops, nsm);
}
