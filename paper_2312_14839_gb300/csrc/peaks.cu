// FMA-throughput microbenchmark: the measured FP32 and FP64 arithmetic peaks that the element
// kernel (FP32 FMA-bound) and the FP64 energy/gradient kernel (FP64-pipe-bound) are reported
// against. Eight independent FMA chains per thread, enough CTAs to fill every SM; the result is
// written only under a condition that never holds, so the chains cannot be removed.
#include <string>

#include "common.cuh"

namespace bhem {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T a, T b, T* out) {
  T x0 = (T)threadIdx.x * (T)1e-6, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == (T)-1.2345) out[blockIdx.x] = s;
}

}  // namespace bhem

using namespace bhem;

extern "C" shell_status shell_measure_fma_peak(int fp64, int iters, void* stream, double* flops_per_s) {
  if (!flops_per_s || iters < 1) return fail(SHELL_ERR_ARG, "invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  BHEM_CUDA(cudaGetDevice(&dev));
  BHEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  void* out = nullptr;
  BHEM_CUDA(cudaMalloc(&out, sizeof(double) * blocks));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  shell_status rc = SHELL_OK;
  float ms = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = fail(SHELL_ERR_CUDA, "cudaEventCreate failed");
  } else {
    for (int rep = 0; rep < 2 && rc == SHELL_OK; ++rep) {   // the first launch warms up
      cudaEventRecord(e0, st);
      if (fp64)
        k_fma_peak<double><<<blocks, threads, 0, st>>>(iters, 0.9999999, 1e-7, (double*)out);
      else
        k_fma_peak<float><<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-4f, (float*)out);
      cudaEventRecord(e1, st);
      const cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess || cudaGetLastError() != cudaSuccess)
        rc = fail(SHELL_ERR_CUDA, std::string("FMA peak kernel: ") + cudaGetErrorString(e));
    }
    if (rc == SHELL_OK) cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != SHELL_OK) return rc;
  const double flops = 2.0 * 8.0 * (double)iters * (double)blocks * (double)threads;
  *flops_per_s = ms > 0.f ? flops / (ms * 1e-3) : 0.0;
  return SHELL_OK;
}
