// Throughput microbenchmarks: the measured FP32 and FP64 arithmetic peaks that the element
// kernel (FP32 FMA-bound) and the FP64 energy/gradient kernel (FP64-pipe-bound) are reported
// against, and the warp-level tensor-core (mma.sync) rates a tensor-core element contraction
// would run at. Eight independent FMA chains per thread, enough CTAs to fill every SM; the result is
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

// Warp-level tensor-core (mma.sync) throughput: four independent accumulator tiles per warp, one
// MMA each per loop iteration, register operands (no memory traffic). kind 0: TF32 m16n8k8 (the
// form a TF32 split of the element contraction would use), kind 1: BF16 m16n8k16.
__global__ void __launch_bounds__(256) k_mma_peak(int kind, int iters, float* out) {
  const unsigned t = threadIdx.x;
  const unsigned a0 = kind == 0 ? __float_as_uint(1.0f + t * 1e-3f) : 0x3f803f80u + t;
  const unsigned a1 = a0 ^ 1u, a2 = a0 ^ 2u, a3 = a0 ^ 3u;
  const unsigned b0 = kind == 0 ? __float_as_uint(0.5f) : 0x3f003f00u, b1 = b0 ^ 1u;
  float c[4][4] = {};
  if (kind == 0) {
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int u = 0; u < 4; ++u)
        asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                     : "+f"(c[u][0]), "+f"(c[u][1]), "+f"(c[u][2]), "+f"(c[u][3])
                     : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  } else {
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int u = 0; u < 4; ++u)
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                     : "+f"(c[u][0]), "+f"(c[u][1]), "+f"(c[u][2]), "+f"(c[u][3])
                     : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float s = 0.f;
#pragma unroll
  for (int u = 0; u < 4; ++u) s += (c[u][0] + c[u][1]) + (c[u][2] + c[u][3]);
  if (s == -1.2345f) out[blockIdx.x] = s;
}

}  // namespace bhem

using namespace bhem;

extern "C" shell_status shell_measure_mma_peak(int kind, int iters, void* stream, double* flops_per_s) {
  if (!flops_per_s || iters < 1 || (kind != 0 && kind != 1)) return fail(SHELL_ERR_ARG, "invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  BHEM_CUDA(cudaGetDevice(&dev));
  BHEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 4, threads = 256;
  void* out = nullptr;
  BHEM_CUDA(cudaMalloc(&out, sizeof(float) * blocks));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  shell_status rc = SHELL_OK;
  float ms = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = fail(SHELL_ERR_CUDA, "cudaEventCreate failed");
  } else {
    for (int rep = 0; rep < 2 && rc == SHELL_OK; ++rep) {   // the first launch warms up
      cudaEventRecord(e0, st);
      k_mma_peak<<<blocks, threads, 0, st>>>(kind, iters, (float*)out);
      cudaEventRecord(e1, st);
      const cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess || cudaGetLastError() != cudaSuccess)
        rc = fail(SHELL_ERR_CUDA, std::string("MMA peak kernel: ") + cudaGetErrorString(e));
    }
    if (rc == SHELL_OK) cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != SHELL_OK) return rc;
  const double mma = 4.0 * (double)iters * (double)blocks * (double)(threads / 32);
  const double flop_per_mma = kind == 0 ? 2.0 * 16 * 8 * 8 : 2.0 * 16 * 8 * 16;
  *flops_per_s = ms > 0.f ? mma * flop_per_mma / (ms * 1e-3) : 0.0;
  return SHELL_OK;
}

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
