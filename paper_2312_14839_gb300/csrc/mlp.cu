// Learned Newton warm start: a per-node MLP 28 -> 256 -> 256 -> 256 -> 12 with GELU, BF16 weights
// and activations, FP32 accumulation on the tensor cores (tcgen05.mma kind::f16 with TMEM
// accumulators, operands staged by TMA; tc_gemm.cuh), trained with an MSE loss and Adam by the
// kernels of this file. The paper has no learning component; the implicit-Euler Newton solve of
// Sec. 6.1 stays the judge of every step.
//
// Node features (28, FP32): the node's 12 DOFs relative to rest (u = q - q_rest), its 12 velocity
// DOFs, and 4 means over its present edge neighbours: of u_nb - u_i for the position DOFs (a
// discrete Laplacian of the displacement, 3 values), and of the neighbours' position speed |v_nb|
// (their previous step's |dq| over dt, 1 value).
// Output (12): the node's update beyond the inertial predictor, q^{n+1} - q^n - dt v^n.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace bhem {
namespace mlp {

constexpr int kIn = 28, kInPad = 32, kHid = 256, kOut = 12, kOutPad = 16, kLayers = 4;
constexpr int kDin[kLayers] = {kInPad, kHid, kHid, kHid};   // padded fan-in
constexpr int kDout[kLayers] = {kHid, kHid, kHid, kOutPad};  // padded fan-out
constexpr int kRin[kLayers] = {kIn, kHid, kHid, kHid};       // fan-in
constexpr int kRout[kLayers] = {kHid, kHid, kHid, kOut};     // fan-out
// normalisation vector: in_mean[28] in_istd[28] out_mean[12] out_std[12] out_istd[12]
constexpr int kNormInMean = 0, kNormInIstd = 28, kNormOutMean = 56, kNormOutStd = 68, kNormOutIstd = 80;
constexpr int kNormSize = 96;

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// ------------------------------------------------------------------------------------------
// Epilogues of the tensor-core GEMM (tc_gemm.cuh): per row and 16 accumulator columns, the values
// of the FP32 output channel (f) and of the BF16 channels (b: row-major and transposed). A
// transposed BF16 copy ([column][row], row stride ldt) is what the weight-gradient GEMMs read as
// their K-contiguous operands.
// ------------------------------------------------------------------------------------------
constexpr int kErrIndex = 1, kErrTimeout = 2;   // bits of the network's error word

// forward layer: Z = acc + bias (FP32 pre-activation; bias = the per-column vector) and, for a
// hidden layer, GELU(Z) for the BF16 channels
struct EpiForward {
  int hidden;
  __device__ void operator()(int, int, const float* bias, const float (&acc)[16], float (&f)[16],
                             float (&b)[16]) const {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      f[j] = acc[j] + bias[j];
      b[j] = hidden ? gelu(f[j]) : f[j];
    }
  }
};

// split-K weight gradient: the FP32 channel adds acc into the zeroed gradient
struct EpiAtomic {
  __device__ void operator()(int, int, const float*, const float (&acc)[16], float (&f)[16], float (&b)[16]) const {
#pragma unroll
    for (int j = 0; j < 16; ++j) f[j] = b[j] = acc[j];
  }
};

// back-propagation through a hidden layer: dZ = (dZ_next W) * GELU'(Z), for all three channels
struct EpiGeluBack {
  const float* Z;
  int ld;
  int rows;
  __device__ void operator()(int row, int col0, const float*, const float (&acc)[16], float (&f)[16],
                             float (&b)[16]) const {
    if (row >= rows) {
#pragma unroll
      for (int j = 0; j < 16; ++j) f[j] = b[j] = 0.f;
      return;
    }
    const float4* zp = reinterpret_cast<const float4*>(Z + (long long)row * ld + col0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 z4 = zp[q];
      f[4 * q] = acc[4 * q] * gelu_grad(z4.x);
      f[4 * q + 1] = acc[4 * q + 1] * gelu_grad(z4.y);
      f[4 * q + 2] = acc[4 * q + 2] * gelu_grad(z4.z);
      f[4 * q + 3] = acc[4 * q + 3] * gelu_grad(z4.w);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) b[j] = f[j];
  }
};

// ------------------------------------------------------------------------------------------
// Element-wise kernels
// ------------------------------------------------------------------------------------------
// normalised BF16 input rows (gathered through idx when given), and their transpose XbT
// ([32][ldt]) when given; an index outside [0, data_rows) gives a zero row and raises the error flag
__global__ void k_input(int rows, const float* __restrict__ X, long long data_rows, const int* __restrict__ idx,
                        const float* __restrict__ norm, bf16* __restrict__ Xb, bf16* __restrict__ XbT,
                        long long ldt, int* err) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * kInPad; e += gridDim.x * blockDim.x) {
    const int r = e / kInPad, c = e % kInPad;
    float v = 0.f;
    const long long src = idx ? (long long)idx[r] : r;
    if (src < 0 || src >= data_rows) {
      if (c == 0) atomicOr(err, kErrIndex);
    } else if (c < kIn) {
      v = (X[src * kIn + c] - norm[kNormInMean + c]) * norm[kNormInIstd + c];
    }
    const bf16 b = __float2bfloat16(v);
    Xb[e] = b;
    if (XbT) XbT[c * ldt + r] = b;
  }
}

// Y = Z * out_std + out_mean over the 12 output columns
__global__ void k_output(int rows, const float* __restrict__ Z, const float* __restrict__ norm, float* __restrict__ Y) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * kOut; e += gridDim.x * blockDim.x) {
    const int r = e / kOut, c = e % kOut;
    Y[e] = Z[(long long)r * kOutPad + c] * norm[kNormOutStd + c] + norm[kNormOutMean + c];
  }
}

// MSE on normalised targets: loss = mean (Z - Tn)^2 over rows x 12; dZ = 2 (Z - Tn) / (rows x 12),
// zero in the padded columns (FP32, BF16, and BF16 transposed [16][ldt])
__global__ void k_loss(int rows, const float* __restrict__ Z, const float* __restrict__ T, long long data_rows,
                       const int* __restrict__ idx, const float* __restrict__ norm, float* __restrict__ dZ,
                       bf16* __restrict__ dZb, bf16* __restrict__ dZbT, long long ldt, double* loss) {
  __shared__ double sbuf[32];
  double part = 0.0;
  const float scale = 2.f / (float)(rows * kOut);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * kOutPad; e += gridDim.x * blockDim.x) {
    const int r = e / kOutPad, c = e % kOutPad;
    const long long src = idx ? (long long)idx[r] : r;
    float d = 0.f;
    if (c < kOut && src >= 0 && src < data_rows) {
      const float tn = (T[src * kOut + c] - norm[kNormOutMean + c]) * norm[kNormOutIstd + c];
      const float diff = Z[e] - tn;
      part += (double)diff * diff;
      d = scale * diff;
    }
    dZ[e] = d;
    dZb[e] = __float2bfloat16(d);
    dZbT[c * ldt + r] = __float2bfloat16(d);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sbuf[w];
    atomicAdd(loss, s / (double)(rows * kOut));
  }
}

// db[n] += sum over rows of dZ[r][n]: CTA (x, y) takes columns 128 x .. 128 x + 127 of the
// 64-row slab y, with eight independent partial sums per thread (eight loads in flight), then one
// atomic per column
constexpr int kColsumRows = 64;

__global__ void k_colsum(int rows, int cols, const float* __restrict__ dZ, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= cols) return;
  const int r0 = blockIdx.y * kColsumRows, r1 = min(rows, r0 + kColsumRows);
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int r = r0;
  for (; r + 8 <= r1; r += 8)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] += dZ[(long long)(r + j) * cols + n];
  for (; r < r1; ++r) acc[0] += dZ[(long long)r * cols + n];
  atomicAdd(&db[n], ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7])));
}

// Adam (Kingma and Ba) on the FP32 master parameters of every tensor of the network in one launch,
// refreshing a tensor's BF16 copy and its transpose (a [rows x cols] matrix stored [cols][rows])
// where given. Padded entries see zero gradients and stay zero.
constexpr int kAdamTensors = 2 * kLayers;
struct AdamSet {
  float* w[kAdamTensors];
  const float* g[kAdamTensors];
  float* m[kAdamTensors];
  float* v[kAdamTensors];
  bf16* wb[kAdamTensors];
  bf16* wbT[kAdamTensors];
  int rows[kAdamTensors], cols[kAdamTensors];
  long long end[kAdamTensors];   // cumulative element counts
};

__global__ void k_adam(AdamSet S, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long total = S.end[kAdamTensors - 1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int t = 0;
    while (e >= S.end[t]) ++t;
    const long long i = e - (t ? S.end[t - 1] : 0);
    const float gr = S.g[t][i];
    const float mm = b1 * S.m[t][i] + (1.f - b1) * gr;
    const float vv = b2 * S.v[t][i] + (1.f - b2) * gr * gr;
    S.m[t][i] = mm;
    S.v[t][i] = vv;
    const float wn = S.w[t][i] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    S.w[t][i] = wn;
    if (S.wb[t]) S.wb[t][i] = __float2bfloat16(wn);
    if (S.wbT[t]) S.wbT[t][(i % S.cols[t]) * S.rows[t] + i / S.cols[t]] = __float2bfloat16(wn);
  }
}

// BF16 copy of a [rows x cols] FP32 matrix, and its transpose [cols][rows] when bT is given
__global__ void k_to_bf16(int rows, int cols, const float* __restrict__ a, bf16* __restrict__ b,
                          bf16* __restrict__ bT) {
  const long long count = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const bf16 h = __float2bfloat16(a[e]);
    b[e] = h;
    if (bT) bT[(e % cols) * rows + e / cols] = h;
  }
}

// per-column sum and sum of squares (FP64) of a [rows x cols] FP32 matrix; one CTA per column
__global__ void k_colstats(long long rows, int cols, const float* __restrict__ X, double* __restrict__ acc) {
  const int c = blockIdx.x;
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (long long r = threadIdx.x; r < rows; r += blockDim.x) {
    const double x = X[r * cols + c];
    a += x;
    b += x * x;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    acc[2 * c] = s1[0];
    acc[2 * c + 1] = s2[0];
  }
}

// ------------------------------------------------------------------------------------------
// Shell-side kernels: node features, training targets, warm start
// ------------------------------------------------------------------------------------------
// the 28 features of node i (shared by the feature kernel and the fused warm start)
__device__ __forceinline__ void node_features_of(int i, int n1, int n2, int per_u, int per_v,
                                                 const double* __restrict__ q, const double* __restrict__ rest,
                                                 const double* __restrict__ v, float* out) {
  double ui[3];
  for (int k = 0; k < 12; ++k) {
    const double u = q[(size_t)i * 12 + k] - rest[(size_t)i * 12 + k];
    if (k < 3) ui[k] = u;
    out[k] = (float)u;
    out[12 + k] = (float)v[(size_t)i * 12 + k];
  }
  const int ii = i % n1, jj = i / n1;
  const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
  double lap[3] = {0.0, 0.0, 0.0}, speed = 0.0;
  int cnt = 0;
  for (int e = 0; e < 4; ++e) {
    int a = ii + di[e], b = jj + dj[e];
    if (per_u) a = (a + n1) % n1;
    if (per_v) b = (b + n2) % n2;
    if (a < 0 || a >= n1 || b < 0 || b >= n2 || (a == ii && b == jj)) continue;
    const size_t o = ((size_t)b * n1 + a) * 12;
    for (int c = 0; c < 3; ++c) lap[c] += (q[o + c] - rest[o + c]) - ui[c];
    speed += sqrt(v[o] * v[o] + v[o + 1] * v[o + 1] + v[o + 2] * v[o + 2]);
    ++cnt;
  }
  for (int c = 0; c < 3; ++c) out[24 + c] = cnt ? (float)(lap[c] / cnt) : 0.f;
  out[27] = cnt ? (float)(speed / cnt) : 0.f;
}

__global__ void k_node_features(int n1, int n2, int per_u, int per_v, const double* __restrict__ q,
                                const double* __restrict__ rest, const double* __restrict__ v,
                                float* __restrict__ X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n1 * n2) return;
  node_features_of(i, n1, n2, per_u, per_v, q, rest, v, X + (size_t)i * kIn);
}

__global__ void k_targets(long long n_dof, const double* __restrict__ q_next, const double* __restrict__ q,
                          const double* __restrict__ v, double dt, float* __restrict__ T) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_dof;
       e += (long long)gridDim.x * blockDim.x)
    T[e] = (float)(q_next[e] - q[e] - dt * v[e]);
}

// warm = q + dt v + out_std * Z + out_mean (the inertial predictor alone when Z is NULL)
__global__ void k_compose(int n_nodes, const double* __restrict__ q, const double* __restrict__ v, double dt,
                          const float* __restrict__ Z, const float* __restrict__ norm, double* __restrict__ warm) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_nodes * kOut; e += gridDim.x * blockDim.x) {
    const int r = e / kOut, c = e % kOut;
    const float y = Z ? Z[(long long)r * kOutPad + c] * norm[kNormOutStd + c] + norm[kNormOutMean + c] : 0.f;
    warm[e] = q[e] + dt * v[e] + (double)y;
  }
}

// ------------------------------------------------------------------------------------------
// Fused warm start: features -> normalised BF16 input -> 4 layers -> q + dt v + output, one
// launch. A CTA takes 128 nodes (one per TMEM lane). The activations stay in shared memory as the
// next layer's A operand (128-byte swizzled K-major tiles, written by the epilogue); each layer's
// weights arrive by TMA into one shared buffer as soon as the previous layer's MMAs are done, and
// one thread issues the layer's tcgen05.mma into a 128 x 256 FP32 TMEM accumulator. Every output
// is accumulated over the same K chunks, in the same order and with the same MMA shapes as the
// GEMM path (shell_mlp_forward), and finished by the same epilogue arithmetic, so the network
// output equals that path's.
// ------------------------------------------------------------------------------------------
constexpr int kWarmThreads = 512;                 // 16 warps: TMEM lane quarter w % 4, column part w / 4
constexpr int kActBytes = 4 * tc::kBM * 128;      // 4 K chunks of 128 rows x 128 bytes
constexpr int kWgtBytes = 4 * kHid * 128;         // 4 K chunks of 256 rows x 128 bytes
constexpr size_t kWarmSmem = (size_t)kActBytes + kWgtBytes + 1024;

struct WarmArgs {
  int n_nodes, n1, n2, per_u, per_v;
  const double* q;
  const double* rest;
  const double* v;
  double dt;
  const float* bias[kLayers];
  const float* norm;
  double* warm;
  int* err;
  unsigned polls;
};

__device__ __forceinline__ uint4 pack_bf16x8(const float* x) {
  unsigned w[4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
    w[j] = (unsigned)__bfloat16_as_ushort(__float2bfloat16(x[2 * j])) |
           ((unsigned)__bfloat16_as_ushort(__float2bfloat16(x[2 * j + 1])) << 16);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__global__ void __launch_bounds__(kWarmThreads, 1)
k_mlp_warm(const __grid_constant__ CUtensorMap tw0, const __grid_constant__ CUtensorMap tw1,
           const __grid_constant__ CUtensorMap tw2, const __grid_constant__ CUtensorMap tw3, WarmArgs A) {
  extern __shared__ unsigned char warm_smem_raw[];
  __shared__ __align__(8) uint64_t bar_w, bar_mma;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  volatile int* abort_flag = &s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t raw = tc::smem_addr(warm_smem_raw);
  const uint32_t act = (raw + 1023u) & ~1023u, wgt = act + kActBytes;
  unsigned char* act_g = warm_smem_raw + (act - raw);   // generic pointer to the activation tiles
  const uint32_t bw = tc::smem_addr(&bar_w), bm = tc::smem_addr(&bar_mma);
  const int r0 = blockIdx.x * tc::kBM;
  if (tid == 0) {
    tc::mbar_init(bw, 1);
    tc::mbar_init(bm, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc<kHid>(tc::smem_addr(&tmem_slot));
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {   // layer-0 weights (K = 32: one 64-column chunk, the rest read as zeros)
    tc::mbar_arrive_expect_tx(bw, kHid * 128);
    tc::tma_load_2d(wgt, &tw0, bw, 0, 0);
  }
  // layer-0 input rows (the arithmetic of k_node_features and k_input): K chunk 0, columns 32..63 zero
  if (tid < tc::kBM) {
    const int i = r0 + tid;
    float f[kIn];
    if (i < A.n_nodes) node_features_of(i, A.n1, A.n2, A.per_u, A.per_v, A.q, A.rest, A.v, f);
    float x[kInPad];
#pragma unroll
    for (int c = 0; c < kInPad; ++c)
      x[c] = (i < A.n_nodes && c < kIn) ? (f[c] - A.norm[kNormInMean + c]) * A.norm[kNormInIstd + c] : 0.f;
    uint4* row = reinterpret_cast<uint4*>(act_g + tid * 128);
#pragma unroll
    for (int p = 0; p < 8; ++p) row[p ^ (tid & 7)] = p < 4 ? pack_bf16x8(x + 8 * p) : make_uint4(0u, 0u, 0u, 0u);
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const int quarter = warp & 3, part = warp >> 2, row = quarter * 32 + lane;
  const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
  int w_inflight = 0;   // thread 0: the layer whose weight copy is in flight, or -1
  int l = 0;
#pragma unroll 1
  for (; l < kLayers; ++l) {
    const int N = l < kLayers - 1 ? kHid : kOutPad;
    const int nch = l == 0 ? 1 : kHid / tc::kBK;
    if (tid == 0) {
      if (!tc::mbar_wait_parity(bw, l & 1, A.polls)) {
        *abort_flag = 1;
      } else {
        w_inflight = -1;
        tc::tc_fence_after();
        const uint32_t idesc = tc::idesc_bf16(tc::kBM, N);
        for (int c = 0; c < nch; ++c)
#pragma unroll
          for (int j = 0; j < tc::kBK / 16; ++j)
            tc::mma_bf16_ss(tmem, tc::smem_desc_sw128(act + c * (tc::kBM * 128) + 32 * j),
                            tc::smem_desc_sw128(wgt + c * (N * 128) + 32 * j), idesc, c > 0 || j > 0);
      }
      tc::mma_commit(bm);
    }
    if (!tc::mbar_wait_parity(bm, l & 1, A.polls)) *abort_flag = 1;
    tc::tc_fence_after();
    __syncthreads();
    if (*abort_flag) break;
    if (tid == 0 && l + 1 < kLayers) {   // the weight buffer is free: fetch the next layer's
      const int N1 = l + 1 < kLayers - 1 ? kHid : kOutPad;
      const CUtensorMap* m = l == 0 ? &tw1 : (l == 1 ? &tw2 : &tw3);
      tc::mbar_arrive_expect_tx(bw, (kHid / tc::kBK) * N1 * 128);
      for (int c = 0; c < kHid / tc::kBK; ++c) tc::tma_load_2d(wgt + c * N1 * 128, m, bw, c * tc::kBK, 0);
      w_inflight = l + 1;
    }
    const float* bias = A.bias[l];
    if (l < kLayers - 1) {
      // epilogue of a hidden layer (the arithmetic of EpiForward): GELU(acc + bias) in BF16,
      // written over the activations as the next layer's A tiles
#pragma unroll 1
      for (int c0 = part * (kHid / 4); c0 < (part + 1) * (kHid / 4); c0 += 16) {
        float v[16];
        tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
        float a[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) a[j] = gelu(v[j] + bias[c0 + j]);
        unsigned char* rp = act_g + (c0 / tc::kBK) * (tc::kBM * 128) + row * 128;
        const int p = (c0 % tc::kBK) / 8;
        *reinterpret_cast<uint4*>(rp + ((p ^ (row & 7)) * 16)) = pack_bf16x8(a);
        *reinterpret_cast<uint4*>(rp + (((p + 1) ^ (row & 7)) * 16)) = pack_bf16x8(a + 8);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      tc::tc_fence_before();
      __syncthreads();
      tc::tc_fence_after();
    } else if (part == 0) {
      // output layer: warm = q + dt v + out_std * (acc + bias) + out_mean (k_output, k_compose)
      float v[16];
      tc::tmem_ld16(lane_addr, v);
      const int i = r0 + row;
      if (i < A.n_nodes) {
#pragma unroll
        for (int c = 0; c < kOut; ++c) {
          const float y = (v[c] + bias[c]) * A.norm[kNormOutStd + c] + A.norm[kNormOutMean + c];
          const size_t gi = (size_t)i * 12 + c;
          A.warm[gi] = A.q[gi] + A.dt * A.v[gi] + (double)y;
        }
      }
    }
  }
  if (tid == 0 && *abort_flag) {
    atomicOr(A.err, kErrTimeout);
    // a weight copy still in flight, and the commit of the stopped layer, land in shared memory:
    // wait for them before the CTA exits
    if (w_inflight >= 0) tc::mbar_wait_parity(bw, w_inflight & 1, tc::kDrainPolls);
    tc::mbar_wait_parity(bm, l & 1, tc::kDrainPolls);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc<kHid>(tmem);
}

}  // namespace mlp
}  // namespace bhem

// ==========================================================================================
// Host side
// ==========================================================================================
using namespace bhem;
using namespace bhem::mlp;

struct shell_mlp_s {
  int max_rows = 0;
  cudaStream_t stream = nullptr;
  unsigned wait_polls = (unsigned)kDefaultWaitPolls;   // bound of the tensor-core pipeline waits
  long long launches = 0;
  int step = 0;
  // parameters (padded; FP32 master copies, BF16 copies for the GEMMs), Adam moments, gradients
  float *W[kLayers] = {}, *b[kLayers] = {}, *gW[kLayers] = {}, *gb[kLayers] = {};
  float *mW[kLayers] = {}, *vW[kLayers] = {}, *mb[kLayers] = {}, *vb[kLayers] = {};
  bf16* Wb[kLayers] = {};
  bf16* WbT[kLayers] = {};   // transposed BF16 weights [fan_in][fan_out] (input-gradient GEMMs)
  CUtensorMap warm_maps[kLayers];   // TMA maps of Wb for the fused warm start (box 64 x fan-out)
  // activations of the last forward pass, and their gradients; the *T arrays are transposed
  // copies [features][ldt] read by the weight-gradient GEMMs
  long long ldt = 0;         // max_rows rounded up to 8 (16-byte rows for TMA)
  bf16 *Xb = nullptr, *XbT = nullptr;
  float* Z[kLayers] = {};
  bf16 *Ab[kLayers] = {}, *AbT[kLayers] = {};
  float* dZ[kLayers] = {};
  bf16 *dZb[kLayers] = {}, *dZbT[kLayers] = {};
  float* Xraw = nullptr;  // [max_rows x 28] features of a warm-start call
  float* norm = nullptr;  // kNormSize floats
  double* loss = nullptr;
  double* stats = nullptr;
  int* err = nullptr;
  double* h_loss = nullptr;  // pinned
  int* h_err = nullptr;      // pinned
};

namespace {

template <typename T>
shell_status malloc_zero(T** p, size_t count, cudaStream_t s) {
  *p = nullptr;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(SHELL_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  BHEM_CUDA(cudaMemsetAsync(*p, 0, sizeof(T) * (count ? count : 1), s));
  return SHELL_OK;
}

void free_mlp(shell_mlp_s* m) {
  for (int l = 0; l < kLayers; ++l) {
    void* ps[] = {m->W[l], m->b[l], m->gW[l], m->gb[l], m->mW[l], m->vW[l], m->mb[l], m->vb[l], m->Wb[l],
                  m->WbT[l], m->Z[l], m->Ab[l], m->AbT[l], m->dZ[l], m->dZb[l], m->dZbT[l]};
    for (void* p : ps)
      if (p) cudaFree(p);
  }
  void* ps[] = {m->Xb, m->XbT, m->Xraw, m->norm, m->loss, m->stats, m->err};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (m->h_loss) cudaFreeHost(m->h_loss);
  if (m->h_err) cudaFreeHost(m->h_err);
  delete m;
}

int eblocks(long long n) { return (int)std::min<long long>(4096, std::max(1LL, (n + 255) / 256)); }

// N tile of the 256-column GEMMs: 128 columns, so that two CTAs share an SM
constexpr int kTileN = 128;

// Outputs of one GEMM (any may be null): FP32 (stored, or added for split K), BF16 row-major,
// BF16 transposed; colvec: the per-column vector handed to the epilogue.
struct GemmOut {
  float* f32 = nullptr;
  long long ldf = 0;
  bool add = false;
  bf16* b16 = nullptr;
  long long ldb = 0;
  bf16* b16t = nullptr;
  long long ldt = 0;
  const float* colvec = nullptr;
};

// C = A B^T on the tensor cores for A [m][k] (row stride lda) and B [n][k] (row stride ldb), both
// BF16 with K contiguous; K split over up to ksplit CTAs per output tile.
template <int BN, class Epi>
shell_status tc_gemm(shell_mlp_s& M, const bf16* A, long long lda, const bf16* B, long long ldb, int m, int n, int k,
                     int ksplit, const GemmOut& o, const Epi& epi, cudaStream_t st) {
  CUtensorMap ma, mb;
  tc::TcOut out;
  std::memset(&out, 0, sizeof(out));
  int mask = 0;
  bool ok = tc::encode_bf16_map(&ma, A, m, k, lda, tc::kBM) && tc::encode_bf16_map(&mb, B, n, k, ldb, BN);
  if (o.f32) {
    ok = ok && tc::encode_out_f32(&out.f32, o.f32, m, n, o.ldf);
    mask |= o.add ? tc::kOutF32Add : tc::kOutF32;
  }
  if (o.b16) {
    ok = ok && tc::encode_out_b16(&out.b16, o.b16, m, n, o.ldb);
    mask |= tc::kOutB16;
  }
  if (o.b16t) {
    ok = ok && tc::encode_out_b16t(&out.b16t, o.b16t, n, m, o.ldt);
    mask |= tc::kOutB16T;
  }
  if (!ok) return fail(SHELL_ERR_CUDA, "tensor map encoding failed (cuTensorMapEncodeTiled)");
  const cudaError_t e = tc::launch_gemm_tc<BN, Epi>(ma, mb, out, mask, o.colvec, m, n, k, ksplit, epi, M.err,
                                                    kErrTimeout, M.wait_polls, st);
  BHEM_CUDA(e);
  ++M.launches;
  return SHELL_OK;
}

// forward pass of the rows staged in M.Xb: Z_l (FP32 pre-activation), Ab_l (BF16 GELU) and, when
// training, the transposed AbT_l
shell_status forward(shell_mlp_s& M, int rows, bool training, cudaStream_t st) {
  const bf16* in = M.Xb;
  for (int l = 0; l < kLayers; ++l) {
    const bool hidden = l < kLayers - 1;
    GemmOut o;
    o.f32 = M.Z[l];
    o.ldf = kDout[l];
    o.colvec = M.b[l];
    if (hidden) {
      o.b16 = M.Ab[l];
      o.ldb = kDout[l];
      if (training) {
        o.b16t = M.AbT[l];
        o.ldt = M.ldt;
      }
    }
    const EpiForward e{hidden ? 1 : 0};
    if (kDout[l] == kHid) BHEM_TRY(tc_gemm<kTileN>(M, in, kDin[l], M.Wb[l], kDin[l], rows, kHid, kDin[l], 1, o, e, st));
    else BHEM_TRY(tc_gemm<kOutPad>(M, in, kDin[l], M.Wb[l], kDin[l], rows, kOutPad, kDin[l], 1, o, e, st));
    in = M.Ab[l];
  }
  return SHELL_OK;
}

// parameter gradients of the loss whose dZ (last layer) k_loss left in M.dZ[3], M.dZb[3], M.dZbT[3]
shell_status backward(shell_mlp_s& M, int rows, cudaStream_t st) {
  int dev = 0, nsm = 0;
  BHEM_CUDA(cudaGetDevice(&dev));
  BHEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int kchunks = (rows + tc::kBK - 1) / tc::kBK;
  for (int l = kLayers - 1; l >= 0; --l) {
    BHEM_CUDA(cudaMemsetAsync(M.gW[l], 0, sizeof(float) * kDout[l] * kDin[l], st));
    BHEM_CUDA(cudaMemsetAsync(M.gb[l], 0, sizeof(float) * kDout[l], st));
    // dW_l = dZ_l^T A_{l-1}: M = fan-out, N = fan-in, K = rows, split over about one CTA per SM
    const bf16* At = l > 0 ? M.AbT[l - 1] : M.XbT;
    const int tiles = (kDout[l] + tc::kBM - 1) / tc::kBM * (kDin[l] == kHid ? kHid / kTileN : 1);
    const int ksplit = std::max(1, std::min(kchunks, 2 * nsm / tiles));
    GemmOut ow;
    ow.f32 = M.gW[l];
    ow.ldf = kDin[l];
    ow.add = true;
    const EpiAtomic ea{};
    if (kDin[l] == kHid)
      BHEM_TRY(tc_gemm<kTileN>(M, M.dZbT[l], M.ldt, At, M.ldt, kDout[l], kHid, rows, ksplit, ow, ea, st));
    else
      BHEM_TRY(tc_gemm<kInPad>(M, M.dZbT[l], M.ldt, At, M.ldt, kDout[l], kInPad, rows, ksplit, ow, ea, st));
    dim3 cg((kDout[l] + 127) / 128, (rows + kColsumRows - 1) / kColsumRows);
    k_colsum<<<cg, 128, 0, st>>>(rows, kDout[l], M.dZ[l], M.gb[l]);
    BHEM_CUDA(cudaGetLastError());
    ++M.launches;
    if (l == 0) break;
    // dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1}): M = rows, N = fan-in, K = fan-out
    GemmOut og;
    og.f32 = M.dZ[l - 1];
    og.ldf = kDout[l - 1];
    og.b16 = M.dZb[l - 1];
    og.ldb = kDout[l - 1];
    og.b16t = M.dZbT[l - 1];
    og.ldt = M.ldt;
    const EpiGeluBack eg{M.Z[l - 1], kDout[l - 1], rows};
    BHEM_TRY(tc_gemm<kTileN>(M, M.dZb[l], kDout[l], M.WbT[l], kDout[l], rows, kHid, kDout[l], 1, og, eg, st));
  }
  return SHELL_OK;
}

shell_status stage_input(shell_mlp_s& M, const float* X, long long data_rows, const int* idx, int rows,
                         bool training, cudaStream_t st) {
  k_input<<<eblocks((long long)rows * kInPad), 256, 0, st>>>(rows, X, data_rows, idx, M.norm, M.Xb,
                                                             training ? M.XbT : nullptr, M.ldt, M.err);
  BHEM_CUDA(cudaGetLastError());
  ++M.launches;
  return SHELL_OK;
}

// waits for the stream, returns the loss when asked, and turns a raised error flag into an error
shell_status finish(shell_mlp_s& M, double* loss) {
  BHEM_CUDA(cudaMemcpyAsync(M.h_err, M.err, sizeof(int), cudaMemcpyDeviceToHost, M.stream));
  if (loss) BHEM_CUDA(cudaMemcpyAsync(M.h_loss, M.loss, sizeof(double), cudaMemcpyDeviceToHost, M.stream));
  BHEM_CUDA(cudaStreamSynchronize(M.stream));
  if (*M.h_err) {
    const int e = *M.h_err;
    BHEM_CUDA(cudaMemsetAsync(M.err, 0, sizeof(int), M.stream));
    BHEM_CUDA(cudaStreamSynchronize(M.stream));
    if (e & kErrTimeout) return fail(SHELL_ERR_TIMEOUT, "a bounded tensor-core pipeline wait expired");
    return fail(SHELL_ERR_ARG, "row index outside [0, data_rows)");
  }
  if (loss) *loss = *M.h_loss;
  return SHELL_OK;
}

long long param_count() {
  long long n = 0;
  for (int l = 0; l < kLayers; ++l) n += (long long)kRout[l] * kRin[l] + kRout[l];
  return n;
}

// host packed layout: per layer W [fan_out x fan_in] row-major, then b [fan_out]
shell_status copy_params(shell_mlp_s& M, float* host_out, const float* host_in, int grads) {
  std::vector<float> buf;
  long long off = 0;
  for (int l = 0; l < kLayers; ++l) {
    float* W = grads ? M.gW[l] : M.W[l];
    float* b = grads ? M.gb[l] : M.b[l];
    const int ro = kRout[l], ri = kRin[l], din = kDin[l];
    buf.assign((size_t)kDout[l] * din, 0.f);
    if (host_in) {
      for (int o = 0; o < ro; ++o)
        for (int i = 0; i < ri; ++i) buf[(size_t)o * din + i] = host_in[off + (long long)o * ri + i];
      BHEM_CUDA(cudaMemcpy(W, buf.data(), sizeof(float) * buf.size(), cudaMemcpyHostToDevice));
      BHEM_CUDA(cudaMemcpy(b, host_in + off + (long long)ro * ri, sizeof(float) * ro, cudaMemcpyHostToDevice));
    } else {
      BHEM_CUDA(cudaMemcpy(buf.data(), W, sizeof(float) * buf.size(), cudaMemcpyDeviceToHost));
      for (int o = 0; o < ro; ++o)
        for (int i = 0; i < ri; ++i) host_out[off + (long long)o * ri + i] = buf[(size_t)o * din + i];
      BHEM_CUDA(cudaMemcpy(host_out + off + (long long)ro * ri, b, sizeof(float) * ro, cudaMemcpyDeviceToHost));
    }
    off += (long long)ro * ri + ro;
  }
  return SHELL_OK;
}

}  // namespace

extern "C" shell_status shell_mlp_create(int max_rows, void* stream, shell_mlp_t** out) {
  if (!out || max_rows < 1 || max_rows > (1 << 24)) return fail(SHELL_ERR_ARG, "invalid argument");
  *out = nullptr;
  shell_mlp_s* M = new shell_mlp_s();
  M->max_rows = max_rows;
  M->stream = (cudaStream_t)stream;
  M->ldt = ((long long)max_rows + 7) / 8 * 8;
  shell_status st = SHELL_OK;
  const size_t R = (size_t)max_rows, RT = (size_t)M->ldt;
  for (int l = 0; l < kLayers && st == SHELL_OK; ++l) {
    const size_t nw = (size_t)kDout[l] * kDin[l], nb = kDout[l];
    float** f32w[] = {&M->W[l], &M->gW[l], &M->mW[l], &M->vW[l]};
    for (float** p : f32w)
      if (st == SHELL_OK) st = malloc_zero(p, nw, M->stream);
    float** f32b[] = {&M->b[l], &M->gb[l], &M->mb[l], &M->vb[l]};
    for (float** p : f32b)
      if (st == SHELL_OK) st = malloc_zero(p, nb, M->stream);
    if (st == SHELL_OK) st = malloc_zero(&M->Wb[l], nw, M->stream);
    if (st == SHELL_OK && l > 0) st = malloc_zero(&M->WbT[l], nw, M->stream);
    if (st == SHELL_OK) st = malloc_zero(&M->Z[l], R * kDout[l], M->stream);
    if (st == SHELL_OK && l < kLayers - 1) st = malloc_zero(&M->Ab[l], R * kDout[l], M->stream);
    if (st == SHELL_OK && l < kLayers - 1) st = malloc_zero(&M->AbT[l], RT * kDout[l], M->stream);
    if (st == SHELL_OK) st = malloc_zero(&M->dZ[l], R * kDout[l], M->stream);
    if (st == SHELL_OK) st = malloc_zero(&M->dZb[l], R * kDout[l], M->stream);
    if (st == SHELL_OK) st = malloc_zero(&M->dZbT[l], RT * kDout[l], M->stream);
  }
  if (st == SHELL_OK) st = malloc_zero(&M->Xb, R * kInPad, M->stream);
  if (st == SHELL_OK) st = malloc_zero(&M->XbT, RT * kInPad, M->stream);
  if (st == SHELL_OK) st = malloc_zero(&M->Xraw, R * kIn, M->stream);
  if (st == SHELL_OK) st = malloc_zero(&M->norm, kNormSize, M->stream);
  if (st == SHELL_OK) st = malloc_zero(&M->loss, 1, M->stream);
  if (st == SHELL_OK) st = malloc_zero(&M->stats, 2 * kIn, M->stream);
  if (st == SHELL_OK) st = malloc_zero(&M->err, 1, M->stream);
  if (st == SHELL_OK && (cudaMallocHost((void**)&M->h_loss, sizeof(double)) != cudaSuccess ||
                         cudaMallocHost((void**)&M->h_err, sizeof(int)) != cudaSuccess)) {
    cudaGetLastError();
    st = fail(SHELL_ERR_OOM, "cudaMallocHost failed");
  }
  for (int l = 0; l < kLayers && st == SHELL_OK; ++l)
    if (!tc::encode_bf16_map(&M->warm_maps[l], M->Wb[l], kDout[l], kDin[l], kDin[l], kDout[l]))
      st = fail(SHELL_ERR_CUDA, "tensor map encoding failed (cuTensorMapEncodeTiled)");
  if (st == SHELL_OK) {
    // identity normalisation until shell_mlp_set_normalization
    float h[kNormSize] = {};
    for (int k = 0; k < kIn; ++k) h[kNormInIstd + k] = 1.f;
    for (int k = 0; k < kOut; ++k) h[kNormOutStd + k] = h[kNormOutIstd + k] = 1.f;
    if (cudaMemcpyAsync(M->norm, h, sizeof(h), cudaMemcpyHostToDevice, M->stream) != cudaSuccess ||
        cudaStreamSynchronize(M->stream) != cudaSuccess)
      st = fail(SHELL_ERR_CUDA, "normalisation upload failed");
  }
  if (st != SHELL_OK) {
    cudaStreamSynchronize(M->stream);
    free_mlp(M);
    return st;
  }
  *out = M;
  return SHELL_OK;
}

extern "C" shell_status shell_mlp_destroy(shell_mlp_t* M) {
  if (!M) return SHELL_OK;
  cudaStreamSynchronize(M->stream);
  free_mlp(M);
  return SHELL_OK;
}

extern "C" shell_status shell_mlp_param_count(long long* count) {
  if (!count) return fail(SHELL_ERR_ARG, "NULL argument");
  *count = param_count();
  return SHELL_OK;
}

extern "C" shell_status shell_mlp_set_params(shell_mlp_t* M, const float* params) {
  if (!M || !params) return fail(SHELL_ERR_ARG, "NULL argument");
  BHEM_CUDA(cudaStreamSynchronize(M->stream));
  BHEM_TRY(copy_params(*M, nullptr, params, 0));
  for (int l = 0; l < kLayers; ++l) {
    const long long n = (long long)kDout[l] * kDin[l];
    k_to_bf16<<<eblocks(n), 256, 0, M->stream>>>(kDout[l], kDin[l], M->W[l], M->Wb[l], M->WbT[l]);
    BHEM_CUDA(cudaGetLastError());
    ++M->launches;
    BHEM_CUDA(cudaMemsetAsync(M->mW[l], 0, sizeof(float) * n, M->stream));
    BHEM_CUDA(cudaMemsetAsync(M->vW[l], 0, sizeof(float) * n, M->stream));
    BHEM_CUDA(cudaMemsetAsync(M->mb[l], 0, sizeof(float) * kDout[l], M->stream));
    BHEM_CUDA(cudaMemsetAsync(M->vb[l], 0, sizeof(float) * kDout[l], M->stream));
  }
  M->step = 0;
  BHEM_CUDA(cudaStreamSynchronize(M->stream));
  return SHELL_OK;
}

extern "C" shell_status shell_mlp_get_params(shell_mlp_t* M, float* params, float* grads) {
  if (!M) return fail(SHELL_ERR_ARG, "NULL argument");
  BHEM_CUDA(cudaStreamSynchronize(M->stream));
  if (params) BHEM_TRY(copy_params(*M, params, nullptr, 0));
  if (grads) BHEM_TRY(copy_params(*M, grads, nullptr, 1));
  return SHELL_OK;
}

extern "C" shell_status shell_mlp_set_normalization(shell_mlp_t* M, const float* in_mean, const float* in_std,
                                                    const float* out_mean, const float* out_std) {
  if (!M || !in_mean || !in_std || !out_mean || !out_std) return fail(SHELL_ERR_ARG, "NULL argument");
  float h[kNormSize] = {};
  for (int k = 0; k < kIn; ++k) {
    h[kNormInMean + k] = in_mean[k];
    h[kNormInIstd + k] = in_std[k] > 0.f ? 1.f / in_std[k] : 1.f;
  }
  for (int k = 0; k < kOut; ++k) {
    h[kNormOutMean + k] = out_mean[k];
    h[kNormOutStd + k] = out_std[k] > 0.f ? out_std[k] : 1.f;
    h[kNormOutIstd + k] = out_std[k] > 0.f ? 1.f / out_std[k] : 1.f;
  }
  BHEM_CUDA(cudaMemcpyAsync(M->norm, h, sizeof(h), cudaMemcpyHostToDevice, M->stream));
  BHEM_CUDA(cudaStreamSynchronize(M->stream));
  return SHELL_OK;
}

extern "C" shell_status shell_mlp_column_stats(shell_mlp_t* M, const float* X, long long rows, int cols,
                                               double* mean, double* stdv) {
  if (!M || !X || rows < 1 || cols < 1 || cols > kIn || !mean || !stdv)
    return fail(SHELL_ERR_ARG, "invalid argument");
  k_colstats<<<cols, 256, 0, M->stream>>>(rows, cols, X, M->stats);
  BHEM_CUDA(cudaGetLastError());
  ++M->launches;
  double h[2 * kIn];
  BHEM_CUDA(cudaMemcpyAsync(h, M->stats, sizeof(double) * 2 * cols, cudaMemcpyDeviceToHost, M->stream));
  BHEM_CUDA(cudaStreamSynchronize(M->stream));
  for (int c = 0; c < cols; ++c) {
    mean[c] = h[2 * c] / (double)rows;
    const double var = h[2 * c + 1] / (double)rows - mean[c] * mean[c];
    stdv[c] = var > 0.0 ? std::sqrt(var) : 0.0;
  }
  return SHELL_OK;
}

extern "C" shell_status shell_mlp_forward(shell_mlp_t* M, const float* X, int rows, float* Y) {
  if (!M || !X || !Y || rows < 1 || rows > M->max_rows) return fail(SHELL_ERR_ARG, "invalid argument");
  BHEM_TRY(stage_input(*M, X, rows, nullptr, rows, false, M->stream));
  BHEM_TRY(forward(*M, rows, false, M->stream));
  k_output<<<eblocks((long long)rows * kOut), 256, 0, M->stream>>>(rows, M->Z[kLayers - 1], M->norm, Y);
  BHEM_CUDA(cudaGetLastError());
  ++M->launches;
  return SHELL_OK;
}

extern "C" shell_status shell_mlp_gradients(shell_mlp_t* M, const float* X, const float* T, long long data_rows,
                                            const int* idx, int rows, double* loss) {
  if (!M || !X || !T || rows < 1 || rows > M->max_rows || data_rows < 1 || (!idx && rows > data_rows))
    return fail(SHELL_ERR_ARG, "invalid argument");
  BHEM_TRY(stage_input(*M, X, data_rows, idx, rows, true, M->stream));
  BHEM_TRY(forward(*M, rows, true, M->stream));
  BHEM_CUDA(cudaMemsetAsync(M->loss, 0, sizeof(double), M->stream));
  k_loss<<<eblocks((long long)rows * kOutPad), 256, 0, M->stream>>>(
      rows, M->Z[kLayers - 1], T, data_rows, idx, M->norm, M->dZ[kLayers - 1], M->dZb[kLayers - 1],
      M->dZbT[kLayers - 1], M->ldt, M->loss);
  BHEM_CUDA(cudaGetLastError());
  ++M->launches;
  BHEM_TRY(backward(*M, rows, M->stream));
  return loss ? finish(*M, loss) : SHELL_OK;
}

extern "C" shell_status shell_mlp_train_step(shell_mlp_t* M, const float* X, const float* T, long long data_rows,
                                             const int* idx, int rows, float lr, double* loss) {
  BHEM_TRY(shell_mlp_gradients(M, X, T, data_rows, idx, rows, nullptr));
  M->step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - std::pow(b1, (float)M->step), c2 = 1.f - std::pow(b2, (float)M->step);
  AdamSet S{};
  long long end = 0;
  for (int l = 0; l < kLayers; ++l) {
    const int t = 2 * l;   // weights, then bias
    S.w[t] = M->W[l];
    S.g[t] = M->gW[l];
    S.m[t] = M->mW[l];
    S.v[t] = M->vW[l];
    S.wb[t] = M->Wb[l];
    S.wbT[t] = M->WbT[l];
    S.rows[t] = kDout[l];
    S.cols[t] = kDin[l];
    S.end[t] = end += (long long)kDout[l] * kDin[l];
    S.w[t + 1] = M->b[l];
    S.g[t + 1] = M->gb[l];
    S.m[t + 1] = M->mb[l];
    S.v[t + 1] = M->vb[l];
    S.rows[t + 1] = 1;
    S.cols[t + 1] = kDout[l];
    S.end[t + 1] = end += kDout[l];
  }
  k_adam<<<eblocks(end), 256, 0, M->stream>>>(S, lr, b1, b2, eps, c1, c2);
  ++M->launches;
  BHEM_CUDA(cudaGetLastError());
  return loss ? finish(*M, loss) : SHELL_OK;
}

extern "C" shell_status shell_mlp_set_wait_budget(shell_mlp_t* M, int polls) {
  if (!M) return fail(SHELL_ERR_ARG, "NULL argument");
  BHEM_CUDA(cudaStreamSynchronize(M->stream));
  M->wait_polls = polls < 0 ? (unsigned)kDefaultWaitPolls : (unsigned)polls;
  return SHELL_OK;
}

extern "C" shell_status shell_mlp_kernel_launches(const shell_mlp_t* M, long long* count) {
  if (!M || !count) return fail(SHELL_ERR_ARG, "NULL argument");
  *count = M->launches;
  return SHELL_OK;
}

extern "C" shell_status shell_node_features(shell_t* shell, const double* q, const double* v, float* X) {
  if (!shell || !q || !v || !X) return fail(SHELL_ERR_ARG, "NULL argument");
  Shell& s = *shell;
  k_node_features<<<(s.n_nodes + 127) / 128, 128, 0, s.stream>>>(s.n1, s.n2, s.grid.periodic_u, s.grid.periodic_v,
                                                                 q, s.d_rest, v, X);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

extern "C" shell_status shell_warm_targets(long long n_dof, const double* q_next, const double* q, const double* v,
                                           double dt, float* T, void* stream) {
  if (n_dof < 1 || !q_next || !q || !v || !T) return fail(SHELL_ERR_ARG, "invalid argument");
  k_targets<<<eblocks(n_dof), 256, 0, (cudaStream_t)stream>>>(n_dof, q_next, q, v, dt, T);
  BHEM_CUDA(cudaGetLastError());
  return SHELL_OK;
}

extern "C" shell_status shell_mlp_warm_start(shell_mlp_t* M, shell_t* shell, const double* q, const double* v,
                                             double dt, double* warm) {
  if (!shell || !q || !v || !warm) return fail(SHELL_ERR_ARG, "NULL argument");
  Shell& s = *shell;
  if (!M) {
    k_compose<<<eblocks((long long)s.n_nodes * kOut), 256, 0, s.stream>>>(s.n_nodes, q, v, dt, nullptr, nullptr,
                                                                          warm);
    BHEM_CUDA(cudaGetLastError());
    ++s.launches;
    return SHELL_OK;
  }
  static bool attr_set[64] = {false};
  if (!attr_set[s.device & 63]) {
    BHEM_CUDA(cudaFuncSetAttribute(k_mlp_warm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWarmSmem));
    attr_set[s.device & 63] = true;
  }
  WarmArgs A{};
  A.n_nodes = s.n_nodes;
  A.n1 = s.n1;
  A.n2 = s.n2;
  A.per_u = s.grid.periodic_u;
  A.per_v = s.grid.periodic_v;
  A.q = q;
  A.rest = s.d_rest;
  A.v = v;
  A.dt = dt;
  for (int l = 0; l < kLayers; ++l) A.bias[l] = M->b[l];
  A.norm = M->norm;
  A.warm = warm;
  A.err = M->err;
  A.polls = M->wait_polls;
  k_mlp_warm<<<(s.n_nodes + tc::kBM - 1) / tc::kBM, kWarmThreads, kWarmSmem, s.stream>>>(
      M->warm_maps[0], M->warm_maps[1], M->warm_maps[2], M->warm_maps[3], A);
  BHEM_CUDA(cudaGetLastError());
  ++M->launches;
  return SHELL_OK;
}
