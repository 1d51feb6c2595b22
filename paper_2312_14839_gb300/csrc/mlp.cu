// Learned Newton warm start: a per-node MLP 28 -> 256 -> 256 -> 256 -> 12 with GELU, BF16 weights
// and activations, FP32 accumulation on the tensor cores (mma.sync m16n8k16, BF16 in, FP32 out),
// trained with an MSE loss and Adam by the kernels of this file. The paper has no learning
// component; the implicit-Euler Newton solve of Sec. 6.1 stays the judge of every step.
//
// Node features (28, FP32): the node's 12 DOFs relative to rest (u = q - q_rest), its 12 velocity
// DOFs, and 4 means over its present edge neighbours: of u_nb - u_i for the position DOFs (a
// discrete Laplacian of the displacement, 3 values), and of the neighbours' position speed |v_nb|
// (their previous step's |dq| over dt, 1 value).
// Output (12): the node's update beyond the inertial predictor, q^{n+1} - q^n - dt v^n.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"

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
// Tensor-core GEMM: C[m][n] = sum_k A(m, k) B(n, k) (+ bias[n]); A, B BF16 with arbitrary element
// strides, FP32 accumulation. 64 x 64 tile per CTA of 4 warps (32 x 32 each), K in chunks of 32,
// split-K over gridDim.z with FP32 atomics into a zeroed C. Optional BF16 copy of GELU(C) or C.
// ------------------------------------------------------------------------------------------
struct GemmArgs {
  int M, N, K;
  const bf16* A;
  long long sAm, sAk;
  const bf16* B;
  long long sBn, sBk;
  float* C;
  long long ldc;
  bf16* Cb;
  long long ldcb;
  const float* bias;
  int gelu;
  int atomic;
};

constexpr int BM = 64, BN = 64, BK = 32, BKP = BK + 8;

__device__ __forceinline__ unsigned pack2(bf16 lo, bf16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// stage a 64 x 32 tile (rows r, columns k) of a strided operand; the loop order follows the unit
// stride so that global loads coalesce
__device__ __forceinline__ void stage_tile(bf16 (*S)[BKP], const bf16* __restrict__ P, long long s_row,
                                           long long s_k, int row0, int rows, int k0, int K, int tid) {
  const bf16 zero = __float2bfloat16(0.f);
  if (s_k == 1) {
    for (int e = tid; e < 64 * BK; e += 128) {
      const int r = e / BK, k = e % BK, gr = row0 + r, gk = k0 + k;
      S[r][k] = (gr < rows && gk < K) ? P[gr * s_row + gk] : zero;
    }
  } else {
    for (int e = tid; e < 64 * BK; e += 128) {
      const int r = e % 64, k = e / 64, gr = row0 + r, gk = k0 + k;
      S[r][k] = (gr < rows && gk < K) ? P[gr * s_row + gk * s_k] : zero;
    }
  }
}

__global__ void __launch_bounds__(128) k_gemm(GemmArgs G) {
  __shared__ bf16 As[BM][BKP];
  __shared__ bf16 Bs[BN][BKP];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kchunks = (G.K + BK - 1) / BK;
  const int per = (kchunks + gridDim.z - 1) / gridDim.z;
  const int kc0 = blockIdx.z * per, kc1 = min(kchunks, kc0 + per);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  for (int kc = kc0; kc < kc1; ++kc) {
    stage_tile(As, G.A, G.sAm, G.sAk, m0, G.M, kc * BK, G.K, tid);
    stage_tile(Bs, G.B, G.sBn, G.sBk, n0, G.N, kc * BK, G.K, tid);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned a[2][4], b[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm * 32 + mt * 16 + g;
        a[mt][0] = pack2(As[r][kk + 2 * t], As[r][kk + 2 * t + 1]);
        a[mt][1] = pack2(As[r + 8][kk + 2 * t], As[r + 8][kk + 2 * t + 1]);
        a[mt][2] = pack2(As[r][kk + 2 * t + 8], As[r][kk + 2 * t + 9]);
        a[mt][3] = pack2(As[r + 8][kk + 2 * t + 8], As[r + 8][kk + 2 * t + 9]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = wn * 32 + nt * 8 + g;
        b[nt][0] = pack2(Bs[c][kk + 2 * t], Bs[c][kk + 2 * t + 1]);
        b[nt][1] = pack2(Bs[c][kk + 2 * t + 8], Bs[c][kk + 2 * t + 9]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a[mt], b[nt]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = m0 + wm * 32 + mt * 16 + g + (e >= 2 ? 8 : 0);
        const int n = n0 + wn * 32 + nt * 8 + 2 * t + (e & 1);
        if (m >= G.M || n >= G.N) continue;
        float v = acc[mt][nt][e];
        if (G.bias && blockIdx.z == 0) v += G.bias[n];
        if (G.C) {
          if (G.atomic) atomicAdd(&G.C[m * G.ldc + n], v);
          else G.C[m * G.ldc + n] = v;
        }
        if (G.Cb) G.Cb[m * G.ldcb + n] = __float2bfloat16(G.gelu ? gelu(v) : v);
      }
}

// ------------------------------------------------------------------------------------------
// Element-wise kernels
// ------------------------------------------------------------------------------------------
// normalised BF16 input rows (gathered through idx when given); an index outside [0, data_rows)
// gives a zero row and raises the error flag
__global__ void k_input(int rows, const float* __restrict__ X, long long data_rows, const int* __restrict__ idx,
                        const float* __restrict__ norm, bf16* __restrict__ Xb, int* err) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * kInPad; e += gridDim.x * blockDim.x) {
    const int r = e / kInPad, c = e % kInPad;
    float v = 0.f;
    const long long src = idx ? (long long)idx[r] : r;
    if (src < 0 || src >= data_rows) {
      if (c == 0) atomicOr(err, 1);
    } else if (c < kIn) {
      v = (X[src * kIn + c] - norm[kNormInMean + c]) * norm[kNormInIstd + c];
    }
    Xb[e] = __float2bfloat16(v);
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
// zero in the padded columns
__global__ void k_loss(int rows, const float* __restrict__ Z, const float* __restrict__ T, long long data_rows,
                       const int* __restrict__ idx, const float* __restrict__ norm, float* __restrict__ dZ,
                       bf16* __restrict__ dZb, double* loss) {
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

// dZ = dA * GELU'(Z) (FP32 and BF16 copies)
__global__ void k_gelu_back(long long count, const float* __restrict__ dA, const float* __restrict__ Z,
                            float* __restrict__ dZ, bf16* __restrict__ dZb) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const float d = dA[e] * gelu_grad(Z[e]);
    dZ[e] = d;
    dZb[e] = __float2bfloat16(d);
  }
}

// db[n] += sum over rows of dZ[r][n]; CTA row y sums the 256-row slabs y, y + gridDim.y, ...
__global__ void k_colsum(int rows, int cols, const float* __restrict__ dZ, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= cols) return;
  float s = 0.f;
  for (int r0 = blockIdx.y * 256; r0 < rows; r0 += gridDim.y * 256) {
    const int r1 = min(rows, r0 + 256);
    for (int r = r0; r < r1; ++r) s += dZ[(long long)r * cols + n];
  }
  atomicAdd(&db[n], s);
}

// Adam (Kingma and Ba) on FP32 master parameters, refreshing the BF16 copy when given. Padded
// entries see zero gradients and stay zero.
__global__ void k_adam(long long count, float* __restrict__ w, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ wb, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const float gr = grad[e];
    const float mm = b1 * m[e] + (1.f - b1) * gr;
    const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    const float wn = w[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    w[e] = wn;
    if (wb) wb[e] = __float2bfloat16(wn);
  }
}

__global__ void k_to_bf16(long long count, const float* __restrict__ a, bf16* __restrict__ b) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    b[e] = __float2bfloat16(a[e]);
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
// launch. A CTA takes 32 nodes; activations stay in shared memory (BF16, as the GEMM path stores
// them), weights are read from L2 (every CTA reads the same 280 KB). Each output element is
// accumulated over K in the same k16 order and with the same epilogue as k_gemm, so the network
// output equals the unfused path's.
// ------------------------------------------------------------------------------------------
constexpr int kFR = 32;                 // nodes per CTA
constexpr int kLdX = kInPad + 8;        // padded row strides (bank-conflict-free fragment loads)
constexpr int kLdA = kHid + 8;

__device__ __forceinline__ unsigned lds_pair(const bf16* p) { return *reinterpret_cast<const unsigned*>(p); }
__device__ __forceinline__ unsigned ldg_pair(const bf16* p) { return __ldg(reinterpret_cast<const unsigned*>(p)); }

__global__ void __launch_bounds__(128)
k_mlp_warm(int n_nodes, int n1, int n2, int per_u, int per_v, const double* __restrict__ q,
           const double* __restrict__ rest, const double* __restrict__ v, double dt,
           const bf16* __restrict__ W0, const bf16* __restrict__ W1, const bf16* __restrict__ W2,
           const bf16* __restrict__ W3, const float* __restrict__ b0, const float* __restrict__ b1,
           const float* __restrict__ b2, const float* __restrict__ b3, const float* __restrict__ norm,
           double* __restrict__ warm) {
  __shared__ __align__(16) bf16 sX[kFR * kLdX];
  __shared__ __align__(16) bf16 sA[2][kFR * kLdA];
  __shared__ float sY[kFR][kOutPad];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  const int r0 = blockIdx.x * kFR;
  // features and normalisation (the arithmetic of k_node_features and k_input)
  if (tid < kFR) {
    const int i = r0 + tid;
    float f[kIn];
    if (i < n_nodes) node_features_of(i, n1, n2, per_u, per_v, q, rest, v, f);
    for (int c = 0; c < kInPad; ++c) {
      float x = 0.f;
      if (i < n_nodes && c < kIn) x = (f[c] - norm[kNormInMean + c]) * norm[kNormInIstd + c];
      sX[tid * kLdX + c] = __float2bfloat16(x);
    }
  }
  __syncthreads();
  // hidden layers: warp w computes output columns [64 w, 64 w + 64) of all 32 rows
  const bf16* in = sX;
  int ldin = kLdX, K = kInPad;
  for (int l = 0; l < kLayers - 1; ++l) {
    const bf16* W = l == 0 ? W0 : l == 1 ? W1 : W2;
    const float* bias = l == 0 ? b0 : l == 1 ? b1 : b2;
    float acc[2][8][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
    for (int kk = 0; kk < K; kk += 16) {
      unsigned a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const bf16* ar = in + (mt * 16 + g) * ldin + kk + 2 * t;
        a[mt][0] = lds_pair(ar);
        a[mt][1] = lds_pair(ar + 8 * ldin);
        a[mt][2] = lds_pair(ar + 8);
        a[mt][3] = lds_pair(ar + 8 * ldin + 8);
      }
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const bf16* br = W + (size_t)(warp * 64 + nt * 8 + g) * K + kk + 2 * t;
        const unsigned b[2] = {ldg_pair(br), ldg_pair(br + 8)};
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][nt], a[mt], b);
      }
    }
    bf16* out = sA[l & 1];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int m = mt * 16 + g + (e >= 2 ? 8 : 0);
          const int n = warp * 64 + nt * 8 + 2 * t + (e & 1);
          out[m * kLdA + n] = __float2bfloat16(gelu(acc[mt][nt][e] + bias[n]));
        }
    __syncthreads();
    in = out;
    ldin = kLdA;
    K = kHid;
  }
  // output layer (16 padded columns): warps 0 and 1 take 8 columns each
  if (warp < 2) {
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    for (int kk = 0; kk < kHid; kk += 16) {
      unsigned a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const bf16* ar = in + (mt * 16 + g) * kLdA + kk + 2 * t;
        a[mt][0] = lds_pair(ar);
        a[mt][1] = lds_pair(ar + 8 * kLdA);
        a[mt][2] = lds_pair(ar + 8);
        a[mt][3] = lds_pair(ar + 8 * kLdA + 8);
      }
      const bf16* br = W3 + (size_t)(warp * 8 + g) * kHid + kk + 2 * t;
      const unsigned b[2] = {ldg_pair(br), ldg_pair(br + 8)};
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt], a[mt], b);
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = mt * 16 + g + (e >= 2 ? 8 : 0);
        const int n = warp * 8 + 2 * t + (e & 1);
        sY[m][n] = acc[mt][e] + b3[n];
      }
  }
  __syncthreads();
  // warm = q + dt v + out_std * y + out_mean (the arithmetic of k_compose)
  for (int e = tid; e < kFR * kOut; e += blockDim.x) {
    const int r = e / kOut, c = e % kOut, i = r0 + r;
    if (i >= n_nodes) continue;
    const size_t gi = (size_t)i * 12 + c;
    const float y = sY[r][c] * norm[kNormOutStd + c] + norm[kNormOutMean + c];
    warm[gi] = q[gi] + dt * v[gi] + (double)y;
  }
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
  long long launches = 0;
  int step = 0;
  // parameters (padded; FP32 master copies, BF16 copies for the GEMMs), Adam moments, gradients
  float *W[kLayers] = {}, *b[kLayers] = {}, *gW[kLayers] = {}, *gb[kLayers] = {};
  float *mW[kLayers] = {}, *vW[kLayers] = {}, *mb[kLayers] = {}, *vb[kLayers] = {};
  bf16* Wb[kLayers] = {};
  // activations of the last forward pass, and their gradients
  bf16* Xb = nullptr;
  float* Z[kLayers] = {};
  bf16* Ab[kLayers] = {};
  float *dZ[kLayers] = {}, *dA = nullptr;
  bf16* dZb[kLayers] = {};
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
                  m->Z[l], m->Ab[l], m->dZ[l], m->dZb[l]};
    for (void* p : ps)
      if (p) cudaFree(p);
  }
  void* ps[] = {m->Xb, m->dA, m->Xraw, m->norm, m->loss, m->stats, m->err};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (m->h_loss) cudaFreeHost(m->h_loss);
  if (m->h_err) cudaFreeHost(m->h_err);
  delete m;
}

int eblocks(long long n) { return (int)std::min<long long>(4096, std::max(1LL, (n + 255) / 256)); }

shell_status gemm(shell_mlp_s& M, const GemmArgs& G, int ksplit, cudaStream_t st) {
  dim3 grid((G.N + BN - 1) / BN, (G.M + BM - 1) / BM, ksplit);
  k_gemm<<<grid, 128, 0, st>>>(G);
  BHEM_CUDA(cudaGetLastError());
  ++M.launches;
  return SHELL_OK;
}

// forward pass of the rows staged in M.Xb: Z_l (FP32 pre-activation), Ab_l (BF16 GELU)
shell_status forward(shell_mlp_s& M, int rows, cudaStream_t st) {
  const bf16* in = M.Xb;
  for (int l = 0; l < kLayers; ++l) {
    GemmArgs G{};
    G.M = rows;
    G.N = kDout[l];
    G.K = kDin[l];
    G.A = in;
    G.sAm = kDin[l];
    G.sAk = 1;
    G.B = M.Wb[l];
    G.sBn = kDin[l];
    G.sBk = 1;
    G.C = M.Z[l];
    G.ldc = kDout[l];
    G.Cb = l < kLayers - 1 ? M.Ab[l] : nullptr;
    G.ldcb = kDout[l];
    G.bias = M.b[l];
    G.gelu = l < kLayers - 1;
    BHEM_TRY(gemm(M, G, 1, st));
    in = M.Ab[l];
  }
  return SHELL_OK;
}

// parameter gradients of the loss whose dZ (last layer) k_loss left in M.dZ[3] / M.dZb[3]
shell_status backward(shell_mlp_s& M, int rows, cudaStream_t st) {
  for (int l = kLayers - 1; l >= 0; --l) {
    BHEM_CUDA(cudaMemsetAsync(M.gW[l], 0, sizeof(float) * kDout[l] * kDin[l], st));
    BHEM_CUDA(cudaMemsetAsync(M.gb[l], 0, sizeof(float) * kDout[l], st));
    // dW_l = dZ_l^T A_{l-1}
    GemmArgs G{};
    G.M = kDout[l];
    G.N = kDin[l];
    G.K = rows;
    G.A = M.dZb[l];
    G.sAm = 1;
    G.sAk = kDout[l];
    G.B = l > 0 ? M.Ab[l - 1] : M.Xb;
    G.sBn = 1;
    G.sBk = kDin[l];
    G.C = M.gW[l];
    G.ldc = kDin[l];
    G.atomic = 1;
    BHEM_TRY(gemm(M, G, std::max(1, std::min(64, rows / 512)), st));
    dim3 cg((kDout[l] + 127) / 128, std::min(1024, (rows + 255) / 256));
    k_colsum<<<cg, 128, 0, st>>>(rows, kDout[l], M.dZ[l], M.gb[l]);
    BHEM_CUDA(cudaGetLastError());
    ++M.launches;
    if (l == 0) break;
    // dA_{l-1} = dZ_l W_l, then dZ_{l-1} = dA_{l-1} GELU'(Z_{l-1})
    GemmArgs H{};
    H.M = rows;
    H.N = kDin[l];
    H.K = kDout[l];
    H.A = M.dZb[l];
    H.sAm = kDout[l];
    H.sAk = 1;
    H.B = M.Wb[l];
    H.sBn = 1;
    H.sBk = kDin[l];
    H.C = M.dA;
    H.ldc = kDin[l];
    BHEM_TRY(gemm(M, H, 1, st));
    const long long cnt = (long long)rows * kDout[l - 1];
    k_gelu_back<<<eblocks(cnt), 256, 0, st>>>(cnt, M.dA, M.Z[l - 1], M.dZ[l - 1], M.dZb[l - 1]);
    BHEM_CUDA(cudaGetLastError());
    ++M.launches;
  }
  return SHELL_OK;
}

shell_status stage_input(shell_mlp_s& M, const float* X, long long data_rows, const int* idx, int rows,
                         cudaStream_t st) {
  k_input<<<eblocks((long long)rows * kInPad), 256, 0, st>>>(rows, X, data_rows, idx, M.norm, M.Xb, M.err);
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
    BHEM_CUDA(cudaMemsetAsync(M.err, 0, sizeof(int), M.stream));
    BHEM_CUDA(cudaStreamSynchronize(M.stream));
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
  shell_status st = SHELL_OK;
  const size_t R = (size_t)max_rows;
  for (int l = 0; l < kLayers && st == SHELL_OK; ++l) {
    const size_t nw = (size_t)kDout[l] * kDin[l], nb = kDout[l];
    float** f32w[] = {&M->W[l], &M->gW[l], &M->mW[l], &M->vW[l]};
    for (float** p : f32w)
      if (st == SHELL_OK) st = malloc_zero(p, nw, M->stream);
    float** f32b[] = {&M->b[l], &M->gb[l], &M->mb[l], &M->vb[l]};
    for (float** p : f32b)
      if (st == SHELL_OK) st = malloc_zero(p, nb, M->stream);
    if (st == SHELL_OK) st = malloc_zero(&M->Wb[l], nw, M->stream);
    if (st == SHELL_OK) st = malloc_zero(&M->Z[l], R * kDout[l], M->stream);
    if (st == SHELL_OK) st = malloc_zero(&M->Ab[l], R * kDout[l], M->stream);
    if (st == SHELL_OK) st = malloc_zero(&M->dZ[l], R * kDout[l], M->stream);
    if (st == SHELL_OK) st = malloc_zero(&M->dZb[l], R * kDout[l], M->stream);
  }
  if (st == SHELL_OK) st = malloc_zero(&M->Xb, R * kInPad, M->stream);
  if (st == SHELL_OK) st = malloc_zero(&M->dA, R * kHid, M->stream);
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
    k_to_bf16<<<eblocks(n), 256, 0, M->stream>>>(n, M->W[l], M->Wb[l]);
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
  BHEM_TRY(stage_input(*M, X, rows, nullptr, rows, M->stream));
  BHEM_TRY(forward(*M, rows, M->stream));
  k_output<<<eblocks((long long)rows * kOut), 256, 0, M->stream>>>(rows, M->Z[kLayers - 1], M->norm, Y);
  BHEM_CUDA(cudaGetLastError());
  ++M->launches;
  return SHELL_OK;
}

extern "C" shell_status shell_mlp_gradients(shell_mlp_t* M, const float* X, const float* T, long long data_rows,
                                            const int* idx, int rows, double* loss) {
  if (!M || !X || !T || rows < 1 || rows > M->max_rows || data_rows < 1 || (!idx && rows > data_rows))
    return fail(SHELL_ERR_ARG, "invalid argument");
  BHEM_TRY(stage_input(*M, X, data_rows, idx, rows, M->stream));
  BHEM_TRY(forward(*M, rows, M->stream));
  BHEM_CUDA(cudaMemsetAsync(M->loss, 0, sizeof(double), M->stream));
  k_loss<<<eblocks((long long)rows * kOutPad), 256, 0, M->stream>>>(rows, M->Z[kLayers - 1], T, data_rows, idx,
                                                                    M->norm, M->dZ[kLayers - 1],
                                                                    M->dZb[kLayers - 1], M->loss);
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
  for (int l = 0; l < kLayers; ++l) {
    const long long nw = (long long)kDout[l] * kDin[l];
    k_adam<<<eblocks(nw), 256, 0, M->stream>>>(nw, M->W[l], M->gW[l], M->mW[l], M->vW[l], M->Wb[l], lr, b1, b2, eps,
                                               c1, c2);
    k_adam<<<eblocks(kDout[l]), 256, 0, M->stream>>>(kDout[l], M->b[l], M->gb[l], M->mb[l], M->vb[l], nullptr, lr,
                                                     b1, b2, eps, c1, c2);
    M->launches += 2;
  }
  BHEM_CUDA(cudaGetLastError());
  return loss ? finish(*M, loss) : SHELL_OK;
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
  k_mlp_warm<<<(s.n_nodes + kFR - 1) / kFR, 128, 0, s.stream>>>(
      s.n_nodes, s.n1, s.n2, s.grid.periodic_u, s.grid.periodic_v, q, s.d_rest, v, dt, M->Wb[0], M->Wb[1],
      M->Wb[2], M->Wb[3], M->b[0], M->b[1], M->b[2], M->b[3], M->norm, warm);
  BHEM_CUDA(cudaGetLastError());
  ++M->launches;
  return SHELL_OK;
}
