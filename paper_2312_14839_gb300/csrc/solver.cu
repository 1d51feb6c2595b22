// Linear-algebra kernels of the implicit-Euler Newton step (Sec. 6.1): 12x12 BSR SpMV, block-
// Jacobi preconditioner, PCG with device-resident scalars, consistent-mass products and the
// Newton residual g = dV/dq + M (q - y)/dt^2 - F. No kernel waits on another CTA: grid
// reductions use the last-CTA ticket of grid_reduce.
#include <algorithm>

#include "common.cuh"

namespace bhem {

int grid_for(long long work, int per_block) {
  long long b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 0x7fffffffLL) b = 0x7fffffffLL;
  return (int)b;
}

// ------------------------------------------------------------------------------------------
// BSR SpMV  y = (A + tau D) p on free DOFs (y = 0 on fixed DOFs), fused with p . y; tau D is
// the regulariser shift per DOF kind (zero without regularisation).
// Each 12x12 block row is read by TPR threads, one 16-byte chunk of one row per thread, so the
// threads of a block row stream the block's 576 (FP32) or 1152 (FP64) bytes contiguously.
// ------------------------------------------------------------------------------------------
template <typename Rm> struct Chunk;
template <> struct Chunk<float> { using T = float4; static constexpr int E = 4; };
template <> struct Chunk<double> { using T = double2; static constexpr int E = 2; };

// dot of one 16-byte matrix chunk with the matching entries of x, both in the matrix precision
// (x is an FP32 copy for FP32 matrices: an FP64->FP32 conversion per product would run on the
// narrow FP64 pipe)
__device__ __forceinline__ float chunk_dot(float4 a, const float* __restrict__ x) {
  const float4 xv = *reinterpret_cast<const float4*>(x);
  return a.x * xv.x + a.y * xv.y + a.z * xv.z + a.w * xv.w;
}
__device__ __forceinline__ double chunk_dot(double2 a, const double* __restrict__ x) {
  const double2 x0 = *reinterpret_cast<const double2*>(x);
  return a.x * x0.x + a.y * x0.y;
}

constexpr int kSpmvThreads = 288;

template <typename Rm>
__global__ void __launch_bounds__(kSpmvThreads)
k_spmv(int n, const int* __restrict__ rp, const int* __restrict__ col, const Rm* __restrict__ val,
       const Rm* __restrict__ x, const double* __restrict__ xd, Shift4 td,
       const unsigned char* __restrict__ mask, double* __restrict__ y, PcgState* st, Reduce red) {
  using CT = typename Chunk<Rm>::T;
  constexpr int E = Chunk<Rm>::E;
  constexpr int NC = 12 / E;            // chunks per row
  constexpr int TPR = 12 * NC;          // threads per block row
  constexpr int RPC = kSpmvThreads / TPR;
  if (st && st->done) return;
  __shared__ Rm sacc[kSpmvThreads];
  const int t = threadIdx.x;
  const int br = t / TPR, w = t % TPR, r = w / NC, cc = w % NC;
  const int i = blockIdx.x * RPC + br;
  Rm acc = 0;
  if (i < n) {
    const int k0 = rp[i], k1 = rp[i + 1];
    // a node of the structured grid couples to at most 9 nodes: issue all block loads first
    constexpr int U = 9;
    CT v[U];
    int j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u;
      if (k < k1) {
        j[u] = col[k];
        v[u] = __ldcs(reinterpret_cast<const CT*>(val + (size_t)k * 144 + r * 12 + cc * E));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < k1) acc += chunk_dot(v[u], x + (size_t)j[u] * 12 + cc * E);
    for (int k = k0 + U; k < k1; ++k) {
      CT w = __ldcs(reinterpret_cast<const CT*>(val + (size_t)k * 144 + r * 12 + cc * E));
      acc += chunk_dot(w, x + (size_t)col[k] * 12 + cc * E);
    }
  }
  sacc[t] = acc;
  __syncthreads();
  double part = 0.0;
  if (i < n && cc == 0) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NC; ++c) s += (double)sacc[t + c];
    const size_t gi = (size_t)i * 12 + r;
    const double xi = xd ? xd[gi] : (double)x[gi];
    double yi = s;
    yi += td.v[r / 3] * xi;
    if (mask && mask[gi]) yi = 0.0;
    y[gi] = yi;
    part = xi * yi;
  }
  if (st) {
    double v1[1] = {part};
    if (grid_reduce<1>(v1, red, &st->pq, gridDim.x) && threadIdx.x == 0) {
      double pq = st->pq;
      if (!(pq > 0.0)) {
        st->negcurv = 1;
        st->done = 1;
        st->alpha = 0.0;
      } else {
        st->alpha = st->rz / pq;
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Block-Jacobi: D_i = (A_ii masked + tau D)^{-1} by Cholesky; a block that is not SPD falls back
// to the inverse of its diagonal. 12 threads per node (one row each), 16 nodes per CTA.
// ------------------------------------------------------------------------------------------
template <typename Rm, typename Rd>
__global__ void __launch_bounds__(192)
k_precond(int n, const int* __restrict__ diag_block, const Rm* __restrict__ val,
          const unsigned char* __restrict__ mask, Shift4 td, Rd* __restrict__ Dinv) {
  __shared__ Rd sL[16][12][13];
  __shared__ Rd sW[16][12][13];
  __shared__ Rd sdiag[16][12];
  __shared__ int sok[16];
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  const bool active = i < n;
  if (active) {
    const Rm* B = val + (size_t)diag_block[i] * 144;
    const bool fa = mask && mask[(size_t)i * 12 + a];
    for (int b = 0; b < 12; ++b) {
      const bool fb = mask && mask[(size_t)i * 12 + b];
      Rd v = (Rd)B[a * 12 + b];
      if (fa || fb) v = (a == b) ? (Rd)1 : (Rd)0;
      else if (a == b) v += (Rd)td.v[a / 3];
      sL[ln][a][b] = v;
    }
    sdiag[ln][a] = sL[ln][a][a];
  }
  if (a == 0) sok[ln] = 1;
  __syncthreads();
  for (int j = 0; j < 12; ++j) {
    if (active && a == j && sok[ln]) {
      Rd sacc = sL[ln][j][j];
      for (int k = 0; k < j; ++k) sacc -= sL[ln][j][k] * sL[ln][j][k];
      if (!(sacc > (Rd)0)) sok[ln] = 0;
      else sL[ln][j][j] = sqrt(sacc);
    }
    __syncthreads();
    if (active && a > j && sok[ln]) {
      Rd u = sL[ln][a][j];
      for (int k = 0; k < j; ++k) u -= sL[ln][a][k] * sL[ln][j][k];
      sL[ln][a][j] = u / sL[ln][j][j];
    }
    __syncthreads();
  }
  const bool ok = active && sok[ln];
  if (ok) {
    // column a of W = L^{-1} (lower triangular) by forward substitution
    for (int r = 0; r < 12; ++r) {
      if (r < a) { sW[ln][r][a] = 0; continue; }
      Rd u = (r == a) ? (Rd)1 : (Rd)0;
      for (int k = a; k < r; ++k) u -= sL[ln][r][k] * sW[ln][k][a];
      sW[ln][r][a] = u / sL[ln][r][r];
    }
  }
  __syncthreads();
  if (!active) return;
  Rd* D = Dinv + (size_t)i * 144 + a * 12;
  if (ok) {
    for (int b = 0; b < 12; ++b) {   // D = W^T W, row a
      Rd sacc = 0;
      for (int k = (a > b ? a : b); k < 12; ++k) sacc += sW[ln][k][a] * sW[ln][k][b];
      D[b] = sacc;
    }
  } else {
    const Rd d = sdiag[ln][a];
    for (int b = 0; b < 12; ++b) D[b] = (a == b) ? (d > (Rd)0 ? (Rd)1 / d : (Rd)1) : (Rd)0;
  }
}

// FP32 block-Jacobi set-up with one thread per node: the same Cholesky, forward substitution and
// W^T W as k_precond, in the same operation order, held in registers, so no step waits on a
// barrier. The 12x12 diagonal block is read as 36 16-byte loads.
__global__ void __launch_bounds__(128)
k_precond32_thread(int n, const int* __restrict__ diag_block, const float* __restrict__ val,
                   const unsigned char* __restrict__ mask, Shift4 td, float* __restrict__ Dinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float L[12][12];
  const float4* B4 = reinterpret_cast<const float4*>(val + (size_t)diag_block[i] * 144);
#pragma unroll
  for (int e4 = 0; e4 < 36; ++e4) {
    const float4 v = B4[e4];
    L[e4 / 3][(e4 % 3) * 4 + 0] = v.x;
    L[e4 / 3][(e4 % 3) * 4 + 1] = v.y;
    L[e4 / 3][(e4 % 3) * 4 + 2] = v.z;
    L[e4 / 3][(e4 % 3) * 4 + 3] = v.w;
  }
  bool fm[12];
#pragma unroll
  for (int a = 0; a < 12; ++a) fm[a] = mask && mask[(size_t)i * 12 + a];
  float dg[12];
#pragma unroll
  for (int a = 0; a < 12; ++a) {
#pragma unroll
    for (int b = 0; b < 12; ++b) {
      if (fm[a] || fm[b]) L[a][b] = (a == b) ? 1.f : 0.f;
      else if (a == b) L[a][b] += (float)td.v[a / 3];
    }
    dg[a] = L[a][a];
  }
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    float sacc = L[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) sacc -= L[j][k] * L[j][k];
    if (!(sacc > 0.f)) ok = false;
    L[j][j] = sqrtf(sacc);
#pragma unroll
    for (int a = j + 1; a < 12; ++a) {
      float u = L[a][j];
#pragma unroll
      for (int k = 0; k < j; ++k) u -= L[a][k] * L[j][k];
      L[a][j] = u / L[j][j];
    }
  }
  float* D = Dinv + (size_t)i * 144;
  if (!ok) {
#pragma unroll
    for (int a = 0; a < 12; ++a)
#pragma unroll
      for (int b = 0; b < 12; ++b) D[a * 12 + b] = (a == b) ? (dg[a] > 0.f ? 1.f / dg[a] : 1.f) : 0.f;
    return;
  }
  // W = L^{-1} (lower triangular) by forward substitution, column by column
  float W[12][12];
#pragma unroll
  for (int a = 0; a < 12; ++a)
#pragma unroll
    for (int r = 0; r < 12; ++r) {
      if (r < a) { W[r][a] = 0.f; continue; }
      float u = (r == a) ? 1.f : 0.f;
#pragma unroll
      for (int k = a; k < r; ++k) u -= L[r][k] * W[k][a];
      W[r][a] = u / L[r][r];
    }
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    float row[12];
#pragma unroll
    for (int b = 0; b < 12; ++b) {
      float sacc = 0.f;
#pragma unroll
      for (int k = (a > b ? a : b); k < 12; ++k) sacc += W[k][a] * W[k][b];
      row[b] = sacc;
    }
    float4* d4 = reinterpret_cast<float4*>(D + a * 12);
    d4[0] = make_float4(row[0], row[1], row[2], row[3]);
    d4[1] = make_float4(row[4], row[5], row[6], row[7]);
    d4[2] = make_float4(row[8], row[9], row[10], row[11]);
  }
}

// Per DOF kind k (x, x_,1, x_,2, x_,12), over free DOFs: sum |A_ii|, count, min A_ii. They give the
// regulariser scale (mean |A_ii| of the kind) and tell which regulariser levels leave a
// non-positive diagonal entry (such a matrix cannot be positive definite).
template <typename Rm>
__global__ void k_diag_check(int n, const int* __restrict__ diag_block, const Rm* __restrict__ val,
                             const unsigned char* __restrict__ mask, double* out12, Reduce red) {
  double v[12];
#pragma unroll
  for (int q = 0; q < 4; ++q) { v[3 * q] = 0.0; v[3 * q + 1] = 0.0; v[3 * q + 2] = INFINITY; }
  // grid-stride over the DOFs, the loads of U strides issued before their use (a few CTAs per SM:
  // the FP64 block reductions below are the expensive part on this GPU)
  constexpr int U = 4;
  const int m = n * 12, stride = gridDim.x * blockDim.x;
  for (int k0 = blockIdx.x * blockDim.x + threadIdx.x; k0 < m; k0 += U * stride) {
    Rm d[U];
    bool use[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * stride;
      use[u] = k < m && !(mask && mask[k]);
      if (use[u]) d[u] = val[(size_t)diag_block[k / 12] * 144 + (k % 12) * 13];
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (use[u]) {
        const int q = ((k0 + u * stride) % 12) / 3;
        const double dd = (double)d[u];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
          if (qq == q) { v[3 * qq] += fabs(dd); v[3 * qq + 1] += 1.0; v[3 * qq + 2] = fmin(v[3 * qq + 2], dd); }
      }
  }
  grid_reduce<12>(v, red, out12, gridDim.x, 0x924u);   // the min entries: 2, 5, 8, 11
}

// ------------------------------------------------------------------------------------------
// PCG kernels: 12 threads per node, 16 nodes per CTA.
// ------------------------------------------------------------------------------------------
constexpr int kNodeThreads = 192;

template <typename Rd>
__device__ __forceinline__ double apply_block(const Rd* __restrict__ D, const Rd* sr, int a) {
  Rd s = 0;
#pragma unroll
  for (int c = 0; c < 12; ++c) s += D[a * 12 + c] * sr[c];
  return (double)s;
}

template <typename Rd>
__global__ void __launch_bounds__(kNodeThreads)
k_pcg_init(int n, const double* __restrict__ rhs, const Rd* __restrict__ Dinv,
           const unsigned char* __restrict__ mask, double* __restrict__ x, double* __restrict__ r,
           double* __restrict__ z, double* __restrict__ p, Rd* __restrict__ pr, double rtol2,
           int fixed, PcgState* st, Reduce red) {
  __shared__ Rd sr[16][12];
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  const size_t gi = (size_t)i * 12 + a;
  double ri = 0.0, zi = 0.0;
  if (i < n) {
    ri = (mask && mask[gi]) ? 0.0 : rhs[gi];
    x[gi] = 0.0;
    r[gi] = ri;
    sr[ln][a] = (Rd)ri;
  }
  __syncthreads();
  if (i < n) {
    zi = (mask && mask[gi]) ? 0.0 : apply_block<Rd>(Dinv + (size_t)i * 144, sr[ln], a);
    z[gi] = zi;
    p[gi] = zi;
    if (pr) pr[gi] = (Rd)zi;
  }
  double v[2] = {ri * zi, ri * ri};
  double out[2];
  if (grid_reduce<2>(v, red, out, gridDim.x) && threadIdx.x == 0) {
    st->rz = out[0];
    st->bb = out[1];
    st->rr = out[1];
    st->rtol2 = rtol2;
    st->fixed = fixed;
    st->iters = 0;
    st->negcurv = 0;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->pq = 0.0;
    st->done = (out[1] == 0.0) ? 1 : 0;
  }
}

template <typename Rd>
__global__ void __launch_bounds__(kNodeThreads)
k_pcg_update(int n, double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
             const double* __restrict__ p, const double* __restrict__ Ap,
             const Rd* __restrict__ Dinv, const unsigned char* __restrict__ mask, PcgState* st,
             Reduce red) {
  if (st->done) return;
  __shared__ Rd sr[16][12];
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  const size_t gi = (size_t)i * 12 + a;
  const double alpha = st->alpha;
  double ri = 0.0, zi = 0.0;
  if (i < n) {
    x[gi] += alpha * p[gi];
    ri = r[gi] - alpha * Ap[gi];
    r[gi] = ri;
    sr[ln][a] = (Rd)ri;
  }
  __syncthreads();
  if (i < n) {
    zi = (mask && mask[gi]) ? 0.0 : apply_block<Rd>(Dinv + (size_t)i * 144, sr[ln], a);
    z[gi] = zi;
  }
  double v[2] = {ri * zi, ri * ri};
  double out[2];
  if (grid_reduce<2>(v, red, out, gridDim.x) && threadIdx.x == 0) {
    const double rz_new = out[0];
    st->rr = out[1];
    st->iters += 1;
    st->beta = rz_new / st->rz;
    st->rz = rz_new;
    if (st->fixed == 0 && out[1] <= st->rtol2 * st->bb) st->done = 1;
    if (rz_new == 0.0) st->done = 1;
  }
}

__global__ void k_pcg_pupdate(int m, const double* __restrict__ z, double* __restrict__ p,
                              float* __restrict__ p32, const PcgState* st) {
  if (st->done) return;
  const double beta = st->beta;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const double v = z[k] + beta * p[k];
    p[k] = v;
    if (p32) p32[k] = (float)v;
  }
}

__global__ void k_to_float(int m, const double* __restrict__ a, float* __restrict__ b) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) b[k] = (float)a[k];
}

// ------------------------------------------------------------------------------------------
// Mixed-precision PCG (FP32 matrix, FP32 vectors, dot products as exact FP32 products summed in
// double-float): no FP64-pipe work per element. 36 threads per block row as in k_spmv.
// ------------------------------------------------------------------------------------------
// Programmatic dependent launch: a kernel of the PCG iteration may be launched while the previous
// kernel of its stream is still finishing (its CTAs are scheduled early); before it reads or
// writes any memory it waits here until the previous kernel has completed and its writes are
// visible. Without such a launch the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Launch of kernel k, with programmatic dependent launch when pdl is set.
template <typename... KArgs, typename... Args>
static cudaError_t launch_k(bool pdl, void (*k)(KArgs...), unsigned grid, unsigned block, cudaStream_t st,
                            Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}
struct Shift4f { float v[4]; };

// acc += a . x as an explicit FMA chain (both FP32 SpMV kernels round identically)
__device__ __forceinline__ float dot4_acc(float acc, const float4 a, const float4 x) {
  acc = __fmaf_rn(a.x, x.x, acc);
  acc = __fmaf_rn(a.y, x.y, acc);
  acc = __fmaf_rn(a.z, x.z, acc);
  return __fmaf_rn(a.w, x.w, acc);
}

__global__ void __launch_bounds__(kSpmvThreads)
k_spmv32(int n, const int* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ val,
         const float* __restrict__ x, Shift4f td, const unsigned char* __restrict__ mask,
         float* __restrict__ y, PcgState* st, Reduce red) {
  constexpr int NC = 3, TPR = 36, RPC = kSpmvThreads / TPR;
  pdl_wait();
  // the solve's stop flag is read together with the row pointers, which the block loads wait
  // for anyway, and tested before those loads: a launch after the solve stopped streams nothing
  // (the flag is written only by the last CTA of a launch, after every CTA read it)
  const int done = st ? st->done : 0;
  __shared__ float sacc[kSpmvThreads];
  const int t = threadIdx.x;
  const int br = t / TPR, w = t % TPR, r = w / NC, cc = w % NC;
  const int i = blockIdx.x * RPC + br;
  const int k0 = i < n ? rp[i] : 0, k1 = i < n ? rp[i + 1] : 0;
  if (done) return;
  float acc = 0.f;
  if (i < n) {
    constexpr int U = 9;
    float4 v[U];
    int j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u;
      if (k < k1) {
        j[u] = col[k];
        v[u] = __ldcs(reinterpret_cast<const float4*>(val + (size_t)k * 144 + r * 12 + cc * 4));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < k1) {
        const float4 xv = *reinterpret_cast<const float4*>(x + (size_t)j[u] * 12 + cc * 4);
        acc = dot4_acc(acc, v[u], xv);
      }
    for (int k = k0 + U; k < k1; ++k) {
      const float4 a = __ldcs(reinterpret_cast<const float4*>(val + (size_t)k * 144 + r * 12 + cc * 4));
      const float4 xv = *reinterpret_cast<const float4*>(x + (size_t)col[k] * 12 + cc * 4);
      acc = dot4_acc(acc, a, xv);
    }
  }
  sacc[t] = acc;
  __syncthreads();
  F2 part{0.f, 0.f};
  if (i < n && cc == 0) {
    const size_t gi = (size_t)i * 12 + r;
    const float xi = x[gi];
    float yi = (sacc[t] + sacc[t + 1]) + sacc[t + 2];
    yi = __fmaf_rn(st ? st->td[r / 3] : td.v[r / 3], xi, yi);   // PCG: the solve's shift
    if (mask && mask[gi]) yi = 0.f;
    y[gi] = yi;
    part = f2_prod(xi, yi);
  }
  if (st) {
    F2 v1[1] = {part};
    double out[1];
    if (grid_reduce_f2<1>(v1, red, out, gridDim.x) && threadIdx.x == 0) {
      st->pq = out[0];
      if (!(out[0] > 0.0)) {
        st->negcurv = 1;
        st->done = 1;
        st->alpha = 0.0;
      } else {
        st->alpha = st->rz / out[0];
      }
    }
  }
}

// k_spmv32 reading each node row's blocks left of the diagonal as transposes (an opt-in form of
// the mixed-precision plain SpMV; Shell::spmv_sym). The row's u-th block left of the diagonal is
// the transpose of block kt[u] = (j, i) of row j < i (the row's transposed-block slots): the same
// values when the assembled matrix is symmetric (exactly with the colour-ordered assembly, whose
// sums over patches run in the same order for (i, j) and (j, i); to rounding with the atomic
// one). Row j read those values moments before (rows run in order across the grid), so they come
// from L2, and DRAM streams only the diagonal and upper blocks. Each thread copies its 16-byte
// pieces of the row's blocks, and the row's first three threads the x pieces they multiply, into
// shared memory with cp.async (L2 only, no registers held while the copies fly, blocks and x in
// one group), and reads them back, the blocks left of the diagonal transposed. The arithmetic and its order per
// row are those of k_spmv32, so the two agree bit for bit on an exactly symmetric matrix.
constexpr int kSymBlocks = 9;   // blocks of a node row staged (a row has at most 9)
// per CTA: the 8 rows' blocks and x pieces, 44,928 B (4 CTAs per SM)
constexpr size_t kSpmvSymSmem = sizeof(float) * (kSpmvThreads / 36) * kSymBlocks * (144 + 12);

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}

__global__ void __launch_bounds__(kSpmvThreads)
k_spmv32_sym(int n, const int* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ val,
             const int* __restrict__ tpos, const int* __restrict__ dg, const float* __restrict__ x, Shift4f td,
             const unsigned char* __restrict__ mask, float* __restrict__ y, PcgState* st, Reduce red) {
  constexpr int NC = 3, TPR = 36, RPC = kSpmvThreads / TPR;
  // the solve's stop flag is read together with the row pointers, which the block loads wait
  // for anyway, and tested before those loads: a launch after the solve stopped streams nothing
  // (the flag is written only by the last CTA of a launch, after every CTA read it)
  const int done = st ? st->done : 0;
  __shared__ float sacc[kSpmvThreads];
  extern __shared__ __align__(16) float sblk[];   // [RPC][kSymBlocks][144]
  const int t = threadIdx.x;
  const int br = t / TPR, w = t % TPR, r = w / NC, cc = w % NC;
  const int i = blockIdx.x * RPC + br;
  const int k0 = i < n ? rp[i] : 0, k1 = i < n ? rp[i + 1] : 0;
  // the diagonal block (blocks before it are left of it) and the row's transposed-block slots,
  // read beside the row pointers
  const int kd = i < n ? dg[i] : k0;
  int4 t0 = make_int4(0, 0, 0, 0), t1 = t0;
  if (i < n) {
    t0 = __ldg(reinterpret_cast<const int4*>(tpos) + 2 * i);
    t1 = __ldg(reinterpret_cast<const int4*>(tpos) + 2 * i + 1);
  }
  if (done) return;
  float* rowb = sblk + (size_t)br * kSymBlocks * 144;
  float* rowx = sblk + (size_t)RPC * kSymBlocks * 144 + (size_t)br * kSymBlocks * 12;
  const int nlow = kd - k0;
  if (i < n) {
    const int kt[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
    for (int u = 0; u < kSymBlocks; ++u) {
      const int k = k0 + u;
      if (k < k1) {
        const int kb = (u < 8 && u < nlow) ? kt[u < 8 ? u : 0] : k;
        cp_async16(rowb + u * 144 + r * 12 + cc * 4, val + (size_t)kb * 144 + r * 12 + cc * 4);
        // the piece x_j[4 cc .. 4 cc + 3] that the row's threads of column piece cc share
        if (r == 0) cp_async16(rowx + u * 12 + cc * 4, x + (size_t)col[k] * 12 + cc * 4);
      }
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  float acc = 0.f;
  if (i < n) {
#pragma unroll
    for (int u = 0; u < kSymBlocks; ++u)
      if (k0 + u < k1) {
        float4 a;
        if (u < nlow) {
          const float* b = rowb + u * 144 + cc * 48 + r;   // block (i, j) = (block (j, i))^T
          a = make_float4(b[0], b[12], b[24], b[36]);
        } else {
          a = *reinterpret_cast<const float4*>(rowb + u * 144 + r * 12 + cc * 4);
        }
        const float4 xv = *reinterpret_cast<const float4*>(rowx + u * 12 + cc * 4);
        acc = dot4_acc(acc, a, xv);
      }
    for (int k = k0 + kSymBlocks; k < k1; ++k) {
      const float4 a = __ldcg(reinterpret_cast<const float4*>(val + (size_t)k * 144 + r * 12 + cc * 4));
      const float4 xv = *reinterpret_cast<const float4*>(x + (size_t)col[k] * 12 + cc * 4);
      acc = dot4_acc(acc, a, xv);
    }
  }
  sacc[t] = acc;
  __syncthreads();
  F2 part{0.f, 0.f};
  if (i < n && cc == 0) {
    const size_t gi = (size_t)i * 12 + r;
    const float xi = x[gi];
    float yi = (sacc[t] + sacc[t + 1]) + sacc[t + 2];
    yi = __fmaf_rn(st ? st->td[r / 3] : td.v[r / 3], xi, yi);   // PCG: the solve's shift
    if (mask && mask[gi]) yi = 0.f;
    y[gi] = yi;
    part = f2_prod(xi, yi);
  }
  if (st) {
    F2 v1[1] = {part};
    double out[1];
    if (grid_reduce_f2<1>(v1, red, out, gridDim.x) && threadIdx.x == 0) {
      st->pq = out[0];
      if (!(out[0] > 0.0)) {
        st->negcurv = 1;
        st->done = 1;
        st->alpha = 0.0;
      } else {
        st->alpha = st->rz / out[0];
      }
    }
  }
}

// The SpMV of a mixed-precision PCG iteration with the search-direction update folded in: it
// gathers z instead of p and forms, per own row, p = z + beta p (the arithmetic of
// k_pcg32_pupdate4) and Ap = (A + tau D) z + beta Ap, which equals (A + tau D) p by linearity, so
// no separate p-update launch is needed; then p.Ap and alpha as in k_spmv32. The recurrence for
// Ap carries its rounding from one iteration to the next instead of recomputing A p. Used for
// shells of at most kFoldMaxNodes nodes, where the saved launch is a large part of an iteration
// (280 x 5: 1.15 against 1.23 ms per Newton iteration; 30 x 30 twist: 532 against 504 steps/s);
// at 256 x 256 the own-row reads at the end of every CTA cost more than the p-update kernel
// (8.20 against 8.06 ms).
__global__ void __launch_bounds__(kSpmvThreads)
k_spmv32_pcg(int n, const int* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ val,
             const float* __restrict__ x, const unsigned char* __restrict__ mask, float* __restrict__ p,
             float* __restrict__ y, PcgState* st, Reduce red) {
  constexpr int NC = 3, TPR = 36, RPC = kSpmvThreads / TPR;
  // the solve's stop flag is read together with the row pointers, which the block loads wait
  // for anyway, and tested before those loads: a launch after the solve stopped streams nothing
  // (the flag is written only by the last CTA of a launch, after every CTA read it)
  const int done = st->done;
  __shared__ float sacc[kSpmvThreads];
  const int t = threadIdx.x;
  const int br = t / TPR, w = t % TPR, r = w / NC, cc = w % NC;
  const int i = blockIdx.x * RPC + br;
  const int k0 = i < n ? rp[i] : 0, k1 = i < n ? rp[i + 1] : 0;
  if (done) return;
  float acc = 0.f;
  if (i < n) {
    constexpr int U = 9;
    float4 v[U];
    int j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u;
      if (k < k1) {
        j[u] = col[k];
        v[u] = __ldcs(reinterpret_cast<const float4*>(val + (size_t)k * 144 + r * 12 + cc * 4));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < k1) {
        const float4 xv = *reinterpret_cast<const float4*>(x + (size_t)j[u] * 12 + cc * 4);
        acc = dot4_acc(acc, v[u], xv);
      }
    for (int k = k0 + U; k < k1; ++k) {
      const float4 a = __ldcs(reinterpret_cast<const float4*>(val + (size_t)k * 144 + r * 12 + cc * 4));
      const float4 xv = *reinterpret_cast<const float4*>(x + (size_t)col[k] * 12 + cc * 4);
      acc = dot4_acc(acc, a, xv);
    }
  }
  sacc[t] = acc;
  __syncthreads();
  F2 part{0.f, 0.f};
  if (i < n && cc == 0) {
    // x is z here: w = (A + tau D) z, then p = z + beta p and q = w + beta q (q = A p by linearity;
    // the first iteration of a solve takes p = z, q = w)
    const size_t gi = (size_t)i * 12 + r;
    const float zi = x[gi];
    float wi = (sacc[t] + sacc[t + 1]) + sacc[t + 2];
    wi = __fmaf_rn(st->td[r / 3], zi, wi);
    if (mask && mask[gi]) wi = 0.f;
    float pi = zi, qi = wi;
    if (st->iters > 0) {
      const float bf = (float)st->beta;
      pi = fmaf(bf, p[gi], zi);
      qi = fmaf(bf, y[gi], wi);
    }
    p[gi] = pi;
    y[gi] = qi;
    part = f2_prod(pi, qi);
  }
  {
    F2 v1[1] = {part};
    double out[1];
    if (grid_reduce_f2<1>(v1, red, out, gridDim.x) && threadIdx.x == 0) {
      st->pq = out[0];
      if (!(out[0] > 0.0)) {
        st->negcurv = 1;
        st->done = 1;
        st->alpha = 0.0;
      } else {
        st->alpha = st->rz / out[0];
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// FP32 BSR SpMV, TMA-pipelined persistent form. A CTA owns a contiguous range of row groups
// (8 block rows each); the values of one group are contiguous in val, so one bulk asynchronous
// copy (cp.async.bulk, completion counted on an mbarrier) moves them into one stage of a
// shared-memory ring. kTmaStages groups are in flight while the CTA computes from the oldest
// stage; x is gathered through L1/L2. Same arithmetic and summation order per row as k_spmv32.
// Every mbarrier wait is bounded: on expiry the kernel raises ERRBIT_TIMEOUT, waits (bounded)
// for the copies it issued, and leaves.
// ------------------------------------------------------------------------------------------
constexpr int kTmaRows = 8, kTmaThreads = kTmaRows * 36, kTmaStages = 4;
constexpr unsigned kTmaChunk = 32768u;   // bytes per bulk copy instruction
constexpr int kWaitPolls = kDefaultWaitPolls;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, int polls = kWaitPolls) {
  for (int i = 0; i < polls; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(kTmaThreads, 1)
k_spmv32_tma(int n, const int* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ val,
             const float* __restrict__ x, Shift4f td, const unsigned char* __restrict__ mask,
             float* __restrict__ y, PcgState* st, Reduce red, int stage_floats, int* err, int polls) {
  extern __shared__ __align__(128) float sval[];
  __shared__ __align__(8) unsigned long long bar[kTmaStages];
  __shared__ float sacc[kTmaThreads];
  if (st && st->done) return;
  const int t = threadIdx.x;
  const int ngroups = (n + kTmaRows - 1) / kTmaRows;
  const int per = (ngroups + gridDim.x - 1) / gridDim.x;
  const int g0 = min(ngroups, blockIdx.x * per), g1 = min(ngroups, g0 + per);
  if (t == 0) {
    for (int q = 0; q < kTmaStages; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bar[q])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();
  // thread 0 issues the copy of group g into stage q
  auto issue = [&](int g, int q) {
    const int i0 = g * kTmaRows, i1 = min(n, i0 + kTmaRows);
    const long long k0 = rp[i0], k1 = rp[i1];
    const unsigned bytes = (unsigned)((k1 - k0) * 576);
    const unsigned b = smem_addr(&bar[q]);
    unsigned long long state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;\n"
                 : "=l"(state)
                 : "r"(b), "r"(bytes)
                 : "memory");
    const char* src = reinterpret_cast<const char*>(val + k0 * 144);
    const unsigned dst = smem_addr(sval + (size_t)q * stage_floats);
    for (unsigned off = 0; off < bytes; off += kTmaChunk) {
      const unsigned sz = min(kTmaChunk, bytes - off);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
              dst + off),
          "l"(src + off), "r"(sz), "r"(b)
          : "memory");
    }
  };
  if (t == 0)
    for (int q = 0; q < kTmaStages && g0 + q < g1; ++q) issue(g0 + q, q);

  const int br = t / 36, w = t % 36, r = w / 3, cc = w % 3;
  F2 part{0.f, 0.f};
  int it = 0;
  bool timed_out = false;
  for (int g = g0; g < g1; ++g, ++it) {
    const int q = it % kTmaStages;
    const bool ok = mbar_wait(smem_addr(&bar[q]), (unsigned)((it / kTmaStages) & 1), polls);
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    const int i0 = g * kTmaRows, i = i0 + br;
    float acc = 0.f;
    if (i < n) {
      const int kbase = rp[i0], k0 = rp[i], k1 = rp[i + 1];
      const float* sv = sval + (size_t)q * stage_floats + (size_t)(k0 - kbase) * 144 + r * 12 + cc * 4;
      constexpr int U = 9;
      int j[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (k0 + u < k1) j[u] = col[k0 + u];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (k0 + u < k1) {
          const float4 a = *reinterpret_cast<const float4*>(sv + u * 144);
          const float4 xv = *reinterpret_cast<const float4*>(x + (size_t)j[u] * 12 + cc * 4);
          acc = dot4_acc(acc, a, xv);
        }
      for (int k = k0 + U; k < k1; ++k) {
        const float4 a = *reinterpret_cast<const float4*>(sv + (k - k0) * 144);
        const float4 xv = *reinterpret_cast<const float4*>(x + (size_t)col[k] * 12 + cc * 4);
        acc = dot4_acc(acc, a, xv);
      }
    }
    sacc[t] = acc;
    __syncthreads();   // stage q fully read; sacc complete
    if (t == 0 && g + kTmaStages < g1) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(g + kTmaStages, q);
    }
    if (i < n && cc == 0) {
      const size_t gi = (size_t)i * 12 + r;
      const float xi = x[gi];
      float yi = (sacc[t] + sacc[t + 1]) + sacc[t + 2];
      yi = __fmaf_rn(st ? st->td[r / 3] : td.v[r / 3], xi, yi);   // PCG: the solve's shift
      if (mask && mask[gi]) yi = 0.f;
      y[gi] = yi;
      part = f2_add(part, f2_prod(xi, yi));
    }
    __syncthreads();   // sacc is rewritten by the next group
  }
  if (timed_out) {
    // raise the error (the host voids the call's results) and drain the copies this CTA issued
    // (local groups it .. it + stages - 1) with the full default budget, whatever the stage
    // waits were given; the grid reduction below still completes
    if (t == 0) {
      atomicOr(err, ERRBIT_TIMEOUT);
      for (int k = it; k < it + kTmaStages && g0 + k < g1; ++k)
        mbar_wait(smem_addr(&bar[k % kTmaStages]), (unsigned)((k / kTmaStages) & 1));
    }
    __syncthreads();
  }
  if (st) {
    F2 v1[1] = {part};
    double out[1];
    if (grid_reduce_f2<1>(v1, red, out, gridDim.x) && threadIdx.x == 0) {
      st->pq = out[0];
      if (!(out[0] > 0.0)) {
        st->negcurv = 1;
        st->done = 1;
        st->alpha = 0.0;
      } else {
        st->alpha = st->rz / out[0];
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Mixed-precision PCG as one persistent cooperative launch: every CTA owns a contiguous range of
// node rows and runs all iterations of the solve, the phases separated by grid barriers:
//   SpMV of its rows (p.Ap partial) | barrier + sum | update x, r, z = D r of its rows (r.z, r.r
//   partials) | barrier + sums | p = z + beta p of its rows | barrier.
// The arithmetic per element is that of k_spmv32, k_pcg32_update and k_pcg32_pupdate4; the
// partial sums are taken per CTA and combined by the last CTA to arrive at the barrier (in CTA
// order), which publishes the totals before it releases the others, so every CTA takes the same
// decisions. Every barrier wait is bounded (Shell::wait_polls polls): on expiry the CTA raises
// ERRBIT_TIMEOUT and returns, and the others then time out at their next barrier. The launch is
// cooperative, so all CTAs are resident and a barrier completes unless a CTA has given up.
// ------------------------------------------------------------------------------------------
struct PersistSync {
  unsigned count, gen;   // barrier arrivals and generation
  double out[4];         // totals published by the last CTA of a reducing barrier
};
constexpr int kPersistMaxCtas = 4096;

// Grid barrier; with nv > 0 the last CTA to arrive first sums the nv per-CTA partials
// part[v * kPersistMaxCtas + b] (b = 0 .. gridDim.x - 1, double-float, in a fixed order) into
// ps->out[v]. Returns false when this CTA's wait ran out (the kernel must return).
__device__ __forceinline__ bool persist_sync(PersistSync* ps, const float2* part, int nv, int polls,
                                             int* err) {
  __shared__ int s_last, s_ok;
  __shared__ unsigned s_gen;
  __shared__ F2 sred[3][32];
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &ps->gen;
    s_gen = *vgen;   // no CTA can release this barrier before this CTA has arrived
    __threadfence();
    s_last = atomicAdd(&ps->count, 1u) == gridDim.x - 1u ? 1 : 0;
    s_ok = 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int v = 0; v < nv; ++v) {
      F2 acc{0.f, 0.f};
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const float2 y = __ldcg(part + (size_t)v * kPersistMaxCtas + b);
        acc = f2_add(acc, F2{y.x, y.y});
      }
      const F2 t = f2_block_sum(acc, sred, v);
      if (threadIdx.x == 0) ps->out[v] = (double)t.hi + (double)t.lo;
    }
    if (threadIdx.x == 0) {
      ps->count = 0u;
      __threadfence();
      atomicAdd(&ps->gen, 1u);
    }
  } else if (threadIdx.x == 0) {
    volatile unsigned* vgen = &ps->gen;
    int i = 0;
    for (; i < polls; ++i) {
      if (*vgen != s_gen) break;
      __nanosleep(32);
    }
    if (i >= polls) {
      atomicOr(err, ERRBIT_TIMEOUT);
      s_ok = 0;
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ double persist_out(PersistSync* ps, int v) {
  return *reinterpret_cast<volatile double*>(&ps->out[v]);
}

__global__ void __launch_bounds__(kSpmvThreads)
k_pcg32_persistent(int n, int per, const int* __restrict__ rp, const int* __restrict__ col,
                   const float* __restrict__ val, const float* __restrict__ Dinv,
                   const unsigned char* __restrict__ mask, float* __restrict__ x, float* __restrict__ r,
                   float* __restrict__ z, float* __restrict__ p, float* __restrict__ Ap, PcgState* st,
                   PersistSync* ps, float2* part, int polls, int* err) {
  constexpr int NC = 3, TPR = 36, RPC = kSpmvThreads / TPR, NPG = kSpmvThreads / 12;
  __shared__ float sacc[kSpmvThreads];
  __shared__ float sr[NPG][12];
  __shared__ F2 sred[2][32];
  const int t = threadIdx.x;
  const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
  const float td[4] = {st->td[0], st->td[1], st->td[2], st->td[3]};
  const int limit = st->limit, fixed = st->fixed;
  const double rtol2 = st->rtol2, bb = st->bb;
  double rz = st->rz, rr = st->rr, pq = 0.0, alpha = 0.0, beta = 0.0;
  int iters = 0, negcurv = 0;
  int done = st->done || limit <= 0;
  const int br = t / TPR, w = t % TPR, rr_ = w / NC, cc = w % NC;
  const int ln = t / 12, a = t % 12;
  while (!done) {
    // y = (A + tau D) p on this CTA's rows and the partial p.y
    F2 part_pq{0.f, 0.f};
    for (int base = i0; base < i1; base += RPC) {
      const int i = base + br;
      float acc = 0.f;
      if (i < i1) {
        const int k0 = rp[i], k1 = rp[i + 1];
        for (int k = k0; k < k1; ++k) {
          const float4 av = __ldcs(reinterpret_cast<const float4*>(val + (size_t)k * 144 + rr_ * 12 + cc * 4));
          const float4 xv = __ldcg(reinterpret_cast<const float4*>(p + (size_t)col[k] * 12 + cc * 4));
          acc = dot4_acc(acc, av, xv);
        }
      }
      sacc[t] = acc;
      __syncthreads();
      if (i < i1 && cc == 0) {
        const size_t gi = (size_t)i * 12 + rr_;
        const float xi = __ldcg(p + gi);
        float yi = (sacc[t] + sacc[t + 1]) + sacc[t + 2];
        yi = __fmaf_rn(td[rr_ / 3], xi, yi);
        if (mask && mask[gi]) yi = 0.f;
        Ap[gi] = yi;
        part_pq = f2_add(part_pq, f2_prod(xi, yi));
      }
      __syncthreads();
    }
    {
      const F2 c = f2_block_sum(part_pq, sred, 0);
      if (t == 0) part[blockIdx.x] = make_float2(c.hi, c.lo);
    }
    if (!persist_sync(ps, part, 1, polls, err)) return;
    pq = persist_out(ps, 0);
    if (!(pq > 0.0)) {
      negcurv = 1;
      alpha = 0.0;
      break;
    }
    alpha = rz / pq;
    // x += alpha p, r -= alpha Ap, z = D r on this CTA's nodes; partials r.z, r.r
    const float af = (float)alpha;
    F2 prz{0.f, 0.f}, prr{0.f, 0.f};
    for (int base = i0; base < i1; base += NPG) {
      const int i = base + ln;
      const size_t gi = (size_t)i * 12 + a;
      float ri = 0.f, zi = 0.f;
      if (i < i1) {
        x[gi] = fmaf(af, p[gi], x[gi]);
        ri = fmaf(-af, Ap[gi], r[gi]);
        r[gi] = ri;
        sr[ln][a] = ri;
      }
      __syncthreads();
      if (i < i1) {
        if (!(mask && mask[gi])) {
          const float* D = Dinv + (size_t)i * 144 + a * 12;
          const float* q = sr[ln];
          zi = __fmaf_rn(D[0], q[0], 0.f);
#pragma unroll
          for (int c = 1; c < 12; ++c) zi = __fmaf_rn(D[c], q[c], zi);
        }
        z[gi] = zi;
      }
      prz = f2_add(prz, f2_prod(ri, zi));
      prr = f2_add(prr, f2_prod(ri, ri));
      __syncthreads();
    }
    {
      const F2 c0 = f2_block_sum(prz, sred, 0);
      const F2 c1 = f2_block_sum(prr, sred, 1);
      if (t == 0) {
        part[kPersistMaxCtas + blockIdx.x] = make_float2(c0.hi, c0.lo);
        part[2 * kPersistMaxCtas + blockIdx.x] = make_float2(c1.hi, c1.lo);
      }
    }
    if (!persist_sync(ps, part + kPersistMaxCtas, 2, polls, err)) return;
    const double rz_new = persist_out(ps, 0);
    rr = persist_out(ps, 1);
    iters += 1;
    beta = rz_new / rz;
    rz = rz_new;
    if (fixed == 0 && rr <= rtol2 * bb) done = 1;
    if (rz_new == 0.0) done = 1;
    if (iters >= limit) done = 1;
    if (done) break;
    // p = z + beta p on this CTA's rows, then every CTA waits before the next SpMV reads them
    const float bf = (float)beta;
    for (int k = i0 * 12 + t; k < i1 * 12; k += blockDim.x) p[k] = fmaf(bf, p[k], z[k]);
    if (!persist_sync(ps, nullptr, 0, polls, err)) return;
  }
  if (blockIdx.x == 0 && t == 0) {
    st->iters = iters;
    st->rz = rz;
    st->rr = rr;
    st->pq = pq;
    st->alpha = alpha;
    st->beta = beta;
    st->negcurv = negcurv;
    st->done = 1;
  }
}

// ------------------------------------------------------------------------------------------
// Mixed-precision PCG of a small shell as one thread-block cluster: the cluster's CTAs (one per
// SM, up to 16) own contiguous ranges of node rows and run all iterations, the phases separated
// by the hardware cluster barrier (barrier.cluster, release/acquire at cluster scope, which also
// orders the global-memory vectors the CTAs exchange). A reduction is one partial per CTA in its
// own shared memory, read by every CTA through distributed shared memory in rank order after the
// barrier, so every CTA holds the same totals and takes the same decisions; the partials are
// double-buffered, since a CTA rewrites one only two barriers later. Per iteration, as in
// k_pcg32_persistent: SpMV (p.Ap) | barrier | update x, r, z = D r (r.z, r.r) | barrier |
// p = z + beta p | barrier. The arithmetic per element is that of k_spmv32, k_pcg32_update and
// k_pcg32_pupdate4. Every CTA runs every barrier (control flow depends only on the shared totals
// and the launch's state), so the barriers cannot wait on a CTA that has left.
// ------------------------------------------------------------------------------------------
constexpr int kClusterRows = 16;                        // node rows per SpMV pass of a CTA
constexpr int kClusterThreads = kClusterRows * 36;      // 576
constexpr int kClusterMaxCtas = 16;

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_ctas() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(r));
  return r;
}

// float2 at a shared-memory address of CTA `rank` of the cluster
__device__ __forceinline__ float2 dsmem_ld_f2(const float2* local, unsigned rank) {
  unsigned addr = (unsigned)__cvta_generic_to_shared(local), remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(remote) : "r"(addr), "r"(rank));
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(remote) : "memory");
  return v;
}

// Totals over the cluster's CTAs of the nv partials in every CTA's slots: lane q of warp 0 reads
// CTA q's slots through distributed shared memory (one remote load per lane, all in flight at
// once), lane 0 sums them in rank order (so every CTA gets the same doubles) and the CTA reads them
// from shared memory. All threads of the CTA must call it.
__device__ __forceinline__ void cluster_totals(const float2* slots, int nv, unsigned nctas, double* s_tot,
                                               double* out) {
  if (threadIdx.x < 32) {
    const unsigned q = threadIdx.x;
    float2 y[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (q < nctas)
      for (int v = 0; v < nv; ++v) y[v] = dsmem_ld_f2(slots + v, q);
    for (int v = 0; v < nv; ++v) {
      F2 acc{0.f, 0.f};
      for (unsigned k = 0; k < nctas; ++k) {
        const float hi = __shfl_sync(0xffffffffu, y[v].x, k), lo = __shfl_sync(0xffffffffu, y[v].y, k);
        acc = f2_add(acc, F2{hi, lo});
      }
      if (q == 0) s_tot[v] = (double)acc.hi + (double)acc.lo;
    }
  }
  __syncthreads();
  for (int v = 0; v < nv; ++v) out[v] = s_tot[v];
}

__global__ void __launch_bounds__(kClusterThreads, 1)
k_pcg32_cluster(int n, int per, const int* __restrict__ rp, const int* __restrict__ col,
                const float* __restrict__ val, const float* __restrict__ Dinv,
                const unsigned char* __restrict__ mask, float* __restrict__ x, float* __restrict__ r,
                float* __restrict__ z, float* __restrict__ p, float* __restrict__ Ap, PcgState* st) {
  constexpr int NC = 3, TPR = 36, NPG = kClusterThreads / 12;
  __shared__ float sacc[kClusterThreads];
  __shared__ float sr[NPG][12];
  __shared__ F2 sred[2][32];
  __shared__ float2 slots[2][2];   // [buffer][value]: this CTA's partials of a reduction
  __shared__ double s_tot[2];
  const int t = threadIdx.x;
  const unsigned rank = cluster_rank(), nctas = cluster_ctas();
  const int i0 = min(n, (int)rank * per), i1 = min(n, i0 + per);
  const float td[4] = {st->td[0], st->td[1], st->td[2], st->td[3]};
  const int limit = st->limit, fixed = st->fixed;
  const double rtol2 = st->rtol2, bb = st->bb;
  double rz = st->rz, rr = st->rr, pq = 0.0, alpha = 0.0, beta = 0.0;
  int iters = 0, negcurv = 0, buf = 0;
  int done = st->done || limit <= 0;
  const int br = t / TPR, w = t % TPR, rr_ = w / NC, cc = w % NC;
  const int ln = t / 12, a = t % 12;
  while (!done) {
    // y = (A + tau D) p on this CTA's rows and the partial p.y
    F2 part_pq{0.f, 0.f};
    for (int base = i0; base < i1; base += kClusterRows) {
      const int i = base + br;
      float acc = 0.f;
      if (i < i1) {
        // up to 9 blocks of the row in flight at once (a node row has at most 9), as in k_spmv32
        const int k0 = rp[i], k1 = rp[i + 1];
        constexpr int U = 9;
        float4 v[U];
        int j[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int k = k0 + u;
          if (k < k1) {
            j[u] = col[k];
            v[u] = __ldcs(reinterpret_cast<const float4*>(val + (size_t)k * 144 + rr_ * 12 + cc * 4));
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k0 + u < k1) {
            const float4 xv = __ldcg(reinterpret_cast<const float4*>(p + (size_t)j[u] * 12 + cc * 4));
            acc = dot4_acc(acc, v[u], xv);
          }
        for (int k = k0 + U; k < k1; ++k) {
          const float4 av = __ldcs(reinterpret_cast<const float4*>(val + (size_t)k * 144 + rr_ * 12 + cc * 4));
          const float4 xv = __ldcg(reinterpret_cast<const float4*>(p + (size_t)col[k] * 12 + cc * 4));
          acc = dot4_acc(acc, av, xv);
        }
      }
      sacc[t] = acc;
      __syncthreads();
      if (i < i1 && cc == 0) {
        const size_t gi = (size_t)i * 12 + rr_;
        const float xi = __ldcg(p + gi);
        float yi = (sacc[t] + sacc[t + 1]) + sacc[t + 2];
        yi = __fmaf_rn(td[rr_ / 3], xi, yi);
        if (mask && mask[gi]) yi = 0.f;
        Ap[gi] = yi;
        part_pq = f2_add(part_pq, f2_prod(xi, yi));
      }
      __syncthreads();
    }
    {
      const F2 c = f2_block_sum(part_pq, sred, 0);
      if (t == 0) slots[buf][0] = make_float2(c.hi, c.lo);
    }
    cluster_barrier();
    cluster_totals(slots[buf], 1, nctas, s_tot, &pq);
    buf ^= 1;
    if (!(pq > 0.0)) {
      negcurv = 1;
      alpha = 0.0;
      break;
    }
    alpha = rz / pq;
    // x += alpha p, r -= alpha Ap, z = D r on this CTA's nodes; partials r.z, r.r
    const float af = (float)alpha;
    F2 prz{0.f, 0.f}, prr{0.f, 0.f};
    for (int base = i0; base < i1; base += NPG) {
      const int i = base + ln;
      const size_t gi = (size_t)i * 12 + a;
      float ri = 0.f, zi = 0.f;
      if (i < i1) {
        x[gi] = fmaf(af, p[gi], x[gi]);
        ri = fmaf(-af, Ap[gi], r[gi]);
        r[gi] = ri;
        sr[ln][a] = ri;
      }
      __syncthreads();
      if (i < i1) {
        if (!(mask && mask[gi])) {
          const float* D = Dinv + (size_t)i * 144 + a * 12;
          const float* q = sr[ln];
          zi = __fmaf_rn(D[0], q[0], 0.f);
#pragma unroll
          for (int c = 1; c < 12; ++c) zi = __fmaf_rn(D[c], q[c], zi);
        }
        z[gi] = zi;
      }
      prz = f2_add(prz, f2_prod(ri, zi));
      prr = f2_add(prr, f2_prod(ri, ri));
      __syncthreads();
    }
    {
      const F2 c0 = f2_block_sum(prz, sred, 0);
      const F2 c1 = f2_block_sum(prr, sred, 1);
      if (t == 0) {
        slots[buf][0] = make_float2(c0.hi, c0.lo);
        slots[buf][1] = make_float2(c1.hi, c1.lo);
      }
    }
    cluster_barrier();
    double tot[2];
    cluster_totals(slots[buf], 2, nctas, s_tot, tot);
    const double rz_new = tot[0];
    rr = tot[1];
    buf ^= 1;
    iters += 1;
    beta = rz_new / rz;
    rz = rz_new;
    if (fixed == 0 && rr <= rtol2 * bb) done = 1;
    if (rz_new == 0.0) done = 1;
    if (iters >= limit) done = 1;
    if (done) break;
    // p = z + beta p on this CTA's rows, then every CTA waits before the next SpMV reads them
    const float bf = (float)beta;
    for (int k = i0 * 12 + t; k < i1 * 12; k += blockDim.x) p[k] = fmaf(bf, p[k], z[k]);
    cluster_barrier();
  }
  // no CTA leaves while another may still read its partials
  cluster_barrier();
  if (rank == 0 && t == 0) {
    st->iters = iters;
    st->rz = rz;
    st->rr = rr;
    st->pq = pq;
    st->alpha = alpha;
    st->beta = beta;
    st->negcurv = negcurv;
    st->done = 1;
  }
}


// row a of a 12x12 block times sr, as the explicit FMA chain of k_pcg32_update
__device__ __forceinline__ float apply_block32(const float* __restrict__ D, const float* sr, int a) {
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 12; ++c) s = __fmaf_rn(D[a * 12 + c], sr[c], s);
  return s;
}

__global__ void __launch_bounds__(kNodeThreads)
k_pcg32_init(int n, const double* __restrict__ rhs, const float* __restrict__ Dinv,
             const unsigned char* __restrict__ mask, float* __restrict__ x, float* __restrict__ r,
             float* __restrict__ z, float* __restrict__ p, double rtol2, int fixed, int limit, Shift4f td,
             PcgState* st, Reduce red) {
  __shared__ float sr[16][12];
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  const size_t gi = (size_t)i * 12 + a;
  float ri = 0.f, zi = 0.f;
  if (i < n) {
    ri = (mask && mask[gi]) ? 0.f : (float)rhs[gi];
    x[gi] = 0.f;
    r[gi] = ri;
    sr[ln][a] = ri;
  }
  __syncthreads();
  if (i < n) {
    zi = (mask && mask[gi]) ? 0.f : apply_block32(Dinv + (size_t)i * 144, sr[ln], a);
    z[gi] = zi;
    p[gi] = zi;
  }
  F2 v[2] = {f2_prod(ri, zi), f2_prod(ri, ri)};
  double out[2];
  if (grid_reduce_f2<2>(v, red, out, gridDim.x) && threadIdx.x == 0) {
    st->rz = out[0];
    st->bb = out[1];
    st->rr = out[1];
    st->rtol2 = rtol2;
    st->fixed = fixed;
    st->limit = limit;
    for (int k = 0; k < 4; ++k) st->td[k] = td.v[k];
    st->iters = 0;
    st->bodies = 0;
    st->negcurv = 0;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->pq = 0.0;
    st->done = (out[1] == 0.0) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(kNodeThreads)
k_pcg32_update(int n, float* __restrict__ x, float* __restrict__ r, float* __restrict__ z,
               const float* __restrict__ p, const float* __restrict__ Ap,
               const float* __restrict__ Dinv, const unsigned char* __restrict__ mask, PcgState* st,
               Reduce red) {
  pdl_wait();
  if (st->done) return;
  const double alpha_d = st->alpha;
  __shared__ float sr[16][12];
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  F2 rz{0.f, 0.f}, rr{0.f, 0.f};
  // this thread's row of the node's 12x12 inverse (48 contiguous bytes) and its DOF of
  // x, p, Ap, r; the next group's are loaded before this group's work, so their latency overlaps it
  struct GroupLoads {
    float4 d0, d1, d2;
    float xv, pv, av, rv;
  };
  GroupLoads cur{}, nxt{};
  auto load = [&](int base, GroupLoads& g) {
    const int i = base + ln;
    if (i < n) {
      const float4* drow = reinterpret_cast<const float4*>(Dinv + (size_t)i * 144 + a * 12);
      g.d0 = __ldg(drow);
      g.d1 = __ldg(drow + 1);
      g.d2 = __ldg(drow + 2);
      const size_t gi = (size_t)i * 12 + a;
      g.xv = x[gi];
      g.pv = p[gi];
      g.av = Ap[gi];
      g.rv = r[gi];
    }
  };
  const int stride = gridDim.x * 16;
  if ((int)blockIdx.x * 16 < n) load(blockIdx.x * 16, cur);
  const float alpha = (float)alpha_d;
  // grid-stride over groups of 16 nodes: a few CTAs per SM, so the last CTA of the grid
  // reduction folds few partials
  for (int base = blockIdx.x * 16; base < n; base += stride) {
    if (base + stride < n) load(base + stride, nxt);
    const int i = base + ln;
    const size_t gi = (size_t)i * 12 + a;
    float ri = 0.f, zi = 0.f;
    if (i < n) {
      x[gi] = fmaf(alpha, cur.pv, cur.xv);
      ri = fmaf(-alpha, cur.av, cur.rv);
      r[gi] = ri;
      sr[ln][a] = ri;
    }
    __syncthreads();
    if (i < n) {
      if (!(mask && mask[gi])) {
        const float* q = sr[ln];
        zi = __fmaf_rn(cur.d0.x, q[0], 0.f);
        zi = __fmaf_rn(cur.d0.y, q[1], zi);
        zi = __fmaf_rn(cur.d0.z, q[2], zi);
        zi = __fmaf_rn(cur.d0.w, q[3], zi);
        zi = __fmaf_rn(cur.d1.x, q[4], zi);
        zi = __fmaf_rn(cur.d1.y, q[5], zi);
        zi = __fmaf_rn(cur.d1.z, q[6], zi);
        zi = __fmaf_rn(cur.d1.w, q[7], zi);
        zi = __fmaf_rn(cur.d2.x, q[8], zi);
        zi = __fmaf_rn(cur.d2.y, q[9], zi);
        zi = __fmaf_rn(cur.d2.z, q[10], zi);
        zi = __fmaf_rn(cur.d2.w, q[11], zi);
      }
      z[gi] = zi;
    }
    rz = f2_add(rz, f2_prod(ri, zi));
    rr = f2_add(rr, f2_prod(ri, ri));
    __syncthreads();   // sr is rewritten by the next group
    cur = nxt;
  }
  F2 v[2] = {rz, rr};
  double out[2];
  if (grid_reduce_f2<2>(v, red, out, gridDim.x) && threadIdx.x == 0) {
    const double rz_new = out[0];
    st->rr = out[1];
    st->iters += 1;
    st->beta = rz_new / st->rz;
    st->rz = rz_new;
    if (st->fixed == 0 && out[1] <= st->rtol2 * st->bb) st->done = 1;
    if (rz_new == 0.0) st->done = 1;
    if (st->iters >= st->limit) st->done = 1;
  }
}

__global__ void k_pcg32_pupdate(int m, const float* __restrict__ z, float* __restrict__ p,
                                const PcgState* st) {
  pdl_wait();
  // z and p (8 bytes a thread) are loaded while the stop flag and beta are in flight; a launch
  // after the solve stopped reads them for nothing
  const int done = st->done;
  const double beta_d = st->beta;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const float pk = p[k], zk = z[k];
    if (done) return;
    p[k] = fmaf((float)beta_d, pk, zk);
  }
}

// The same update four DOFs at a time (m4 = m / 4; m = 12 n is a multiple of 4 and the vectors
// are cudaMalloc'd, so every float4 is aligned): a quarter of the threads for this short pass.
__global__ void k_pcg32_pupdate4(int m4, const float4* __restrict__ z, float4* __restrict__ p,
                                 const PcgState* st) {
  pdl_wait();
  const int done = st->done;
  const double beta_d = st->beta;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m4; k += gridDim.x * blockDim.x) {
    const float4 pk = p[k], zk = z[k];
    if (done) return;
    const float b = (float)beta_d;
    p[k] = make_float4(fmaf(b, pk.x, zk.x), fmaf(b, pk.y, zk.y), fmaf(b, pk.z, zk.z), fmaf(b, pk.w, zk.w));
  }
}

__global__ void k_to_double(int m, const float* __restrict__ a, double* __restrict__ b) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) b[k] = (double)a[k];
}

// ------------------------------------------------------------------------------------------
// Consistent mass products (4x4 scalar blocks (x) I3), FP64.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double mass_row(const int* __restrict__ rp, const int* __restrict__ col,
                                           const double* __restrict__ mass, const double* __restrict__ w,
                                           const double* __restrict__ wsub, int i, int r, int c) {
  double s = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = col[k];
    const double* mb = mass + (size_t)k * 16 + r * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double wv = w[(size_t)j * 12 + q * 3 + c];
      if (wsub) wv -= wsub[(size_t)j * 12 + q * 3 + c];
      s += mb[q] * wv;
    }
  }
  return s;
}

__global__ void __launch_bounds__(kNodeThreads)
k_mass_mult(int n, const int* __restrict__ rp, const int* __restrict__ col,
            const double* __restrict__ mass, const double* __restrict__ x, double* __restrict__ y) {
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  if (i >= n) return;
  y[(size_t)i * 12 + a] = mass_row(rp, col, mass, x, nullptr, i, a / 3, a % 3);
}

// g = grad_el + M (q - y) / dt^2 - F (masked to 0 on fixed DOFs), gin = the inertial/external
// part; |g|^2 reduced into *gn2.
__global__ void __launch_bounds__(kNodeThreads)
k_grad_finish(int n, const int* __restrict__ rp, const int* __restrict__ col,
              const double* __restrict__ mass, const double* __restrict__ fgrav,
              const double* __restrict__ q, const double* __restrict__ yv, double inv_dt2,
              double gx, double gy, double gz, const unsigned char* __restrict__ mask,
              double* __restrict__ g, double* __restrict__ gin, double* gn2, Reduce red,
              int* err) {
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  double part = 0.0;
  if (i < n) {
    const size_t gi = (size_t)i * 12 + a;
    const int r = a / 3, c = a % 3;
    const double grav = c == 0 ? gx : c == 1 ? gy : gz;
    double gi_in = mass_row(rp, col, mass, q, yv, i, r, c) * inv_dt2 - fgrav[(size_t)i * 4 + r] * grav;
    double gv = g[gi] + gi_in;
    if (mask && mask[gi]) { gv = 0.0; gi_in = 0.0; }
    if (!isfinite(gv)) atomicOr(err, ERRBIT_NONFINITE);
    g[gi] = gv;
    if (gin) gin[gi] = gi_in;
    part = gv * gv;
  }
  double v[1] = {part};
  grid_reduce<1>(v, red, gn2, gridDim.x);
}

// Residual after a step q' = q + alpha d when the elastic gradient at q' is already in g: the
// inertial part is linear in q, M (q' - y) / dt^2 - F = gin + alpha M d / dt^2 with M d from the
// line search, so no second mass product is formed. c = alpha / dt^2; fixed DOFs get zero.
__global__ void k_grad_linear(int m, const double* __restrict__ Md, double c,
                              const unsigned char* __restrict__ mask, double* __restrict__ g,
                              double* __restrict__ gin, double* gn2, Reduce red, int* err) {
  double part = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    double gi_in = __fma_rn(c, Md[k], gin[k]);
    double gv = g[k] + gi_in;
    if (mask && mask[k]) { gv = 0.0; gi_in = 0.0; }
    if (!isfinite(gv)) atomicOr(err, ERRBIT_NONFINITE);
    g[k] = gv;
    gin[k] = gi_in;
    part += gv * gv;
  }
  double v[1] = {part};
  grid_reduce<1>(v, red, gn2, gridDim.x);
}

__global__ void k_dots3(int m, const double* __restrict__ a0, const double* __restrict__ b0,
                        const double* __restrict__ a1, const double* __restrict__ b1,
                        const double* __restrict__ a2, const double* __restrict__ b2, double* out,
                        Reduce red) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    v[0] += a0[k] * b0[k];
    v[1] += a1[k] * b1[k];
    v[2] += a2[k] * b2[k];
  }
  grid_reduce<3>(v, red, out, gridDim.x);
}

__global__ void k_diff(int m, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) c[k] = a[k] - b[k];
}

__global__ void k_axpy(int m, double* __restrict__ q, const double* __restrict__ d, double alpha) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) q[k] = __fma_rn(alpha, d[k], q[k]);
}

__global__ void k_overwrite_fixed(int m, double* __restrict__ dst, const double* __restrict__ src,
                                  const unsigned char* __restrict__ mask,
                                  const double* __restrict__ fixed_vals) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
    dst[k] = (mask && mask[k]) ? fixed_vals[k] : src[k];
}

__global__ void k_predictor(int m, const double* __restrict__ qn, const double* __restrict__ v,
                            double dt, double* __restrict__ y) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) y[k] = qn[k] + dt * v[k];
}

__global__ void k_velocity(int m, const double* __restrict__ q, const double* __restrict__ qn,
                           double inv_dt, double* __restrict__ v) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) v[k] = (q[k] - qn[k]) * inv_dt;
}

__global__ void k_negate(int m, const double* __restrict__ a, double* __restrict__ b) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) b[k] = -a[k];
}

// ------------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------------
static int vec_blocks(int m) {
  int b = grid_for(m, 256);
  return b > 4096 ? 4096 : b;
}

shell_status launch_grad_finish(Shell& s, const double* q, const double* y, double dt,
                                const double grav[3], const unsigned char* mask, double* g,
                                double* gin, double* gnorm2_out) {
  int blocks = grid_for(s.n_nodes, 16);
  if (blocks > s.red.stride) return fail(SHELL_ERR_ARG, "too many nodes for one reduction");
  // q - y once per DOF: the mass product then takes one FP64 FMA per term instead of a
  // subtraction and an FMA (it is bound by the FP64 pipe); same values, same sums
  k_diff<<<vec_blocks(s.n_dof), 256, 0, s.stream>>>(s.n_dof, q, y, s.d_qmy);
  ++s.launches;
  k_grad_finish<<<blocks, kNodeThreads, 0, s.stream>>>(s.n_nodes, s.d_row_ptr, s.d_col, s.d_mass,
                                                       s.d_fgrav, s.d_qmy, nullptr, 1.0 / (dt * dt), grav[0],
                                                       grav[1], grav[2], mask, g, gin, gnorm2_out,
                                                       s.red, s.d_err);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_grad_linear(Shell& s, const double* Md, double alpha, double dt,
                                const unsigned char* mask, double* g, double* gin, double* gnorm2_out) {
  const int blocks = std::min(vec_blocks(s.n_dof), 1024);
  k_grad_linear<<<blocks, 256, 0, s.stream>>>(s.n_dof, Md, alpha / (dt * dt), mask, g, gin, gnorm2_out,
                                              s.red, s.d_err);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_mass_mult(Shell& s, const double* x, double* y) {
  k_mass_mult<<<grid_for(s.n_nodes, 16), kNodeThreads, 0, s.stream>>>(s.n_nodes, s.d_row_ptr,
                                                                     s.d_col, s.d_mass, x, y);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_dots3(Shell& s, int m, const double* a0, const double* b0, const double* a1,
                          const double* b1, const double* a2, const double* b2, double* out3) {
  int blocks = std::min(vec_blocks(m), 1024);
  k_dots3<<<blocks, 256, 0, s.stream>>>(m, a0, b0, a1, b1, a2, b2, out3, s.red);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_precond_setup(Shell& s, const unsigned char* mask, const double td[4]) {
  int blocks = grid_for(s.n_nodes, 16);
  Shift4 sh{{td[0], td[1], td[2], td[3]}};
  if (s.val_fp64)
    k_precond<double, double><<<blocks, 192, 0, s.stream>>>(s.n_nodes, s.d_diag_block,
        (const double*)s.d_val, mask, sh, (double*)s.d_Dinv);
  else
    k_precond32_thread<<<grid_for(s.n_nodes, 128), 128, 0, s.stream>>>(s.n_nodes, s.d_diag_block,
        (const float*)s.d_val, mask, sh, (float*)s.d_Dinv);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

// Local part of the Sec. 6.1 regulariser: every free diagonal entry A_ii <= 0 (DOF kind k) becomes
// max(-A_ii, floor_k), floor_k = 1e-8 D_k; the number of entries changed is added to *count.
template <typename Rm>
__global__ void k_fix_diag(int m, const int* __restrict__ diag_block, Rm* __restrict__ val,
                           const unsigned char* __restrict__ mask, Shift4 floor, int* count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m || (mask && mask[k])) return;
  Rm* a = &val[(size_t)diag_block[k / 12] * 144 + (k % 12) * 13];
  const Rm v = *a;
  if (v <= Rm(0)) {
    const Rm f = (Rm)floor.v[(k % 12) / 3];
    *a = -v > f ? -v : f;
    atomicAdd(count, 1);
  }
}

shell_status launch_fix_diag(Shell& s, const unsigned char* mask, const double floor4[4], int* count) {
  Shift4 f{{floor4[0], floor4[1], floor4[2], floor4[3]}};
  const int blocks = (s.n_dof + 255) / 256;
  if (s.val_fp64)
    k_fix_diag<double><<<blocks, 256, 0, s.stream>>>(s.n_dof, s.d_diag_block, (double*)s.d_val, mask, f, count);
  else
    k_fix_diag<float><<<blocks, 256, 0, s.stream>>>(s.n_dof, s.d_diag_block, (float*)s.d_val, mask, f, count);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_diag_check(Shell& s, const unsigned char* mask, double* out12, bool aux) {
  // aux: beside other reducing kernels, on the shell's second workspace
  const Reduce& red = aux ? s.red_aux : s.red;
  int blocks = grid_for(s.n_dof, 256 * 4);
  if (blocks > 2 * std::max(1, s.num_sms)) blocks = 2 * std::max(1, s.num_sms);
  if (blocks > red.stride) return fail(SHELL_ERR_ARG, "reduction workspace too small");
  if (s.val_fp64)
    k_diag_check<double><<<blocks, 256, 0, s.stream>>>(s.n_nodes, s.d_diag_block,
        (const double*)s.d_val, mask, out12, red);
  else
    k_diag_check<float><<<blocks, 256, 0, s.stream>>>(s.n_nodes, s.d_diag_block,
        (const float*)s.d_val, mask, out12, red);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_pcg_init(Shell& s, const unsigned char* mask, const double* rhs, double rtol,
                             int fixed, int limit, const double td[4]) {
  int blocks = grid_for(s.n_nodes, 16);
  if (blocks > s.red.stride) return fail(SHELL_ERR_ARG, "too many nodes for one reduction");
  double rtol2 = fixed > 0 ? 0.0 : rtol * rtol;
  if (!s.val_fp64) {
    Shift4f sh{{(float)td[0], (float)td[1], (float)td[2], (float)td[3]}};
    k_pcg32_init<<<blocks, kNodeThreads, 0, s.stream>>>(s.n_nodes, rhs, (const float*)s.d_Dinv, mask,
        s.d_x32, s.d_r32, s.d_z32, s.d_p32, rtol2, fixed, limit, sh, s.d_pcg, s.red);
    BHEM_CUDA(cudaGetLastError());
    ++s.launches;
    return SHELL_OK;
  }
  if (s.val_fp64)
    k_pcg_init<double><<<blocks, kNodeThreads, 0, s.stream>>>(
        s.n_nodes, rhs, (const double*)s.d_Dinv, mask, s.d_x, s.d_r, s.d_z, s.d_p, nullptr, rtol2,
        fixed, s.d_pcg, s.red);
  else
    k_pcg_init<float><<<blocks, kNodeThreads, 0, s.stream>>>(
        s.n_nodes, rhs, (const float*)s.d_Dinv, mask, s.d_x, s.d_r, s.d_z, s.d_p, s.d_p32, rtol2,
        fixed, s.d_pcg, s.red);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

static shell_status launch_spmv_impl(Shell& s, const void* x, const double* xd,
                                     const unsigned char* mask, const double td[4], double* y,
                                     PcgState* st) {
  Shift4 sh{{td[0], td[1], td[2], td[3]}};
  const int n = s.n_nodes;
  if (s.val_fp64) {
    constexpr int RPC = kSpmvThreads / 72;
    int blocks = grid_for(n, RPC);
    if (st && blocks > s.red.stride) return fail(SHELL_ERR_ARG, "too many nodes for one reduction");
    k_spmv<double><<<blocks, kSpmvThreads, 0, s.stream>>>(n, s.d_row_ptr, s.d_col,
        (const double*)s.d_val, (const double*)x, xd, sh, mask, y, st, s.red);
  } else {
    constexpr int RPC = kSpmvThreads / 36;
    int blocks = grid_for(n, RPC);
    if (st && blocks > s.red.stride) return fail(SHELL_ERR_ARG, "too many nodes for one reduction");
    k_spmv<float><<<blocks, kSpmvThreads, 0, s.stream>>>(n, s.d_row_ptr, s.d_col,
        (const float*)s.d_val, (const float*)x, xd, sh, mask, y, st, s.red);
  }
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

static shell_status launch_spmv32(Shell& s, const float* x, Shift4f sh, const unsigned char* mask, float* y,
                                  PcgState* st);

shell_status launch_spmv(Shell& s, const void* x, int x_fp32, void* y) {
  // every SpMV kernel reads x in 16-byte vector loads
  if (reinterpret_cast<uintptr_t>(x) & 15) return fail(SHELL_ERR_ARG, "x must be 16-byte aligned");
  const double zero[4] = {0.0, 0.0, 0.0, 0.0};
  if (s.val_fp64) return launch_spmv_impl(s, x, nullptr, nullptr, zero, (double*)y, nullptr);
  const float* xs = (const float*)x;
  float* ys = (float*)y;
  if (!x_fp32) {
    // FP64 in and out: convert through the shell's FP32 vectors
    k_to_float<<<vec_blocks(s.n_dof), 256, 0, s.stream>>>(s.n_dof, (const double*)x, s.d_z32);
    BHEM_CUDA(cudaGetLastError());
    ++s.launches;
    xs = s.d_z32;
    ys = s.d_Ap32;
  }
  BHEM_TRY(launch_spmv32(s, xs, Shift4f{{0.f, 0.f, 0.f, 0.f}}, nullptr, ys, nullptr));
  if (!x_fp32) {
    k_to_double<<<vec_blocks(s.n_dof), 256, 0, s.stream>>>(s.n_dof, s.d_Ap32, (double*)y);
    BHEM_CUDA(cudaGetLastError());
    ++s.launches;
  }
  return SHELL_OK;
}

shell_status setup_spmv(Shell& s) {
  s.spmv_tma = 0;
  {
    int d = 0;
    BHEM_CUDA(cudaGetDevice(&d));
    BHEM_CUDA(cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, d));
  }
  if (s.val_fp64) return SHELL_OK;
  const size_t stage_floats = (size_t)kTmaRows * std::max(1, s.max_row) * 144;
  const size_t smem = stage_floats * sizeof(float) * kTmaStages;
  int dev = 0, max_optin = 0, sms = 0;
  BHEM_CUDA(cudaGetDevice(&dev));
  BHEM_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  BHEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t static_smem = 8 * kTmaStages + sizeof(float) * kTmaThreads + 512;
  const bool fits = smem + static_smem <= (size_t)max_optin;
  if (s.opt.spmv == SHELL_SPMV_TMA && !fits)
    return fail(SHELL_ERR_ARG, "SHELL_SPMV_TMA: 8 block rows of the longest row do not fit in shared memory");
  // AUTO takes the plain kernel: on GB300 it reaches 0.87 of the measured HBM copy bandwidth at
  // 256x256 (4 CTAs per SM keep every block load of 36 rows in flight), the bulk-copy ring 0.42
  // (one CTA per SM computes too few groups at a time to cover the latency of the x gathers)
  if (s.opt.spmv != SHELL_SPMV_TMA || !fits) return SHELL_OK;
  BHEM_CUDA(cudaFuncSetAttribute(k_spmv32_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int ngroups = (s.n_nodes + kTmaRows - 1) / kTmaRows;
  s.spmv_tma = 1;
  s.spmv_stage_floats = (int)stage_floats;
  s.spmv_smem = smem;
  s.spmv_grid = std::max(1, std::min(ngroups, sms));
  if (s.spmv_grid > s.red.stride) return fail(SHELL_ERR_ARG, "reduction workspace too small");
  return SHELL_OK;
}

static shell_status launch_spmv32(Shell& s, const float* x, Shift4f sh, const unsigned char* mask, float* y,
                                  PcgState* st) {
  const int n = s.n_nodes;
  if (s.spmv_tma) {
    k_spmv32_tma<<<s.spmv_grid, kTmaThreads, s.spmv_smem, s.stream>>>(
        n, s.d_row_ptr, s.d_col, (const float*)s.d_val, x, sh, mask, y, st, s.red, s.spmv_stage_floats, s.d_err,
        s.wait_polls);
  } else {
    const int blocks = grid_for(n, kSpmvThreads / 36);
    if (st && blocks > s.red.stride) return fail(SHELL_ERR_ARG, "too many nodes for one reduction");
    if (s.spmv_sym)
      k_spmv32_sym<<<blocks, kSpmvThreads, kSpmvSymSmem, s.stream>>>(
          n, s.d_row_ptr, s.d_col, (const float*)s.d_val, s.d_tpos, s.d_diag_block, x, sh, mask, y, st, s.red);
    else
      BHEM_CUDA(launch_k(s.pdl && st, k_spmv32, blocks, kSpmvThreads, s.stream, n, (const int*)s.d_row_ptr,
                         (const int*)s.d_col, (const float*)s.d_val, x, sh, mask, y, st, s.red));
  }
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_pcg_iteration(Shell& s, const unsigned char* mask, const double td[4]) {
  const int n = s.n_nodes, m = s.n_dof;
  if (!s.val_fp64) {
    Shift4f sh{{(float)td[0], (float)td[1], (float)td[2], (float)td[3]}};
    const bool fold = pcg_folds_pupdate(s);
    if (fold) {
      const int blocks = grid_for(n, kSpmvThreads / 36);
      if (blocks > s.red.stride) return fail(SHELL_ERR_ARG, "too many nodes for one reduction");
      k_spmv32_pcg<<<blocks, kSpmvThreads, 0, s.stream>>>(n, s.d_row_ptr, s.d_col, (const float*)s.d_val, s.d_z32,
                                                          mask, s.d_p32, s.d_Ap32, s.d_pcg, s.red);
      BHEM_CUDA(cudaGetLastError());
      ++s.launches;
    } else {
      BHEM_TRY(launch_spmv32(s, s.d_p32, sh, mask, s.d_Ap32, s.d_pcg));
    }
    if (s.update_grid <= 0) {   // the resident CTAs: a CTA waiting for a free SM would run its groups last
      int occ = 0;
      BHEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg32_update, kNodeThreads, 0));
      s.update_grid = std::max(1, std::min(grid_for(n, 16), std::max(1, occ) * std::max(1, s.num_sms)));
    }
    BHEM_CUDA(launch_k(s.pdl, k_pcg32_update, s.update_grid, kNodeThreads, s.stream, n, s.d_x32, s.d_r32,
                       s.d_z32, (const float*)s.d_p32, (const float*)s.d_Ap32, (const float*)s.d_Dinv, mask,
                       s.d_pcg, s.red));
    BHEM_CUDA(cudaGetLastError());
    ++s.launches;
    if (fold) return SHELL_OK;   // the next iteration's SpMV forms p
    if (m % 4 == 0)
      BHEM_CUDA(launch_k(s.pdl, k_pcg32_pupdate4, vec_blocks(m / 4), 256, s.stream, m / 4,
                         reinterpret_cast<const float4*>(s.d_z32), reinterpret_cast<float4*>(s.d_p32),
                         (const PcgState*)s.d_pcg));
    else
      BHEM_CUDA(launch_k(s.pdl, k_pcg32_pupdate, vec_blocks(m), 256, s.stream, m, (const float*)s.d_z32, s.d_p32,
                         (const PcgState*)s.d_pcg));
    BHEM_CUDA(cudaGetLastError());
    ++s.launches;
    return SHELL_OK;
  }
  const void* px = (const void*)s.d_p;
  BHEM_TRY(launch_spmv_impl(s, px, s.d_p, mask, td, s.d_Ap, s.d_pcg));
  k_pcg_update<double><<<grid_for(n, 16), kNodeThreads, 0, s.stream>>>(
      n, s.d_x, s.d_r, s.d_z, s.d_p, s.d_Ap, (const double*)s.d_Dinv, mask, s.d_pcg, s.red);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  k_pcg_pupdate<<<vec_blocks(m), 256, 0, s.stream>>>(m, s.d_z, s.d_p, nullptr, s.d_pcg);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

// Iterations per body of the device-side PCG loop: the body's fixed cost (condition kernel and
// relaunch, about 4.6 us) is shared by kLoopUnroll iterations, and at most kLoopUnroll - 1
// iterations launched after the solve stopped exit at once. On the 256^2 sheet's Newton
// iteration: 8.31 ms with one iteration per body, 8.15 with 4, 8.23 with 8.
constexpr int kLoopUnroll = 4;

// Condition of the device-side PCG loop, after each body: go on while the solve runs, and never
// past st->limit iterations (so the loop ends even if no kernel stopped it).
__global__ void k_pcg_loop_cond(PcgState* st, cudaGraphConditionalHandle loop) {
  const int bodies = ++st->bodies;
  cudaGraphSetConditional(loop, (!st->done && bodies * kLoopUnroll < st->limit) ? 1u : 0u);
}

int pcg_loop_unroll() { return kLoopUnroll; }

constexpr int kFoldMaxNodes = 16384;
bool pcg_folds_pupdate(const Shell& s) {
  return !s.val_fp64 && !s.spmv_tma && s.pcg_fold_pupdate && s.n_nodes <= kFoldMaxNodes;
}
int pcg_kernels_per_iteration(const Shell& s) { return pcg_folds_pupdate(s) ? 2 : 3; }

void drop_pcg_graphs(Shell& s) {
  for (auto& gph : s.pcg_graphs) {
    if (gph.exec) cudaGraphExecDestroy(gph.exec);
    gph = Shell::PcgGraph{};
  }
  s.pcg_graph_next = 0;
}

// The whole mixed-precision solve as one cooperative launch (k_pcg32_persistent), after
// launch_precond_setup and launch_pcg_init. Grid: one CTA per 24 nodes, at most as many as can be
// resident (occupancy x SMs) and kPersistMaxCtas.
shell_status launch_pcg_persistent(Shell& s, const unsigned char* mask) {
  if (s.val_fp64) return fail(SHELL_ERR_ARG, "the persistent PCG is for mixed precision");
  if (!s.d_persist) {
    const cudaError_t e = cudaMalloc(&s.d_persist, sizeof(PersistSync) + sizeof(float2) * 3 * kPersistMaxCtas);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s.d_persist = nullptr;
      return fail(SHELL_ERR_OOM, std::string("persistent PCG workspace: ") + cudaGetErrorString(e));
    }
    int occ = 0;
    BHEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg32_persistent, kSpmvThreads, 0));
    s.persist_max_ctas = std::min(kPersistMaxCtas, std::max(1, occ) * std::max(1, s.num_sms));
  }
  const int n = s.n_nodes;
  int G = std::max(1, std::min(s.persist_max_ctas, (n + 23) / 24));
  int per = (n + G - 1) / G;
  G = (n + per - 1) / per;
  PersistSync* ps = reinterpret_cast<PersistSync*>(s.d_persist);
  float2* part = reinterpret_cast<float2*>(reinterpret_cast<char*>(s.d_persist) + sizeof(PersistSync));
  BHEM_CUDA(cudaMemsetAsync(&ps->count, 0, sizeof(unsigned), s.stream));
  const int* rp = s.d_row_ptr;
  const int* col = s.d_col;
  const float* val = (const float*)s.d_val;
  const float* Dinv = (const float*)s.d_Dinv;
  int polls = s.wait_polls;
  void* args[] = {(void*)&n, (void*)&per, (void*)&rp, (void*)&col, (void*)&val, (void*)&Dinv, (void*)&mask,
                  (void*)&s.d_x32, (void*)&s.d_r32, (void*)&s.d_z32, (void*)&s.d_p32, (void*)&s.d_Ap32,
                  (void*)&s.d_pcg, (void*)&ps, (void*)&part, (void*)&polls, (void*)&s.d_err};
  BHEM_CUDA(cudaLaunchCooperativeKernel((const void*)k_pcg32_persistent, dim3(G), dim3(kSpmvThreads), args, 0,
                                        s.stream));
  ++s.launches;
  return SHELL_OK;
}

// Cluster size for the cluster PCG (16 where the device runs such a cluster, else 8; 0 if none),
// decided once per device.
static int cluster_pcg_ctas(int device) {
  static int cached[64] = {0};
  static bool known[64] = {false};
  const int d = device & 63;
  if (known[d]) return cached[d];
  int best = 0;
  if (cudaFuncSetAttribute(k_pcg32_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    cudaGetLastError();
  for (int c : {kClusterMaxCtas, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kClusterThreads);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_pcg32_cluster, &cfg) == cudaSuccess && nclusters > 0) {
      best = c;
      break;
    }
    cudaGetLastError();
  }
  cached[d] = best;
  known[d] = true;
  return best;
}

shell_status launch_pcg_cluster(Shell& s, const unsigned char* mask) {
  if (s.val_fp64) return fail(SHELL_ERR_ARG, "the cluster PCG is for mixed precision");
  const int C = cluster_pcg_ctas(s.device);
  if (C <= 0) return fail(SHELL_ERR_CUDA, "no thread-block cluster fits this device");
  const int n = s.n_nodes;
  const int per = (n + C - 1) / C;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.stream = s.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  BHEM_CUDA(cudaLaunchKernelEx(&cfg, k_pcg32_cluster, n, per, (const int*)s.d_row_ptr, (const int*)s.d_col,
                               (const float*)s.d_val, (const float*)s.d_Dinv, mask, s.d_x32, s.d_r32, s.d_z32,
                               s.d_p32, s.d_Ap32, s.d_pcg));
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_pcg_loop_graph(Shell& s, const unsigned char* mask) {
  if (s.val_fp64) return fail(SHELL_ERR_ARG, "PCG graphs are for mixed precision");
  Shell::PcgGraph* hit = nullptr;
  for (auto& gph : s.pcg_graphs)
    if (gph.exec && gph.mask == mask && gph.iters == -1) hit = &gph;
  if (!hit) {
    if (!s.cap_stream) BHEM_CUDA(cudaStreamCreateWithFlags(&s.cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    BHEM_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle loop;
    cudaError_t e = cudaGraphConditionalHandleCreate(&loop, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = loop;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return fail(SHELL_ERR_CUDA, std::string("PCG loop graph: ") + cudaGetErrorString(e));
    }
    // the body: kLoopUnroll iterations and the condition, captured on a private stream
    const double zero[4] = {0.0, 0.0, 0.0, 0.0};
    cudaStream_t keep = s.stream;
    const long long keep_launches = s.launches;
    s.stream = s.cap_stream;
    e = cudaStreamBeginCaptureToGraph(s.cap_stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    shell_status st = SHELL_OK;
    if (e == cudaSuccess) {
      for (int k = 0; k < kLoopUnroll && st == SHELL_OK; ++k) st = launch_pcg_iteration(s, mask, zero);
      if (st == SHELL_OK) {
        k_pcg_loop_cond<<<1, 1, 0, s.cap_stream>>>(s.d_pcg, loop);
        if (cudaGetLastError() != cudaSuccess) st = fail(SHELL_ERR_CUDA, "PCG loop condition launch");
      }
      cudaGraph_t body = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(s.cap_stream, &body);
      if (e2 != cudaSuccess && st == SHELL_OK) st = fail(SHELL_ERR_CUDA, std::string("PCG loop capture: ") + cudaGetErrorString(e2));
    } else {
      st = fail(SHELL_ERR_CUDA, std::string("PCG loop capture: ") + cudaGetErrorString(e));
    }
    s.stream = keep;
    s.launches = keep_launches;
    if (st != SHELL_OK) {
      cudaGraphDestroy(graph);
      return st;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) return fail(SHELL_ERR_CUDA, std::string("PCG loop instantiate: ") + cudaGetErrorString(e3));
    hit = &s.pcg_graphs[s.pcg_graph_next];
    if (hit->exec) cudaGraphExecDestroy(hit->exec);
    *hit = Shell::PcgGraph{mask, -1, exec};
    s.pcg_graph_next = (s.pcg_graph_next + 1) % Shell::kGraphSlots;
  }
  BHEM_CUDA(cudaGraphLaunch(hit->exec, s.stream));
  return SHELL_OK;
}


// Solution of the last PCG solve as FP64 in s.d_x (converted from the FP32 vector of a mixed
// shell).
shell_status launch_pcg_result(Shell& s) {
  if (s.val_fp64) return SHELL_OK;
  k_to_double<<<vec_blocks(s.n_dof), 256, 0, s.stream>>>(s.n_dof, s.d_x32, s.d_x);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_axpy_fixed(Shell& s, double* q, const double* d, double alpha) {
  k_axpy<<<vec_blocks(s.n_dof), 256, 0, s.stream>>>(s.n_dof, q, d, alpha);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_overwrite_fixed(Shell& s, double* dst, const double* src,
                                    const unsigned char* mask, const double* fixed_vals) {
  k_overwrite_fixed<<<vec_blocks(s.n_dof), 256, 0, s.stream>>>(s.n_dof, dst, src, mask, fixed_vals);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_predictor(Shell& s, const double* qn, const double* v, double dt, double* y) {
  k_predictor<<<vec_blocks(s.n_dof), 256, 0, s.stream>>>(s.n_dof, qn, v, dt, y);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_velocity(Shell& s, const double* q, const double* qn, double dt, double* v) {
  k_velocity<<<vec_blocks(s.n_dof), 256, 0, s.stream>>>(s.n_dof, q, qn, 1.0 / dt, v);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_negate(Shell& s, const double* a, double* b) {
  k_negate<<<vec_blocks(s.n_dof), 256, 0, s.stream>>>(s.n_dof, a, b);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

}  // namespace bhem
