// Linear-algebra kernels of the implicit-Euler Newton step (Sec. 6.1): 12x12 BSR SpMV, block-
// Jacobi preconditioner, PCG with device-resident scalars, consistent-mass products and the
// Newton residual g = dV/dq + M (q - y)/dt^2 - F. No kernel waits on another CTA: grid
// reductions use the last-CTA ticket of grid_reduce.
#include "common.cuh"

namespace bhem {

int grid_for(long long work, int per_block) {
  long long b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 0x7fffffffLL) b = 0x7fffffffLL;
  return (int)b;
}

// ------------------------------------------------------------------------------------------
// BSR SpMV  y = (A + tau |diag(A)|) p on free DOFs (y = 0 on fixed DOFs), fused with p . y.
// Each 12x12 block row is read by TPR threads, one 16-byte chunk of one row per thread, so the
// threads of a block row stream the block's 576 (FP32) or 1152 (FP64) bytes contiguously.
// ------------------------------------------------------------------------------------------
template <typename Rm> struct Chunk;
template <> struct Chunk<float> { using T = float4; static constexpr int E = 4; };
template <> struct Chunk<double> { using T = double2; static constexpr int E = 2; };

// dot of one 16-byte matrix chunk with the matching FP64 entries of x, in the matrix precision
__device__ __forceinline__ float chunk_dot(float4 a, const double* __restrict__ x) {
  const double2 x0 = *reinterpret_cast<const double2*>(x);
  const double2 x1 = *reinterpret_cast<const double2*>(x + 2);
  return a.x * (float)x0.x + a.y * (float)x0.y + a.z * (float)x1.x + a.w * (float)x1.y;
}
__device__ __forceinline__ double chunk_dot(double2 a, const double* __restrict__ x) {
  const double2 x0 = *reinterpret_cast<const double2*>(x);
  return a.x * x0.x + a.y * x0.y;
}

constexpr int kSpmvThreads = 288;

template <typename Rm>
__global__ void __launch_bounds__(kSpmvThreads)
k_spmv(int n, const int* __restrict__ rp, const int* __restrict__ col, const Rm* __restrict__ val,
       const double* __restrict__ x, const double* __restrict__ diagA, double tau,
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
    for (int k = k0; k < k1; ++k) {
      const int j = col[k];
      CT v = __ldcs(reinterpret_cast<const CT*>(val + (size_t)k * 144 + r * 12 + cc * E));
      acc += chunk_dot(v, x + (size_t)j * 12 + cc * E);
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
    const double xi = x[gi];
    double yi = s;
    if (tau != 0.0) yi += tau * fabs(diagA[gi]) * xi;
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
// Block-Jacobi: D_i = (A_ii masked + tau |diag|)^{-1} by Cholesky; a block that is not SPD falls
// back to the inverse of its diagonal. Also records diag(A). One thread per node.
// ------------------------------------------------------------------------------------------
template <typename Rm, typename Rd>
__global__ void k_precond(int n, const int* __restrict__ diag_block, const Rm* __restrict__ val,
                          const unsigned char* __restrict__ mask, double tau,
                          double* __restrict__ diagA, Rd* __restrict__ Dinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Rm* B = val + (size_t)diag_block[i] * 144;
  Rd L[144];
  bool fixed[12];
  for (int a = 0; a < 12; ++a) {
    fixed[a] = mask && mask[(size_t)i * 12 + a];
    diagA[(size_t)i * 12 + a] = (double)B[a * 13];
  }
  for (int a = 0; a < 12; ++a)
    for (int b = 0; b < 12; ++b) {
      Rd v = (Rd)B[a * 12 + b];
      if (fixed[a] || fixed[b]) v = (a == b) ? (Rd)1 : (Rd)0;
      else if (a == b) v += (Rd)(tau * fabs((double)B[a * 13]));
      L[a * 12 + b] = v;
    }
  Rd diag[12];
  for (int a = 0; a < 12; ++a) diag[a] = L[a * 13];
  bool ok = true;
  // in-place Cholesky, lower triangle
  for (int j = 0; j < 12 && ok; ++j) {
    Rd s = L[j * 13];
    for (int k = 0; k < j; ++k) s -= L[j * 12 + k] * L[j * 12 + k];
    if (!(s > (Rd)0)) { ok = false; break; }
    Rd d = sqrt(s);
    L[j * 13] = d;
    for (int a = j + 1; a < 12; ++a) {
      Rd u = L[a * 12 + j];
      for (int k = 0; k < j; ++k) u -= L[a * 12 + k] * L[j * 12 + k];
      L[a * 12 + j] = u / d;
    }
  }
  Rd* D = Dinv + (size_t)i * 144;
  if (!ok) {
    for (int a = 0; a < 12; ++a)
      for (int b = 0; b < 12; ++b)
        D[a * 12 + b] = (a == b) ? (diag[a] > (Rd)0 ? (Rd)1 / diag[a] : (Rd)1) : (Rd)0;
    return;
  }
  // W = L^{-1} (lower), stored in the upper triangle's mirror: compute column by column
  Rd Wm[144];
  for (int c = 0; c < 12; ++c) {
    for (int a = 0; a < 12; ++a) {
      if (a < c) { Wm[a * 12 + c] = 0; continue; }
      Rd u = (a == c) ? (Rd)1 : (Rd)0;
      for (int k = c; k < a; ++k) u -= L[a * 12 + k] * Wm[k * 12 + c];
      Wm[a * 12 + c] = u / L[a * 13];
    }
  }
  // D = W^T W
  for (int a = 0; a < 12; ++a)
    for (int b = a; b < 12; ++b) {
      Rd s = 0;
      for (int k = (a > b ? a : b); k < 12; ++k) s += Wm[k * 12 + a] * Wm[k * 12 + b];
      D[a * 12 + b] = s;
      D[b * 12 + a] = s;
    }
}

// ------------------------------------------------------------------------------------------
// PCG kernels: 12 threads per node, 16 nodes per CTA.
// ------------------------------------------------------------------------------------------
constexpr int kNodeThreads = 192;

template <typename Rd>
__device__ __forceinline__ double apply_block(const Rd* __restrict__ D, const double* sr, int a) {
  Rd s = 0;
#pragma unroll
  for (int c = 0; c < 12; ++c) s += D[a * 12 + c] * (Rd)sr[c];
  return (double)s;
}

template <typename Rd>
__global__ void __launch_bounds__(kNodeThreads)
k_pcg_init(int n, const double* __restrict__ rhs, const Rd* __restrict__ Dinv,
           const unsigned char* __restrict__ mask, double* __restrict__ x, double* __restrict__ r,
           double* __restrict__ z, double* __restrict__ p, double rtol2,
           int fixed, PcgState* st, Reduce red) {
  __shared__ double sr[16][12];
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  const size_t gi = (size_t)i * 12 + a;
  double ri = 0.0, zi = 0.0;
  if (i < n) {
    ri = (mask && mask[gi]) ? 0.0 : rhs[gi];
    x[gi] = 0.0;
    r[gi] = ri;
    sr[ln][a] = ri;
  }
  __syncthreads();
  if (i < n) {
    zi = (mask && mask[gi]) ? 0.0 : apply_block<Rd>(Dinv + (size_t)i * 144, sr[ln], a);
    z[gi] = zi;
    p[gi] = zi;
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
  __shared__ double sr[16][12];
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  const size_t gi = (size_t)i * 12 + a;
  const double alpha = st->alpha;
  double ri = 0.0, zi = 0.0;
  if (i < n) {
    x[gi] += alpha * p[gi];
    ri = r[gi] - alpha * Ap[gi];
    r[gi] = ri;
    sr[ln][a] = ri;
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
                              const PcgState* st) {
  if (st->done) return;
  const double beta = st->beta;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
    p[k] = z[k] + beta * p[k];
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

__global__ void k_axpy(int m, double* __restrict__ q, const double* __restrict__ d, double alpha) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) q[k] += alpha * d[k];
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
  if (blocks > kMaxPartials) return fail(SHELL_ERR_ARG, "too many nodes for one reduction");
  k_grad_finish<<<blocks, kNodeThreads, 0, s.stream>>>(s.n_nodes, s.d_row_ptr, s.d_col, s.d_mass,
                                                       s.d_fgrav, q, y, 1.0 / (dt * dt), grav[0],
                                                       grav[1], grav[2], mask, g, gin, gnorm2_out,
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
  int blocks = vec_blocks(m);
  k_dots3<<<blocks, 256, 0, s.stream>>>(m, a0, b0, a1, b1, a2, b2, out3, s.red);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_precond_setup(Shell& s, const unsigned char* mask, double tau) {
  int blocks = grid_for(s.n_nodes, 64);
  if (s.val_fp64)
    k_precond<double, double><<<blocks, 64, 0, s.stream>>>(s.n_nodes, s.d_diag_block,
        (const double*)s.d_val, mask, tau, s.d_diagA, (double*)s.d_Dinv);
  else
    k_precond<float, float><<<blocks, 64, 0, s.stream>>>(s.n_nodes, s.d_diag_block,
        (const float*)s.d_val, mask, tau, s.d_diagA, (float*)s.d_Dinv);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_pcg_init(Shell& s, const unsigned char* mask, const double* rhs, double rtol,
                             int fixed) {
  int blocks = grid_for(s.n_nodes, 16);
  if (blocks > kMaxPartials) return fail(SHELL_ERR_ARG, "too many nodes for one reduction");
  double rtol2 = fixed > 0 ? 0.0 : rtol * rtol;
  if (s.val_fp64)
    k_pcg_init<double><<<blocks, kNodeThreads, 0, s.stream>>>(
        s.n_nodes, rhs, (const double*)s.d_Dinv, mask, s.d_x, s.d_r, s.d_z, s.d_p, rtol2, fixed,
        s.d_pcg, s.red);
  else
    k_pcg_init<float><<<blocks, kNodeThreads, 0, s.stream>>>(
        s.n_nodes, rhs, (const float*)s.d_Dinv, mask, s.d_x, s.d_r, s.d_z, s.d_p, rtol2, fixed,
        s.d_pcg, s.red);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

static shell_status launch_spmv_impl(Shell& s, const double* x, const unsigned char* mask,
                                     double tau, double* y, PcgState* st) {
  const int n = s.n_nodes;
  if (s.val_fp64) {
    constexpr int RPC = kSpmvThreads / 72;
    int blocks = grid_for(n, RPC);
    if (st && blocks > kMaxPartials) return fail(SHELL_ERR_ARG, "too many nodes for one reduction");
    k_spmv<double><<<blocks, kSpmvThreads, 0, s.stream>>>(n, s.d_row_ptr, s.d_col,
        (const double*)s.d_val, x, s.d_diagA, tau, mask, y, st, s.red);
  } else {
    constexpr int RPC = kSpmvThreads / 36;
    int blocks = grid_for(n, RPC);
    if (st && blocks > kMaxPartials) return fail(SHELL_ERR_ARG, "too many nodes for one reduction");
    k_spmv<float><<<blocks, kSpmvThreads, 0, s.stream>>>(n, s.d_row_ptr, s.d_col,
        (const float*)s.d_val, x, s.d_diagA, tau, mask, y, st, s.red);
  }
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

shell_status launch_spmv(Shell& s, const double* x, double* y) {
  return launch_spmv_impl(s, x, nullptr, 0.0, y, nullptr);
}

shell_status launch_pcg_iteration(Shell& s, const unsigned char* mask, double tau) {
  const int n = s.n_nodes, m = s.n_dof;
  BHEM_TRY(launch_spmv_impl(s, s.d_p, mask, tau, s.d_Ap, s.d_pcg));
  if (s.val_fp64)
    k_pcg_update<double><<<grid_for(n, 16), kNodeThreads, 0, s.stream>>>(
        n, s.d_x, s.d_r, s.d_z, s.d_p, s.d_Ap, (const double*)s.d_Dinv, mask, s.d_pcg, s.red);
  else
    k_pcg_update<float><<<grid_for(n, 16), kNodeThreads, 0, s.stream>>>(
        n, s.d_x, s.d_r, s.d_z, s.d_p, s.d_Ap, (const float*)s.d_Dinv, mask, s.d_pcg, s.red);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  k_pcg_pupdate<<<vec_blocks(m), 256, 0, s.stream>>>(m, s.d_z, s.d_p, s.d_pcg);
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
