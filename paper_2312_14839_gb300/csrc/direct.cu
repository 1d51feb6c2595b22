// Direct solver for the Newton systems (the paper's solver in Sec. 6.1 is a sparse LDL^T). The
// regular patch grid makes A block tridiagonal over the node rows: with the nodes ordered row by
// row along one grid direction, a node couples only with nodes of its own row and of the two
// neighbouring rows (Sec. 4.3: two nodes couple iff they share a patch). So the Cholesky factor
// is banded: A = L L^T with L block lower bidiagonal, and no fill-in outside the bands,
//   L_00 L_00^T = A_00,   L_{j+1,j} = A_{j+1,j} L_jj^{-T},
//   L_{j+1,j+1} L_{j+1,j+1}^T = A_{j+1,j+1} - L_{j+1,j} L_{j+1,j}^T,
// in FP64. For the positive-definite systems Newton needs, L L^T is the LDL^T factorisation with
// D = diag(L)^2. Every dense row block (12 x nodes-per-row unknowns) is factorised by a right-
// looking blocked Cholesky (32-column panels: diagonal block, panel solve, trailing update), all
// hand-written kernels. A pivot that is not positive means A + tau D is not positive definite,
// which the Newton loop treats like negative curvature met by PCG (tau grows tenfold).
//
// The rows run along the grid direction that gives the narrower rows and is not periodic (a
// periodic direction would couple the first and the last row); shells periodic in both
// directions are rejected, as are rows of more than kMaxBand unknowns.
#include <algorithm>
#include <cmath>
#include <string>

#include "common.cuh"

namespace bhem {
namespace {

constexpr int kNb = 32;           // panel width of the blocked Cholesky
constexpr int kMaxBand = 4096;    // unknowns per row block
constexpr size_t kMaxBytes = 8ull << 30;

struct Band {
  int along_v;   // 1: rows are node rows j (node = j * n1 + i); 0: rows are node columns i
  int rows, B;   // row blocks and unknowns per row block
  int n1;
};

__device__ __forceinline__ void node_rowpos(const Band& b, int node, int* row, int* pos) {
  if (b.along_v) { *row = node / b.n1; *pos = node % b.n1; }
  else { *row = node % b.n1; *pos = node / b.n1; }
}

// global DOF of unknown l of row block j
__device__ __forceinline__ long long dof_of(const Band& b, int j, int l) {
  const int pos = l / 12, k = l % 12;
  const long long node = b.along_v ? (long long)j * b.n1 + pos : (long long)pos * b.n1 + j;
  return node * 12 + k;
}

// One CTA per node, one thread per entry of a 12 x 12 block: the diagonal row blocks Ad[j] and
// the sub-diagonal blocks Ao[j] (rows of row block j + 1, columns of row block j), row-major
// B x B, prescribed rows and columns replaced by the identity, the free diagonal shifted by td.
template <typename T>
__global__ void __launch_bounds__(144) k_band_blocks(int n, Band b, const int* __restrict__ row_ptr,
                                                     const int* __restrict__ col, const T* __restrict__ val,
                                                     const unsigned char* __restrict__ mask, Shift4 td,
                                                     double* __restrict__ Ad, double* __restrict__ Ao) {
  const int I = blockIdx.x, e = threadIdx.x, r = e / 12, c = e % 12;
  if (I >= n) return;
  int jI, pI;
  node_rowpos(b, I, &jI, &pI);
  const long long gi = 12LL * I + r;
  const size_t BB = (size_t)b.B * b.B;
  for (int k = row_ptr[I]; k < row_ptr[I + 1]; ++k) {
    const int J = col[k];
    int jJ, pJ;
    node_rowpos(b, J, &jJ, &pJ);
    const long long gj = 12LL * J + c;
    double v = (double)val[(size_t)k * 144 + e];
    if (mask && (mask[gi] || mask[gj])) v = gi == gj ? 1.0 : 0.0;
    else if (gi == gj) v += td.v[r / 3];
    const size_t at = (size_t)(pI * 12 + r) * b.B + pJ * 12 + c;
    if (jJ == jI) Ad[(size_t)jI * BB + at] = v;
    else if (jI == jJ + 1) Ao[(size_t)jJ * BB + at] = v;
  }
}

// Cholesky of the nb x nb diagonal block at (k, k) of S (row-major, leading dimension ld), in
// shared memory by one CTA, lower triangle written back. A pivot that is not positive (or not
// finite) raises *flag, and every later kernel of the factorisation returns at once.
__global__ void __launch_bounds__(256) k_potf2(double* __restrict__ S, int ld, int k, int nb, int* flag) {
  __shared__ double a[kNb][kNb + 1];
  if (*flag) return;
  const int t = threadIdx.x;
  for (int e = t; e < nb * nb; e += blockDim.x) a[e / nb][e % nb] = S[(size_t)(k + e / nb) * ld + k + e % nb];
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    const double d = a[c][c];
    if (!(d > 0.0) || !isfinite(d)) {   // uniform: every thread reads the same value
      if (t == 0) atomicExch(flag, 1);
      return;
    }
    const double l = sqrt(d);
    __syncthreads();
    if (t == 0) a[c][c] = l;
    for (int i = c + 1 + t; i < nb; i += blockDim.x) a[i][c] /= l;
    __syncthreads();
    for (int e = t; e < (nb - c - 1) * (nb - c - 1); e += blockDim.x) {
      const int i = c + 1 + e / (nb - c - 1), j = c + 1 + e % (nb - c - 1);
      if (j <= i) a[i][j] -= a[i][c] * a[j][c];
    }
    __syncthreads();
  }
  for (int e = t; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    if (j <= i) S[(size_t)(k + i) * ld + k + j] = a[i][j];
  }
}

// Panel solve below the diagonal block: rows i >= k + nb of columns k .. k + nb - 1 become
// S[i, k:] L_kk^{-T} (forward substitution with the factored diagonal block, one thread a row).
__global__ void __launch_bounds__(128) k_trsm_panel(double* __restrict__ S, int ld, int m, int k, int nb, int* flag) {
  __shared__ double L[kNb][kNb + 1];
  if (*flag) return;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x)
    L[e / nb][e % nb] = S[(size_t)(k + e / nb) * ld + k + e % nb];
  __syncthreads();
  const int i = k + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double x[kNb];
  double* row = S + (size_t)i * ld + k;
#pragma unroll
  for (int c = 0; c < kNb; ++c) x[c] = c < nb ? row[c] : 0.0;
#pragma unroll
  for (int c = 0; c < kNb; ++c) {
    if (c >= nb) break;
    double s = x[c];
#pragma unroll
    for (int t = 0; t < kNb; ++t)
      if (t < c) s -= x[t] * L[c][t];
    x[c] = s / L[c][c];
  }
#pragma unroll
  for (int c = 0; c < kNb; ++c)
    if (c < nb) row[c] = x[c];
}

// Symmetric rank-K downdate of the lower triangle: C[i][j] -= sum_t P[i][t] P[j][t] for
// 0 <= j <= i < m. One CTA per 32 x 32 tile of the lower triangle (blockIdx.y = tile row,
// blockIdx.x = tile column), 256 threads, 4 outputs each; K is staged in 32-wide slices.
__global__ void __launch_bounds__(256) k_syrk_lower(double* __restrict__ C, int ldc, const double* __restrict__ P,
                                                    int ldp, int m, int K, const int* flag) {
  __shared__ double Pi[32][33], Pj[32][33];
  if (*flag) return;
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (tj > ti) return;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 32 x 8
  const int i0 = ti * 32, j0 = tj * 32;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t0 = 0; t0 < K; t0 += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int r = e / 32, t = e % 32;
      Pi[r][t] = (i0 + r < m && t0 + t < K) ? P[(size_t)(i0 + r) * ldp + t0 + t] : 0.0;
      Pj[r][t] = (j0 + r < m && t0 + t < K) ? P[(size_t)(j0 + r) * ldp + t0 + t] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
      const double pj = Pj[tx][t];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += Pi[ty + 8 * u][t] * pj;
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty + 8 * u, j = j0 + tx;
    if (i < m && j < m && j <= i) C[(size_t)i * ldc + j] -= acc[u];
  }
}

// X <- X L^{-T} for the B x B sub-diagonal block X = A_{j+1,j} (L = L_jj lower): each row of X is
// one forward substitution, one warp per row (lanes split the dot products).
__global__ void __launch_bounds__(256) k_trsm_rows(double* __restrict__ X, const double* __restrict__ L, int B,
                                                   const int* flag) {
  if (*flag) return;
  const int lane = threadIdx.x & 31, r = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= B) return;
  double* x = X + (size_t)r * B;
  for (int c = 0; c < B; ++c) {
    const double* Lc = L + (size_t)c * B;
    double s = 0.0;
    for (int t = lane; t < c; t += 32) s += x[t] * Lc[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[c] = (x[c] - s) / Lc[c];
    __syncwarp();
  }
}

// Forward substitution of row block j: y_j = L_jj^{-1} (b_j - L_{j,j-1} y_{j-1}); b is the
// right-hand side in DOF order (prescribed DOFs read as 0), y is the row-block-ordered work
// vector. One CTA; the row block's residual is kept in shared memory.
__global__ void __launch_bounds__(512) k_solve_fwd(Band b, int j, const double* __restrict__ Ad,
                                                   const double* __restrict__ Ao, const double* __restrict__ rhs,
                                                   const unsigned char* __restrict__ mask, double* __restrict__ y) {
  extern __shared__ double r[];
  const int B = b.B, t = threadIdx.x;
  const size_t BB = (size_t)B * B;
  const double* L = Ad + (size_t)j * BB;
  for (int i = t; i < B; i += blockDim.x) {
    const long long g = dof_of(b, j, i);
    double v = (mask && mask[g]) ? 0.0 : rhs[g];
    if (j > 0) {
      const double* Lo = Ao + (size_t)(j - 1) * BB + (size_t)i * B;
      const double* yp = y + (size_t)(j - 1) * B;
      for (int s = 0; s < B; ++s) v -= Lo[s] * yp[s];
    }
    r[i] = v;
  }
  __syncthreads();
  for (int c = 0; c < B; ++c) {
    const double yc = r[c] / L[(size_t)c * B + c];
    __syncthreads();
    if (t == 0) r[c] = yc;
    for (int i = c + 1 + t; i < B; i += blockDim.x) r[i] -= L[(size_t)i * B + c] * yc;
    __syncthreads();
  }
  for (int i = t; i < B; i += blockDim.x) y[(size_t)j * B + i] = r[i];
}

// Back substitution of row block j: x_j = L_jj^{-T} (y_j - L_{j+1,j}^T x_{j+1}); writes the DOF-
// ordered solution (prescribed DOFs 0) and keeps the row block's values in xr for row j - 1.
__global__ void __launch_bounds__(512) k_solve_bwd(Band b, int j, const double* __restrict__ Ad,
                                                   const double* __restrict__ Ao, const double* __restrict__ y,
                                                   const unsigned char* __restrict__ mask, double* __restrict__ xr,
                                                   double* __restrict__ x) {
  extern __shared__ double r[];
  const int B = b.B, t = threadIdx.x;
  const size_t BB = (size_t)B * B;
  const double* L = Ad + (size_t)j * BB;
  for (int i = t; i < B; i += blockDim.x) {
    double v = y[(size_t)j * B + i];
    if (j + 1 < b.rows) {
      const double* Lo = Ao + (size_t)j * BB;   // rows of row block j + 1, columns of j
      const double* xn = xr + (size_t)(j + 1) * B;
      for (int s = 0; s < B; ++s) v -= Lo[(size_t)s * B + i] * xn[s];
    }
    r[i] = v;
  }
  __syncthreads();
  for (int c = B - 1; c >= 0; --c) {
    const double xc = r[c] / L[(size_t)c * B + c];
    __syncthreads();
    if (t == 0) r[c] = xc;
    for (int i = t; i < c; i += blockDim.x) r[i] -= L[(size_t)c * B + i] * xc;
    __syncthreads();
  }
  for (int i = t; i < B; i += blockDim.x) {
    xr[(size_t)j * B + i] = r[i];
    const long long g = dof_of(b, j, i);
    x[g] = (mask && mask[g]) ? 0.0 : r[i];
  }
}

Band band_of(const Shell& s) {
  Band b{};
  const shell_grid& g = s.grid;
  const bool v_ok = !g.periodic_v, u_ok = !g.periodic_u;
  // rows along v: row blocks of n1 nodes; rows along u: row blocks of n2 nodes
  b.along_v = v_ok && (!u_ok || s.n1 <= s.n2) ? 1 : 0;
  b.n1 = s.n1;
  b.rows = b.along_v ? s.n2 : s.n1;
  b.B = 12 * (b.along_v ? s.n1 : s.n2);
  if (!v_ok && !u_ok) b.rows = 0;
  return b;
}

}  // namespace

void destroy_direct(Shell& s) {
  if (s.d_dense) cudaFree(s.d_dense);
  s.d_dense = nullptr;
}

// Solves (A + tau D) x = rhs on the free DOFs (x = 0 on prescribed ones) into s.d_x. *not_pd is
// set, and s.d_x left unspecified, when a Cholesky pivot is not positive.
shell_status run_direct(Shell& s, const unsigned char* mask, const double td[4], const double* rhs, int* not_pd) {
  const Band b = band_of(s);
  if (b.rows == 0) return fail(SHELL_ERR_ARG, "the direct solver needs a grid that is not periodic in both directions");
  if (b.B > kMaxBand) return fail(SHELL_ERR_ARG, "the direct solver takes rows of at most 4096 unknowns");
  const size_t BB = (size_t)b.B * b.B;
  const size_t bytes = sizeof(double) * (BB * (2 * (size_t)b.rows) + 2 * (size_t)b.rows * b.B) + 256;
  if (bytes > kMaxBytes) return fail(SHELL_ERR_ARG, "the direct solver's factor would exceed 8 GB");
  *not_pd = 0;
  if (!s.d_dense) {
    const cudaError_t e = cudaMalloc((void**)&s.d_dense, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s.d_dense = nullptr;
      return fail(SHELL_ERR_OOM, std::string("banded factor: ") + cudaGetErrorString(e));
    }
  }
  double* Ad = s.d_dense;
  double* Ao = Ad + BB * b.rows;
  double* yv = Ao + BB * b.rows;
  double* xr = yv + (size_t)b.rows * b.B;
  int* flag = reinterpret_cast<int*>(xr + (size_t)b.rows * b.B);
  BHEM_CUDA(cudaMemsetAsync(Ad, 0, sizeof(double) * BB * 2 * b.rows, s.stream));
  BHEM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s.stream));
  const Shift4 sh{{td[0], td[1], td[2], td[3]}};
  if (s.val_fp64)
    k_band_blocks<double><<<s.n_nodes, 144, 0, s.stream>>>(s.n_nodes, b, s.d_row_ptr, s.d_col,
                                                           (const double*)s.d_val, mask, sh, Ad, Ao);
  else
    k_band_blocks<float><<<s.n_nodes, 144, 0, s.stream>>>(s.n_nodes, b, s.d_row_ptr, s.d_col,
                                                          (const float*)s.d_val, mask, sh, Ad, Ao);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  const int B = b.B;
  for (int j = 0; j < b.rows; ++j) {
    double* S = Ad + (size_t)j * BB;
    for (int k = 0; k < B; k += kNb) {
      const int nb = std::min(kNb, B - k), rest = B - k - nb;
      k_potf2<<<1, 256, 0, s.stream>>>(S, B, k, nb, flag);
      ++s.launches;
      if (rest > 0) {
        k_trsm_panel<<<(rest + 127) / 128, 128, 0, s.stream>>>(S, B, B, k, nb, flag);
        const int tiles = (rest + 31) / 32;
        k_syrk_lower<<<dim3(tiles, tiles), 256, 0, s.stream>>>(S + (size_t)(k + nb) * B + k + nb, B,
                                                               S + (size_t)(k + nb) * B + k, B, rest, nb, flag);
        s.launches += 2;
      }
    }
    if (j + 1 < b.rows) {
      double* X = Ao + (size_t)j * BB;
      k_trsm_rows<<<(B + 7) / 8, 256, 0, s.stream>>>(X, S, B, flag);
      const int tiles = (B + 31) / 32;
      k_syrk_lower<<<dim3(tiles, tiles), 256, 0, s.stream>>>(Ad + (size_t)(j + 1) * BB, B, X, B, B, B, flag);
      s.launches += 2;
    }
    BHEM_CUDA(cudaGetLastError());
  }
  int h_flag = 0;
  BHEM_CUDA(cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s.stream));
  BHEM_CUDA(cudaStreamSynchronize(s.stream));
  if (h_flag) {
    *not_pd = 1;
    return SHELL_OK;
  }
  const size_t smem = sizeof(double) * B;
  if (smem > 48 * 1024) {
    BHEM_CUDA(cudaFuncSetAttribute(k_solve_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BHEM_CUDA(cudaFuncSetAttribute(k_solve_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  for (int j = 0; j < b.rows; ++j) k_solve_fwd<<<1, 512, smem, s.stream>>>(b, j, Ad, Ao, rhs, mask, yv);
  for (int j = b.rows - 1; j >= 0; --j) k_solve_bwd<<<1, 512, smem, s.stream>>>(b, j, Ad, Ao, yv, mask, xr, s.d_x);
  s.launches += 2LL * b.rows;
  BHEM_CUDA(cudaGetLastError());
  return SHELL_OK;
}

}  // namespace bhem
