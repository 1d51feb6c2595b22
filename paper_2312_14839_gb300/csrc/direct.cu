// Direct solver for the Newton systems (the paper's solver in Sec. 6.1 is a sparse LDL^T): the
// assembled BSR matrix plus the diagonal regulariser tau D is expanded into a dense FP64 matrix
// and factorised by Cholesky (cuSOLVER potrf; for the positive-definite systems Newton needs,
// A = L L^T is the LDL^T factorisation with D = diag(L)^2), then solved (potrs). A failed
// factorisation means A + tau D is not positive definite, which the Newton loop treats like
// negative curvature met by PCG: tau grows tenfold and the system is solved again. This is a
// comparator for the iterative path, for systems of up to kMaxDense unknowns.
#include <cusolverDn.h>

#include <string>

#include "common.cuh"

namespace bhem {
namespace {

constexpr int kMaxDense = 65536;

// One CTA per block row of the BSR, one thread per entry of a 12 x 12 block: A[gi, gj]
// (column-major, n x n) = the block entry, prescribed rows and columns replaced by the identity,
// the free diagonal shifted by td[kind].
template <typename T>
__global__ void __launch_bounds__(144) k_bsr_dense(int n, const int* __restrict__ row_ptr, const int* __restrict__ col,
                                                   const T* __restrict__ val, const unsigned char* __restrict__ mask,
                                                   Shift4 td, double* __restrict__ A) {
  const int i = blockIdx.x, e = threadIdx.x, r = e / 12, c = e % 12;
  const long long gi = 12LL * i + r;
  for (int b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
    const long long gj = 12LL * col[b] + c;
    double v = (double)val[(size_t)b * 144 + e];
    if (mask && (mask[gi] || mask[gj])) v = gi == gj ? 1.0 : 0.0;
    else if (gi == gj) v += td.v[r / 3];
    A[gj * n + gi] = v;
  }
}

__global__ void k_masked_copy(int n, const double* __restrict__ src, const unsigned char* __restrict__ mask,
                              double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (mask && mask[i]) ? 0.0 : src[i];
}

}  // namespace

void destroy_direct(Shell& s) {
  if (s.cusolver) cusolverDnDestroy((cusolverDnHandle_t)s.cusolver);
  if (s.d_dense) cudaFree(s.d_dense);
  if (s.d_dense_work) cudaFree(s.d_dense_work);
  s.cusolver = nullptr;
  s.d_dense = nullptr;
  s.d_dense_work = nullptr;
}

// Solves (A + tau D) x = rhs on the free DOFs (x = 0 on prescribed ones) into s.d_x. *not_pd is
// set, and s.d_x left unspecified, when the Cholesky factorisation fails.
shell_status run_direct(Shell& s, const unsigned char* mask, const double td[4], const double* rhs, int* not_pd) {
  const int n = s.n_dof;
  if (n > kMaxDense) return fail(SHELL_ERR_ARG, "the direct solver takes at most 65,536 DOF");
  *not_pd = 0;
  if (!s.cusolver) {
    cusolverDnHandle_t h = nullptr;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return fail(SHELL_ERR_CUDA, "cusolverDnCreate failed");
    s.cusolver = h;
  }
  cusolverDnHandle_t h = (cusolverDnHandle_t)s.cusolver;
  if (cusolverDnSetStream(h, s.stream) != CUSOLVER_STATUS_SUCCESS) return fail(SHELL_ERR_CUDA, "cusolverDnSetStream");
  if (!s.d_dense) {
    const cudaError_t e = cudaMalloc((void**)&s.d_dense, sizeof(double) * (size_t)n * n + sizeof(int) * 2);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s.d_dense = nullptr;
      return fail(SHELL_ERR_OOM, std::string("dense matrix: ") + cudaGetErrorString(e));
    }
    int lwork = 0;
    if (cusolverDnDpotrf_bufferSize(h, CUBLAS_FILL_MODE_LOWER, n, s.d_dense, n, &lwork) != CUSOLVER_STATUS_SUCCESS)
      return fail(SHELL_ERR_CUDA, "cusolverDnDpotrf_bufferSize failed");
    const cudaError_t e2 = cudaMalloc((void**)&s.d_dense_work, sizeof(double) * (size_t)(lwork > 0 ? lwork : 1));
    if (e2 != cudaSuccess) {
      cudaGetLastError();
      s.d_dense_work = nullptr;
      return fail(SHELL_ERR_OOM, std::string("dense workspace: ") + cudaGetErrorString(e2));
    }
    s.dense_lwork = lwork;
  }
  int* d_info = (int*)(s.d_dense + (size_t)n * n);
  BHEM_CUDA(cudaMemsetAsync(s.d_dense, 0, sizeof(double) * (size_t)n * n, s.stream));
  const Shift4 sh{{td[0], td[1], td[2], td[3]}};
  if (s.val_fp64)
    k_bsr_dense<double><<<s.n_nodes, 144, 0, s.stream>>>(n, s.d_row_ptr, s.d_col, (const double*)s.d_val, mask, sh,
                                                         s.d_dense);
  else
    k_bsr_dense<float><<<s.n_nodes, 144, 0, s.stream>>>(n, s.d_row_ptr, s.d_col, (const float*)s.d_val, mask, sh,
                                                        s.d_dense);
  k_masked_copy<<<grid_for(n, 256), 256, 0, s.stream>>>(n, rhs, mask, s.d_x);
  s.launches += 2;
  BHEM_CUDA(cudaGetLastError());
  if (cusolverDnDpotrf(h, CUBLAS_FILL_MODE_LOWER, n, s.d_dense, n, s.d_dense_work, s.dense_lwork, d_info) !=
      CUSOLVER_STATUS_SUCCESS)
    return fail(SHELL_ERR_CUDA, "cusolverDnDpotrf failed");
  int info = 0;
  BHEM_CUDA(cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, s.stream));
  BHEM_CUDA(cudaStreamSynchronize(s.stream));
  if (info > 0) {
    *not_pd = 1;
    return SHELL_OK;
  }
  if (info < 0) return fail(SHELL_ERR_CUDA, "cusolverDnDpotrf: invalid argument " + std::to_string(-info));
  if (cusolverDnDpotrs(h, CUBLAS_FILL_MODE_LOWER, n, 1, s.d_dense, n, s.d_x, n, d_info + 1) != CUSOLVER_STATUS_SUCCESS)
    return fail(SHELL_ERR_CUDA, "cusolverDnDpotrs failed");
  return SHELL_OK;
}

}  // namespace bhem
