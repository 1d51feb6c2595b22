// Element kernels of the BHEM hot path: per-patch energy, 48-DOF gradient and 48x48 Hessian
// (App. B) with the 4x4 Gauss rule (App. A.2), and their scatter into the 12x12 BSR matrix.
//
// Factorisation used by the Hessian kernel. At one Gauss point every term of App. B.2 is a sum
// of products phi_k^I phi_l^J B_kl over five shape-derivative kinds k, l in {,1 ,2 ,11 ,22 ,12}:
//   K_IJ = sum_g sum_{k,l} phi_gk^I phi_gl^J M_g[k,l],   M_g[k,l] in R^{3x3}
// where M_g (15x15, symmetric) collects h (d alpha)^T H (d alpha) + h^3/12 (d beta)^T H (d beta),
// the (H alpha) second-derivative term of alpha and, for the exact Hessian, the
// (H beta) second-derivative term of beta. The latter is linear in a_{a,b}, so the three Voigt
// components merge into one vector c~ = sum_i w_i a_{(i)} (w = (m1, m2, 2 m3), m = H beta) and
// one set of D^{gamma delta}(c~) matrices. The kernel then forms T = phi^T M_g per row I and
// K += T phi per column J.
#include "element_impl.cuh"

namespace bhem {

// Shape table and Gauss weights of one shell, built once (FP64 arithmetic) into global memory.
__global__ void k_shape_table(double d1, double d2, double* __restrict__ t64, float* __restrict__ t32) {
  __shared__ double sphi[kPhiSize];
  for (int e = threadIdx.x; e < kPhiSize; e += blockDim.x) sphi[e] = 0.0;
  __syncthreads();
  build_shape_table<double>(sphi, d1, d2);
  __syncthreads();
  for (int e = threadIdx.x; e < kPhiTable; e += blockDim.x) {
    double v = e < kPhiSize ? sphi[e] : gauss_weight(e - kPhiSize, d1, d2);
    t64[e] = v;
    t32[e] = (float)v;
  }
}

// ------------------------------------------------------------------------------------------
// Rest data per Gauss point (FP64, once per shell): a_bar_{ab}, b_bar_{ab}, Voigt H, W sqrt(a_bar)
// SoA: restgp[f * (np * 16) + p * 16 + g], f = 0..12.
// ------------------------------------------------------------------------------------------
__global__ void k_rest_setup(int np, const int4* __restrict__ pnodes, const double* __restrict__ rest,
                             const double* __restrict__ table, double lam, double mu,
                             double* __restrict__ restgp, int* err) {
  __shared__ double sphi[kPhiTable];
  load_shape_table<double>(sphi, table);
  __syncthreads();
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)np * 16) return;
  int p = (int)(t >> 4), g = (int)(t & 15);
  int4 pn = pnodes[p];
  int nd[4] = {pn.x, pn.y, pn.z, pn.w};
  double qb[48];
  for (int l = 0; l < 48; ++l) qb[l] = rest[(size_t)nd[l / 12] * 12 + (l % 12)];
  V3<double> v[5];
  interp5<double, double>(sphi, qb, g, v);
  V3<double> a1 = v[0], a2 = v[1];
  double a11 = dot(a1, a1), a22 = dot(a2, a2), a12 = dot(a1, a2);
  double det = a11 * a22 - a12 * a12;
  if (!(det > 1e-300)) { atomicOr(err, ERRBIT_DEGENERATE); det = 1.0; }
  double sq = sqrt(det);
  V3<double> a3 = (1.0 / sq) * cross(a1, a2);
  double ai11 = a22 / det, ai22 = a11 / det, ai12 = -a12 / det;
  size_t S = (size_t)np * 16, o = (size_t)p * 16 + g;
  restgp[0 * S + o] = a11;
  restgp[1 * S + o] = a22;
  restgp[2 * S + o] = a12;
  restgp[3 * S + o] = dot(v[2], a3);
  restgp[4 * S + o] = dot(v[3], a3);
  restgp[5 * S + o] = dot(v[4], a3);
  // Voigt H of App. B.1
  restgp[6 * S + o] = (lam + 2 * mu) * ai11 * ai11;
  restgp[7 * S + o] = lam * ai11 * ai22 + 2 * mu * ai12 * ai12;
  restgp[8 * S + o] = (lam + 2 * mu) * ai11 * ai12;
  restgp[9 * S + o] = (lam + 2 * mu) * ai22 * ai22;
  restgp[10 * S + o] = (lam + 2 * mu) * ai12 * ai22;
  restgp[11 * S + o] = (lam + mu) * ai12 * ai12 + mu * ai11 * ai22;
  restgp[12 * S + o] = sphi[kPhiSize + g] * sq;
}

// Consistent mass (Eq. mass) as 4x4 scalar blocks and gravity load factors (Sec. 4.3).
// One warp per patch; atomic scatter (once per shell).
__global__ void k_mass(int np, const int* __restrict__ pblocks, const int4* __restrict__ pnodes,
                       const double* __restrict__ restgp, const double* __restrict__ table,
                       double rho_h, double* __restrict__ mass, double* __restrict__ fgrav) {
  __shared__ double sphi[kPhiTable];
  load_shape_table<double>(sphi, table);
  __syncthreads();
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  size_t S = (size_t)np * 16;
  for (int p = warp; p < np; p += nwarps) {
    double w[16];
    for (int g = 0; g < 16; ++g) w[g] = rho_h * restgp[12 * S + (size_t)p * 16 + g];
    for (int e = lane; e < 256 + 16; e += 32) {
      if (e < 256) {
        int I = e >> 4, J = e & 15;
        double s = 0.0;
        for (int g = 0; g < 16; ++g) s += w[g] * sphi[I * kPhiStride + g] * sphi[J * kPhiStride + g];
        int kb = pblocks[p * 16 + (I >> 2) * 4 + (J >> 2)];
        atomicAdd(&mass[(size_t)kb * 16 + (I & 3) * 4 + (J & 3)], s);
      } else {
        int I = e - 256;
        double s = 0.0;
        for (int g = 0; g < 16; ++g) s += w[g] * sphi[I * kPhiStride + g];
        int4 pn = pnodes[p];
        int nd[4] = {pn.x, pn.y, pn.z, pn.w};
        atomicAdd(&fgrav[(size_t)nd[I >> 2] * 4 + (I & 3)], s);
      }
    }
  }
}

shell_status launch_rest_setup(Shell& s) {
  int np = s.n_patches;
  long long threads = (long long)np * 16;
  int blocks = (int)((threads + 255) / 256);
  k_shape_table<<<1, 256, 0, s.stream>>>(s.grid.dxi1, s.grid.dxi2, s.d_phi64, s.d_phi32);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  k_rest_setup<<<blocks, 256, 0, s.stream>>>(np, s.d_patch_nodes, s.d_rest, s.d_phi64, s.lam, s.mu,
                                             s.d_restgp, s.d_err);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  BHEM_CUDA(cudaMemsetAsync(s.d_mass, 0, sizeof(double) * 16 * (size_t)s.n_blocks, s.stream));
  BHEM_CUDA(cudaMemsetAsync(s.d_fgrav, 0, sizeof(double) * 4 * (size_t)s.n_nodes, s.stream));
  int mblocks = grid_for((long long)np * 32, 256);
  k_mass<<<mblocks, 256, 0, s.stream>>>(np, s.d_patch_blocks, s.d_patch_nodes, s.d_restgp,
                                        s.d_phi64, s.mat.density * s.mat.thickness, s.d_mass,
                                        s.d_fgrav);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

// ------------------------------------------------------------------------------------------
// Light FP64 kernel: energy (and gradient) per patch, half a warp per patch, lane = Gauss point.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
k_energy_grad64(int np, const int4* __restrict__ pnodes, const double* __restrict__ q,
                const double* __restrict__ dir, double step, const double* __restrict__ restgp,
                double dxi1, double dxi2, double h, double* __restrict__ energy_p,
                const double* __restrict__ energy_ref, double* __restrict__ grad, Reduce red,
                double* scal_out, int* err) {
  __shared__ double w1[kHerm1D], w2[kHerm1D];
  __shared__ double sq[kEgPatches][48];
  __shared__ double sT[kEgPatches][144];
  __shared__ double sG[kEgPatches][16][15];
  build_hermite_1d(w1, dxi1, threadIdx.x, blockDim.x);
  build_hermite_1d(w2, dxi2, threadIdx.x, blockDim.x);
  __syncthreads();
  const int hw = threadIdx.x >> 4, g = threadIdx.x & 15;
  const int p = blockIdx.x * kEgPatches + hw;
  const bool active = p < np;
  int nd[4] = {0, 0, 0, 0};
  if (active) {
    int4 pn = pnodes[p];
    nd[0] = pn.x; nd[1] = pn.y; nd[2] = pn.z; nd[3] = pn.w;
  }
  const double ep = eg64_patch(w1, w2, sq[hw], sT[hw], sG[hw], p, active, g, nd, q, dir, step, restgp,
                               (size_t)np * 16, h, grad, err);
  double contrib = 0.0;
  if (active && g == 0) {
    if (!isfinite(ep)) atomicOr(err, ERRBIT_NONFINITE);
    if (energy_ref) contrib = ep - energy_ref[p];
    else contrib = ep;
    if (energy_p) energy_p[p] = ep;
  }
  if (scal_out) {
    double vv[1] = {contrib};
    grid_reduce<1>(vv, red, scal_out, gridDim.x);
  }
}

shell_status launch_energy_grad64(Shell& s, const double* q, const double* dir, double step,
                                  double* energy_p, const double* energy_ref, double* grad,
                                  double* scal_out) {
  int blocks = (s.n_patches + kEgPatches - 1) / kEgPatches;
  if (blocks > s.red.stride) return fail(SHELL_ERR_ARG, "too many patches for one reduction");
  k_energy_grad64<<<blocks, 128, 0, s.stream>>>(s.n_patches, s.d_patch_nodes, q, dir, step,
                                                s.d_restgp, s.grid.dxi1, s.grid.dxi2,
                                                s.mat.thickness, energy_p, energy_ref, grad, s.red,
                                                scal_out, s.d_err);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

// ------------------------------------------------------------------------------------------
// Heavy kernel: one warp per patch computes E, gradient and the 48x48 Hessian.
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(32 * ElemCfg<R>::kWarps)
k_element_full(ElemArgs A) {
  constexpr int NW = ElemCfg<R>::kWarps;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sphi = reinterpret_cast<R*>(smem_raw);
  R* w1d = sphi + ((kPhiTable + 3) & ~3);
  WarpSmem<R>* Ws = reinterpret_cast<WarpSmem<R>*>(smem_raw + sizeof(R) * elem_table_elems<R>());
  R* sphg = w1d + 2 * kHerm1D;
  load_shape_table<R>(sphi, reinterpret_cast<const R*>(A.phi));
  build_hermite_1d<R>(w1d, A.d1, threadIdx.x, blockDim.x);
  build_hermite_1d<R>(w1d + kHerm1D, A.d2, threadIdx.x, blockDim.x);
  __syncthreads();
  if constexpr (sizeof(R) == 4) {
    build_phi_gauss(sphg, sphi, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpSmem<R>& W = Ws[wid];
  const int total = A.plist ? A.plist_n : A.np;
  const int stride = gridDim.x * NW;
  if constexpr (sizeof(R) == 4) {
    if (A.grad64) {
      // FP64 energy and gradient at the same q (the arithmetic of k_energy_grad64) in the warps of
      // the FP32 Hessian: the FP64 pipe works while other warps issue the FP32 pass. Every second
      // patch of a warp, its two half-warps evaluate that patch and the warp's next one, in the
      // warp's Gauss-point-matrix area (free between patches; 2 x 432 doubles).
      __shared__ double w1_64[kHerm1D], w2_64[kHerm1D];
      build_hermite_1d<double>(w1_64, A.d1, threadIdx.x, blockDim.x);
      build_hermite_1d<double>(w2_64, A.d2, threadIdx.x, blockDim.x);
      __syncthreads();
      static_assert(sizeof(W.M) >= 2 * 432 * sizeof(double), "FP64 scratch fits the M_g area");
      const int hw = lane >> 4, g = lane & 15;
      double* scratch = reinterpret_cast<double*>(&W.M[0][0]) + hw * 432;
      int k = 0;
      for (int it = blockIdx.x * NW + wid; it < total; it += stride, ++k) {
        if ((k & 1) == 0) {
          const int itp = it + hw * stride;
          const bool active = itp < total;
          const int pp = active ? (A.plist ? A.plist[itp] : itp) : 0;
          int nd[4] = {0, 0, 0, 0};
          if (active) {
            const int4 pn = A.pnodes[pp];
            nd[0] = pn.x;
            nd[1] = pn.y;
            nd[2] = pn.z;
            nd[3] = pn.w;
          }
          const double ep = eg64_patch(w1_64, w2_64, scratch, scratch + 48,
                                       reinterpret_cast<double(*)[15]>(scratch + 192), pp, active, g, nd, A.q,
                                       nullptr, 0.0, A.restgp, (size_t)A.np * 16, A.h, A.grad64, A.err);
          if (active && g == 0) {
            if (!isfinite(ep)) atomicOr(A.err, ERRBIT_NONFINITE);
            A.energy64[pp] = ep;
          }
          __syncwarp();
        }
        element_patch<R>(sphi, w1d, sphg, W, A.plist ? A.plist[it] : it, A, lane);
      }
      return;
    }
  }
  for (int it = blockIdx.x * NW + wid; it < total; it += stride)
    element_patch<R>(sphi, w1d, sphg, W, A.plist ? A.plist[it] : it, A, lane);
}

template <typename R>
static size_t elem_smem_bytes() {
  return sizeof(R) * elem_table_elems<R>() + sizeof(WarpSmem<R>) * ElemCfg<R>::kWarps;
}

template <typename R>
static shell_status launch_full_t(Shell& s, const ElemArgs& A, int work) {
  constexpr int NW = ElemCfg<R>::kWarps;
  size_t smem = elem_smem_bytes<R>();
  static bool attr_done[64] = {false};
  int dev = s.device < 64 ? s.device : 63;
  if (!attr_done[dev]) {
    BHEM_CUDA(cudaFuncSetAttribute(k_element_full<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_done[dev] = true;
  }
  if (work <= 0) return SHELL_OK;
  int blocks = (work + NW - 1) / NW;
  int nsm = 0;
  BHEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s.device));
  int occ = 0;
  BHEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_element_full<R>, 32 * NW, smem));
  int cap = nsm * (occ > 0 ? occ : 1) * 8;
  if (blocks > cap) blocks = cap;
  k_element_full<R><<<blocks, 32 * NW, smem, s.stream>>>(A);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

// element_tc.cu: the FP32 pass with the tensor-core contraction (same arguments and outputs)
shell_status launch_full_tc(Shell& s, const ElemArgs& A, int work);

template <typename R>
static shell_status launch_full_pick(Shell& s, const ElemArgs& A, int work) {
  if constexpr (sizeof(R) == 4) {
    if (s.elem_tc) return launch_full_tc(s, A, work);
  }
  return launch_full_t<R>(s, A, work);
}

shell_status launch_element_full(Shell& s, const double* q, bool fp64, const ElemOutputs& out) {
  ElemArgs A{};
  A.np = s.n_patches;
  A.phi = fp64 ? (const void*)s.d_phi64 : (const void*)s.d_phi32;
  A.pnodes = s.d_patch_nodes;
  A.pblocks = s.d_patch_blocks;
  A.q = q;
  A.rest = s.d_rest;
  A.d1 = s.grid.dxi1;
  A.d2 = s.grid.dxi2;
  A.lam = s.lam;
  A.mu = s.mu;
  A.h = s.mat.thickness;
  A.rho_h = s.mat.density * s.mat.thickness;
  A.mass_scale = out.mass_scale;
  A.pseudo = out.pseudo;
  A.energy_p = out.energy_p;
  A.grad_p = out.grad_p;
  A.hess_p = out.hess_p;
  A.hess_vec = ((uintptr_t)out.hess_p & 15u) == 0;
  A.bsr = out.bsr;
  A.err = s.d_err;
  if (!fp64 && out.grad64) {
    A.restgp = s.d_restgp;
    A.energy64 = out.energy64;
    A.grad64 = out.grad64;
  }
  if (out.bsr && s.opt.assembly == SHELL_ASM_COLOR) {
    // colour-ordered: patches of one colour share no node, plain read-modify-write
    A.bsr_atomic = 0;
    for (int c = 0; c < 9; ++c) {
      int b = s.h_color_patches[c], e = s.h_color_patches[c + 1];
      if (e <= b) continue;
      ElemArgs Ac = A;
      Ac.plist = s.d_color_list + b;
      Ac.plist_n = e - b;
      BHEM_TRY(fp64 ? launch_full_t<double>(s, Ac, e - b) : launch_full_pick<float>(s, Ac, e - b));
    }
    return SHELL_OK;
  }
  A.bsr_atomic = 1;
  return fp64 ? launch_full_t<double>(s, A, A.np) : launch_full_pick<float>(s, A, A.np);
}

}  // namespace bhem
