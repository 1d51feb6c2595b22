// Batched BHEM: many independent shells of uneven sizes and materials stepped together.
//
// All shells live in one concatenation: node, patch and block arrays are shell after shell, and
// the BSR matrix is block diagonal across shells. Each phase of a Newton iteration (FP64
// residual, FP32 element Hessians + assembly, block-Jacobi set-up, PCG iterations, line-search
// energy trials, update) is one persistent launch over all shells. Per-shell scalars (Newton
// state, regulariser level, PCG alpha/beta, line-search alpha) live in device memory and are
// advanced by one-thread-per-shell controller kernels, so every shell runs its own Newton to its
// own 1e-8 residual with the same policies as the single-shell solver (Sec. 6.1 readings). The
// host only reads a few counters between phases; PCG iterations are replayed from a CUDA graph.
//
// Element kernels take work items (shell, first, last) of at most `ppi` patches of one shell, so
// a CTA can hold that shell's shape table in shared memory; ppi and the assembly scheme (atomic
// or colour-ordered) are chosen by shell_batch_autotune.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "element_impl.cuh"

namespace bhem {
namespace batch {

struct ShellPar {
  double lam, mu, h, rho_h;
  int node_off, node_end, patch_off, patch_end;
};

struct ShellState {
  // Newton
  double gref, gn;
  int active, status, newton_iters, first;
  // PCG
  double rz, pq, rr, bb, alpha, beta, rtol2;
  int pcg_done, pcg_iters, pcg_iters_total, negcurv, restart, reg_level, regularizations, limit;
  double tau;
  float td[4];
  double dbar[4], dmin[4], dcount[4];
  // line search
  double dMd, dgin, gd, ls_alpha, ls_prev_alpha, ls_prev_phi, dV;
  int searching, ls_trials, ls_backtracks, diag_fixes;
  // reduction accumulators, zeroed by the controllers before use
  double acc[4];
  double acc2[12];
};

struct Counters { int n_active, n_running, n_restart, n_searching; };

// Device-side loop state of the captured Newton step (one CUDA graph per step: WHILE nodes for
// the Newton iterations, the regulariser rounds, the PCG chunks and the line-search trials, each
// condition set by a one-thread kernel from the counters), and the body executions of each loop
// for the launch count.
struct LoopState {
  int newton_it, round, pcg_iters, trial;
  long long n_newton, n_reg, n_pcg, n_ls;
};
// Per-step input written by the host before each step (a graph replays with new values)
struct StepInput { double tau_carry; };
constexpr int kGraphPcgChunk = 4;   // PCG iterations per body of the PCG WHILE node

constexpr int kRowNodes = 8;          // block rows per SpMV CTA (36 threads each)
constexpr int kSpmvThreads = 288;
constexpr int kNodeThreads = 192;     // 12 threads per node, 16 nodes per CTA

// ------------------------------------------------------------------------------------------
// Segmented CTA reductions: the rows of one CTA span at most two shells (every shell has at
// least 4 nodes per patch row and the CTAs hold <= 16 nodes of consecutive shells... the
// two-segment split is checked by the host at set-up: every shell has >= 16 nodes).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double block_sum_d(double v, double* sbuf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sbuf[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += sbuf[w];
  return s;
}

// The rows of one CTA belong to at most two consecutive shells s0 <= s1 (every shell has at
// least 16 nodes, checked at set-up). A thread's value v belongs to the shell of its row (v = 0
// for rows without work); the CTA sums each segment and adds it with one FP64 atomic into acc
// of that shell, when the CTA-uniform flag use0 / use1 says the shell takes part.
__device__ __forceinline__ void seg_add_d(double v, int sh, int s0, int s1, bool use0, bool use1,
                                          ShellState* st, int slot) {
  __shared__ double sbuf[32];
  const double a = block_sum_d(sh == s0 ? v : 0.0, sbuf);
  const double b = block_sum_d(sh != s0 ? v : 0.0, sbuf);
  if (threadIdx.x == 0) {
    if (use0 && s0 >= 0) atomicAdd(&st[s0].acc[slot], a);
    if (use1 && s1 >= 0 && s1 != s0) atomicAdd(&st[s1].acc[slot], b);
  }
}

__device__ __forceinline__ void seg_add_f2(F2 v, int sh, int s0, int s1, bool use0, bool use1,
                                           ShellState* st, int slot) {
  __shared__ F2 sbuf2[1][32];
  const F2 z{0.f, 0.f};
  const F2 a = f2_block_sum(sh == s0 ? v : z, sbuf2, 0);
  const F2 b = f2_block_sum(sh != s0 ? v : z, sbuf2, 0);
  if (threadIdx.x == 0) {
    if (use0 && s0 >= 0) atomicAdd(&st[s0].acc[slot], (double)a.hi + (double)a.lo);
    if (use1 && s1 >= 0 && s1 != s0) atomicAdd(&st[s1].acc[slot], (double)b.hi + (double)b.lo);
  }
}

// ------------------------------------------------------------------------------------------
// Set-up kernels
// ------------------------------------------------------------------------------------------
__global__ void k_tables(int S, const double* __restrict__ dxi, double* __restrict__ t64,
                         float* __restrict__ t32) {
  __shared__ double sphi[kPhiSize];
  const int s = blockIdx.x;
  if (s >= S) return;
  for (int e = threadIdx.x; e < kPhiSize; e += blockDim.x) sphi[e] = 0.0;
  __syncthreads();
  build_shape_table<double>(sphi, dxi[2 * s], dxi[2 * s + 1]);
  __syncthreads();
  for (int e = threadIdx.x; e < kPhiTable; e += blockDim.x) {
    double v = e < kPhiSize ? sphi[e] : gauss_weight(e - kPhiSize, dxi[2 * s], dxi[2 * s + 1]);
    t64[(size_t)s * kPhiTable + e] = v;
    t32[(size_t)s * kPhiTable + e] = (float)v;
  }
}

__global__ void k_rest(int P, const int* __restrict__ pshell, const ShellPar* __restrict__ par,
                       const int4* __restrict__ pnodes, const double* __restrict__ rest,
                       const double* __restrict__ t64, double* __restrict__ restgp, int* err) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)P * 16) return;
  const int p = (int)(t >> 4), g = (int)(t & 15);
  const int s = pshell[p];
  const double* tab = t64 + (size_t)s * kPhiTable;
  const int4 pn = pnodes[p];
  const int nd[4] = {pn.x, pn.y, pn.z, pn.w};
  double qb[48];
  for (int l = 0; l < 48; ++l) qb[l] = rest[(size_t)nd[l / 12] * 12 + (l % 12)];
  V3<double> v[5];
  interp5<double, double>(tab, qb, g, v);
  const double a11 = dot(v[0], v[0]), a22 = dot(v[1], v[1]), a12 = dot(v[0], v[1]);
  double det = a11 * a22 - a12 * a12;
  if (!(det > 1e-300)) { atomicOr(err, ERRBIT_DEGENERATE); det = 1.0; }
  const double sq = sqrt(det);
  const V3<double> a3 = (1.0 / sq) * cross(v[0], v[1]);
  const double ai11 = a22 / det, ai22 = a11 / det, ai12 = -a12 / det;
  const double lam = par[s].lam, mu = par[s].mu;
  const size_t SS = (size_t)P * 16, o = (size_t)p * 16 + g;
  restgp[0 * SS + o] = a11;
  restgp[1 * SS + o] = a22;
  restgp[2 * SS + o] = a12;
  restgp[3 * SS + o] = dot(v[2], a3);
  restgp[4 * SS + o] = dot(v[3], a3);
  restgp[5 * SS + o] = dot(v[4], a3);
  restgp[6 * SS + o] = (lam + 2 * mu) * ai11 * ai11;
  restgp[7 * SS + o] = lam * ai11 * ai22 + 2 * mu * ai12 * ai12;
  restgp[8 * SS + o] = (lam + 2 * mu) * ai11 * ai12;
  restgp[9 * SS + o] = (lam + 2 * mu) * ai22 * ai22;
  restgp[10 * SS + o] = (lam + 2 * mu) * ai12 * ai22;
  restgp[11 * SS + o] = (lam + mu) * ai12 * ai12 + mu * ai11 * ai22;
  restgp[12 * SS + o] = tab[kPhiSize + g] * sq;
}

__global__ void k_mass(int P, const int* __restrict__ pshell, const ShellPar* __restrict__ par,
                       const int* __restrict__ pblocks, const int4* __restrict__ pnodes,
                       const double* __restrict__ restgp, const double* __restrict__ t64,
                       double* __restrict__ mass, double* __restrict__ fgrav) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const size_t SS = (size_t)P * 16;
  for (int p = warp; p < P; p += nwarps) {
    const int s = pshell[p];
    const double* tab = t64 + (size_t)s * kPhiTable;
    double w[16];
    for (int g = 0; g < 16; ++g) w[g] = par[s].rho_h * restgp[12 * SS + (size_t)p * 16 + g];
    for (int e = lane; e < 256 + 16; e += 32) {
      if (e < 256) {
        const int I = e >> 4, J = e & 15;
        double sum = 0.0;
        for (int g = 0; g < 16; ++g) sum += w[g] * tab[I * kPhiStride + g] * tab[J * kPhiStride + g];
        const int kb = pblocks[(size_t)p * 16 + (I >> 2) * 4 + (J >> 2)];
        atomicAdd(&mass[(size_t)kb * 16 + (I & 3) * 4 + (J & 3)], sum);
      } else {
        const int I = e - 256;
        double sum = 0.0;
        for (int g = 0; g < 16; ++g) sum += w[g] * tab[I * kPhiStride + g];
        const int4 pn = pnodes[p];
        const int nd[4] = {pn.x, pn.y, pn.z, pn.w};
        atomicAdd(&fgrav[(size_t)nd[I >> 2] * 4 + (I & 3)], sum);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Element kernels over work items (shell, first, last) of one shell each
// ------------------------------------------------------------------------------------------
struct ElemBatchArgs {
  int n_items;
  const int4* items;
  const int* plist;            // patch ids (colour order) the items index, or null (identity)
  const ShellPar* par;
  const ShellState* st;
  const float* t32;
  const double* dxi;           // [2 * shells] parameter extents of one patch
  const int4* pnodes;
  const int* pblocks;
  const double* q;
  const double* rest;
  double mass_scale;
  float* bsr;
  int bsr_atomic;
  int* err;
};

__global__ void __launch_bounds__(32 * ElemCfg<float>::kWarps)
k_element(ElemBatchArgs B) {
  constexpr int NW = ElemCfg<float>::kWarps;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sphi = reinterpret_cast<float*>(smem_raw);
  float* w1d = sphi + ((kPhiTable + 3) & ~3);
  WarpSmem<float>* Ws = reinterpret_cast<WarpSmem<float>*>(smem_raw + sizeof(float) * elem_table_elems<float>());
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < B.n_items; it += gridDim.x) {
    const int4 item = B.items[it];
    const int s = item.x;
    if (!B.st[s].active) continue;   // uniform over the CTA
    __syncthreads();
    load_shape_table<float>(sphi, B.t32 + (size_t)s * kPhiTable);
    build_hermite_1d<float>(w1d, B.dxi[2 * s], threadIdx.x, blockDim.x);
    build_hermite_1d<float>(w1d + kHerm1D, B.dxi[2 * s + 1], threadIdx.x, blockDim.x);
    __syncthreads();
    build_phi_gauss(w1d + 2 * kHerm1D, sphi, threadIdx.x, blockDim.x);
    __syncthreads();
    ElemArgs A{};
    A.pnodes = B.pnodes;
    A.pblocks = B.pblocks;
    A.q = B.q;
    A.rest = B.rest;
    A.lam = B.par[s].lam;
    A.mu = B.par[s].mu;
    A.h = B.par[s].h;
    A.rho_h = B.par[s].rho_h;
    A.mass_scale = B.mass_scale;
    A.bsr = B.bsr;
    A.bsr_atomic = B.bsr_atomic;
    A.err = B.err;
    for (int k = item.y + wid; k < item.z; k += NW) {
      const int p = B.plist ? B.plist[k] : k;
      element_patch<float>(sphi, w1d, w1d + 2 * kHerm1D, Ws[wid], p, A, lane);
    }
  }
}

// FP64 energy/gradient per patch over items of <= 8 patches of one shell.
// mode 0: grad += dE/dq, Ep[p] = E_p (shells with active != 0)
// mode 1: acc[3] += E_p(q + alpha_s d) - Ep[p] (shells with searching != 0)
__global__ void __launch_bounds__(128)
k_eg64(int n_items, const int4* __restrict__ items, int P, const ShellPar* __restrict__ par,
       ShellState* st, const double* __restrict__ dxi, const int4* __restrict__ pnodes,
       const double* __restrict__ q, const double* __restrict__ dir,
       const double* __restrict__ restgp, double* __restrict__ Ep, double* __restrict__ grad,
       int mode, int* err) {
  __shared__ double w1[kHerm1D], w2[kHerm1D];
  __shared__ double sq[kEgPatches][48];
  __shared__ double sT[kEgPatches][144];
  __shared__ double sG[kEgPatches][16][15];
  __shared__ double sbuf[32];
  const int hw = threadIdx.x >> 4, g = threadIdx.x & 15;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4 item = items[it];
    const int s = item.x;
    const bool run = mode == 0 ? st[s].active != 0 : st[s].searching != 0;
    if (!run) continue;   // uniform over the CTA
    __syncthreads();
    build_hermite_1d(w1, dxi[2 * s], threadIdx.x, blockDim.x);
    build_hermite_1d(w2, dxi[2 * s + 1], threadIdx.x, blockDim.x);
    __syncthreads();
    const int p = item.y + hw;
    const bool active = p < item.z;
    int nd[4] = {0, 0, 0, 0};
    if (active) {
      const int4 pn = pnodes[p];
      nd[0] = pn.x; nd[1] = pn.y; nd[2] = pn.z; nd[3] = pn.w;
    }
    const double step = mode == 1 ? st[s].ls_alpha : 0.0;
    const double ep = eg64_patch(w1, w2, sq[hw], sT[hw], sG[hw], p, active, g, nd, q, mode == 1 ? dir : nullptr,
                                 step, restgp, (size_t)P * 16, par[s].h, mode == 0 ? grad : nullptr, err);
    double contrib = 0.0;
    if (active && g == 0) {
      if (!isfinite(ep)) atomicOr(err, ERRBIT_NONFINITE);
      if (mode == 0) { Ep[p] = ep; contrib = ep; }
      else contrib = ep - Ep[p];
    }
    if (mode == 1) {
      const double tot = block_sum_d(contrib, sbuf);
      if (threadIdx.x == 0) atomicAdd(&st[s].acc[3], tot);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Row kernels (12 threads per node, 16 nodes per CTA)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void cta_shells(int n, const int* __restrict__ nshell, int first_node,
                                           int count, int* s0, int* s1) {
  const int last = min(first_node + count, n) - 1;
  *s0 = first_node < n ? nshell[first_node] : -1;
  *s1 = last >= first_node ? nshell[last] : -1;
}

// g = grad_el + M (q - y)/dt^2 - F (masked), gin; acc[0] += |g|^2 (shells with active != 0)
__global__ void __launch_bounds__(kNodeThreads)
k_grad_finish(int n, const int* __restrict__ nshell, ShellState* st, const int* __restrict__ rp,
              const int* __restrict__ col, const double* __restrict__ mass,
              const double* __restrict__ fgrav, const double* __restrict__ q,
              const double* __restrict__ yv, double inv_dt2, double gx, double gy, double gz,
              const unsigned char* __restrict__ mask, double* __restrict__ g,
              double* __restrict__ gin, int* err) {
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  int s0, s1;
  cta_shells(n, nshell, blockIdx.x * 16, 16, &s0, &s1);
  double part = 0.0;
  int sh = -1;
  if (i < n) {
    sh = nshell[i];
    if (st[sh].active) {
      const size_t gi = (size_t)i * 12 + a;
      const int r = a / 3, c = a % 3;
      const double grav = c == 0 ? gx : c == 1 ? gy : gz;
      double sum = 0.0;
      for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = col[k];
        const double* mb = mass + (size_t)k * 16 + r * 4;
        for (int qq = 0; qq < 4; ++qq) sum += mb[qq] * (q[(size_t)j * 12 + qq * 3 + c] - yv[(size_t)j * 12 + qq * 3 + c]);
      }
      double gi_in = sum * inv_dt2 - fgrav[(size_t)i * 4 + r] * grav;
      double gv = g[gi] + gi_in;
      if (mask && mask[gi]) { gv = 0.0; gi_in = 0.0; }
      if (!isfinite(gv)) atomicOr(err, ERRBIT_NONFINITE);
      g[gi] = gv;
      gin[gi] = gi_in;
      part = gv * gv;
    }
  }
  seg_add_d(part, sh, s0, s1, true, true, st, 0);
}

// Per shell and DOF kind over free DOFs: sum |A_ii| (acc2[3k]), count (acc2[3k+1]) and min A_ii
// (acc2[3k+2], by an order-preserving integer atomicMin on the float value).
__device__ __forceinline__ int float_order(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float order_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void __launch_bounds__(kNodeThreads)
k_diag_stats(int n, const int* __restrict__ nshell, ShellState* st, const int* __restrict__ diag_block,
             const float* __restrict__ val, const unsigned char* __restrict__ mask,
             int* __restrict__ dmin_bits) {
  __shared__ double ssum[2][4], scnt[2][4];
  __shared__ int smin[2][4];
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12, kind = a / 3;
  const int i = blockIdx.x * 16 + ln;
  int s0, s1;
  cta_shells(n, nshell, blockIdx.x * 16, 16, &s0, &s1);
  if (threadIdx.x < 8) {
    ssum[threadIdx.x / 4][threadIdx.x % 4] = 0.0;
    scnt[threadIdx.x / 4][threadIdx.x % 4] = 0.0;
    smin[threadIdx.x / 4][threadIdx.x % 4] = 0x7fffffff;
  }
  __syncthreads();
  if (i < n && !(mask && mask[(size_t)i * 12 + a])) {
    const int sh = nshell[i];
    if (st[sh].active) {
      const float d = val[(size_t)diag_block[i] * 144 + a * 13];
      const int seg = sh == s0 ? 0 : 1;
      atomicAdd(&ssum[seg][kind], (double)fabsf(d));
      atomicAdd(&scnt[seg][kind], 1.0);
      atomicMin(&smin[seg][kind], float_order(d));
    }
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int seg = threadIdx.x / 4, k = threadIdx.x % 4;
    const int sh = seg == 0 ? s0 : s1;
    if (sh >= 0 && (seg == 0 || s1 != s0) && scnt[seg][k] > 0.0) {
      atomicAdd(&st[sh].acc2[3 * k], ssum[seg][k]);
      atomicAdd(&st[sh].acc2[3 * k + 1], scnt[seg][k]);
      atomicMin(&dmin_bits[4 * sh + k], smin[seg][k]);
    }
  }
}

__global__ void __launch_bounds__(192)
k_precond(int n, const int* __restrict__ nshell, const ShellState* st,
          const int* __restrict__ diag_block, const float* __restrict__ val,
          const unsigned char* __restrict__ mask, float* __restrict__ Dinv, int only_restart) {
  __shared__ float sL[16][12][13];
  __shared__ float sW[16][12][13];
  __shared__ float sdiag[16][12];
  __shared__ int sok[16];
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  bool active = i < n;
  int s = 0;
  if (active) {
    s = nshell[i];
    active = st[s].active && !st[s].pcg_done && (!only_restart || st[s].restart);
  }
  if (active) {
    const float* Bv = val + (size_t)diag_block[i] * 144;
    const bool fa = mask && mask[(size_t)i * 12 + a];
    for (int b = 0; b < 12; ++b) {
      const bool fb = mask && mask[(size_t)i * 12 + b];
      float v = Bv[a * 12 + b];
      if (fa || fb) v = (a == b) ? 1.f : 0.f;
      else if (a == b) v += st[s].td[a / 3];
      sL[ln][a][b] = v;
    }
    sdiag[ln][a] = sL[ln][a][a];
  }
  if (a == 0) sok[ln] = 1;
  __syncthreads();
  for (int j = 0; j < 12; ++j) {
    if (active && a == j && sok[ln]) {
      float acc = sL[ln][j][j];
      for (int k = 0; k < j; ++k) acc -= sL[ln][j][k] * sL[ln][j][k];
      if (!(acc > 0.f)) sok[ln] = 0;
      else sL[ln][j][j] = sqrtf(acc);
    }
    __syncthreads();
    if (active && a > j && sok[ln]) {
      float u = sL[ln][a][j];
      for (int k = 0; k < j; ++k) u -= sL[ln][a][k] * sL[ln][j][k];
      sL[ln][a][j] = u / sL[ln][j][j];
    }
    __syncthreads();
  }
  const bool ok = active && sok[ln];
  if (ok) {
    for (int r = 0; r < 12; ++r) {
      if (r < a) { sW[ln][r][a] = 0.f; continue; }
      float u = (r == a) ? 1.f : 0.f;
      for (int k = a; k < r; ++k) u -= sL[ln][r][k] * sW[ln][k][a];
      sW[ln][r][a] = u / sL[ln][r][r];
    }
  }
  __syncthreads();
  if (!active) return;
  float* D = Dinv + (size_t)i * 144 + a * 12;
  if (ok) {
    for (int b = 0; b < 12; ++b) {
      float acc = 0.f;
      for (int k = (a > b ? a : b); k < 12; ++k) acc += sW[ln][k][a] * sW[ln][k][b];
      D[b] = acc;
    }
  } else {
    const float d = sdiag[ln][a];
    for (int b = 0; b < 12; ++b) D[b] = (a == b) ? (d > 0.f ? 1.f / d : 1.f) : 0.f;
  }
}

__device__ __forceinline__ float apply_block(const float* __restrict__ D, const float* sr, int a) {
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 12; ++c) s += D[a * 12 + c] * sr[c];
  return s;
}

// PCG init for shells that start (or restart) a solve: x = 0, r = rhs, z = D r, p = z;
// acc[0] += r.z, acc[1] += r.r
__global__ void __launch_bounds__(kNodeThreads)
k_pcg_init(int n, const int* __restrict__ nshell, ShellState* st, const double* __restrict__ rhs,
           const float* __restrict__ Dinv, const unsigned char* __restrict__ mask,
           float* __restrict__ x, float* __restrict__ r, float* __restrict__ z, float* __restrict__ p,
           int only_restart) {
  __shared__ float sr[16][12];
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  int s0, s1;
  cta_shells(n, nshell, blockIdx.x * 16, 16, &s0, &s1);
  const size_t gi = (size_t)i * 12 + a;
  bool act = false;
  int sh = -1;
  float ri = 0.f, zi = 0.f;
  if (i < n) {
    sh = nshell[i];
    act = st[sh].active && !st[sh].pcg_done && (!only_restart || st[sh].restart);
    if (act) {
      ri = (mask && mask[gi]) ? 0.f : (float)rhs[gi];
      x[gi] = 0.f;
      r[gi] = ri;
      sr[ln][a] = ri;
    }
  }
  __syncthreads();
  if (act) {
    zi = (mask && mask[gi]) ? 0.f : apply_block(Dinv + (size_t)i * 144, sr[ln], a);
    z[gi] = zi;
    p[gi] = zi;
  }
  auto starts = [&](int s) { return s >= 0 && st[s].active && !st[s].pcg_done && (!only_restart || st[s].restart); };
  const bool use0 = starts(s0), use1 = starts(s1);
  seg_add_f2(f2_prod(ri, zi), sh, s0, s1, use0, use1, st, 0);
  seg_add_f2(f2_prod(ri, ri), sh, s0, s1, use0, use1, st, 1);
}

__device__ __forceinline__ bool pcg_running(const ShellState& S) { return S.active && !S.pcg_done; }

// y = (A + tau D) p on rows of running shells; acc[0] += p.y
// x is z: per running shell's own rows, p = z + beta p (the first iteration of a solve: p = z)
// and y = Ap = (A + tau D) z + beta Ap, equal to (A + tau D) p by linearity, so no separate
// p-update launch follows the update
__global__ void __launch_bounds__(kSpmvThreads)
k_spmv(int n, const int* __restrict__ nshell, ShellState* st, const int* __restrict__ rp,
       const int* __restrict__ col, const float* __restrict__ val, const float* __restrict__ x,
       const unsigned char* __restrict__ mask, float* __restrict__ p, float* __restrict__ y) {
  __shared__ float sacc[kSpmvThreads];
  const int t = threadIdx.x;
  const int br = t / 36, w = t % 36, r = w / 3, cc = w % 3;
  const int i = blockIdx.x * kRowNodes + br;
  int s0, s1;
  cta_shells(n, nshell, blockIdx.x * kRowNodes, kRowNodes, &s0, &s1);
  const bool run0 = s0 >= 0 && pcg_running(st[s0]), run1 = s1 >= 0 && pcg_running(st[s1]);
  if (!run0 && !run1) return;   // uniform over the CTA
  int sh = -1;
  bool run = false;
  float acc = 0.f;
  if (i < n) {
    sh = nshell[i];
    run = pcg_running(st[sh]);
    if (run) {
      const int k0 = rp[i], k1 = rp[i + 1];
      for (int k = k0; k < k1; ++k) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(val + (size_t)k * 144 + r * 12 + cc * 4));
        const float4 xv = *reinterpret_cast<const float4*>(x + (size_t)col[k] * 12 + cc * 4);
        acc += a.x * xv.x + a.y * xv.y + a.z * xv.z + a.w * xv.w;
      }
    }
  }
  sacc[t] = acc;
  __syncthreads();
  F2 part{0.f, 0.f};
  if (run && cc == 0) {
    const size_t gi = (size_t)i * 12 + r;
    const float zi = x[gi];
    float wi = (sacc[t] + sacc[t + 1]) + sacc[t + 2];
    wi += st[sh].td[r / 3] * zi;
    if (mask && mask[gi]) wi = 0.f;
    float pi = zi, qi = wi;
    if (st[sh].pcg_iters > 0) {
      const float bf = (float)st[sh].beta;
      pi = fmaf(bf, p[gi], zi);
      qi = fmaf(bf, y[gi], wi);
    }
    p[gi] = pi;
    y[gi] = qi;
    part = f2_prod(pi, qi);
  }
  seg_add_f2(part, sh, s0, s1, run0, run1, st, 0);
}

// x += alpha p, r -= alpha Ap, z = D r on running shells; acc[0] += r.z, acc[1] += r.r
__global__ void __launch_bounds__(kNodeThreads)
k_pcg_update(int n, const int* __restrict__ nshell, ShellState* st, float* __restrict__ x,
             float* __restrict__ r, float* __restrict__ z, const float* __restrict__ p,
             const float* __restrict__ Ap, const float* __restrict__ Dinv,
             const unsigned char* __restrict__ mask) {
  __shared__ float sr[16][12];
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  int s0, s1;
  cta_shells(n, nshell, blockIdx.x * 16, 16, &s0, &s1);
  const bool run0 = s0 >= 0 && pcg_running(st[s0]), run1 = s1 >= 0 && pcg_running(st[s1]);
  if (!run0 && !run1) return;
  const size_t gi = (size_t)i * 12 + a;
  bool run = false;
  int sh = -1;
  float ri = 0.f, zi = 0.f;
  if (i < n) {
    sh = nshell[i];
    run = pcg_running(st[sh]);
    if (run) {
      const float al = (float)st[sh].alpha;
      x[gi] = fmaf(al, p[gi], x[gi]);
      ri = fmaf(-al, Ap[gi], r[gi]);
      r[gi] = ri;
      sr[ln][a] = ri;
    }
  }
  __syncthreads();
  if (run) {
    zi = (mask && mask[gi]) ? 0.f : apply_block(Dinv + (size_t)i * 144, sr[ln], a);
    z[gi] = zi;
  }
  seg_add_f2(f2_prod(ri, zi), sh, s0, s1, run0, run1, st, 0);
  seg_add_f2(f2_prod(ri, ri), sh, s0, s1, run0, run1, st, 1);
}


// ------------------------------------------------------------------------------------------
// Controllers: one thread per shell
// ------------------------------------------------------------------------------------------
// After k_pcg_init: rz, bb from acc[0..1]
__global__ void k_ctrl_pcg_start(int S, ShellState* st, Counters* cnt, int only_restart,
                                 double rtol, int pcg_max, int fixed) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  ShellState& T = st[s];
  const bool started = T.active && !T.pcg_done && (!only_restart || T.restart);
  if (started) {
    T.rz = T.acc[0];
    T.bb = T.acc[1];
    T.rr = T.acc[1];
    T.rtol2 = fixed > 0 ? 0.0 : rtol * rtol;
    T.limit = fixed > 0 ? fixed : pcg_max;
    T.pcg_iters = 0;
    T.negcurv = 0;
    T.restart = 0;
    if (T.bb == 0.0 || T.limit == 0) T.pcg_done = 1;
  }
  T.acc[0] = 0.0;
  T.acc[1] = 0.0;
  if (T.active && !T.pcg_done) atomicAdd(&cnt->n_running, 1);
}

__global__ void k_ctrl_count_running(int S, const ShellState* st, Counters* cnt) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S && st[s].active && !st[s].pcg_done) atomicAdd(&cnt->n_running, 1);
}

// After k_spmv: alpha = rz / p.Ap, or negative curvature
__global__ void k_ctrl_alpha(int S, ShellState* st) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  ShellState& T = st[s];
  if (T.active && !T.pcg_done) {
    const double pq = T.acc[0];
    T.pq = pq;
    if (!(pq > 0.0)) {
      T.negcurv = 1;
      T.pcg_done = 1;
      T.alpha = 0.0;
    } else {
      T.alpha = T.rz / pq;
    }
  }
  T.acc[0] = 0.0;
}

// After k_pcg_update: beta, convergence, iteration limit
__global__ void k_ctrl_beta(int S, ShellState* st) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  ShellState& T = st[s];
  if (T.active && !T.pcg_done) {
    const double rz_new = T.acc[0];
    T.rr = T.acc[1];
    T.pcg_iters += 1;
    T.pcg_iters_total += 1;
    T.beta = rz_new / T.rz;
    T.rz = rz_new;
    if (T.rtol2 > 0.0 && T.rr <= T.rtol2 * T.bb) T.pcg_done = 1;
    if (rz_new == 0.0) T.pcg_done = 1;
    if (T.pcg_iters >= T.limit) T.pcg_done = 1;
  }
  T.acc[0] = 0.0;
  T.acc[1] = 0.0;
}

// After k_diag_stats: per-kind scale, first admissible regulariser level, PCG not done
__global__ void k_ctrl_reg_init(int S, ShellState* st, const int* __restrict__ dmin_bits) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  ShellState& T = st[s];
  for (int k = 0; k < 4; ++k) {
    T.dcount[k] = T.acc2[3 * k + 1];
    T.dbar[k] = T.dcount[k] > 0 ? T.acc2[3 * k] / T.dcount[k] : 1.0;
    T.dmin[k] = (double)order_float(dmin_bits[4 * s + k]);
    T.acc2[3 * k] = T.acc2[3 * k + 1] = T.acc2[3 * k + 2] = 0.0;
  }
  if (!T.active) return;
  T.pcg_done = 0;
  T.restart = 1;   // the solve (re)starts: the PCG set-up kernels take the shells with this flag
  // Sec. 6.1 regulariser: tau starts at a tenth of the previous Newton iteration's tau (T.tau;
  // at the first, of the level carried into the step; 0 when a tenth is below 1e-8)
  double tau = T.tau / 10.0;
  if (tau < 1e-8) tau = 0.0;
  if (tau > 0.0) T.regularizations += 1;
  T.tau = tau;
  for (int k = 0; k < 4; ++k) T.td[k] = (float)(tau * T.dbar[k]);
}

// Local part of the regulariser, after k_ctrl_reg_init: every free diagonal entry A_ii <= 0 of an
// active shell becomes max(-A_ii, 1e-8 D_k) of that shell (D_k from the diagonal before the fix).
__global__ void k_fix_diag(int m, const int* __restrict__ nshell, ShellState* st, const int* __restrict__ diag_block,
                           float* __restrict__ val, const unsigned char* __restrict__ mask) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    if (mask && mask[k]) continue;
    const int i = k / 12, a = k % 12;
    float* d = &val[(size_t)diag_block[i] * 144 + a * 13];
    const float v = *d;
    if (v > 0.f) continue;
    ShellState& T = st[nshell[i]];
    if (!T.active) continue;
    const float f = (float)(1e-8 * T.dbar[a / 3]);
    *d = -v > f ? -v : f;
    atomicAdd(&T.diag_fixes, 1);
  }
}

// Between PCG chunks: shells that met negative curvature restart with tau x 10 (at least 1e-8);
// beyond 1e4 the shell's step gives up.
__global__ void k_ctrl_restart(int S, ShellState* st, Counters* cnt) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  ShellState& T = st[s];
  if (!(T.active && T.pcg_done && T.negcurv)) return;
  T.negcurv = 0;
  T.tau = fmax(10.0 * T.tau, 1e-8);
  if (T.tau > 1e4) {
    T.status = SHELL_ERR_INDEFINITE;
    T.active = 0;
    return;
  }
  T.regularizations += 1;   // the restarted solve runs with tau > 0
  for (int k = 0; k < 4; ++k) T.td[k] = (float)(T.tau * T.dbar[k]);
  T.pcg_done = 0;
  T.restart = 1;
  atomicAdd(&cnt->n_restart, 1);
}

// After the residual: Newton convergence per shell
__global__ void k_ctrl_newton(int S, ShellState* st, Counters* cnt, double rtol, int newton_max,
                              int set_ref) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  ShellState& T = st[s];
  if (T.active) {
    T.gn = sqrt(T.acc[0]);
    if (set_ref) T.gref = T.gn;
    if (T.gn <= rtol * T.gref) {
      T.active = 0;
    } else if (T.newton_iters >= newton_max) {
      T.active = 0;
      T.status = SHELL_ERR_NOT_CONVERGED;
    }
  }
  T.acc[0] = 0.0;
  if (T.active) atomicAdd(&cnt->n_active, 1);
}

// Line search start: dots (acc2[0..2] = d.Md, d.gin, g.d) -> alpha = 1, searching per shell
__global__ void k_ctrl_ls_start(int S, ShellState* st, Counters* cnt, double inv_dt2) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  ShellState& T = st[s];
  const double dMd = T.acc2[0] * inv_dt2, dgin = T.acc2[1], gd = T.acc2[2];
  T.acc2[0] = T.acc2[1] = T.acc2[2] = 0.0;
  T.acc[3] = 0.0;
  T.searching = 0;
  if (!T.active) return;
  T.ls_alpha = 1.0;
  T.ls_trials = 0;
  if (T.gn > 1e-6 * T.gref) {
    if (!(gd < 0.0)) {
      T.status = SHELL_ERR_LINESEARCH;
      T.active = 0;
      return;
    }
    T.dMd = dMd;
    T.dgin = dgin;
    T.gd = gd;
    T.searching = 1;
    atomicAdd(&cnt->n_searching, 1);
  }
}

// After a trial energy pass: Armijo test, else the next alpha (quadratic, then cubic)
__global__ void k_ctrl_ls_step(int S, ShellState* st, Counters* cnt) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  ShellState& T = st[s];
  const double dV = T.acc[3];
  T.acc[3] = 0.0;
  if (!T.searching) return;
  const double alpha = T.ls_alpha, gd = T.gd;
  const double phi = dV + alpha * T.dgin + 0.5 * alpha * alpha * T.dMd;
  if (isfinite(phi) && phi <= 1e-4 * alpha * gd) {
    T.searching = 0;
    return;
  }
  T.ls_backtracks += 1;
  double a_new;
  if (!isfinite(phi)) {
    a_new = 0.5 * alpha;
  } else if (T.ls_trials == 0) {
    a_new = -gd * alpha * alpha / (2.0 * (phi - gd * alpha));
  } else {
    const double a0 = T.ls_prev_alpha, a1 = alpha;
    const double r1 = phi - gd * a1, r0 = T.ls_prev_phi - gd * a0;
    const double den = a0 * a0 * a1 * a1 * (a1 - a0);
    const double ca = (a0 * a0 * r1 - a1 * a1 * r0) / den;
    const double cb = (-a0 * a0 * a0 * r1 + a1 * a1 * a1 * r0) / den;
    const double disc = cb * cb - 3.0 * ca * gd;
    a_new = (ca == 0.0 || disc < 0.0) ? 0.5 * alpha : (-cb + sqrt(disc)) / (3.0 * ca);
  }
  if (!(a_new >= 0.1 * alpha)) a_new = 0.1 * alpha;
  if (a_new > 0.5 * alpha) a_new = 0.5 * alpha;
  T.ls_prev_alpha = alpha;
  T.ls_prev_phi = phi;
  T.ls_alpha = a_new;
  T.ls_trials += 1;
  if (T.ls_trials >= 20) {
    T.searching = 0;
    T.status = SHELL_ERR_LINESEARCH;
    T.active = 0;
    return;
  }
  atomicAdd(&cnt->n_searching, 1);
}

// ------------------------------------------------------------------------------------------
// Conditions of the captured step's WHILE nodes (one thread). Each mirrors a loop bound of the
// host-driven step: Newton while a shell is active and it <= newton_max; regulariser rounds while
// a shell restarts, at most 16; PCG chunks while a shell runs and the iterations are below the
// limit; line-search trials while a shell searches, at most 20.
// ------------------------------------------------------------------------------------------
__global__ void k_cond_newton(const Counters* cnt, LoopState* L, int newton_max, cudaGraphConditionalHandle h,
                              int first) {
  if (first) *L = LoopState{};
  const bool go = cnt->n_active > 0 && L->newton_it <= newton_max;
  if (go) {
    L->newton_it += 1;
    L->n_newton += 1;
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_cond_reg(const Counters* cnt, LoopState* L, cudaGraphConditionalHandle h, int first) {
  bool go;
  if (first) {
    L->round = 0;
    go = true;
  } else {
    L->round += 1;
    go = cnt->n_restart > 0 && L->round < 16;
  }
  if (go) L->n_reg += 1;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_cond_pcg(const Counters* cnt, LoopState* L, int limit, cudaGraphConditionalHandle h, int first) {
  if (first) L->pcg_iters = 0;
  else L->pcg_iters += kGraphPcgChunk;
  const bool go = cnt->n_running > 0 && L->pcg_iters < limit;
  if (go) L->n_pcg += 1;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_cond_ls(const Counters* cnt, LoopState* L, cudaGraphConditionalHandle h, int first) {
  if (first) L->trial = 0;
  else L->trial += 1;
  const bool go = cnt->n_searching > 0 && L->trial < 20;
  if (go) L->n_ls += 1;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// ------------------------------------------------------------------------------------------
// Vector kernels over all DOFs (with per-shell coefficients)
// ------------------------------------------------------------------------------------------
__global__ void k_dots3(int n, const int* __restrict__ nshell, ShellState* st,
                        const double* __restrict__ d, const double* __restrict__ Md,
                        const double* __restrict__ gin, const double* __restrict__ g) {
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  int s0, s1;
  cta_shells(n, nshell, blockIdx.x * 16, 16, &s0, &s1);
  int sh = -1;
  double v0 = 0.0, v1 = 0.0, v2 = 0.0;
  if (i < n) {
    sh = nshell[i];
    if (st[sh].active) {
      const size_t gi = (size_t)i * 12 + a;
      v0 = d[gi] * Md[gi];
      v1 = d[gi] * gin[gi];
      v2 = g[gi] * d[gi];
    }
  }
  // accumulate into acc2[0..2]
  __shared__ double sbuf[32];
  const double a0 = block_sum_d(sh == s0 ? v0 : 0.0, sbuf), b0 = block_sum_d(sh >= 0 && sh != s0 ? v0 : 0.0, sbuf);
  const double a1 = block_sum_d(sh == s0 ? v1 : 0.0, sbuf), b1 = block_sum_d(sh >= 0 && sh != s0 ? v1 : 0.0, sbuf);
  const double a2 = block_sum_d(sh == s0 ? v2 : 0.0, sbuf), b2 = block_sum_d(sh >= 0 && sh != s0 ? v2 : 0.0, sbuf);
  if (threadIdx.x == 0) {
    if (s0 >= 0) {
      atomicAdd(&st[s0].acc2[0], a0); atomicAdd(&st[s0].acc2[1], a1); atomicAdd(&st[s0].acc2[2], a2);
    }
    if (s1 >= 0 && s1 != s0) {
      atomicAdd(&st[s1].acc2[0], b0); atomicAdd(&st[s1].acc2[1], b1); atomicAdd(&st[s1].acc2[2], b2);
    }
  }
}

__global__ void k_mass_mult(int n, const int* __restrict__ rp, const int* __restrict__ col,
                            const double* __restrict__ mass, const double* __restrict__ x,
                            double* __restrict__ y) {
  const int ln = threadIdx.x / 12, a = threadIdx.x % 12;
  const int i = blockIdx.x * 16 + ln;
  if (i >= n) return;
  const int r = a / 3, c = a % 3;
  double sum = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = col[k];
    for (int qq = 0; qq < 4; ++qq) sum += mass[(size_t)k * 16 + r * 4 + qq] * x[(size_t)j * 12 + qq * 3 + c];
  }
  y[(size_t)i * 12 + a] = sum;
}

__global__ void k_dir(int m, const int* __restrict__ nshell, const ShellState* st,
                      const float* __restrict__ x32, const double* __restrict__ g,
                      double* __restrict__ d, double* __restrict__ rhs, int mode) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    if (mode == 0) rhs[k] = -g[k];
    else d[k] = st[nshell[k / 12]].active ? (double)x32[k] : 0.0;
  }
}

__global__ void k_update(int m, const int* __restrict__ nshell, const ShellState* st,
                         double* __restrict__ q, const double* __restrict__ d) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const ShellState& T = st[nshell[k / 12]];
    if (T.active) q[k] += T.ls_alpha * d[k];
  }
}

__global__ void k_count_newton(int S, ShellState* st) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S && st[s].active) st[s].newton_iters += 1;
}

__global__ void k_begin_step(int S, ShellState* st, const StepInput* in) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  st[s] = ShellState{};
  st[s].active = 1;
  st[s].tau = in ? in->tau_carry : 0.0;   // the regulariser level carried in (the first solve starts at a tenth)
}

__global__ void k_predict(int m, const double* __restrict__ q, const double* __restrict__ v, double dt,
                          double* __restrict__ qn, double* __restrict__ y) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    qn[k] = q[k];
    y[k] = q[k] + dt * v[k];
  }
}

__global__ void k_fix(int m, double* __restrict__ q, const double* __restrict__ src,
                      const unsigned char* __restrict__ mask, const double* __restrict__ qfix) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
    q[k] = (mask && mask[k]) ? qfix[k] : src[k];
}

__global__ void k_velocity(int m, const int* __restrict__ nshell, const ShellState* st,
                           double* __restrict__ q, const double* __restrict__ qn, double inv_dt,
                           double* __restrict__ v) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const int status = st[nshell[k / 12]].status;
    if (status == SHELL_OK || status == SHELL_ERR_NOT_CONVERGED) v[k] = (q[k] - qn[k]) * inv_dt;
    else q[k] = qn[k];
  }
}

}  // namespace batch
}  // namespace bhem

// ==========================================================================================
// Host side
// ==========================================================================================
using namespace bhem;
using namespace bhem::batch;

struct shell_batch_s {
  int S = 0, N = 0, P = 0, NB = 0, M = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int ppi = 8, assembly = SHELL_ASM_ATOMIC;
  std::vector<ShellPar> hpar;
  std::vector<int> node_off;
  std::vector<int> color_off;      // offsets of the 9 colour classes in the colour-ordered list
  // device
  ShellPar* par = nullptr;
  ShellState* st = nullptr;
  Counters* cnt = nullptr;
  Counters* h_cnt = nullptr;
  ShellState* h_st = nullptr;
  int *nshell = nullptr, *pshell = nullptr, *row_ptr = nullptr, *col = nullptr, *diag = nullptr;
  int *pblocks = nullptr, *plist_color = nullptr, *dmin_bits = nullptr;
  int4 *pnodes = nullptr, *items = nullptr, *eg_items = nullptr;
  int n_items = 0, n_eg_items = 0;
  std::vector<int> color_item_off;  // items of each colour in the colour-ordered item list
  int4* color_items = nullptr;
  int n_color_items = 0;
  double *dxi = nullptr, *t64 = nullptr, *rest = nullptr, *restgp = nullptr, *mass = nullptr, *fgrav = nullptr;
  float *t32 = nullptr, *val = nullptr, *Dinv = nullptr;
  float *x32 = nullptr, *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *Ap32 = nullptr;
  double *qn = nullptr, *y = nullptr, *g = nullptr, *gin = nullptr, *d = nullptr, *Md = nullptr;
  double *rhs = nullptr, *Ep = nullptr, *qwork = nullptr, *vwork = nullptr, *qfix = nullptr, *warm = nullptr;
  unsigned char* mask = nullptr;
  int* err = nullptr;
  int* h_err = nullptr;
  long long launches = 0;
  cudaGraphExec_t pcg_graph = nullptr;
  int pcg_graph_iters = 0;
  const unsigned char* pcg_graph_mask = nullptr;
  // the captured whole-step graph, its key, capture streams and loop state
  cudaGraphExec_t step_graph = nullptr;
  std::vector<unsigned char> step_key;
  cudaStream_t cap[4] = {nullptr, nullptr, nullptr, nullptr};
  LoopState* loop = nullptr;
  LoopState* h_loop = nullptr;
  StepInput* input = nullptr;      // device copy of the step's inputs (regulariser level)
  StepInput* h_input = nullptr;    // pinned
  long long k_fixed = 0, k_newton = 0, k_reg = 0, k_pcg = 0, k_ls = 0;   // kernels per body
};

namespace {

template <typename T>
shell_status balloc(T** p, size_t count) {
  *p = nullptr;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(SHELL_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return SHELL_OK;
}

void bfree_all(shell_batch_s* b) {
  void* ptrs[] = {b->par, b->st, b->cnt, b->nshell, b->pshell, b->row_ptr, b->col, b->diag, b->pblocks,
                  b->plist_color, b->dmin_bits, b->pnodes, b->items, b->eg_items, b->color_items, b->dxi,
                  b->t64, b->rest, b->restgp, b->mass, b->fgrav, b->t32, b->val, b->Dinv, b->x32, b->r32,
                  b->z32, b->p32, b->Ap32, b->qn, b->y, b->g, b->gin, b->d, b->Md, b->rhs, b->Ep,
                  b->qwork, b->vwork, b->qfix, b->warm, b->mask, b->err, b->loop, b->input};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->h_cnt) cudaFreeHost(b->h_cnt);
  if (b->h_st) cudaFreeHost(b->h_st);
  if (b->h_err) cudaFreeHost(b->h_err);
  if (b->pcg_graph) cudaGraphExecDestroy(b->pcg_graph);
  if (b->step_graph) cudaGraphExecDestroy(b->step_graph);
  if (b->h_loop) cudaFreeHost(b->h_loop);
  if (b->h_input) cudaFreeHost(b->h_input);
  for (cudaStream_t c : b->cap)
    if (c) cudaStreamDestroy(c);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

int blocks_for(long long work, int per) {
  long long v = (work + per - 1) / per;
  return (int)std::max(1LL, std::min(v, 1LL << 30));
}

int vblocks(long long m) { return (int)std::min<long long>(4096, std::max(1LL, (m + 255) / 256)); }

#define BL(b) (++(b).launches)

shell_status check_err(shell_batch_s& b) {
  BHEM_CUDA(cudaMemcpyAsync(b.h_err, b.err, sizeof(int), cudaMemcpyDeviceToHost, b.stream));
  BHEM_CUDA(cudaStreamSynchronize(b.stream));
  const int bits = *b.h_err;
  if (bits) {
    BHEM_CUDA(cudaMemsetAsync(b.err, 0, sizeof(int), b.stream));
    BHEM_CUDA(cudaStreamSynchronize(b.stream));
  }
  if (bits & ERRBIT_DEGENERATE) return fail(SHELL_ERR_DEGENERATE, "degenerate surface normal at a Gauss point");
  if (bits & ERRBIT_NONFINITE) return fail(SHELL_ERR_NONFINITE, "non-finite energy or residual");
  return SHELL_OK;
}

shell_status read_counters(shell_batch_s& b) {
  BHEM_CUDA(cudaMemcpyAsync(b.h_cnt, b.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, b.stream));
  BHEM_CUDA(cudaStreamSynchronize(b.stream));
  return SHELL_OK;
}

shell_status zero_counters(shell_batch_s& b) {
  BHEM_CUDA(cudaMemsetAsync(b.cnt, 0, sizeof(Counters), b.stream));
  return SHELL_OK;
}

size_t elem_smem() { return sizeof(float) * elem_table_elems<float>() + sizeof(WarpSmem<float>) * ElemCfg<float>::kWarps; }

// The element kernel's dynamic shared memory limit, set once per device (outside any capture)
shell_status element_attr(int device) {
  static bool done[128] = {false};
  if (!done[device & 127]) {
    BHEM_CUDA(cudaFuncSetAttribute(k_element, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)elem_smem()));
    done[device & 127] = true;
  }
  return SHELL_OK;
}

// FP32 element Hessians of active shells assembled into the BSR (+ mass_scale M)
shell_status assemble(shell_batch_s& b, const double* q, double mass_scale) {
  BHEM_CUDA(cudaMemsetAsync(b.val, 0, sizeof(float) * 144 * (size_t)b.NB, b.stream));
  BHEM_TRY(element_attr(b.device));
  int nsm = 0;
  BHEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b.device));
  ElemBatchArgs A{};
  A.par = b.par;
  A.st = b.st;
  A.t32 = b.t32;
  A.dxi = b.dxi;
  A.pnodes = b.pnodes;
  A.pblocks = b.pblocks;
  A.q = q;
  A.rest = b.rest;
  A.mass_scale = mass_scale;
  A.bsr = b.val;
  A.err = b.err;
  if (b.assembly == SHELL_ASM_COLOR) {
    A.bsr_atomic = 0;
    A.plist = b.plist_color;
    for (int c = 0; c < 9; ++c) {
      const int i0 = b.color_item_off[c], i1 = b.color_item_off[c + 1];
      if (i1 <= i0) continue;
      A.items = b.color_items + i0;
      A.n_items = i1 - i0;
      k_element<<<std::min(A.n_items, nsm * 8), 32 * ElemCfg<float>::kWarps, elem_smem(), b.stream>>>(A);
      BHEM_CUDA(cudaGetLastError());
      BL(b);
    }
    return SHELL_OK;
  }
  A.bsr_atomic = 1;
  A.items = b.items;
  A.n_items = b.n_items;
  A.plist = nullptr;
  k_element<<<std::min(A.n_items, nsm * 8), 32 * ElemCfg<float>::kWarps, elem_smem(), b.stream>>>(A);
  BHEM_CUDA(cudaGetLastError());
  BL(b);
  return SHELL_OK;
}

// Work items of at most ppi patches of one shell (identity order and colour order)
void build_items(shell_batch_s& b, std::vector<int4>& items, std::vector<int4>& citems,
                 std::vector<int>& coff, const std::vector<int>& color_of, int ppi) {
  items.clear();
  for (int s = 0; s < b.S; ++s)
    for (int p = b.hpar[s].patch_off; p < b.hpar[s].patch_end; p += ppi)
      items.push_back(make_int4(s, p, std::min(p + ppi, b.hpar[s].patch_end), 0));
  // colour order: patches sorted by (colour, shell); items index that list
  citems.clear();
  coff.assign(10, 0);
  std::vector<std::vector<int>> per(9);
  for (int c = 0; c < 9; ++c) {
    coff[c] = (int)citems.size();
    for (int s = 0; s < b.S; ++s) {
      // contiguous positions of colour c within shell s in the colour-ordered list
      const int base = b.color_off[c * (b.S + 1) + s], end = b.color_off[c * (b.S + 1) + s + 1];
      for (int k = base; k < end; k += ppi) citems.push_back(make_int4(s, k, std::min(k + ppi, end), 0));
    }
  }
  coff[9] = (int)citems.size();
  (void)color_of;
}

shell_status upload_items(shell_batch_s& b, int ppi) {
  if (b.step_graph) {   // its element launches hold the previous items
    cudaGraphExecDestroy(b.step_graph);
    b.step_graph = nullptr;
    b.step_key.clear();
  }
  std::vector<int4> items, citems;
  std::vector<int> coff;
  build_items(b, items, citems, coff, std::vector<int>(), ppi);
  if (b.items) cudaFree(b.items);
  if (b.color_items) cudaFree(b.color_items);
  b.items = nullptr;
  b.color_items = nullptr;
  BHEM_TRY(balloc(&b.items, items.size()));
  BHEM_TRY(balloc(&b.color_items, citems.size()));
  BHEM_CUDA(cudaMemcpy(b.items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
  BHEM_CUDA(cudaMemcpy(b.color_items, citems.data(), sizeof(int4) * citems.size(), cudaMemcpyHostToDevice));
  b.n_items = (int)items.size();
  b.n_color_items = (int)citems.size();
  b.color_item_off = coff;
  b.ppi = ppi;
  return SHELL_OK;
}

// FP64 residual of active shells: g, gin, Ep; k_ctrl_newton updates the Newton state.
shell_status residual(shell_batch_s& b, const double* q, const shell_step_params& P,
                      const unsigned char* mask, int set_ref) {
  BHEM_CUDA(cudaMemsetAsync(b.g, 0, sizeof(double) * b.M, b.stream));
  int nsm = 0;
  BHEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b.device));
  k_eg64<<<std::min(b.n_eg_items, nsm * 16), 128, 0, b.stream>>>(b.n_eg_items, b.eg_items, b.P, b.par, b.st,
      b.dxi, b.pnodes, q, nullptr, b.restgp, b.Ep, b.g, 0, b.err);
  BHEM_CUDA(cudaGetLastError());
  BL(b);
  k_grad_finish<<<blocks_for(b.N, 16), kNodeThreads, 0, b.stream>>>(b.N, b.nshell, b.st, b.row_ptr, b.col,
      b.mass, b.fgrav, q, b.y, 1.0 / (P.dt * P.dt), P.gravity[0], P.gravity[1], P.gravity[2], mask, b.g,
      b.gin, b.err);
  BHEM_CUDA(cudaGetLastError());
  BL(b);
  BHEM_TRY(zero_counters(b));
  k_ctrl_newton<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt, P.newton_rtol, P.newton_max, set_ref);
  BHEM_CUDA(cudaGetLastError());
  BL(b);
  BHEM_TRY(check_err(b));
  return read_counters(b);
}

constexpr int kPcgKernels = 4;   // per PCG iteration: SpMV (with the p-update), alpha, update, beta

shell_status pcg_chunk(shell_batch_s& b, const unsigned char* mask, int iters) {
  for (int k = 0; k < iters; ++k) {
    k_spmv<<<blocks_for(b.N, kRowNodes), kSpmvThreads, 0, b.stream>>>(b.N, b.nshell, b.st, b.row_ptr, b.col,
                                                                        b.val, b.z32, mask, b.p32, b.Ap32);
    k_ctrl_alpha<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st);
    k_pcg_update<<<blocks_for(b.N, 16), kNodeThreads, 0, b.stream>>>(b.N, b.nshell, b.st, b.x32, b.r32, b.z32,
                                                                      b.p32, b.Ap32, b.Dinv, mask);
    k_ctrl_beta<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st);
  }
  BHEM_CUDA(cudaGetLastError());
  return SHELL_OK;
}

// A chunk of PCG iterations, replayed from a CUDA graph (captured on first use).
shell_status pcg_chunk_graph(shell_batch_s& b, const unsigned char* mask, int iters) {
  if (!b.pcg_graph || b.pcg_graph_iters != iters || b.pcg_graph_mask != mask) {
    if (b.pcg_graph) cudaGraphExecDestroy(b.pcg_graph);
    b.pcg_graph = nullptr;
    cudaGraph_t graph;
    BHEM_CUDA(cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeThreadLocal));
    shell_status st = pcg_chunk(b, mask, iters);
    cudaError_t e = cudaStreamEndCapture(b.stream, &graph);
    if (st != SHELL_OK) return st;
    if (e != cudaSuccess) return fail(SHELL_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b.pcg_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(SHELL_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    b.pcg_graph_iters = iters;
    b.pcg_graph_mask = mask;
  }
  BHEM_CUDA(cudaGraphLaunch(b.pcg_graph, b.stream));
  b.launches += (long long)kPcgKernels * iters;
  return SHELL_OK;
}

shell_status solve_directions(shell_batch_s& b, const shell_step_params& P, const unsigned char* mask) {
  // rhs = -g; regulariser scale and first admissible level per shell
  k_dir<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, b.nshell, b.st, b.x32, b.g, b.d, b.rhs, 0);
  BL(b);
  BHEM_CUDA(cudaMemsetAsync(b.dmin_bits, 0x7f, sizeof(int) * 4 * (size_t)b.S, b.stream));
  k_diag_stats<<<blocks_for(b.N, 16), kNodeThreads, 0, b.stream>>>(b.N, b.nshell, b.st, b.diag, b.val, mask,
                                                                     b.dmin_bits);
  BL(b);
  k_ctrl_reg_init<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.dmin_bits);
  BL(b);
  k_fix_diag<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, b.nshell, b.st, b.diag, b.val, mask);
  BL(b);
  int only_restart = 0;
  for (int round = 0; round < 16; ++round) {
    k_precond<<<blocks_for(b.N, 16), 192, 0, b.stream>>>(b.N, b.nshell, b.st, b.diag, b.val, mask, b.Dinv,
                                                          only_restart);
    k_pcg_init<<<blocks_for(b.N, 16), kNodeThreads, 0, b.stream>>>(b.N, b.nshell, b.st, b.rhs, b.Dinv, mask,
                                                                    b.x32, b.r32, b.z32, b.p32, only_restart);
    BHEM_TRY(zero_counters(b));
    k_ctrl_pcg_start<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt, only_restart, P.pcg_rtol,
                                                                 P.pcg_max, P.pcg_fixed_iters);
    b.launches += 3;
    BHEM_CUDA(cudaGetLastError());
    BHEM_TRY(read_counters(b));
    int chunk = 4;
    const int limit = P.pcg_fixed_iters > 0 ? P.pcg_fixed_iters : P.pcg_max;
    int done_iters = 0;
    while (b.h_cnt->n_running > 0 && done_iters < limit) {
      const int c = std::min(chunk, limit - done_iters);
      BHEM_TRY(pcg_chunk_graph(b, mask, c));
      done_iters += c;
      chunk = std::min(chunk * 2, 32);
      BHEM_TRY(zero_counters(b));
      k_ctrl_count_running<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt);
      BL(b);
      BHEM_TRY(read_counters(b));
    }
    // negative curvature: move those shells up the regulariser ladder and restart them
    BHEM_TRY(zero_counters(b));
    k_ctrl_restart<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt);
    BL(b);
    BHEM_TRY(read_counters(b));
    if (b.h_cnt->n_restart == 0) break;
    only_restart = 1;
  }
  k_dir<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, b.nshell, b.st, b.x32, b.g, b.d, b.rhs, 1);
  BL(b);
  BHEM_CUDA(cudaGetLastError());
  return SHELL_OK;
}

shell_status line_search(shell_batch_s& b, const shell_step_params& P, const double* q) {
  k_mass_mult<<<blocks_for(b.N, 16), kNodeThreads, 0, b.stream>>>(b.N, b.row_ptr, b.col, b.mass, b.d, b.Md);
  k_dots3<<<blocks_for(b.N, 16), kNodeThreads, 0, b.stream>>>(b.N, b.nshell, b.st, b.d, b.Md, b.gin, b.g);
  BHEM_TRY(zero_counters(b));
  k_ctrl_ls_start<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt, 1.0 / (P.dt * P.dt));
  b.launches += 3;
  BHEM_CUDA(cudaGetLastError());
  BHEM_TRY(read_counters(b));
  int nsm = 0;
  BHEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b.device));
  for (int trial = 0; trial < 20 && b.h_cnt->n_searching > 0; ++trial) {
    k_eg64<<<std::min(b.n_eg_items, nsm * 16), 128, 0, b.stream>>>(b.n_eg_items, b.eg_items, b.P, b.par, b.st,
        b.dxi, b.pnodes, q, b.d, b.restgp, b.Ep, nullptr, 1, b.err);
    BHEM_TRY(zero_counters(b));
    k_ctrl_ls_step<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt);
    b.launches += 2;
    BHEM_CUDA(cudaGetLastError());
    BHEM_TRY(read_counters(b));
  }
  return SHELL_OK;
}

// ------------------------------------------------------------------------------------------
// The whole implicit-Euler step as one CUDA graph: the same kernels as the host-driven step, in
// the same order, with the host's loop decisions moved into WHILE conditional nodes whose
// conditions one-thread kernels set from the device counters. One graph launch per step, no
// host round trip between the phases.
// ------------------------------------------------------------------------------------------
// Creates a condition handle on the graph being captured on s.
shell_status cap_handle(cudaStream_t s, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  BHEM_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive || !g) return fail(SHELL_ERR_CUDA, "step graph: no active capture");
  BHEM_CUDA(cudaGraphConditionalHandleCreate(h, g, 0, 0));
  return SHELL_OK;
}

// Appends a WHILE node with handle h at the capture point of s; later captured work depends on
// it. *body receives the node's body graph.
shell_status cap_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  BHEM_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
  std::vector<cudaGraphNode_t> dv(deps, deps + nd);
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  BHEM_CUDA(cudaGraphAddNode(&node, g, dv.empty() ? nullptr : dv.data(), nullptr, dv.size(), &np));
  BHEM_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  *body = np.conditional.phGraph_out[0];
  return SHELL_OK;
}

// Runs fn with b.stream set to capture stream `level` capturing into graph `body`.
template <typename F>
shell_status cap_body(shell_batch_s& b, int level, cudaGraph_t body, F fn) {
  cudaStream_t keep = b.stream;
  cudaStream_t s = b.cap[level];
  BHEM_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  b.stream = s;
  shell_status st = fn();
  b.stream = keep;
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &out);
  if (st != SHELL_OK) return st;
  if (e != cudaSuccess) return fail(SHELL_ERR_CUDA, std::string("step graph capture: ") + cudaGetErrorString(e));
  return SHELL_OK;
}

// FP64 residual without the host's error check and counter read (those follow the graph)
shell_status enqueue_residual(shell_batch_s& b, const double* q, const shell_step_params& P,
                              const unsigned char* mask, int set_ref, int nsm) {
  BHEM_CUDA(cudaMemsetAsync(b.g, 0, sizeof(double) * b.M, b.stream));
  k_eg64<<<std::min(b.n_eg_items, nsm * 16), 128, 0, b.stream>>>(b.n_eg_items, b.eg_items, b.P, b.par, b.st,
      b.dxi, b.pnodes, q, nullptr, b.restgp, b.Ep, b.g, 0, b.err);
  k_grad_finish<<<blocks_for(b.N, 16), kNodeThreads, 0, b.stream>>>(b.N, b.nshell, b.st, b.row_ptr, b.col,
      b.mass, b.fgrav, q, b.y, 1.0 / (P.dt * P.dt), P.gravity[0], P.gravity[1], P.gravity[2], mask, b.g,
      b.gin, b.err);
  BHEM_TRY(zero_counters(b));
  k_ctrl_newton<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt, P.newton_rtol, P.newton_max, set_ref);
  b.launches += 3;
  BHEM_CUDA(cudaGetLastError());
  return SHELL_OK;
}

// One Newton iteration's body: assembly, regularised PCG direction, line search, update and the
// residual at the new iterate (then the Newton condition).
shell_status enqueue_newton_body(shell_batch_s& b, const shell_step_params& P, const unsigned char* mask,
                                 double* dq, int nsm, cudaGraphConditionalHandle h_newton) {
  const long long l0 = b.launches;
  BHEM_TRY(assemble(b, dq, 1.0 / (P.dt * P.dt)));
  k_dir<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, b.nshell, b.st, b.x32, b.g, b.d, b.rhs, 0);
  BHEM_CUDA(cudaMemsetAsync(b.dmin_bits, 0x7f, sizeof(int) * 4 * (size_t)b.S, b.stream));
  k_diag_stats<<<blocks_for(b.N, 16), kNodeThreads, 0, b.stream>>>(b.N, b.nshell, b.st, b.diag, b.val, mask,
                                                                     b.dmin_bits);
  k_ctrl_reg_init<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.dmin_bits);
  k_fix_diag<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, b.nshell, b.st, b.diag, b.val, mask);
  b.launches += 4;
  cudaGraphConditionalHandle h_reg;
  BHEM_TRY(cap_handle(b.stream, &h_reg));
  k_cond_reg<<<1, 1, 0, b.stream>>>(b.cnt, b.loop, h_reg, 1);
  BL(b);
  cudaGraph_t reg_body = nullptr;
  BHEM_TRY(cap_while(b.stream, h_reg, &reg_body));
  const int limit = P.pcg_fixed_iters > 0 ? P.pcg_fixed_iters : P.pcg_max;
  BHEM_TRY(cap_body(b, 2, reg_body, [&]() -> shell_status {
    const long long r0 = b.launches;
    k_precond<<<blocks_for(b.N, 16), 192, 0, b.stream>>>(b.N, b.nshell, b.st, b.diag, b.val, mask, b.Dinv, 1);
    k_pcg_init<<<blocks_for(b.N, 16), kNodeThreads, 0, b.stream>>>(b.N, b.nshell, b.st, b.rhs, b.Dinv, mask,
                                                                    b.x32, b.r32, b.z32, b.p32, 1);
    BHEM_TRY(zero_counters(b));
    k_ctrl_pcg_start<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt, 1, P.pcg_rtol, P.pcg_max,
                                                                 P.pcg_fixed_iters);
    b.launches += 3;
    cudaGraphConditionalHandle h_pcg;
    BHEM_TRY(cap_handle(b.stream, &h_pcg));
    k_cond_pcg<<<1, 1, 0, b.stream>>>(b.cnt, b.loop, limit, h_pcg, 1);
    BL(b);
    cudaGraph_t pcg_body = nullptr;
    BHEM_TRY(cap_while(b.stream, h_pcg, &pcg_body));
    BHEM_TRY(cap_body(b, 3, pcg_body, [&]() -> shell_status {
      const long long p0 = b.launches;
      BHEM_TRY(pcg_chunk(b, mask, kGraphPcgChunk));
      b.launches += (long long)kPcgKernels * kGraphPcgChunk;
      BHEM_TRY(zero_counters(b));
      k_ctrl_count_running<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt);
      k_cond_pcg<<<1, 1, 0, b.stream>>>(b.cnt, b.loop, limit, h_pcg, 0);
      b.launches += 2;
      BHEM_CUDA(cudaGetLastError());
      b.k_pcg = b.launches - p0;
      return SHELL_OK;
    }));
    BHEM_TRY(zero_counters(b));
    k_ctrl_restart<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt);
    k_cond_reg<<<1, 1, 0, b.stream>>>(b.cnt, b.loop, h_reg, 0);
    b.launches += 2;
    BHEM_CUDA(cudaGetLastError());
    b.k_reg = (b.launches - r0) - b.k_pcg;
    return SHELL_OK;
  }));
  k_dir<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, b.nshell, b.st, b.x32, b.g, b.d, b.rhs, 1);
  // line search
  k_mass_mult<<<blocks_for(b.N, 16), kNodeThreads, 0, b.stream>>>(b.N, b.row_ptr, b.col, b.mass, b.d, b.Md);
  k_dots3<<<blocks_for(b.N, 16), kNodeThreads, 0, b.stream>>>(b.N, b.nshell, b.st, b.d, b.Md, b.gin, b.g);
  BHEM_TRY(zero_counters(b));
  k_ctrl_ls_start<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt, 1.0 / (P.dt * P.dt));
  b.launches += 4;
  cudaGraphConditionalHandle h_ls;
  BHEM_TRY(cap_handle(b.stream, &h_ls));
  k_cond_ls<<<1, 1, 0, b.stream>>>(b.cnt, b.loop, h_ls, 1);
  BL(b);
  cudaGraph_t ls_body = nullptr;
  BHEM_TRY(cap_while(b.stream, h_ls, &ls_body));
  BHEM_TRY(cap_body(b, 2, ls_body, [&]() -> shell_status {
    const long long s0 = b.launches;
    k_eg64<<<std::min(b.n_eg_items, nsm * 16), 128, 0, b.stream>>>(b.n_eg_items, b.eg_items, b.P, b.par, b.st,
        b.dxi, b.pnodes, dq, b.d, b.restgp, b.Ep, nullptr, 1, b.err);
    BHEM_TRY(zero_counters(b));
    k_ctrl_ls_step<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.cnt);
    k_cond_ls<<<1, 1, 0, b.stream>>>(b.cnt, b.loop, h_ls, 0);
    b.launches += 3;
    BHEM_CUDA(cudaGetLastError());
    b.k_ls = b.launches - s0;
    return SHELL_OK;
  }));
  k_update<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, b.nshell, b.st, dq, b.d);
  k_count_newton<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st);
  b.launches += 2;
  BHEM_TRY(enqueue_residual(b, dq, P, mask, 0, nsm));
  k_cond_newton<<<1, 1, 0, b.stream>>>(b.cnt, b.loop, P.newton_max, h_newton, 0);
  BL(b);
  BHEM_CUDA(cudaGetLastError());
  b.k_newton = (b.launches - l0) - b.k_reg - b.k_pcg - b.k_ls;
  return SHELL_OK;
}

// Captures (or reuses) the graph of one whole step for these pointers and parameters.
shell_status step_graph(shell_batch_s& b, const shell_step_params& P, const unsigned char* mask,
                        const double* qfix, const double* warm, double* dq, double* dv) {
  // the key: every value the captured kernels take by value (the regulariser level carried into
  // the step is read from device memory instead, so it needs no new capture)
  const double fp[7] = {P.dt, P.gravity[0], P.gravity[1], P.gravity[2], P.newton_rtol, P.pcg_rtol, 0.0};
  const int ip[5] = {P.newton_max, P.pcg_max, P.pcg_fixed_iters, b.ppi, b.assembly};
  const void* ptrs[6] = {mask, qfix, warm, dq, dv, b.items};
  std::vector<unsigned char> key(sizeof(fp) + sizeof(ip) + sizeof(ptrs));
  std::memcpy(key.data(), fp, sizeof(fp));
  std::memcpy(key.data() + sizeof(fp), ip, sizeof(ip));
  std::memcpy(key.data() + sizeof(fp) + sizeof(ip), ptrs, sizeof(ptrs));
  if (b.step_graph && key == b.step_key) return SHELL_OK;
  if (b.step_graph) cudaGraphExecDestroy(b.step_graph);
  b.step_graph = nullptr;
  for (int l = 0; l < 4; ++l)
    if (!b.cap[l]) BHEM_CUDA(cudaStreamCreateWithFlags(&b.cap[l], cudaStreamNonBlocking));
  if (!b.loop) {
    BHEM_TRY(balloc(&b.loop, 1));
    BHEM_CUDA(cudaMallocHost((void**)&b.h_loop, sizeof(LoopState)));
  }
  BHEM_TRY(element_attr(b.device));
  int nsm = 0;
  BHEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b.device));
  cudaGraph_t graph = nullptr;
  BHEM_CUDA(cudaGraphCreate(&graph, 0));
  const long long keep_launches = b.launches;
  shell_status st = cap_body(b, 0, graph, [&]() -> shell_status {
    const long long f0 = b.launches;
    k_begin_step<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.input);
    k_predict<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, dq, dv, P.dt, b.qn, b.y);
    k_fix<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, dq, b.qn, mask, qfix);
    b.launches += 3;
    BHEM_TRY(enqueue_residual(b, dq, P, mask, 1, nsm));
    if (warm) {
      k_fix<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, dq, warm, mask, qfix);
      BL(b);
      BHEM_TRY(enqueue_residual(b, dq, P, mask, 0, nsm));
    }
    cudaGraphConditionalHandle h_newton;
    BHEM_TRY(cap_handle(b.stream, &h_newton));
    k_cond_newton<<<1, 1, 0, b.stream>>>(b.cnt, b.loop, P.newton_max, h_newton, 1);
    BL(b);
    const long long f1 = b.launches;
    cudaGraph_t newton_body = nullptr;
    BHEM_TRY(cap_while(b.stream, h_newton, &newton_body));
    BHEM_TRY(cap_body(b, 1, newton_body, [&]() { return enqueue_newton_body(b, P, mask, dq, nsm, h_newton); }));
    const long long f2 = b.launches;
    k_velocity<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, b.nshell, b.st, dq, b.qn, 1.0 / P.dt, dv);
    BL(b);
    BHEM_CUDA(cudaGetLastError());
    b.k_fixed = (f1 - f0) + (b.launches - f2);
    return SHELL_OK;
  });
  b.launches = keep_launches;
  if (st != SHELL_OK) {
    cudaGraphDestroy(graph);
    return st;
  }
  const cudaError_t e = cudaGraphInstantiate(&b.step_graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b.step_graph = nullptr;
    return fail(SHELL_ERR_CUDA, std::string("step graph instantiate: ") + cudaGetErrorString(e));
  }
  b.step_key = key;
  return SHELL_OK;
}

bool is_dev(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" shell_status shell_batch_create(int n_shells, const shell_grid* grids,
                                           const shell_material* materials, const double* rest_dofs,
                                           const shell_options* options, void* stream,
                                           shell_batch_t** out) {
  if (n_shells < 1 || !grids || !materials || !rest_dofs || !out) return fail(SHELL_ERR_ARG, "NULL argument or no shells");
  *out = nullptr;
  if (options && options->precision != SHELL_PREC_MIXED)
    return fail(SHELL_ERR_ARG, "batches run in SHELL_PREC_MIXED precision only");
  shell_batch_s* b = new shell_batch_s();
  b->S = n_shells;
  b->stream = (cudaStream_t)stream;
  if (!b->stream) {
    // the PCG iterations are replayed from a CUDA graph, which cannot be captured on the legacy
    // default stream: use a private blocking stream (it orders with the legacy stream)
    if (cudaStreamCreate(&b->stream) != cudaSuccess) {
      delete b;
      return fail(SHELL_ERR_CUDA, "cudaStreamCreate failed");
    }
    b->own_stream = true;
  }
  cudaGetDevice(&b->device);
  if (options) b->assembly = options->assembly;
  // per-shell topology, concatenated
  std::vector<int4> pnodes;
  std::vector<int> row_ptr(1, 0), col, pblocks, diag, nshell, pshell;
  std::vector<double> dxi;
  b->hpar.resize(n_shells);
  b->node_off.assign(n_shells + 1, 0);
  std::vector<std::vector<int>> color_lists(9 * n_shells);
  int node0 = 0, patch0 = 0;
  for (int s = 0; s < n_shells; ++s) {
    const shell_grid& g = grids[s];
    const shell_material& m = materials[s];
    if (g.nu < 1 || g.nv < 1 || (g.periodic_u && g.nu < 2) || (g.periodic_v && g.nv < 2) || !(g.dxi1 > 0) ||
        !(g.dxi2 > 0) || !(m.thickness > 0) || !(m.young > 0) || !(m.poisson > -1 && m.poisson < 1)) {
      if (b->own_stream) cudaStreamDestroy(b->stream);
      delete b;
      return fail(SHELL_ERR_ARG, "invalid grid or material of shell " + std::to_string(s));
    }
    const int n1 = g.periodic_u ? g.nu : g.nu + 1, n2 = g.periodic_v ? g.nv : g.nv + 1;
    const int n = n1 * n2, np = g.nu * g.nv;
    if (n < 16) {
      if (b->own_stream) cudaStreamDestroy(b->stream);
      delete b;
      return fail(SHELL_ERR_ARG, "every shell of a batch needs at least 16 nodes");
    }
    ShellPar& sp = b->hpar[s];
    sp.lam = m.young * m.poisson / (1.0 - m.poisson * m.poisson);
    sp.mu = m.young / (2.0 * (1.0 + m.poisson));
    sp.h = m.thickness;
    sp.rho_h = m.density * m.thickness;
    sp.node_off = node0;
    sp.node_end = node0 + n;
    sp.patch_off = patch0;
    sp.patch_end = patch0 + np;
    dxi.push_back(g.dxi1);
    dxi.push_back(g.dxi2);
    std::vector<std::vector<int>> nb(n);
    for (int pv = 0; pv < g.nv; ++pv)
      for (int pu = 0; pu < g.nu; ++pu) {
        const int i0 = pu % n1, i1 = (pu + 1) % n1, j0 = pv % n2, j1 = (pv + 1) % n2;
        int4 pn = make_int4(node0 + j0 * n1 + i0, node0 + j0 * n1 + i1, node0 + j1 * n1 + i0, node0 + j1 * n1 + i1);
        pnodes.push_back(pn);
        pshell.push_back(s);
        const int nd[4] = {pn.x - node0, pn.y - node0, pn.z - node0, pn.w - node0};
        for (int a = 0; a < 4; ++a)
          for (int c = 0; c < 4; ++c) nb[nd[a]].push_back(nd[c]);
        color_lists[patch_colour(g, pu, pv) * n_shells + s].push_back(patch0 + pv * g.nu + pu);
      }
    const int blk0 = (int)col.size();
    for (int i = 0; i < n; ++i) {
      auto& v = nb[i];
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
      for (int c : v) col.push_back(node0 + c);
      row_ptr.push_back((int)col.size());
      nshell.push_back(s);
    }
    auto find = [&](int r, int c) {
      auto bgn = col.begin() + row_ptr[r], end = col.begin() + row_ptr[r + 1];
      return (int)(std::lower_bound(bgn, end, c) - col.begin());
    };
    for (int p = 0; p < np; ++p) {
      const int4 pn = pnodes[patch0 + p];
      const int nd[4] = {pn.x, pn.y, pn.z, pn.w};
      for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 4; ++c) pblocks.push_back(find(nd[a], nd[c]));
    }
    for (int i = 0; i < n; ++i) diag.push_back(find(node0 + i, node0 + i));
    (void)blk0;
    node0 += n;
    patch0 += np;
    b->node_off[s + 1] = node0;
  }
  b->N = node0;
  b->P = patch0;
  b->NB = (int)col.size();
  b->M = 12 * b->N;
  // colour-ordered patch list and per-(colour, shell) offsets
  std::vector<int> plist;
  b->color_off.assign(9 * (n_shells + 1), 0);
  for (int c = 0; c < 9; ++c) {
    for (int s = 0; s < n_shells; ++s) {
      b->color_off[c * (n_shells + 1) + s] = (int)plist.size();
      for (int p : color_lists[c * n_shells + s]) plist.push_back(p);
    }
    b->color_off[c * (n_shells + 1) + n_shells] = (int)plist.size();
  }
  std::vector<int4> eg;
  for (int s = 0; s < n_shells; ++s)
    for (int p = b->hpar[s].patch_off; p < b->hpar[s].patch_end; p += kEgPatches)
      eg.push_back(make_int4(s, p, std::min(p + kEgPatches, b->hpar[s].patch_end), 0));
  b->n_eg_items = (int)eg.size();

  const size_t S = n_shells, N = b->N, P = b->P, NB = b->NB, M = b->M;
  shell_status st = SHELL_OK;
#define BA(ptr, count) \
  if (st == SHELL_OK) st = balloc(&(ptr), (size_t)(count))
  BA(b->par, S); BA(b->st, S); BA(b->cnt, 1); BA(b->nshell, N); BA(b->pshell, P); BA(b->row_ptr, N + 1);
  BA(b->col, NB); BA(b->diag, N); BA(b->pblocks, P * 16); BA(b->plist_color, P); BA(b->dmin_bits, 4 * S);
  BA(b->pnodes, P); BA(b->eg_items, eg.size()); BA(b->dxi, 2 * S); BA(b->t64, S * kPhiTable);
  BA(b->t32, S * kPhiTable); BA(b->rest, M); BA(b->restgp, 13 * P * 16); BA(b->mass, NB * 16);
  BA(b->fgrav, N * 4); BA(b->val, NB * 144); BA(b->Dinv, N * 144); BA(b->x32, M); BA(b->r32, M);
  BA(b->z32, M); BA(b->p32, M); BA(b->Ap32, M); BA(b->qn, M); BA(b->y, M); BA(b->g, M); BA(b->gin, M);
  BA(b->d, M); BA(b->Md, M); BA(b->rhs, M); BA(b->Ep, P); BA(b->qwork, M); BA(b->vwork, M);
  BA(b->qfix, M); BA(b->warm, M); BA(b->mask, M); BA(b->err, 1);
#undef BA
  if (st == SHELL_OK) {
    if (cudaMallocHost((void**)&b->h_cnt, sizeof(Counters)) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_st, sizeof(ShellState) * S) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_err, sizeof(int)) != cudaSuccess)
      st = fail(SHELL_ERR_OOM, "cudaMallocHost failed");
  }
  if (st != SHELL_OK) {
    bfree_all(b);
    return st;
  }
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, b->stream);
  };
  up(b->par, b->hpar.data(), sizeof(ShellPar) * S);
  up(b->nshell, nshell.data(), sizeof(int) * N);
  up(b->pshell, pshell.data(), sizeof(int) * P);
  up(b->row_ptr, row_ptr.data(), sizeof(int) * (N + 1));
  up(b->col, col.data(), sizeof(int) * NB);
  up(b->diag, diag.data(), sizeof(int) * N);
  up(b->pblocks, pblocks.data(), sizeof(int) * P * 16);
  up(b->plist_color, plist.data(), sizeof(int) * P);
  up(b->pnodes, pnodes.data(), sizeof(int4) * P);
  up(b->eg_items, eg.data(), sizeof(int4) * eg.size());
  up(b->dxi, dxi.data(), sizeof(double) * 2 * S);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->rest, rest_dofs, sizeof(double) * M, cudaMemcpyDefault, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->st, 0, sizeof(ShellState) * S, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->mass, 0, sizeof(double) * NB * 16, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->fgrav, 0, sizeof(double) * N * 4, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    bfree_all(b);
    return fail(SHELL_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
  }
  st = upload_items(*b, b->ppi);
  if (st == SHELL_OK) {
    k_tables<<<n_shells, 256, 0, b->stream>>>(n_shells, b->dxi, b->t64, b->t32);
    k_rest<<<blocks_for((long long)P * 16, 256), 256, 0, b->stream>>>(b->P, b->pshell, b->par, b->pnodes, b->rest,
                                                                      b->t64, b->restgp, b->err);
    k_mass<<<blocks_for((long long)P * 32, 256), 256, 0, b->stream>>>(b->P, b->pshell, b->par, b->pblocks,
                                                                      b->pnodes, b->restgp, b->t64, b->mass,
                                                                      b->fgrav);
    b->launches += 3;
    if (cudaGetLastError() != cudaSuccess) st = fail(SHELL_ERR_CUDA, "batch set-up launch failed");
  }
  if (st == SHELL_OK) st = check_err(*b);
  if (st != SHELL_OK) {
    bfree_all(b);
    return st;
  }
  *out = b;
  return SHELL_OK;
}

extern "C" shell_status shell_batch_destroy(shell_batch_t* batch) {
  if (!batch) return SHELL_OK;
  cudaStreamSynchronize(batch->stream);
  bfree_all(batch);
  return SHELL_OK;
}

extern "C" shell_status shell_batch_info(const shell_batch_t* b, shell_batch_info_t* info, int* node_offsets) {
  if (!b || !info) return fail(SHELL_ERR_ARG, "NULL argument");
  info->n_shells = b->S;
  info->n_nodes = b->N;
  info->n_patches = b->P;
  info->n_blocks = b->NB;
  info->n_dof = b->M;
  info->patches_per_item = b->ppi;
  info->assembly = b->assembly;
  info->kernel_launches = b->launches;
  if (node_offsets) std::memcpy(node_offsets, b->node_off.data(), sizeof(int) * (b->S + 1));
  return SHELL_OK;
}

extern "C" shell_status shell_batch_autotune(shell_batch_t* batch, const double* q, int repeats) {
  if (!batch || !q) return fail(SHELL_ERR_ARG, "NULL argument");
  shell_batch_s& b = *batch;
  if (repeats < 1) repeats = 3;
  // every shell active for the trial assemblies
  k_begin_step<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, nullptr);
  BL(b);
  const int ppis[4] = {4, 8, 16, 32};
  const int schemes[2] = {SHELL_ASM_ATOMIC, SHELL_ASM_COLOR};
  cudaEvent_t e0, e1;
  BHEM_CUDA(cudaEventCreate(&e0));
  BHEM_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_ppi = b.ppi, best_asm = b.assembly;
  for (int ppi : ppis) {
    BHEM_TRY(upload_items(b, ppi));
    for (int sch : schemes) {
      b.assembly = sch;
      BHEM_TRY(assemble(b, q, 1.0));   // warm-up
      BHEM_CUDA(cudaEventRecord(e0, b.stream));
      for (int r = 0; r < repeats; ++r) BHEM_TRY(assemble(b, q, 1.0));
      BHEM_CUDA(cudaEventRecord(e1, b.stream));
      BHEM_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      BHEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_ppi = ppi;
        best_asm = sch;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BHEM_TRY(upload_items(b, best_ppi));
  b.assembly = best_asm;
  return SHELL_OK;
}

extern "C" shell_status shell_batch_newton_step(shell_batch_t* batch, const shell_step_params* params,
                                                const unsigned char* fixed_mask, const double* q_fixed,
                                                double* q, double* v, const double* warm_start,
                                                shell_step_stats* stats) {
  if (!batch || !params || !q || !v || !stats) return fail(SHELL_ERR_ARG, "NULL argument");
  if ((fixed_mask == nullptr) != (q_fixed == nullptr)) return fail(SHELL_ERR_ARG, "fixed_mask and q_fixed go together");
  const shell_step_params& P = *params;
  if (!(P.dt > 0) || P.newton_max < 0 || P.pcg_max < 0 || P.pcg_fixed_iters < 0 || !(P.tau_carry >= 0) ||
      !std::isfinite(P.tau_carry))
    return fail(SHELL_ERR_ARG, "invalid step parameters");
  shell_batch_s& b = *batch;
  const size_t bytes = sizeof(double) * b.M;
  const bool q_dev = is_dev(q), v_dev = is_dev(v);
  double* dq = q_dev ? q : b.qwork;
  double* dv = v_dev ? v : b.vwork;
  if (!q_dev) BHEM_CUDA(cudaMemcpyAsync(dq, q, bytes, cudaMemcpyHostToDevice, b.stream));
  if (!v_dev) BHEM_CUDA(cudaMemcpyAsync(dv, v, bytes, cudaMemcpyHostToDevice, b.stream));
  const unsigned char* mask = nullptr;
  const double* qfix = nullptr;
  if (fixed_mask) {   // internal copies keep the captured PCG graph's pointers stable
    BHEM_CUDA(cudaMemcpyAsync(b.mask, fixed_mask, b.M, cudaMemcpyDefault, b.stream));
    BHEM_CUDA(cudaMemcpyAsync(b.qfix, q_fixed, bytes, cudaMemcpyDefault, b.stream));
    mask = b.mask;
    qfix = b.qfix;
  }
  const double* warm = nullptr;
  if (warm_start) {
    BHEM_CUDA(cudaMemcpyAsync(b.warm, warm_start, bytes, cudaMemcpyDefault, b.stream));
    warm = b.warm;
  }
  const bool host_loop = std::getenv("BHEM_BATCH_HOST_LOOP") != nullptr;
  if (!b.input) {
    BHEM_TRY(balloc(&b.input, 1));
    BHEM_CUDA(cudaMallocHost((void**)&b.h_input, sizeof(StepInput)));
  }
  b.h_input->tau_carry = P.tau_carry;   // the previous step has synchronised: the buffer is free
  BHEM_CUDA(cudaMemcpyAsync(b.input, b.h_input, sizeof(StepInput), cudaMemcpyHostToDevice, b.stream));
  if (!host_loop) {
    // the whole step is one graph launch; its device-side loops replace the host's decisions
    BHEM_TRY(step_graph(b, P, mask, qfix, warm, dq, dv));
    BHEM_CUDA(cudaGraphLaunch(b.step_graph, b.stream));
    BHEM_CUDA(cudaMemcpyAsync(b.h_loop, b.loop, sizeof(LoopState), cudaMemcpyDeviceToHost, b.stream));
    BHEM_TRY(check_err(b));   // synchronises the stream
    const LoopState& L = *b.h_loop;
    b.launches += b.k_fixed + L.n_newton * b.k_newton + L.n_reg * b.k_reg + L.n_pcg * b.k_pcg + L.n_ls * b.k_ls;
  } else {
    // host-driven step (BHEM_BATCH_HOST_LOOP set): the same kernels, each loop decided on the
    // host from the counters; profilers list every kernel of this form
    k_begin_step<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st, b.input);
    k_predict<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, dq, dv, P.dt, b.qn, b.y);
    k_fix<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, dq, b.qn, mask, qfix);
    b.launches += 3;
    BHEM_CUDA(cudaGetLastError());
    BHEM_TRY(residual(b, dq, P, mask, 1));
    if (warm) {
      k_fix<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, dq, warm, mask, qfix);
      BL(b);
      BHEM_TRY(residual(b, dq, P, mask, 0));
    }
    for (int it = 0; it <= P.newton_max && b.h_cnt->n_active > 0; ++it) {
      BHEM_TRY(assemble(b, dq, 1.0 / (P.dt * P.dt)));
      BHEM_TRY(solve_directions(b, P, mask));
      BHEM_TRY(line_search(b, P, dq));
      k_update<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, b.nshell, b.st, dq, b.d);
      k_count_newton<<<blocks_for(b.S, 128), 128, 0, b.stream>>>(b.S, b.st);
      b.launches += 2;
      BHEM_CUDA(cudaGetLastError());
      BHEM_TRY(residual(b, dq, P, mask, 0));
    }
    k_velocity<<<vblocks(b.M), 256, 0, b.stream>>>(b.M, b.nshell, b.st, dq, b.qn, 1.0 / P.dt, dv);
    BL(b);
  }
  if (!q_dev) BHEM_CUDA(cudaMemcpyAsync(q, dq, bytes, cudaMemcpyDeviceToHost, b.stream));
  if (!v_dev) BHEM_CUDA(cudaMemcpyAsync(v, dv, bytes, cudaMemcpyDeviceToHost, b.stream));
  BHEM_CUDA(cudaMemcpyAsync(b.h_st, b.st, sizeof(ShellState) * b.S, cudaMemcpyDeviceToHost, b.stream));
  BHEM_CUDA(cudaStreamSynchronize(b.stream));
  shell_status worst = SHELL_OK;
  for (int s = 0; s < b.S; ++s) {
    const ShellState& T = b.h_st[s];
    shell_step_stats& o = stats[s];
    o.newton_iters = T.newton_iters;
    o.pcg_iters_total = T.pcg_iters_total;
    o.ls_backtracks = T.ls_backtracks;
    o.regularizations = T.regularizations;
    o.status = T.status;
    o.diag_fixes = T.diag_fixes;
    o.tau_final = T.tau;
    o.res0 = T.gref;
    o.res_final = T.gn;
    if (T.status != SHELL_OK && worst == SHELL_OK) worst = (shell_status)T.status;
  }
  if (worst != SHELL_OK) set_error("at least one shell of the batch did not finish its step");
  return worst;
}
