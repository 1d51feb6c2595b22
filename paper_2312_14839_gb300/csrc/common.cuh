// Internal declarations of libbhem (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "bhem.h"

namespace bhem {

// ------------------------------------------------------------------------------------------
// Error handling: every entry point returns a shell_status and records a thread-local message.
// ------------------------------------------------------------------------------------------
void set_error(const std::string& msg);
shell_status fail(shell_status st, const std::string& msg);

#define BHEM_CUDA(call)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return ::bhem::fail(SHELL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define BHEM_TRY(call)                          \
  do {                                          \
    shell_status s_ = (call);                   \
    if (s_ != SHELL_OK) return s_;              \
  } while (0)

// ------------------------------------------------------------------------------------------
// Patch colours of the colour-ordered assembly: two patches of one colour share no node.
// Along one direction, patches p and p +- 1 share a node column (and, when periodic, the seam
// patch n - 1 shares one with patch 0), so a proper colouring of that path or cycle is p % 2,
// except on an odd cycle, whose seam patch takes the third colour. A 2D colour is the pair
// (u colour, v colour) numbered u + 3 v, so colour ids lie in [0, 9) (some may be empty).
// ------------------------------------------------------------------------------------------
inline int patch_colour_1d(int p, int n, int periodic) {
  return (periodic && (n & 1) && p == n - 1) ? 2 : (p & 1);
}
inline int patch_colour(const shell_grid& g, int pu, int pv) {
  return patch_colour_1d(pu, g.nu, g.periodic_u) + 3 * patch_colour_1d(pv, g.nv, g.periodic_v);
}
constexpr int kColours = 9;

// Polls of a bounded device-side wait (an mbarrier of the bulk-copy SpMV) before it gives up.
constexpr int kDefaultWaitPolls = 1 << 20;

// Device-side error bits (OR-ed into Shell::d_err, read back at synchronising calls).
enum : int { ERRBIT_DEGENERATE = 1, ERRBIT_NONFINITE = 2, ERRBIT_TIMEOUT = 4 };

// ------------------------------------------------------------------------------------------
// Deterministic grid reductions: each CTA writes a partial, the last CTA to arrive (atomic
// ticket, no waiting) sums the partials in CTA order and resets the ticket.
// ------------------------------------------------------------------------------------------
constexpr int kMaxRed = 16;             // values reduced together
constexpr int kMaxPartials = 1 << 17;   // CTAs per reduced kernel (checked at launch)

struct Reduce {
  double* partials;    // [kMaxRed * stride]
  unsigned* ticket;    // one counter
  int stride;          // partials per reduced value (>= the CTAs of any reducing launch)
};

// Scalars of one PCG solve, resident in device memory.
struct PcgState {
  double rz, pq, alpha, beta, rr, bb;
  double rtol2;        // rtol^2 (0 disables the residual test)
  int iters, done, negcurv, fixed;
  int limit;           // iteration cap (mixed precision: enforced on the device)
  float td[4];         // regulariser shift tau * D_k per DOF kind (mixed precision)
  int bodies;          // loop bodies run by the device-side PCG loop (mixed precision)
};

// Scalars of one Newton step.
struct NewtonScalars {
  double gnorm2;       // |g_free|^2
  double dots[3];      // d.Md, d.g_inert, d.g
  double dV;           // sum_p (E_p(q + a d) - E_p(q))
  double energy;       // assembled elastic energy
  double diag_stats[12];  // per DOF kind: sum |A_ii|, count, min A_ii over free DOFs
  int diag_fixes;      // free diagonal entries changed by the regulariser's local part (per step)
  int pad_;
};

// ------------------------------------------------------------------------------------------
// Shell: everything lives in device memory owned by the library.
// ------------------------------------------------------------------------------------------
struct Shell {
  shell_grid grid;
  shell_material mat;
  shell_options opt;
  cudaStream_t stream = nullptr;
  int device = 0;
  int n1 = 0, n2 = 0, n_nodes = 0, n_patches = 0, n_blocks = 0, n_dof = 0;
  double lam = 0, mu = 0;

  // topology
  int4* d_patch_nodes = nullptr;    // [np] corner node ids 00, 10, 01, 11
  int* d_patch_blocks = nullptr;    // [np * 16] BSR block of corner pair (a, b) at a * 4 + b
  int* d_row_ptr = nullptr;         // [n_nodes + 1]
  int* d_col = nullptr;             // [n_blocks]
  int* d_diag_block = nullptr;      // [n_nodes]
  int* d_tpos = nullptr;            // [n_nodes][8]: the blocks (j, i) of row i's blocks (i, j) left of its diagonal
  int* d_color_start = nullptr;     // unused by the atomic path
  int* h_color_patches = nullptr;   // host copy of the colour offsets (kColours + 1 ints)
  int* d_color_list = nullptr;      // [np] patches ordered by colour

  // reference configuration
  double* d_rest = nullptr;         // [n_dof]
  double* d_restgp = nullptr;       // [13 * np * 16] per-Gauss-point rest data (SoA)
  double* d_phi64 = nullptr;        // shape table + Gauss weights (kPhiTable doubles)
  float* d_phi32 = nullptr;         // the same in FP32
  double* d_mass = nullptr;         // [n_blocks * 16] consistent mass, 4x4 scalar blocks
  double* d_qmy = nullptr;          // [n_dof] q - y of the residual's inertial term
  double* d_fgrav = nullptr;        // [n_nodes * 4] gravity load factors

  // assembled matrix
  void* d_val = nullptr;            // [n_blocks * 144] FP32 or FP64
  int val_fp64 = 0;

  // PCG workspace
  double *d_x = nullptr, *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_Ap = nullptr;
  float* d_p32 = nullptr;           // FP32 PCG vectors of a mixed-precision shell
  float *d_x32 = nullptr, *d_r32 = nullptr, *d_z32 = nullptr, *d_Ap32 = nullptr;
  void* d_Dinv = nullptr;           // [n_nodes * 144] block-Jacobi inverses (FP32 or FP64)
  PcgState* d_pcg = nullptr;

  // Newton workspace
  double *d_qn = nullptr, *d_y = nullptr, *d_g = nullptr, *d_gin = nullptr, *d_d = nullptr;
  double *d_Md = nullptr, *d_Ep = nullptr, *d_qwork = nullptr, *d_vwork = nullptr;
  double *d_qfix = nullptr, *d_warm = nullptr, *d_rhs = nullptr;
  double *d_g2 = nullptr, *d_Ep2 = nullptr;  // elastic gradient / patch energies at the first line-search trial
  unsigned char* d_mask = nullptr;
  NewtonScalars* d_ns = nullptr;
  NewtonScalars* h_ns = nullptr;    // pinned
  PcgState* h_pcg = nullptr;        // pinned
  int* d_err = nullptr;
  int* h_err = nullptr;             // pinned
  double* d_energy_tmp = nullptr;

  // Sec. 5 searches (rays.cu, ccd.cu), allocated by their first call: d_search holds the 128
  // global candidate heaps, two counters and the redo list (shared: calls on one shell do not
  // overlap); d_ray_nets the ray search's Bezier nets [np][3][4][4] and boxes [np][8];
  // d_ccd_nets the collision search's start and displacement nets and swept boxes [np][104]
  void* d_search = nullptr;
  // direct solver (direct.cu): the banded Cholesky factor (row blocks), solve vectors and a flag
  double* d_dense = nullptr;
  double* d_ray_nets = nullptr;
  double* d_ccd_nets = nullptr;

  Reduce red{};
  Reduce red_aux{};                 // grid reductions of work on aux_stream (diagonal statistics)
  long long launches = 0;           // kernels launched by this shell (introspection)

  // FP32 SpMV variant: TMA-pipelined persistent kernel when its row-group stages fit in shared
  // memory (max_row = most blocks in one block row)
  int num_sms = 0;                  // multiprocessors of the shell's device (grid sizes)
  int update_grid = 0;              // CTAs of the mixed-precision PCG update (resident at once)
  // BHEM_PCG_HOST_LOOP set: mixed-precision PCG iterations are launched from the host in chunks
  // (as in FP64) instead of the device-side graph loop, whose kernels a profiler cannot list
  int pcg_host_loop = 0;
  // mixed-precision solve form: 1 the device-side graph loop (the default), 0 one persistent
  // cooperative launch per solve (BHEM_PCG_LOOP=persistent), 2 host chunks (BHEM_PCG_LOOP=host or
  // BHEM_PCG_HOST_LOOP)
  int pcg_mode = 1;
  void* d_persist = nullptr;        // persistent PCG: barrier, published totals, per-CTA partials
  int persist_max_ctas = 0;
  int max_row = 0;
  int spmv_tma = 0, spmv_grid = 0, spmv_stage_floats = 0;
  size_t spmv_smem = 0;
  int wait_polls = kDefaultWaitPolls;   // budget of each bounded device-side wait (shell_set_wait_budget)
  // mixed precision: a step's first residual and Hessian in one element launch (default; the
  // environment variable BHEM_FUSE_FIRST_HESSIAN=0 at shell creation selects separate launches)
  bool fuse_first_hessian = true;
  // mixed precision: the FP32 element Hessian's contraction on the tensor cores (tcgen05, TF32
  // head-and-tail products; default), or on the FP32 FMA pipe (the environment variable
  // BHEM_ELEMENT=ffma at shell creation)
  bool elem_tc = true;
  // mixed precision, plain SpMV: k_spmv32_sym reads each node row's diagonal and upper blocks and
  // takes its lower blocks as the transposes of the upper blocks of earlier rows (d_tpos), which
  // those rows have just brought into L2, so DRAM sees each off-diagonal pair once (the
  // environment variable BHEM_SPMV_SYM=1 at shell creation); default k_spmv32, which streams both
  // triangles and was faster (60 against 72 us per launch at 256 x 256)
  bool spmv_sym = false;
  // mixed-precision PCG iterations (plain SpMV, update, direction update) launched with
  // programmatic dependent launch, so each kernel's CTAs are scheduled while the previous one
  // finishes (default; the environment variable BHEM_PDL=0 at shell creation: plain launches)
  bool pdl = true;
  // mixed precision: shells of at most this many nodes solve PCG as one thread-block cluster
  // (default 0: never, the graph loop was faster on every workload; BHEM_PCG_LOOP=cluster: always)
  int pcg_cluster_max_nodes = 0;
  // mixed precision, plain SpMV, shells of at most 16,384 nodes: the p-update folded into the next
  // iteration's SpMV (default; the environment variable BHEM_PCG_PUPDATE=1 at shell creation keeps
  // the separate p-update kernel)
  bool pcg_fold_pupdate = true;

  // CUDA graphs of the mixed-precision PCG loop, keyed by mask (iters = -1)
  struct PcgGraph { const unsigned char* mask; int iters; cudaGraphExec_t exec; };
  static constexpr int kGraphSlots = 12;
  PcgGraph pcg_graphs[kGraphSlots] = {};
  int pcg_graph_next = 0;
  cudaStream_t cap_stream = nullptr;
  // the first Newton iteration's Hessian is assembled on aux_stream while the FP64 residual runs
  // on the shell's stream (ev_q: q ready; ev_hess: Hessian assembled)
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_q = nullptr, ev_hess = nullptr;
  // work was enqueued on aux_stream and no error-free check of the shell's stream has joined it
  // since (a step that failed in between): the next step and shell_destroy synchronise it first
  bool aux_unjoined = false;

  // optional phase trace of shell_newton_step (environment BHEM_TRACE_PHASES=1): CUDA events and
  // host times at phase boundaries, printed to stderr at the end of each step
  int trace = 0;
  int trace_n = 0;
  static constexpr int kTraceMax = 256;
  cudaEvent_t trace_ev[kTraceMax] = {};
  const char* trace_name[kTraceMax] = {};
  double trace_host[kTraceMax] = {};
};

// ------------------------------------------------------------------------------------------
// Kernels launchers (element.cu, solver.cu)
// ------------------------------------------------------------------------------------------
// rest per-Gauss-point data, mass, gravity factors (once per shell)
shell_status launch_rest_setup(Shell& s);
// chooses the FP32 SpMV variant (opt.spmv) and prepares its launch (solver.cu)
shell_status setup_spmv(Shell& s);
// dense Cholesky solve of the regularised Newton system into s.d_x (direct.cu)
shell_status run_direct(Shell& s, const unsigned char* mask, const double td[4], const double* rhs, int* not_pd);
void destroy_direct(Shell& s);
// the shared search scratch of the Sec. 5 searches (allocated on first use; rays.cu)
shell_status search_scratch(Shell& s, void** heaps, int** counters, int** redo_list);
// regulariser shift tau * dbar per DOF kind, as kernel argument
struct Shift4 { double v[4]; };

// Heavy element kernel: energy/gradient/Hessian per patch (one warp per patch).
//   hess_out: unassembled [np*2304] of R, or nullptr; bsr: assembled BSR (R) or nullptr.
struct ElemOutputs {
  double* energy_p = nullptr;   // [np]
  double* grad_p = nullptr;     // [np * 48]
  void* hess_p = nullptr;       // [np * 2304]
  void* bsr = nullptr;          // assembled values
  double mass_scale = 0.0;      // adds mass_scale * M to the assembled / unassembled Hessian
  int pseudo = 0;               // drop the second derivative of beta
  // FP32 kernel only: also the FP64 patch energies and the assembled FP64 gradient at q (the
  // results of launch_energy_grad64 without its energy total), in the same launch; grad64 zeroed
  double* energy64 = nullptr;   // [np]
  double* grad64 = nullptr;     // [n_dof]
};
shell_status launch_element_full(Shell& s, const double* q, bool fp64, const ElemOutputs& out);

// Light FP64 kernel: per-patch energy (and assembled gradient) at q + step * dir.
//   mode 0: energy_p[p] = E_p, grad += dE/dq (grad may be null), total -> scal_out
//   mode 1: total of (E_p(q + step dir) - energy_ref[p]) -> scal_out (no gradient)
shell_status launch_energy_grad64(Shell& s, const double* q, const double* dir, double step,
                                  double* energy_p, const double* energy_ref, double* grad,
                                  double* scal_out);

// Solver kernels (solver.cu)
shell_status launch_grad_finish(Shell& s, const double* q, const double* y, double dt,
                                const double grav[3], const unsigned char* mask, double* g,
                                double* gin, double* gnorm2_out);
shell_status launch_mass_mult(Shell& s, const double* x, double* y);
shell_status launch_grad_linear(Shell& s, const double* Md, double alpha, double dt,
                                const unsigned char* mask, double* g, double* gin, double* gnorm2_out);
shell_status launch_dots3(Shell& s, int n, const double* a0, const double* b0, const double* a1,
                          const double* b1, const double* a2, const double* b2, double* out3);
shell_status launch_precond_setup(Shell& s, const unsigned char* mask, const double td[4]);
// PCG start; limit caps the iterations (the mixed-precision kernels stop there on the device)
shell_status launch_pcg_init(Shell& s, const unsigned char* mask, const double* rhs,
                             double rtol, int fixed, int limit, const double td[4]);
shell_status launch_pcg_iteration(Shell& s, const unsigned char* mask, const double td[4]);
// `iters` mixed-precision PCG iterations replayed from a cached CUDA graph (captured on first use
// for this mask and count); the shift comes from the PCG state
// the whole mixed-precision solve as one graph: a conditional WHILE node around one iteration
shell_status launch_pcg_loop_graph(Shell& s, const unsigned char* mask);
shell_status launch_pcg_persistent(Shell& s, const unsigned char* mask);
// kernels per mixed-precision PCG iteration, and whether the p-update rides in the SpMV
bool pcg_folds_pupdate(const Shell& s);
int pcg_kernels_per_iteration(const Shell& s);
// the whole mixed-precision solve as one thread-block cluster (small shells)
shell_status launch_pcg_cluster(Shell& s, const unsigned char* mask);
int pcg_loop_unroll();   // PCG iterations per loop body
shell_status launch_spmv(Shell& s, const void* x, int x_fp32, void* y);
shell_status launch_pcg_result(Shell& s);
shell_status launch_diag_check(Shell& s, const unsigned char* mask, double* out12, bool aux = false);
shell_status launch_fix_diag(Shell& s, const unsigned char* mask, const double floor4[4], int* count);
void drop_pcg_graphs(Shell& s);
shell_status launch_axpy_fixed(Shell& s, double* q, const double* d, double alpha);
shell_status launch_overwrite_fixed(Shell& s, double* dst, const double* src,
                                    const unsigned char* mask, const double* fixed_vals);
shell_status launch_predictor(Shell& s, const double* qn, const double* v, double dt, double* y);
shell_status launch_velocity(Shell& s, const double* q, const double* qn, double dt, double* v);
shell_status launch_negate(Shell& s, const double* a, double* b);

int grid_for(long long work, int per_block);

// ------------------------------------------------------------------------------------------
// Double-float arithmetic on the FP32 pipe (GB300's FP64 pipe is narrow): a value is hi + lo.
// Products of two floats are exact as (p, fma(a, b, -p)); sums use two-sum.
// ------------------------------------------------------------------------------------------
struct F2 { float hi, lo; };

__device__ __forceinline__ F2 f2_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const F2 s = f2_two_sum(a.hi, b.hi);
  const float lo = __fadd_rn(__fadd_rn(s.lo, a.lo), b.lo);
  const float hi = __fadd_rn(s.hi, lo);
  return {hi, __fsub_rn(lo, __fsub_rn(hi, s.hi))};
}
__device__ __forceinline__ F2 f2_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}

// Grid reduction of NV double-float sums, entirely on the FP32 pipe: per-CTA partials are stored
// as (hi, lo) pairs and the last CTA (ticket, no waiting) combines them in a fixed order; only the
// final value is converted to FP64. Same contract as grid_reduce.
__device__ __forceinline__ F2 f2_block_sum(F2 x, F2 (*sred)[32], int i) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    F2 y;
    y.hi = __shfl_xor_sync(0xffffffffu, x.hi, o);
    y.lo = __shfl_xor_sync(0xffffffffu, x.lo, o);
    x = f2_add(x, y);
  }
  if (lane == 0) sred[i][wid] = x;
  __syncthreads();
  F2 s = sred[i][0];
  for (int w = 1; w < nw; ++w) s = f2_add(s, sred[i][w]);
  __syncthreads();
  return s;
}

template <int NV>
__device__ __forceinline__ bool grid_reduce_f2(const F2 (&v)[NV], Reduce red, double* out,
                                               int nblocks) {
  __shared__ F2 sred2[NV][32];
  __shared__ int last2;
  float2* part = reinterpret_cast<float2*>(red.partials);
  for (int i = 0; i < NV; ++i) {
    const F2 s = f2_block_sum(v[i], sred2, i);
    if (threadIdx.x == 0) part[(size_t)i * red.stride + blockIdx.x] = make_float2(s.hi, s.lo);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t = atomicAdd(red.ticket, 1u);
    last2 = (t == (unsigned)nblocks - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!last2) return false;
  __threadfence();
  for (int i = 0; i < NV; ++i) {
    // partials b = tid, tid + bd, ... summed in that order; 4 L2 loads in flight at a time
    F2 s{0.f, 0.f};
    const float2* pi = part + (size_t)i * red.stride;
    const int bd = blockDim.x;
    int b = threadIdx.x;
    for (; b + 3 * bd < nblocks; b += 4 * bd) {
      float2 y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) y[u] = __ldcg(pi + b + u * bd);   // L2: other CTAs' writes
#pragma unroll
      for (int u = 0; u < 4; ++u) s = f2_add(s, F2{y[u].x, y[u].y});
    }
    for (; b < nblocks; b += bd) {
      const float2 y = __ldcg(pi + b);
      s = f2_add(s, F2{y.x, y.y});
    }
    const F2 t = f2_block_sum(s, sred2, i);
    if (threadIdx.x == 0) out[i] = (double)t.hi + (double)t.lo;
  }
  if (threadIdx.x == 0) *red.ticket = 0u;
  __syncthreads();
  return true;
}

// ------------------------------------------------------------------------------------------
// Deterministic grid reduction of NV doubles (every thread of every CTA must call it): the
// per-CTA sums go to red.partials; the last CTA to take a ticket sums them in CTA order into
// out[0..NV) and returns true (in all of its threads). Nothing waits on other CTAs.
// ------------------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ bool grid_reduce(const double (&v)[NV], Reduce red, double* out,
                                            int nblocks, unsigned minmask = 0u) {
  __shared__ double sred[NV][32];
  __shared__ int last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  double x[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const bool mn = (minmask >> i) & 1u;
    x[i] = v[i];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x[i], o);
      x[i] = mn ? fmin(x[i], y) : x[i] + y;
    }
  }
  if (lane == 0)
    for (int i = 0; i < NV; ++i) sred[i][wid] = x[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < NV; ++i) {
      const bool mn = (minmask >> i) & 1u;
      double s = sred[i][0];
      for (int w = 1; w < nw; ++w) s = mn ? fmin(s, sred[i][w]) : s + sred[i][w];
      red.partials[(size_t)i * red.stride + blockIdx.x] = s;
    }
    __threadfence();
    unsigned t = atomicAdd(red.ticket, 1u);
    last = (t == (unsigned)nblocks - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int i = 0; i < NV; ++i) {
    const bool mn = (minmask >> i) & 1u;
    double s = mn ? INFINITY : 0.0;
    // partials b = tid, tid + bd, ... combined in that order; 8 L2 loads in flight at a time
    const double* pi = red.partials + (size_t)i * red.stride;
    const int bd = blockDim.x;
    int b = threadIdx.x;
    for (; b + 7 * bd < nblocks; b += 8 * bd) {
      double y[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) y[u] = __ldcg(pi + b + u * bd);   // L2: other CTAs' writes
#pragma unroll
      for (int u = 0; u < 8; ++u) s = mn ? fmin(s, y[u]) : s + y[u];
    }
    for (; b < nblocks; b += bd) {
      const double y = __ldcg(pi + b);
      s = mn ? fmin(s, y) : s + y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, s, o);
      s = mn ? fmin(s, y) : s + y;
    }
    __syncthreads();
    if (lane == 0) sred[i][wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = sred[i][0];
      for (int w = 1; w < nw; ++w) tot = mn ? fmin(tot, sred[i][w]) : tot + sred[i][w];
      out[i] = tot;
    }
  }
  if (threadIdx.x == 0) *red.ticket = 0u;
  __syncthreads();
  return true;
}

}  // namespace bhem

// The opaque handle of the C ABI.
struct shell_s : public bhem::Shell {};
