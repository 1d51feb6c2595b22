// C ABI of libbhem: shell set-up, element evaluation, assembly, PCG and the implicit-Euler Newton
// step (Sec. 6.1). Host code here only orchestrates; every arithmetic step of the hot path runs
// in the kernels of element.cu and solver.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace bhem {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

shell_status fail(shell_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

template <typename T>
static shell_status dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(SHELL_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return SHELL_OK;
}

static void dfree(void* p) {
  if (p) cudaFree(p);
}

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------------------------------
// Topology of the structured patch grid (Sec. 4.1) with periodic wrap (Sec. 4.2).
// ------------------------------------------------------------------------------------------
struct HostTopo {
  std::vector<int4> pnodes;
  std::vector<int> row_ptr, col, pblocks, diag, color_list, tpos;
  int color_off[10];
};

static void build_topology(const shell_grid& g, int n1, int n2, HostTopo& T) {
  const int np = g.nu * g.nv, n = n1 * n2;
  T.pnodes.resize(np);
  for (int pv = 0; pv < g.nv; ++pv)
    for (int pu = 0; pu < g.nu; ++pu) {
      int i0 = pu % n1, i1 = (pu + 1) % n1, j0 = pv % n2, j1 = (pv + 1) % n2;
      T.pnodes[pv * g.nu + pu] = make_int4(j0 * n1 + i0, j0 * n1 + i1, j1 * n1 + i0, j1 * n1 + i1);
    }
  std::vector<std::vector<int>> nb(n);
  for (int p = 0; p < np; ++p) {
    int nd[4] = {T.pnodes[p].x, T.pnodes[p].y, T.pnodes[p].z, T.pnodes[p].w};
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) nb[nd[a]].push_back(nd[b]);
  }
  T.row_ptr.assign(n + 1, 0);
  T.col.clear();
  for (int i = 0; i < n; ++i) {
    auto& v = nb[i];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    T.row_ptr[i] = (int)T.col.size();
    T.col.insert(T.col.end(), v.begin(), v.end());
  }
  T.row_ptr[n] = (int)T.col.size();
  auto find = [&](int r, int c) {
    auto b = T.col.begin() + T.row_ptr[r], e = T.col.begin() + T.row_ptr[r + 1];
    return (int)(std::lower_bound(b, e, c) - T.col.begin());
  };
  T.pblocks.resize((size_t)np * 16);
  for (int p = 0; p < np; ++p) {
    int nd[4] = {T.pnodes[p].x, T.pnodes[p].y, T.pnodes[p].z, T.pnodes[p].w};
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) T.pblocks[(size_t)p * 16 + a * 4 + b] = find(nd[a], nd[b]);
  }
  T.diag.resize(n);
  for (int i = 0; i < n; ++i) T.diag[i] = find(i, i);
  // transposed lower blocks: for node row i, slot u < (diag - row start) holds the index of block
  // (col[row start + u], i), the transpose of the row's u-th block left of the diagonal (a row
  // has at most 8 such blocks); 8 slots per row, so a kernel reads them with the row index alone
  T.tpos.assign((size_t)n * 8, 0);
  for (int i = 0; i < n; ++i)
    for (int k = T.row_ptr[i]; k < T.diag[i]; ++k) T.tpos[(size_t)i * 8 + (k - T.row_ptr[i])] = find(T.col[k], i);
  // colours: patches of one colour share no node (patch_colour)
  std::vector<int> cnt(10, 0);
  std::vector<int> colr(np);
  for (int p = 0; p < np; ++p) {
    colr[p] = patch_colour(g, p % g.nu, p / g.nu);
    cnt[colr[p] + 1]++;
  }
  for (int c = 0; c < 9; ++c) cnt[c + 1] += cnt[c];
  for (int c = 0; c < 10; ++c) T.color_off[c] = cnt[c];
  T.color_list.assign(np, 0);
  std::vector<int> pos(cnt.begin(), cnt.begin() + 9);
  for (int p = 0; p < np; ++p) T.color_list[pos[colr[p]]++] = p;
}

static void destroy_shell(shell_s* s) {
  if (!s) return;
  for (int i = 0; i < Shell::kTraceMax; ++i)
    if (s->trace_ev[i]) cudaEventDestroy(s->trace_ev[i]);
  for (auto& gph : s->pcg_graphs)
    if (gph.exec) cudaGraphExecDestroy(gph.exec);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->aux_stream) cudaStreamDestroy(s->aux_stream);
  if (s->ev_q) cudaEventDestroy(s->ev_q);
  if (s->ev_hess) cudaEventDestroy(s->ev_hess);
  destroy_direct(*s);
  void* ptrs[] = {s->d_patch_nodes, s->d_patch_blocks, s->d_row_ptr, s->d_col, s->d_diag_block, s->d_tpos,
                  s->d_color_list, s->d_rest, s->d_restgp, s->d_mass, s->d_fgrav, s->d_val,
                  s->d_x, s->d_r, s->d_z, s->d_p, s->d_Ap, s->d_p32, s->d_x32, s->d_r32, s->d_z32, s->d_Ap32, s->d_Dinv, s->d_phi64, s->d_phi32,
                  s->d_pcg, s->d_qn, s->d_y, s->d_g, s->d_gin, s->d_d, s->d_Md, s->d_Ep,
                  s->d_qwork, s->d_vwork, s->d_qfix, s->d_warm, s->d_mask, s->d_ns, s->d_err, s->d_qmy,
                  s->d_energy_tmp, s->red.partials, s->red.ticket, s->red_aux.partials, s->red_aux.ticket, s->d_rhs, s->d_g2, s->d_Ep2,
                  s->d_search, s->d_ray_nets, s->d_ccd_nets, s->d_persist};
  for (void* p : ptrs) dfree(p);
  if (s->h_ns) cudaFreeHost(s->h_ns);
  if (s->h_pcg) cudaFreeHost(s->h_pcg);
  if (s->h_err) cudaFreeHost(s->h_err);
  delete[] s->h_color_patches;
  delete s;
}

// Phase trace (BHEM_TRACE_PHASES=1): one CUDA event and one host time per mark.
static void mark(Shell& s, const char* name) {
  if (!s.trace || s.trace_n >= Shell::kTraceMax) return;
  const int i = s.trace_n++;
  if (!s.trace_ev[i]) cudaEventCreate(&s.trace_ev[i]);
  cudaEventRecord(s.trace_ev[i], s.stream);
  s.trace_name[i] = name;
  s.trace_host[i] = std::chrono::duration<double, std::micro>(
                        std::chrono::steady_clock::now().time_since_epoch()).count();
}

static void trace_report(Shell& s) {
  if (!s.trace || s.trace_n < 2) { s.trace_n = 0; return; }
  cudaEventSynchronize(s.trace_ev[s.trace_n - 1]);
  std::fprintf(stderr, "[bhem trace] %d marks\n", s.trace_n);
  for (int i = 1; i < s.trace_n; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s.trace_ev[i - 1], s.trace_ev[i]);
    std::fprintf(stderr, "[bhem trace] %-22s device %9.1f us  host %9.1f us\n", s.trace_name[i], ms * 1e3,
                 s.trace_host[i] - s.trace_host[i - 1]);
  }
  s.trace_n = 0;
}

static shell_status sync_and_check(Shell& s) {
  BHEM_CUDA(cudaMemcpyAsync(s.h_err, s.d_err, sizeof(int), cudaMemcpyDeviceToHost, s.stream));
  BHEM_CUDA(cudaStreamSynchronize(s.stream));
  const int bits = *s.h_err;
  if (bits) {
    BHEM_CUDA(cudaMemsetAsync(s.d_err, 0, sizeof(int), s.stream));
    BHEM_CUDA(cudaStreamSynchronize(s.stream));
  }
  if (bits & ERRBIT_DEGENERATE) return fail(SHELL_ERR_DEGENERATE, "degenerate surface normal at a Gauss point");
  if (bits & ERRBIT_NONFINITE) return fail(SHELL_ERR_NONFINITE, "non-finite energy or residual");
  if (bits & ERRBIT_TIMEOUT)
    return fail(SHELL_ERR_TIMEOUT, "a bounded device-side wait expired (bulk copy, grid barrier or tensor-core MMA)");
  return SHELL_OK;
}

}  // namespace bhem

using namespace bhem;

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" const char* shell_last_error(void) { return g_last_error.c_str(); }

extern "C" shell_status shell_create(const shell_grid* grid, const shell_material* material,
                                     const double* rest_dofs, const shell_options* options,
                                     void* stream, shell_t** out) {
  if (!grid || !material || !rest_dofs || !out) return fail(SHELL_ERR_ARG, "NULL argument");
  *out = nullptr;
  const shell_grid& g = *grid;
  if (g.nu < 1 || g.nv < 1 || (g.periodic_u && g.nu < 2) || (g.periodic_v && g.nv < 2))
    return fail(SHELL_ERR_ARG, "grid needs nu, nv >= 1 (>= 2 along a periodic direction)");
  if (!(g.dxi1 > 0) || !(g.dxi2 > 0)) return fail(SHELL_ERR_ARG, "dxi1, dxi2 must be > 0");
  if (!(material->thickness > 0) || !(material->young > 0) || !(material->density >= 0) ||
      !(material->poisson > -1.0 && material->poisson < 1.0))
    return fail(SHELL_ERR_ARG, "invalid material");
  shell_options opt{SHELL_PREC_MIXED, SHELL_HESS_EXACT, SHELL_ASM_ATOMIC, 0, SHELL_SOLVER_PCG};
  if (options) opt = *options;
  if ((opt.precision != SHELL_PREC_FP64 && opt.precision != SHELL_PREC_MIXED) ||
      (opt.hessian != SHELL_HESS_EXACT && opt.hessian != SHELL_HESS_PSEUDO) ||
      (opt.assembly != SHELL_ASM_ATOMIC && opt.assembly != SHELL_ASM_COLOR) ||
      (opt.spmv != SHELL_SPMV_AUTO && opt.spmv != SHELL_SPMV_PLAIN && opt.spmv != SHELL_SPMV_TMA) ||
      (opt.solver != SHELL_SOLVER_PCG && opt.solver != SHELL_SOLVER_DIRECT))
    return fail(SHELL_ERR_ARG, "invalid options");
  long long np_ll = (long long)g.nu * g.nv;
  if (np_ll > (1LL << 26)) return fail(SHELL_ERR_ARG, "grid too large");

  shell_s* s = new shell_s();
  s->grid = g;
  s->mat = *material;
  s->opt = opt;
  s->stream = (cudaStream_t)stream;
  cudaGetDevice(&s->device);
  s->n1 = g.periodic_u ? g.nu : g.nu + 1;
  s->n2 = g.periodic_v ? g.nv : g.nv + 1;
  s->n_nodes = s->n1 * s->n2;
  s->n_patches = (int)np_ll;
  s->n_dof = 12 * s->n_nodes;
  s->lam = material->young * material->poisson / (1.0 - material->poisson * material->poisson);
  s->mu = material->young / (2.0 * (1.0 + material->poisson));
  s->val_fp64 = opt.precision == SHELL_PREC_FP64;
  s->pcg_host_loop = getenv("BHEM_PCG_HOST_LOOP") != nullptr;
  {
    const char* m = getenv("BHEM_PCG_LOOP");
    s->pcg_mode = s->pcg_host_loop ? 2 : 1;
    if (m && std::strcmp(m, "persistent") == 0) s->pcg_mode = 0;
    if (m && std::strcmp(m, "host") == 0) s->pcg_mode = 2;
    if (m && std::strcmp(m, "graph") == 0) s->pcg_cluster_max_nodes = 0;
    if (m && std::strcmp(m, "cluster") == 0) s->pcg_cluster_max_nodes = 1 << 30;
    s->pcg_host_loop = s->pcg_mode == 2;
    const char* pu = getenv("BHEM_PCG_PUPDATE");
    s->pcg_fold_pupdate = !(pu && std::strcmp(pu, "1") == 0);
    const char* f = getenv("BHEM_FUSE_FIRST_HESSIAN");
    s->fuse_first_hessian = !(f && std::strcmp(f, "0") == 0);
    const char* el = getenv("BHEM_ELEMENT");
    s->elem_tc = !(el && std::strcmp(el, "ffma") == 0);
    const char* sy = getenv("BHEM_SPMV_SYM");
    s->spmv_sym = sy && std::strcmp(sy, "1") == 0;
    const char* pd = getenv("BHEM_PDL");
    s->pdl = !(pd && std::strcmp(pd, "0") == 0);
  }

  HostTopo T;
  build_topology(g, s->n1, s->n2, T);
  s->n_blocks = (int)T.col.size();
  for (int i = 0; i < s->n1 * s->n2; ++i) s->max_row = std::max(s->max_row, T.row_ptr[i + 1] - T.row_ptr[i]);
  s->h_color_patches = new int[10];
  std::memcpy(s->h_color_patches, T.color_off, sizeof(int) * 10);

  const int n = s->n_nodes, np = s->n_patches, nb = s->n_blocks, m = s->n_dof;
  shell_status st = SHELL_OK;
#define A(ptr, count) \
  if (st == SHELL_OK) st = dalloc(&(ptr), (size_t)(count))
  A(s->d_patch_nodes, np);
  A(s->d_patch_blocks, (size_t)np * 16);
  A(s->d_row_ptr, n + 1);
  A(s->d_col, nb);
  A(s->d_diag_block, n);
  if (s->spmv_sym) A(s->d_tpos, (size_t)n * 8);   // read by the opt-in symmetric SpMV only
  A(s->d_color_list, np);
  A(s->d_rest, m);
  A(s->d_restgp, (size_t)13 * np * 16);
  A(s->d_mass, (size_t)nb * 16);
  A(s->d_fgrav, (size_t)n * 4);
  if (st == SHELL_OK) {
    if (s->val_fp64) {
      double* v = nullptr;
      st = dalloc(&v, (size_t)nb * 144);
      s->d_val = v;
      double* d = nullptr;
      if (st == SHELL_OK) st = dalloc(&d, (size_t)n * 144);
      s->d_Dinv = d;
    } else {
      float* v = nullptr;
      st = dalloc(&v, (size_t)nb * 144);
      s->d_val = v;
      float* d = nullptr;
      if (st == SHELL_OK) st = dalloc(&d, (size_t)n * 144);
      s->d_Dinv = d;
    }
  }
  A(s->d_x, m); A(s->d_r, m); A(s->d_z, m); A(s->d_p, m); A(s->d_Ap, m);
  A(s->d_pcg, 1); A(s->d_p32, m); A(s->d_x32, m); A(s->d_r32, m); A(s->d_z32, m); A(s->d_Ap32, m);
  A(s->d_phi64, 1568); A(s->d_phi32, 1568);
  A(s->d_qn, m); A(s->d_y, m); A(s->d_g, m); A(s->d_gin, m); A(s->d_d, m); A(s->d_Md, m);
  A(s->d_rhs, m); A(s->d_Ep, np); A(s->d_qwork, m); A(s->d_vwork, m); A(s->d_qfix, m); A(s->d_qmy, m);
  A(s->d_warm, m); A(s->d_mask, m); A(s->d_ns, 1); A(s->d_err, 1); A(s->d_energy_tmp, 1);
  A(s->d_g2, m); A(s->d_Ep2, np);
  // partials: one per CTA of the largest reducing launch (8 patches, 4 FP64 block rows, 16 nodes or
  // 1024 vector CTAs per CTA) per reduced value
  s->red.stride = std::max(1024, std::max(np / 8, n / 4) + 64);
  A(s->red.partials, (size_t)kMaxRed * s->red.stride);
  A(s->red.ticket, 1);
  s->red_aux.stride = 1024;
  A(s->red_aux.partials, (size_t)kMaxRed * s->red_aux.stride);
  A(s->red_aux.ticket, 1);
#undef A
  if (st == SHELL_OK) {
    cudaError_t e1 = cudaMallocHost((void**)&s->h_ns, sizeof(NewtonScalars));
    cudaError_t e2 = cudaMallocHost((void**)&s->h_pcg, sizeof(PcgState));
    cudaError_t e3 = cudaMallocHost((void**)&s->h_err, sizeof(int));
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) st = fail(SHELL_ERR_OOM, "cudaMallocHost failed");
  }
  if (st != SHELL_OK) {
    destroy_shell(s);
    return st;
  }
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream);
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = up(s->d_patch_nodes, T.pnodes.data(), sizeof(int4) * np);
  if (e == cudaSuccess) e = up(s->d_patch_blocks, T.pblocks.data(), sizeof(int) * T.pblocks.size());
  if (e == cudaSuccess) e = up(s->d_row_ptr, T.row_ptr.data(), sizeof(int) * (n + 1));
  if (e == cudaSuccess) e = up(s->d_col, T.col.data(), sizeof(int) * nb);
  if (e == cudaSuccess) e = up(s->d_diag_block, T.diag.data(), sizeof(int) * n);
  if (e == cudaSuccess && s->d_tpos) e = up(s->d_tpos, T.tpos.data(), sizeof(int) * T.tpos.size());
  if (e == cudaSuccess) e = up(s->d_color_list, T.color_list.data(), sizeof(int) * np);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_rest, rest_dofs, sizeof(double) * m, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->red.ticket, 0, sizeof(unsigned), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->red_aux.ticket, 0, sizeof(unsigned), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_pcg, 0, sizeof(PcgState), s->stream);
  if (e != cudaSuccess) {
    destroy_shell(s);
    return fail(SHELL_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
  }
  {
    const char* tv = std::getenv("BHEM_TRACE_PHASES");
    s->trace = (tv && tv[0] == '1') ? 1 : 0;
  }
  st = setup_spmv(*s);
  if (st == SHELL_OK) st = launch_rest_setup(*s);
  if (st == SHELL_OK) st = sync_and_check(*s);
  if (st != SHELL_OK) {
    destroy_shell(s);
    return st;
  }
  *out = s;
  return SHELL_OK;
}

extern "C" shell_status shell_destroy(shell_t* shell) {
  if (!shell) return SHELL_OK;
  cudaStreamSynchronize(shell->stream);
  if (shell->aux_unjoined) cudaStreamSynchronize(shell->aux_stream);
  destroy_shell(shell);
  return SHELL_OK;
}

extern "C" shell_status shell_info(const shell_t* shell, shell_info_t* info) {
  if (!shell || !info) return fail(SHELL_ERR_ARG, "NULL argument");
  info->n_nodes = shell->n_nodes;
  info->n_patches = shell->n_patches;
  info->n_blocks = shell->n_blocks;
  info->n_dof = shell->n_dof;
  return SHELL_OK;
}

extern "C" shell_status shell_set_wait_budget(shell_t* shell, int polls) {
  if (!shell) return fail(SHELL_ERR_ARG, "NULL argument");
  cudaStreamSynchronize(shell->stream);   // no launch in flight uses the graphs dropped below
  shell->wait_polls = polls < 0 ? kDefaultWaitPolls : polls;
  drop_pcg_graphs(*shell);   // captured launches hold the previous budget
  return SHELL_OK;
}

extern "C" shell_status shell_grid_colours(const shell_grid* grid, int* colour) {
  if (!grid || !colour) return fail(SHELL_ERR_ARG, "NULL argument");
  if (grid->nu < 1 || grid->nv < 1) return fail(SHELL_ERR_ARG, "empty grid");
  for (int pv = 0; pv < grid->nv; ++pv)
    for (int pu = 0; pu < grid->nu; ++pu) colour[pv * grid->nu + pu] = patch_colour(*grid, pu, pv);
  return SHELL_OK;
}

extern "C" shell_status shell_element_egh(shell_t* shell, const double* q, int precision,
                                          double* energy_p, double* grad_p, void* hess_p) {
  if (!shell || !q) return fail(SHELL_ERR_ARG, "NULL argument");
  if (precision != SHELL_PREC_FP64 && precision != SHELL_PREC_MIXED) return fail(SHELL_ERR_ARG, "precision");
  ElemOutputs o;
  o.energy_p = energy_p;
  o.grad_p = grad_p;
  o.hess_p = hess_p;
  o.pseudo = shell->opt.hessian == SHELL_HESS_PSEUDO;
  return launch_element_full(*shell, q, precision == SHELL_PREC_FP64, o);
}

namespace bhem {
static shell_status assemble_hessian(Shell& s, const double* q, double mass_scale) {
  size_t bytes = (size_t)s.n_blocks * 144 * (s.val_fp64 ? sizeof(double) : sizeof(float));
  BHEM_CUDA(cudaMemsetAsync(s.d_val, 0, bytes, s.stream));
  ElemOutputs o;
  o.bsr = s.d_val;
  o.mass_scale = mass_scale;
  o.pseudo = s.opt.hessian == SHELL_HESS_PSEUDO;
  return launch_element_full(s, q, s.val_fp64 != 0, o);
}

static shell_status elastic_energy_grad(Shell& s, const double* q, double* energy, double* grad) {
  if (grad) BHEM_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * s.n_dof, s.stream));
  return launch_energy_grad64(s, q, nullptr, 0.0, s.d_Ep, nullptr, grad, energy ? energy : s.d_energy_tmp);
}
}  // namespace bhem

extern "C" shell_status shell_energy_grad_hess(shell_t* shell, const double* q, double mass_scale,
                                               double* energy, double* grad, int want_hessian) {
  if (!shell || !q) return fail(SHELL_ERR_ARG, "NULL argument");
  if (energy || grad) BHEM_TRY(elastic_energy_grad(*shell, q, energy, grad));
  if (want_hessian) BHEM_TRY(assemble_hessian(*shell, q, mass_scale));
  return SHELL_OK;
}

extern "C" shell_status shell_get_bsr(shell_t* shell, const int** row_ptr, const int** col,
                                      const void** val, int* val_is_fp64) {
  if (!shell) return fail(SHELL_ERR_ARG, "NULL argument");
  if (row_ptr) *row_ptr = shell->d_row_ptr;
  if (col) *col = shell->d_col;
  if (val) *val = shell->d_val;
  if (val_is_fp64) *val_is_fp64 = shell->val_fp64;
  return SHELL_OK;
}

extern "C" shell_status shell_get_mass(shell_t* shell, const double** mass_blocks,
                                       const double** gravity_factors) {
  if (!shell) return fail(SHELL_ERR_ARG, "NULL argument");
  if (mass_blocks) *mass_blocks = shell->d_mass;
  if (gravity_factors) *gravity_factors = shell->d_fgrav;
  return SHELL_OK;
}

namespace bhem {
// Runs the PCG kernels on the assembled matrix; the solution is left in s.d_x.
static shell_status run_pcg(Shell& s, const unsigned char* mask, const double td[4],
                            const double* rhs, double rtol, int max_iter, int fixed, int* iters,
                            int* neg) {
  const int limit = fixed > 0 ? fixed : max_iter;
  BHEM_TRY(launch_precond_setup(s, mask, td));
  BHEM_TRY(launch_pcg_init(s, mask, rhs, rtol, fixed, limit, td));
  mark(s, "pcg_setup_enqueued");
  int launched = 0, chunk = 4;
  *s.h_pcg = PcgState{};
  if (!s.val_fp64 && s.pcg_mode == 0) {
    // mixed precision, BHEM_PCG_LOOP=persistent: the whole solve is one persistent cooperative
    // launch (measured slower than the graph loop below on every workload of the bench)
    if (limit > 0) BHEM_TRY(launch_pcg_persistent(s, mask));
    BHEM_CUDA(cudaMemcpyAsync(s.h_pcg, s.d_pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, s.stream));
    BHEM_CUDA(cudaStreamSynchronize(s.stream));
    mark(s, "pcg_persistent");
    launched = limit;
  } else if (!s.val_fp64 && s.pcg_mode == 1 && s.n_nodes <= s.pcg_cluster_max_nodes) {
    // mixed precision, small shell: the whole solve in one thread-block cluster
    if (limit > 0) BHEM_TRY(launch_pcg_cluster(s, mask));
    BHEM_CUDA(cudaMemcpyAsync(s.h_pcg, s.d_pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, s.stream));
    BHEM_CUDA(cudaStreamSynchronize(s.stream));
    mark(s, "pcg_cluster");
    launched = limit;
  } else if (!s.val_fp64 && s.pcg_mode == 1) {
    // mixed precision: the whole solve loops on the device (one graph with a conditional WHILE
    // node around a few iterations; the kernels stop it, at the latest after `limit` iterations)
    if (limit > 0) BHEM_TRY(launch_pcg_loop_graph(s, mask));
    BHEM_CUDA(cudaMemcpyAsync(s.h_pcg, s.d_pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, s.stream));
    BHEM_CUDA(cudaStreamSynchronize(s.stream));
    // per body: the PCG kernels of each iteration (2 with the folded p-update, else 3) and the loop condition
    s.launches += ((long long)pcg_kernels_per_iteration(s) * pcg_loop_unroll() + 1) * s.h_pcg->bodies;
    mark(s, "pcg_loop");
    launched = limit;
  } else {
    BHEM_CUDA(cudaMemcpyAsync(s.h_pcg, s.d_pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, s.stream));
    BHEM_CUDA(cudaStreamSynchronize(s.stream));
    mark(s, "pcg_setup_synced");
  }
  while (launched < limit && !s.h_pcg->done) {   // FP64 (or BHEM_PCG_HOST_LOOP): host chunks
    const int c = std::min(chunk, limit - launched);
    for (int k = 0; k < c; ++k) BHEM_TRY(launch_pcg_iteration(s, mask, td));
    launched += c;
    BHEM_CUDA(cudaMemcpyAsync(s.h_pcg, s.d_pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, s.stream));
    BHEM_CUDA(cudaStreamSynchronize(s.stream));
    mark(s, "pcg_chunk");
    chunk = std::min(chunk * 2, 64);
  }
  *iters = s.h_pcg->iters;
  *neg = s.h_pcg->negcurv;
  BHEM_TRY(sync_and_check(s));
  mark(s, "pcg_checked");
  return launch_pcg_result(s);
}
}  // namespace bhem

namespace bhem {
// Per-kind regulariser scale dbar[k] = mean |A_ii| over free DOFs of kind k (1 if none) and the
// per-kind minimum of A_ii, from the assembled matrix.
struct KindStats { double dbar[4], dmin[4], count[4]; };
static void kind_stats_from_host(const Shell& s, KindStats& K) {
  for (int q = 0; q < 4; ++q) {
    K.count[q] = s.h_ns->diag_stats[3 * q + 1];
    K.dbar[q] = K.count[q] > 0 ? s.h_ns->diag_stats[3 * q] / K.count[q] : 1.0;
    K.dmin[q] = s.h_ns->diag_stats[3 * q + 2];
  }
}

static shell_status kind_stats(Shell& s, const unsigned char* mask, KindStats& K) {
  BHEM_TRY(launch_diag_check(s, mask, s.d_ns->diag_stats));
  BHEM_CUDA(cudaMemcpyAsync(s.h_ns, s.d_ns, sizeof(NewtonScalars), cudaMemcpyDeviceToHost, s.stream));
  BHEM_CUDA(cudaStreamSynchronize(s.stream));
  kind_stats_from_host(s, K);
  return SHELL_OK;
}
// Sec. 6.1 diagonal regulariser, local part: when some free diagonal entry is <= 0, each such
// entry A_ii of kind k becomes max(-A_ii, 1e-8 D_k) (in place, counted in d_ns->diag_fixes).
static shell_status fix_diagonal(Shell& s, const unsigned char* mask, const KindStats& K) {
  bool any = false;
  for (int q = 0; q < 4; ++q) any = any || (K.count[q] > 0 && K.dmin[q] <= 0.0);
  if (!any) return SHELL_OK;
  const double floor4[4] = {1e-8 * K.dbar[0], 1e-8 * K.dbar[1], 1e-8 * K.dbar[2], 1e-8 * K.dbar[3]};
  return launch_fix_diag(s, mask, floor4, &s.d_ns->diag_fixes);
}
}  // namespace bhem

extern "C" shell_status shell_pcg_solve(shell_t* shell, const unsigned char* fixed_mask, double tau,
                                        const double* rhs, double* x, double rtol, int max_iter,
                                        int fixed_iters, int* iters, int* neg_curv) {
  if (!shell || !rhs || !x) return fail(SHELL_ERR_ARG, "NULL argument");
  if (max_iter < 0 || fixed_iters < 0 || !(tau >= 0.0)) return fail(SHELL_ERR_ARG, "invalid PCG limits");
  int it = 0, neg = 0;
  KindStats K;
  BHEM_TRY(kind_stats(*shell, fixed_mask, K));
  const double td[4] = {tau * K.dbar[0], tau * K.dbar[1], tau * K.dbar[2], tau * K.dbar[3]};
  BHEM_TRY(run_pcg(*shell, fixed_mask, td, rhs, rtol, max_iter, fixed_iters, &it, &neg));
  BHEM_CUDA(cudaMemcpyAsync(x, shell->d_x, sizeof(double) * shell->n_dof, cudaMemcpyDeviceToDevice, shell->stream));
  BHEM_TRY(sync_and_check(*shell));
  if (iters) *iters = it;
  if (neg_curv) *neg_curv = neg;
  return SHELL_OK;
}

namespace bhem {
// |g| at q; leaves g in s.d_g, the inertial part in s.d_gin and E_p(q) in s.d_Ep.
// also_wait: an event of work running beside the residual (the first Hessian), joined before the
// error check so that one check sees the error bits of both
static shell_status residual(Shell& s, const double* q, const shell_step_params& P,
                             const unsigned char* mask, double* gnorm, cudaEvent_t also_wait = nullptr) {
  BHEM_CUDA(cudaMemsetAsync(s.d_g, 0, sizeof(double) * s.n_dof, s.stream));
  BHEM_TRY(launch_energy_grad64(s, q, nullptr, 0.0, s.d_Ep, nullptr, s.d_g, &s.d_ns->energy));
  BHEM_TRY(launch_grad_finish(s, q, s.d_y, P.dt, P.gravity, mask, s.d_g, s.d_gin, &s.d_ns->gnorm2));
  if (also_wait) BHEM_CUDA(cudaStreamWaitEvent(s.stream, also_wait, 0));
  BHEM_CUDA(cudaMemcpyAsync(s.h_ns, s.d_ns, sizeof(NewtonScalars), cudaMemcpyDeviceToHost, s.stream));
  BHEM_TRY(sync_and_check(s));
  *gnorm = std::sqrt(s.h_ns->gnorm2);
  return SHELL_OK;
}

// |g| at q together with the first Hessian at q (mixed precision) in one element launch: the warps
// of the FP32 Hessian also evaluate the FP64 patch energies and the FP64 elastic gradient, so the
// FP64 pipe works under the FP32 pass instead of after it. The Hessian's diagonal statistics ride
// on the residual's host copy of the Newton scalars. (The total elastic energy, unused by the step,
// is not formed on this path.)
static shell_status residual_with_hessian(Shell& s, const double* q, const shell_step_params& P,
                                          const unsigned char* mask, double inv_dt2, double* gnorm) {
  BHEM_CUDA(cudaMemsetAsync(s.d_g, 0, sizeof(double) * s.n_dof, s.stream));
  BHEM_CUDA(cudaMemsetAsync(s.d_val, 0, (size_t)s.n_blocks * 144 * sizeof(float), s.stream));
  ElemOutputs o;
  o.bsr = s.d_val;
  o.mass_scale = inv_dt2;
  o.pseudo = s.opt.hessian == SHELL_HESS_PSEUDO;
  o.energy64 = s.d_Ep;
  o.grad64 = s.d_g;
  BHEM_TRY(launch_element_full(s, q, false, o));
  BHEM_TRY(launch_diag_check(s, mask, s.d_ns->diag_stats, true));
  BHEM_TRY(launch_grad_finish(s, q, s.d_y, P.dt, P.gravity, mask, s.d_g, s.d_gin, &s.d_ns->gnorm2));
  BHEM_CUDA(cudaMemcpyAsync(s.h_ns, s.d_ns, sizeof(NewtonScalars), cudaMemcpyDeviceToHost, s.stream));
  BHEM_TRY(sync_and_check(s));
  *gnorm = std::sqrt(s.h_ns->gnorm2);
  return SHELL_OK;
}

// Residual at q = q_prev + d when the elastic gradient and patch energies at q are already in
// d_g / d_Ep (from the accepted first line-search trial, alpha = 1): the inertial part follows from
// the previous one and M d (d_Md, formed for the line search), without a second mass product.
static shell_status residual_reuse(Shell& s, const shell_step_params& P, const unsigned char* mask,
                                   double* gnorm) {
  BHEM_TRY(launch_grad_linear(s, s.d_Md, 1.0, P.dt, mask, s.d_g, s.d_gin, &s.d_ns->gnorm2));
  BHEM_CUDA(cudaMemcpyAsync(s.h_ns, s.d_ns, sizeof(NewtonScalars), cudaMemcpyDeviceToHost, s.stream));
  BHEM_TRY(sync_and_check(s));
  *gnorm = std::sqrt(s.h_ns->gnorm2);
  return SHELL_OK;
}

static shell_status newton_core(Shell& s, const shell_step_params& P, const unsigned char* mask,
                                const double* qfix, double* q, const double* v_in,
                                const double* warm, double* v_out, shell_step_stats& st) {
  const int m = s.n_dof;
  if (s.aux_unjoined) {   // the previous step failed while its first Hessian was in flight
    BHEM_CUDA(cudaStreamSynchronize(s.aux_stream));
    s.aux_unjoined = false;
  }
  s.trace_n = 0;
  mark(s, "start");
  BHEM_CUDA(cudaMemcpyAsync(s.d_qn, q, sizeof(double) * m, cudaMemcpyDeviceToDevice, s.stream));
  BHEM_TRY(launch_predictor(s, s.d_qn, v_in, P.dt, s.d_y));
  if (mask) BHEM_TRY(launch_overwrite_fixed(s, q, s.d_qn, mask, qfix));
  double gref = 0.0, gn = 0.0, tau_carry = P.tau_carry;
  const double inv_dt2 = 1.0 / (P.dt * P.dt);
  BHEM_CUDA(cudaMemsetAsync(&s.d_ns->diag_fixes, 0, sizeof(int), s.stream));
  // The first iteration's Hessian at q does not depend on the residual: it is assembled on the
  // auxiliary stream, enqueued before the FP64 residual, so that the residual's CTAs take over the
  // SMs as the element kernel's retire (7.83 against 7.85 ms per Newton iteration on the 256^2
  // sheet; capping the element grid to make room for them side by side was slower, 8.2 ms).
  // The shell's stream joins it before the residual's error check, so the step continues only
  // when both are complete and error-free; a step that is converged at q leaves it unused.
  // Only for large shells: on small ones every kernel is short, the step is launch- and sync-bound,
  // and the second stream's fixed costs outweigh the overlap (30 x 30 patches: 3% slower).
  constexpr int kOverlapMinPatches = 16384;
  bool hess_pending = false, hess_ready = false;
  if (!warm && P.newton_max > 0 && !s.val_fp64 && s.fuse_first_hessian) {
    // mixed precision: residual and first Hessian in one element launch (residual_with_hessian)
    BHEM_TRY(residual_with_hessian(s, q, P, mask, inv_dt2, &gref));
    hess_ready = true;
  } else if (!warm && P.newton_max > 0 && s.n_patches >= kOverlapMinPatches) {
    if (!s.aux_stream) {
      BHEM_CUDA(cudaStreamCreateWithFlags(&s.aux_stream, cudaStreamNonBlocking));
      BHEM_CUDA(cudaEventCreateWithFlags(&s.ev_q, cudaEventDisableTiming));
      BHEM_CUDA(cudaEventCreateWithFlags(&s.ev_hess, cudaEventDisableTiming));
    }
    BHEM_CUDA(cudaEventRecord(s.ev_q, s.stream));
    BHEM_CUDA(cudaStreamWaitEvent(s.aux_stream, s.ev_q, 0));
    s.aux_unjoined = true;
    cudaStream_t keep = s.stream;
    s.stream = s.aux_stream;
    shell_status sa = assemble_hessian(s, q, inv_dt2);
    // its diagonal statistics too: the residual's host copy of the Newton scalars carries them
    if (sa == SHELL_OK) sa = launch_diag_check(s, mask, s.d_ns->diag_stats, true);
    s.stream = keep;
    BHEM_TRY(sa);
    BHEM_CUDA(cudaEventRecord(s.ev_hess, s.aux_stream));
    hess_pending = true;
  }
  if (!hess_ready) BHEM_TRY(residual(s, q, P, mask, &gref, hess_pending ? s.ev_hess : nullptr));
  s.aux_unjoined = false;   // the residual's synchronised check waited for ev_hess
  mark(s, "residual0");
  st.res0 = gref;
  if (warm) BHEM_TRY(launch_overwrite_fixed(s, q, warm, mask, qfix));
  shell_status status = SHELL_OK;
  // The first line-search trial (alpha = 1) also computes the elastic gradient and patch energies
  // at q + d; when it is accepted, q + d is the next iterate (the same FP64 sum), so the next
  // residual reuses them instead of evaluating the elements again.
  bool reuse = false;
  for (int it = 0;; ++it) {
    if (reuse) BHEM_TRY(residual_reuse(s, P, mask, &gn));
    else if (it > 0 || warm) BHEM_TRY(residual(s, q, P, mask, &gn));
    else gn = gref;
    mark(s, "residual");
    reuse = false;
    if (gn <= P.newton_rtol * gref) break;
    if (it >= P.newton_max) { status = SHELL_ERR_NOT_CONVERGED; break; }
    // Sec. 6.1 diagonal regulariser: the non-positive free diagonal entries fixed in place, then
    // A + tau D (D = per-kind mean |A_ii| before the fix) with tau from a tenth of the previous
    // iteration's tau; each negative curvature met by PCG multiplies tau by 10 (at least 1e-8),
    // beyond 1e4 the step gives up.
    KindStats K;
    const bool from_pending = hess_pending || hess_ready;
    if (hess_pending) {   // assembled and its statistics read with the residual (joined there)
      BHEM_CUDA(cudaStreamWaitEvent(s.stream, s.ev_hess, 0));
      hess_pending = false;
    } else if (hess_ready) {   // assembled in the residual's launch
      hess_ready = false;
    } else {
      BHEM_TRY(assemble_hessian(s, q, inv_dt2));
    }
    mark(s, "assemble_enqueued");
    BHEM_TRY(launch_negate(s, s.d_g, s.d_rhs));
    if (from_pending) kind_stats_from_host(s, K);
    else BHEM_TRY(kind_stats(s, mask, K));
    mark(s, "kind_stats");
    BHEM_TRY(fix_diagonal(s, mask, K));
    double tau = tau_carry / 10.0;
    if (tau < 1e-8) tau = 0.0;
    for (;;) {
      if (tau > 1e4) { status = SHELL_ERR_INDEFINITE; break; }
      int pit = 0, neg = 0;
      const double td[4] = {tau * K.dbar[0], tau * K.dbar[1], tau * K.dbar[2], tau * K.dbar[3]};
      if (s.opt.solver == SHELL_SOLVER_DIRECT)
        BHEM_TRY(run_direct(s, mask, td, s.d_rhs, &neg));
      else
        BHEM_TRY(run_pcg(s, mask, td, s.d_rhs, P.pcg_rtol, P.pcg_max, P.pcg_fixed_iters, &pit, &neg));
      st.pcg_iters_total += pit;
      if (tau > 0.0) st.regularizations++;
      if (!neg) break;
      tau = std::max(10.0 * tau, 1e-8);
    }
    if (status != SHELL_OK) break;
    tau_carry = tau;
    BHEM_CUDA(cudaMemcpyAsync(s.d_d, s.d_x, sizeof(double) * m, cudaMemcpyDeviceToDevice, s.stream));
    // line search on phi(a) = Pi(q + a d) - Pi(q) = dV(a) + a d.g_in + a^2/2 d^T M d / dt^2
    double alpha = 1.0;
    if (gn > 1e-6 * gref) {
      BHEM_TRY(launch_mass_mult(s, s.d_d, s.d_Md));
      BHEM_TRY(launch_dots3(s, m, s.d_d, s.d_Md, s.d_d, s.d_gin, s.d_g, s.d_d, s.d_ns->dots));
      BHEM_CUDA(cudaMemcpyAsync(s.h_ns, s.d_ns, sizeof(NewtonScalars), cudaMemcpyDeviceToHost, s.stream));
      BHEM_CUDA(cudaStreamSynchronize(s.stream));
      mark(s, "ls_dots");
      const double dMd = s.h_ns->dots[0] * inv_dt2, dgin = s.h_ns->dots[1], gd = s.h_ns->dots[2];
      if (!(gd < 0.0)) { status = SHELL_ERR_LINESEARCH; break; }
      double a_prev = 0.0, f_prev = 0.0;
      bool ok = false;
      for (int trial = 0; trial < 20; ++trial) {
        if (trial == 0) {
          BHEM_CUDA(cudaMemsetAsync(s.d_g2, 0, sizeof(double) * m, s.stream));
          BHEM_TRY(launch_energy_grad64(s, q, s.d_d, alpha, s.d_Ep2, s.d_Ep, s.d_g2, &s.d_ns->dV));
        } else {
          BHEM_TRY(launch_energy_grad64(s, q, s.d_d, alpha, nullptr, s.d_Ep, nullptr, &s.d_ns->dV));
        }
        BHEM_CUDA(cudaMemcpyAsync(&s.h_ns->dV, &s.d_ns->dV, sizeof(double), cudaMemcpyDeviceToHost, s.stream));
        BHEM_CUDA(cudaStreamSynchronize(s.stream));
        mark(s, "ls_trial");
        const double phi = s.h_ns->dV + alpha * dgin + 0.5 * alpha * alpha * dMd;
        if (std::isfinite(phi) && phi <= 1e-4 * alpha * gd) {
          ok = true;
          reuse = trial == 0;
          break;
        }
        st.ls_backtracks++;
        double a_new;
        if (!std::isfinite(phi)) {
          a_new = 0.5 * alpha;
        } else if (trial == 0) {
          a_new = -gd * alpha * alpha / (2.0 * (phi - gd * alpha));   // quadratic model minimiser
        } else {
          // cubic through phi(0), phi'(0), phi(a_prev), phi(alpha) (Nocedal-Wright Sec. 3.5)
          const double a0 = a_prev, a1 = alpha;
          const double r1 = phi - gd * a1, r0 = f_prev - gd * a0;
          const double den = a0 * a0 * a1 * a1 * (a1 - a0);
          const double ca = (a0 * a0 * r1 - a1 * a1 * r0) / den;
          const double cb = (-a0 * a0 * a0 * r1 + a1 * a1 * a1 * r0) / den;
          const double disc = cb * cb - 3.0 * ca * gd;
          a_new = (ca == 0.0 || disc < 0.0) ? 0.5 * alpha : (-cb + std::sqrt(disc)) / (3.0 * ca);
        }
        if (!(a_new >= 0.1 * alpha)) a_new = 0.1 * alpha;
        if (a_new > 0.5 * alpha) a_new = 0.5 * alpha;
        a_prev = alpha;
        f_prev = phi;
        alpha = a_new;
      }
      if (!ok) { status = SHELL_ERR_LINESEARCH; break; }
    }
    BHEM_TRY(launch_axpy_fixed(s, q, s.d_d, alpha));
    if (reuse) {
      std::swap(s.d_g, s.d_g2);
      std::swap(s.d_Ep, s.d_Ep2);
    }
    st.newton_iters++;
  }
  if (hess_pending) BHEM_CUDA(cudaStreamWaitEvent(s.stream, s.ev_hess, 0));   // unused, but finished in order
  st.res_final = gn;
  BHEM_CUDA(cudaMemcpyAsync(&s.h_ns->diag_fixes, &s.d_ns->diag_fixes, sizeof(int), cudaMemcpyDeviceToHost,
                            s.stream));
  BHEM_CUDA(cudaStreamSynchronize(s.stream));
  st.diag_fixes = s.h_ns->diag_fixes;
  st.tau_final = tau_carry;
  if (status == SHELL_OK || status == SHELL_ERR_NOT_CONVERGED) {
    BHEM_TRY(launch_velocity(s, q, s.d_qn, P.dt, v_out));
  } else {
    // leave q unchanged on failure
    BHEM_CUDA(cudaMemcpyAsync(q, s.d_qn, sizeof(double) * m, cudaMemcpyDeviceToDevice, s.stream));
  }
  mark(s, "end");
  trace_report(s);
  return status;
}
}  // namespace bhem

extern "C" shell_status shell_newton_step(shell_t* shell, const shell_step_params* params,
                                          const unsigned char* fixed_mask, const double* q_fixed,
                                          double* q, double* v, const double* warm_start,
                                          shell_step_stats* stats) {
  if (!shell || !params || !q || !v || !stats) return fail(SHELL_ERR_ARG, "NULL argument");
  if ((fixed_mask == nullptr) != (q_fixed == nullptr)) return fail(SHELL_ERR_ARG, "fixed_mask and q_fixed go together");
  const shell_step_params& P = *params;
  if (!(P.dt > 0) || P.newton_max < 0 || P.pcg_max < 0 || P.pcg_fixed_iters < 0 || !(P.newton_rtol >= 0) ||
      !(P.tau_carry >= 0) || !std::isfinite(P.tau_carry))
    return fail(SHELL_ERR_ARG, "invalid step parameters");
  Shell& s = *shell;
  std::memset(stats, 0, sizeof(*stats));
  const size_t bytes = sizeof(double) * s.n_dof;
  const bool q_dev = is_device_ptr(q), v_dev = is_device_ptr(v);
  double* dq = q;
  double* dv = v;
  if (!q_dev) {
    dq = s.d_qwork;
    BHEM_CUDA(cudaMemcpyAsync(dq, q, bytes, cudaMemcpyHostToDevice, s.stream));
  }
  if (!v_dev) {
    dv = s.d_vwork;
    BHEM_CUDA(cudaMemcpyAsync(dv, v, bytes, cudaMemcpyHostToDevice, s.stream));
  }
  const unsigned char* dmask = fixed_mask;
  const double* dqfix = q_fixed;
  if (fixed_mask && !is_device_ptr(fixed_mask)) {
    BHEM_CUDA(cudaMemcpyAsync(s.d_mask, fixed_mask, s.n_dof, cudaMemcpyHostToDevice, s.stream));
    dmask = s.d_mask;
  }
  if (q_fixed && !is_device_ptr(q_fixed)) {
    BHEM_CUDA(cudaMemcpyAsync(s.d_qfix, q_fixed, bytes, cudaMemcpyHostToDevice, s.stream));
    dqfix = s.d_qfix;
  }
  const double* dwarm = warm_start;
  if (warm_start && !is_device_ptr(warm_start)) {
    BHEM_CUDA(cudaMemcpyAsync(s.d_warm, warm_start, bytes, cudaMemcpyHostToDevice, s.stream));
    dwarm = s.d_warm;
  }
  shell_status st = newton_core(s, P, dmask, dqfix, dq, dv, dwarm, dv, *stats);
  stats->status = st;
  if (!q_dev) BHEM_CUDA(cudaMemcpyAsync(q, dq, bytes, cudaMemcpyDeviceToHost, s.stream));
  if (!v_dev) BHEM_CUDA(cudaMemcpyAsync(v, dv, bytes, cudaMemcpyDeviceToHost, s.stream));
  BHEM_CUDA(cudaStreamSynchronize(s.stream));
  if (st != SHELL_OK) {
    if (st == SHELL_ERR_NOT_CONVERGED) set_error("Newton did not reach the residual tolerance");
    else if (st == SHELL_ERR_LINESEARCH) set_error("line search failed");
    else if (st == SHELL_ERR_INDEFINITE) set_error("negative curvature persisted beyond tau = 1e4");
  }
  return st;
}

extern "C" shell_status shell_spmv(shell_t* shell, const void* x, int x_is_fp32, void* y) {
  if (!shell || !x || !y) return fail(SHELL_ERR_ARG, "NULL argument");
  if (x_is_fp32 && shell->val_fp64) return fail(SHELL_ERR_ARG, "an FP64 shell takes FP64 x");
  if ((reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(y) & 7))
    return fail(SHELL_ERR_ARG, "x must be 16-byte aligned and y 8-byte aligned");
  return launch_spmv(*shell, x, x_is_fp32, y);
}

extern "C" shell_status shell_kernel_launches(const shell_t* shell, long long* count) {
  if (!shell || !count) return fail(SHELL_ERR_ARG, "NULL argument");
  *count = shell->launches;
  return SHELL_OK;
}
