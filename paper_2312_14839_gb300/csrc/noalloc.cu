// Elastic energy and gradient of a shell with no device allocation at all.
//
// Everything here is self-contained: the kernel derives the patch topology from the grid, the
// shape table and the rest geometry from the rest DOFs, and keeps its only scratch (per-CTA
// partial sums for the energy, the shape table, a ticket counter) in one file-scope device
// array. The caller passes inputs and outputs; no shell object is needed.
#include <mutex>

#include "common.cuh"

namespace bhem {
namespace noalloc {

constexpr int kPatchesPerCta = 8;                          // half a warp per patch
constexpr int kMaxCtas = 16384;
constexpr int kMaxPatches = kPatchesPerCta * kMaxCtas;     // 131072 patches (e.g. 362 x 362)
constexpr int kTable = 16 * 97 + 16;                       // shape table + Gauss weights
constexpr int kStride = 97;

struct Scratch {
  double partials[kMaxCtas];   // per-CTA energy sums (fully rewritten by every call)
  double table[kTable];        // shape table of the current call (rewritten by every call)
  unsigned ticket;             // last-CTA counter: must be 0 when a call starts
};

// The only scratch memory of this entry point: about 141 KB, held by every GPU that loads the
// library until the process exits.
static __device__ __align__(256) unsigned char g_scratch[sizeof(Scratch)];

// ---- App. A.1 / A.2 ---------------------------------------------------------------------
__device__ __forceinline__ double hermite(int p, int r, double t, int d) {
  const double s = p ? 1.0 - t : t;
  double v;
  if (r == 0) v = d == 0 ? (2 * s - 3) * s * s + 1 : d == 1 ? 6 * s * s - 6 * s : 12 * s - 6;
  else        v = d == 0 ? ((s - 2) * s + 1) * s : d == 1 ? (3 * s - 4) * s + 1 : 6 * s - 4;
  if (p == 1 && r == 1) v = -v;
  if (p == 1 && (d & 1)) v = -v;
  return v;
}

__global__ void k_table(double d1, double d2, double* __restrict__ table) {
  const double xi = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
  const double xo = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
  const double th[4] = {0.5 * (1 - xo), 0.5 * (1 - xi), 0.5 * (1 + xi), 0.5 * (1 + xo)};
  const double wi = (18.0 + sqrt(30.0)) / 72.0, wo = (18.0 - sqrt(30.0)) / 72.0;
  const double wt[4] = {wo, wi, wi, wo};
  const int dd1[6] = {0, 1, 0, 2, 0, 1}, dd2[6] = {0, 0, 1, 0, 2, 1};
  for (int e = threadIdx.x; e < kTable; e += blockDim.x) {
    if (e >= 16 * kStride) {
      const int g = e - 16 * kStride;
      table[e] = d1 * d2 * wt[g & 3] * wt[g >> 2];
      continue;
    }
    const int I = e / kStride, rem = e % kStride;
    if (rem >= 96) { table[e] = 0.0; continue; }
    const int k = rem / 16, g = rem % 16;
    const int corner = I >> 2, kind = I & 3;
    const int p = corner & 1, q = corner >> 1, r = kind & 1, s = kind >> 1;
    double v = hermite(p, r, th[g & 3], dd1[k]) * hermite(q, s, th[g >> 2], dd2[k]);
    v *= (r ? d1 : 1.0) * (s ? d2 : 1.0);
    for (int i = 0; i < dd1[k]; ++i) v /= d1;
    for (int i = 0; i < dd2[k]; ++i) v /= d2;
    table[e] = v;
  }
}

struct D3 { double x, y, z; };
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 operator*(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cross(D3 a, D3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// a_1, a_2, a_{1,1}, a_{2,2}, a_{1,2} at Gauss point g from 16 DOF triples
__device__ __forceinline__ void derivs(const double* sphi, const double* qv, int g, D3 out[5]) {
  for (int k = 0; k < 5; ++k) out[k] = {0.0, 0.0, 0.0};
  for (int I = 0; I < 16; ++I) {
    const D3 v = {qv[I * 3], qv[I * 3 + 1], qv[I * 3 + 2]};
    for (int k = 0; k < 5; ++k) out[k] = out[k] + sphi[I * kStride + (k + 1) * 16 + g] * v;
  }
}

// Half a warp per patch, lane = Gauss point: St. Venant-Kirchhoff membrane + bending energy
// (thickness-integrated) and its gradient per generalised coordinate.
__global__ void __launch_bounds__(128)
k_energy_grad(int nu, int nv, int per_u, int per_v, const double* __restrict__ rest,
              const double* __restrict__ q, double lam, double mu, double h,
              double* __restrict__ grad, double* __restrict__ energy_out, Scratch* S) {
  __shared__ double sphi[kTable];
  __shared__ double sq[kPatchesPerCta][48];
  __shared__ double sr[kPatchesPerCta][48];
  __shared__ double sG[kPatchesPerCta][16][15];
  __shared__ double sred[4];
  __shared__ int last;
  for (int e = threadIdx.x; e < kTable; e += blockDim.x) sphi[e] = S->table[e];
  const int n1 = per_u ? nu : nu + 1, n2 = per_v ? nv : nv + 1;
  const int np = nu * nv;
  const int hw = threadIdx.x >> 4, g = threadIdx.x & 15;
  const int p = blockIdx.x * kPatchesPerCta + hw;
  const bool active = p < np;
  int nd[4] = {0, 0, 0, 0};
  if (active) {
    const int pu = p % nu, pv = p / nu;
    for (int c = 0; c < 4; ++c) nd[c] = ((pv + (c >> 1)) % n2) * n1 + (pu + (c & 1)) % n1;
    for (int l = g; l < 48; l += 16) {
      const size_t a = (size_t)nd[l / 12] * 12 + (l % 12);
      sq[hw][l] = q[a];
      sr[hw][l] = rest[a];
    }
  }
  __syncthreads();
  double e = 0.0;
  if (active) {
    D3 v[5], w[5];
    derivs(sphi, sq[hw], g, v);
    derivs(sphi, sr[hw], g, w);
    // rest metric, curvature, contravariant metric, Voigt H
    const double ab11 = dot(w[0], w[0]), ab22 = dot(w[1], w[1]), ab12 = dot(w[0], w[1]);
    const double det = ab11 * ab22 - ab12 * ab12;
    const double sqab = sqrt(det);
    const D3 ab3 = (1.0 / sqab) * cross(w[0], w[1]);
    const double bb[3] = {dot(w[2], ab3), dot(w[3], ab3), dot(w[4], ab3)};
    const double ai11 = ab22 / det, ai22 = ab11 / det, ai12 = -ab12 / det;
    const double H00 = (lam + 2 * mu) * ai11 * ai11, H01 = lam * ai11 * ai22 + 2 * mu * ai12 * ai12;
    const double H02 = (lam + 2 * mu) * ai11 * ai12, H11 = (lam + 2 * mu) * ai22 * ai22;
    const double H12 = (lam + 2 * mu) * ai12 * ai22, H22 = (lam + mu) * ai12 * ai12 + mu * ai11 * ai22;
    const double wgt = sphi[16 * kStride + g] * sqab;
    // deformed geometry and strains
    const D3 a1 = v[0], a2 = v[1];
    const D3 n = cross(a1, a2);
    const double sqa = sqrt(dot(n, n));
    const D3 a3 = (1.0 / sqa) * n;
    const double al[3] = {0.5 * (dot(a1, a1) - ab11), 0.5 * (dot(a2, a2) - ab22), dot(a1, a2) - ab12};
    const double be[3] = {dot(v[2], a3) - bb[0], dot(v[3], a3) - bb[1], 2.0 * (dot(v[4], a3) - bb[2])};
    const double sg[3] = {H00 * al[0] + H01 * al[1] + H02 * al[2], H01 * al[0] + H11 * al[1] + H12 * al[2],
                          H02 * al[0] + H12 * al[1] + H22 * al[2]};
    const double mm[3] = {H00 * be[0] + H01 * be[1] + H02 * be[2], H01 * be[0] + H11 * be[1] + H12 * be[2],
                          H02 * be[0] + H12 * be[1] + H22 * be[2]};
    const double h3 = h * h * h, s = h3 / 12.0;
    e = wgt * (0.5 * h * (al[0] * sg[0] + al[1] * sg[1] + al[2] * sg[2]) +
               h3 / 24.0 * (be[0] * mm[0] + be[1] * mm[1] + be[2] * mm[2]));
    if (grad) {
      const D3 ct = mm[0] * v[2] + mm[1] * v[3] + (2.0 * mm[2]) * v[4];
      const double bt = dot(ct, a3);
      const D3 t1 = cross(a2, a3), t2 = cross(a3, a1);
      const D3 e1 = (1.0 / sqa) * (cross(a2, ct) - bt * t1);
      const D3 e2 = (1.0 / sqa) * (cross(ct, a1) - bt * t2);
      D3 G[5];
      G[0] = wgt * (h * (sg[0] * a1 + sg[2] * a2) + s * e1);
      G[1] = wgt * (h * (sg[1] * a2 + sg[2] * a1) + s * e2);
      G[2] = (wgt * s * mm[0]) * a3;
      G[3] = (wgt * s * mm[1]) * a3;
      G[4] = (wgt * s * 2.0 * mm[2]) * a3;
      for (int k = 0; k < 5; ++k) {
        sG[hw][g][k * 3 + 0] = G[k].x;
        sG[hw][g][k * 3 + 1] = G[k].y;
        sG[hw][g][k * 3 + 2] = G[k].z;
      }
    }
  }
  __syncthreads();
  if (active && grad) {
    for (int l = g; l < 48; l += 16) {
      const int I = l / 3, c = l % 3;
      double acc = 0.0;
      for (int gg = 0; gg < 16; ++gg)
        for (int k = 0; k < 5; ++k) acc += sphi[I * kStride + (k + 1) * 16 + gg] * sG[hw][gg][k * 3 + c];
      atomicAdd(&grad[(size_t)nd[I >> 2] * 12 + (I & 3) * 3 + c], acc);
    }
  }
  // energy: CTA sum in a fixed order, then the last CTA sums the partials in CTA order
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    S->partials[blockIdx.x] = sred[0] + sred[1] + sred[2] + sred[3];
    __threadfence();
    last = atomicAdd(&S->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += ((volatile double*)S->partials)[b];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    *energy_out = sred[0] + sred[1] + sred[2] + sred[3];
    S->ticket = 0u;
  }
}

// Device address of g_scratch, looked up once per device (with that device current) and kept for
// the life of the process; a cudaDeviceReset on that device invalidates it (documented in bhem.h).
static std::mutex g_mutex;
static Scratch* g_addr[128] = {nullptr};

static shell_status scratch_for_current_device(Scratch** out) {
  int dev = 0;
  BHEM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(SHELL_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return fail(SHELL_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = reinterpret_cast<Scratch*>(p);
  }
  *out = g_addr[dev];
  return SHELL_OK;
}

}  // namespace noalloc
}  // namespace bhem

using namespace bhem;

extern "C" shell_status shell_energy_grad_noalloc(const shell_grid* grid, const shell_material* material,
                                                  const double* rest_dofs, const double* q,
                                                  double* energy, double* grad, void* stream) {
  using namespace bhem::noalloc;
  if (!grid || !material || !rest_dofs || !q || !energy) return fail(SHELL_ERR_ARG, "NULL argument");
  const shell_grid& g = *grid;
  if (g.nu < 1 || g.nv < 1 || (g.periodic_u && g.nu < 2) || (g.periodic_v && g.nv < 2) ||
      !(g.dxi1 > 0) || !(g.dxi2 > 0))
    return fail(SHELL_ERR_ARG, "invalid grid");
  const long long np = (long long)g.nu * g.nv;
  if (np > kMaxPatches)
    return fail(SHELL_ERR_ARG, "grid has " + std::to_string(np) + " patches; the allocation-free entry "
                               "point handles at most " + std::to_string(kMaxPatches));
  if (!(material->thickness > 0) || !(material->young > 0) ||
      !(material->poisson > -1.0 && material->poisson < 1.0))
    return fail(SHELL_ERR_ARG, "invalid material");
  Scratch* S = nullptr;
  BHEM_TRY(scratch_for_current_device(&S));
  cudaStream_t st = (cudaStream_t)stream;
  const long long n1 = g.periodic_u ? g.nu : g.nu + 1, n2 = g.periodic_v ? g.nv : g.nv + 1;
  BHEM_CUDA(cudaMemsetAsync(&S->ticket, 0, sizeof(unsigned), st));
  if (grad) BHEM_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * 12 * n1 * n2, st));
  k_table<<<1, 256, 0, st>>>(g.dxi1, g.dxi2, S->table);
  BHEM_CUDA(cudaGetLastError());
  const double lam = material->young * material->poisson / (1.0 - material->poisson * material->poisson);
  const double mu = material->young / (2.0 * (1.0 + material->poisson));
  const int blocks = (int)((np + kPatchesPerCta - 1) / kPatchesPerCta);
  k_energy_grad<<<blocks, 128, 0, st>>>(g.nu, g.nv, g.periodic_u, g.periodic_v, rest_dofs, q, lam, mu,
                                        material->thickness, grad, energy, S);
  BHEM_CUDA(cudaGetLastError());
  return SHELL_OK;
}
