// Static ray-patch intersection (Sec. 5, Eq. ray, Eq. ineqray): nearest hit of each ray with the
// bicubic Hermite shell by subdivision of the patches' Bezier forms.
//
//   k_ray_nets   one thread per patch: Bezier control net (Hermite data b0 = a, b1 = a + a'/3,
//                b2 = b - b'/3, b3 = b per direction, tensor product) and its box.
//   k_ray_groups the box of every kGroup consecutive patches, to skip groups a ray misses.
//   k_trace_rays one ray per thread, FP64: all patch boxes are tested in patch order (staged
//                through shared memory, one chunk at a time for the whole CTA), hits go into a
//                binary min-heap in local memory keyed by the box's entry time tau_min; the top
//                candidate is refined (box at most kEpsTau on every side: an intersection at the
//                midpoint of its tau interval), or split into four sub-patches, at the parameter
//                midpoint (Fig. submid) or, in the Newton variant, around a Newton root of
//                x(u, v) = o + tau d that is abandoned together with its neighbourhood
//                (Fig. subany). The search ends when the heap's top cannot beat the best tau.
//                The children's boxes (4 children x 3 coordinates per split, most of a split's
//                FP64 work) are pooled over the warp: lanes whose rays are done or need no split
//                take jobs of the lanes that do, so a long search left alone in its warp runs
//                its 12 box jobs side by side instead of one after another.
//                A ray whose local heap fills moves it into one of kRedoThreads larger heaps
//                in global memory and continues.
//   k_trace_rays_redo  the rays that found no free global heap, traced again from the start
//                with one (the search is deterministic, so the result is the one an unbounded
//                heap gives).
//
// Sub-patches are cut from the patch's net by blossoming (each restricted curve's points are
// f(a,a,a), f(a,a,b), f(a,b,b), f(b,b,b), De Casteljau with one parameter per level) and only
// their box is kept: per coordinate the 4 theta1-curves are restricted, then the 4 theta2-curves,
// folded straight into the slab test. This file is compiled without mul-add contraction: each
// product and sum is rounded separately, in the order written, so every decision of the search
// (slab intervals, heap order, refinement, Newton convergence) is that of the same sequence of
// IEEE FP64 operations in any plain sequential program.
#include <cmath>

#include "bezier.cuh"
#include "common.cuh"

namespace bhem {
namespace {

using namespace bz;

constexpr double kEpsTau = 1e-9;     // refinement size (positions' units; unit directions)
constexpr int kNetBlock = 128;
constexpr int kRayBlock = 128;
constexpr int kRootChunk = 32;       // group boxes staged in shared memory per pass
constexpr int kGroup = 32;           // consecutive patches per group box

// Min and max of coordinate c of the sub-patch [u0, u1] x [v0, v1] of the net P ([c][i][j]).
__device__ __forceinline__ void sub_range(const double* __restrict__ P, int c, double u0, double u1, double v0,
                                          double v1, double& mn, double& mx) {
  const double* Pc = P + 16 * c;
  double T[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const double in[4] = {__ldg(Pc + j), __ldg(Pc + 4 + j), __ldg(Pc + 8 + j), __ldg(Pc + 12 + j)};
    double o[4];
    curve_restrict(in, u0, u1, o);
#pragma unroll
    for (int i = 0; i < 4; ++i) T[i][j] = o[i];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double o[4];
    curve_restrict(T[i], v0, v1, o);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double s = o[j];
      if (i == 0 && j == 0) {
        mn = s;
        mx = s;
      }
      if (s < mn) mn = s;
      if (s > mx) mx = s;
    }
  }
}

// One axis of the slab test (Eq. ineqray): narrows [lo, hi]; false when the ray misses.
__device__ __forceinline__ bool slab(double mn, double mx, double o, double d, double inv, double& lo,
                                     double& hi) {
  if (d == 0.0) return !(o < mn || o > mx);
  double a = (mn - o) * inv, b = (mx - o) * inv;
  if (a > b) {
    const double t = a;
    a = b;
    b = t;
  }
  if (a > lo) lo = a;
  if (b < hi) hi = b;
  return true;
}

// Box of each group of kGroup consecutive patches (min xyz, max xyz of its patches' boxes). A ray
// that misses a group's box misses every member's: FP64 subtraction and multiplication by the
// same 1/d are monotone, so the group's slab interval contains each member's.
__global__ void k_ray_groups(int np, const double* __restrict__ boxes, double* __restrict__ gboxes) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  const int p0 = gi * kGroup;
  if (p0 >= np) return;
  const int p1 = min(np, p0 + kGroup);
  double mn[3], mx[3];
  for (int c = 0; c < 3; ++c) {
    mn[c] = boxes[(size_t)p0 * 8 + c];
    mx[c] = boxes[(size_t)p0 * 8 + 3 + c];
  }
  for (int p = p0 + 1; p < p1; ++p)
    for (int c = 0; c < 3; ++c) {
      const double a = boxes[(size_t)p * 8 + c], b = boxes[(size_t)p * 8 + 3 + c];
      if (a < mn[c]) mn[c] = a;
      if (b > mx[c]) mx[c] = b;
    }
  double* G = gboxes + (size_t)gi * 8;
  for (int c = 0; c < 3; ++c) {
    G[c] = mn[c];
    G[3 + c] = mx[c];
  }
  G[6] = 0.0;
  G[7] = 0.0;
}

__global__ void __launch_bounds__(kNetBlock) k_ray_nets(int np, const int4* __restrict__ pnodes,
                                                        const double* __restrict__ q, double dxi1, double dxi2,
                                                        double* __restrict__ nets, double* __restrict__ boxes) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int4 n4 = pnodes[p];
  const int nd[4] = {n4.x, n4.y, n4.z, n4.w};
  double* P = nets + (size_t)p * 48;
  patch_net(q, nd, dxi1, dxi2, P);
  // the root box is the box of the net cut to [0, 1]^2, as for every other candidate
  double e = 0.0;
  double* B = boxes + (size_t)p * 8;
  for (int c = 0; c < 3; ++c) {
    double mn, mx;
    sub_range(P, c, 0.0, 1.0, 0.0, 1.0, mn, mx);
    B[c] = mn;
    B[3 + c] = mx;
    if (mx - mn > e) e = mx - mn;
  }
  B[6] = e;
  B[7] = 0.0;
}

// Newton's method on F(u, v, tau) = x(u, v) - o - tau d, Jacobian [x_u | x_v | -d] by Cramer's
// rule. True with the root in (u, v, tau) on convergence; gives up when an iterate leaves the
// window win (the candidate's rectangle widened by its extent on each side).
__device__ bool newton_root(const double* __restrict__ P, const double o[3], const double d[3], double on,
                            const double win[4], double& u, double& v, double& tau, int& iters) {
  double uu = u, vv = v, tt = tau;
  for (int it = 0; it < kNewtonIters; ++it) {
    double x[3], xu[3], xv[3], F[3];
    ++iters;
    bezier_eval(P, uu, vv, x, xu, xv);
#pragma unroll
    for (int c = 0; c < 3; ++c) F[c] = (x[c] - o[c]) - tt * d[c];
    const double fn = sqrt((F[0] * F[0] + F[1] * F[1]) + F[2] * F[2]);
    if (fn <= 1e-12 * ((1.0 + on) + fabs(tt))) {
      u = uu;
      v = vv;
      tau = tt;
      return true;
    }
    const double J[3][3] = {{xu[0], xv[0], -d[0]}, {xu[1], xv[1], -d[1]}, {xu[2], xv[2], -d[2]}};
    const double det = det3(J);
    if (!(fabs(det) > 1e-300)) return false;
    double delta[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double M[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s) M[r][s] = s == k ? -F[r] : J[r][s];
      delta[k] = det3(M) / det;
    }
    uu += delta[0];
    vv += delta[1];
    tt += delta[2];
    if (!isfinite(uu) || !isfinite(vv) || !isfinite(tt)) return false;
    if (uu < win[0] || uu > win[1] || vv < win[2] || vv > win[3]) return false;   // left the window
  }
  return false;
}

struct Ray {
  double o[3], d[3], inv[3];
};

__device__ __forceinline__ void load_ray(const double* __restrict__ origins, const double* __restrict__ dirs,
                                         long long k, Ray& r) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    r.o[c] = origins[3 * k + c];
    r.d[c] = dirs[3 * k + c];
    r.inv[c] = r.d[c] != 0.0 ? 1.0 / r.d[c] : 0.0;
  }
}

// Root candidate: the whole patch p with box B = (min xyz, max xyz, largest side).
__device__ __forceinline__ void root_push(Heap& h, const double* B, int p, const Ray& r) {
  double lo = 0.0, hi = INFINITY;
  bool in = true;
#pragma unroll
  for (int c = 0; c < 3; ++c)
    if (in) in = slab(B[c], B[3 + c], r.o[c], r.d[c], r.inv[c], lo, hi);
  if (in && !(lo > hi)) h.push(Cand{lo, hi, B[6], 0.0, 1.0, 0.0, 1.0, p});
}

// Per-lane state of one ray's search.
struct Search {
  double best = INFINITY, bu = 0.0, bv = 0.0, on = 0.0;
  int bp = -1, nexp = 0, flags = 0, newton_iters = 0;
  bool live = false;
};

// Shared-memory exchange of one warp: the children each lane produced in the current split and
// the coordinate ranges computed for them by whichever lanes took those jobs.
struct WarpSmem {
  double rect[32][4][4];        // child rectangles u0, u1, v0, v1 in push order
  double range[32][12][2];      // (child * 3 + coordinate): min, max
  int patch[32];
  unsigned short jobs[32 * 12]; // lane * 12 + child * 3 + coordinate
};

__device__ __forceinline__ void put_rect(WarpSmem& sm, int lane, int& nch, double u0, double u1, double v0,
                                         double v1) {
  if (!(u1 > u0) || !(v1 > v0)) return;   // degenerate pieces of a pinwheel split
  double* R = sm.rect[lane][nch++];
  R[0] = u0;
  R[1] = u1;
  R[2] = v0;
  R[3] = v1;
}

// The search over the candidates already in each lane's heap, all 32 lanes of the warp together
// (lanes without a ray pass live = false). Every iteration each live lane takes its top
// candidate and, when it splits it, lists its children; the 3 coordinate ranges of every child
// of every lane are then computed as one pool of jobs spread over the warp's lanes, and each
// lane finishes its own children (slab test, push) in order. A ray stops early once its heap
// overflows.
__device__ void search(Heap& h, const Ray& r, const double* __restrict__ nets, int use_newton, Search& S,
                       WarpSmem& sm, int lane) {
  S.on = sqrt((r.o[0] * r.o[0] + r.o[1] * r.o[1]) + r.o[2] * r.o[2]);
  while (__any_sync(0xffffffffu, S.live)) {
    int nch = 0;
    if (S.live) {
      if (h.n == 0 || h.overflow) {
        S.live = false;
      } else {
        const Cand c = h.pop();
        if (c.t0 >= S.best - kEpsTau) {                                    // nothing left can be closer
          S.live = false;
        } else if (c.ext <= kEpsTau || (c.u1 - c.u0 < 1e-13 && c.v1 - c.v0 < 1e-13)) {   // refined
          const double t = 0.5 * (c.t0 + c.t1);
          if (t < S.best - kEpsTau) {
            S.best = t;
            S.bp = c.patch;
            S.bu = 0.5 * (c.u0 + c.u1);
            S.bv = 0.5 * (c.v0 + c.v1);
          }
        } else if (S.nexp == kMaxExpansions) {
          S.flags |= SHELL_RAY_LIMIT;
          S.live = false;
        } else {
          ++S.nexp;
          const double* P = nets + (size_t)c.patch * 48;
          const double um = 0.5 * (c.u0 + c.u1), vm = 0.5 * (c.v0 + c.v1);
          bool pinwheel = false;
          if (use_newton) {
            double x[3], xu[3], xv[3];
            bezier_eval(P, um, vm, x, xu, xv);
            double u = um, v = vm;
            double t = ((x[0] - r.o[0]) * r.d[0] + (x[1] - r.o[1]) * r.d[1]) + (x[2] - r.o[2]) * r.d[2];
            const double wu = c.u1 - c.u0, wv = c.v1 - c.v0;
            const double win[4] = {c.u0 - wu, c.u1 + wu, c.v0 - wv, c.v1 + wv};
            if (newton_root(P, r.o, r.d, S.on, win, u, v, t, S.newton_iters) && u >= c.u0 && u <= c.u1 &&
                v >= c.v0 && v <= c.v1 && t >= 0.0) {
              if (t < S.best) {
                S.best = t;
                S.bp = c.patch;
                S.bu = u;
                S.bv = v;
              }
              // Fig. subany: drop [a1, a2] x [b1, b2] around the root, four rectangles remain
              const double hu = kNbhd * (c.u1 - c.u0), hv = kNbhd * (c.v1 - c.v0);
              const double a1 = fmax(c.u0, u - hu), a2 = fmin(c.u1, u + hu);
              const double b1 = fmax(c.v0, v - hv), b2 = fmin(c.v1, v + hv);
              put_rect(sm, lane, nch, c.u0, a1, b1, c.v1);
              put_rect(sm, lane, nch, a1, c.u1, b2, c.v1);
              put_rect(sm, lane, nch, c.u0, a2, c.v0, b1);
              put_rect(sm, lane, nch, a2, c.u1, c.v0, b2);
              pinwheel = true;
            }
          }
          if (!pinwheel) {   // Fig. submid: four quarters at the parameter midpoint
            put_rect(sm, lane, nch, c.u0, um, vm, c.v1);
            put_rect(sm, lane, nch, um, c.u1, vm, c.v1);
            put_rect(sm, lane, nch, c.u0, um, c.v0, vm);
            put_rect(sm, lane, nch, um, c.u1, c.v0, vm);
          }
          sm.patch[lane] = c.patch;
          h.boxes += nch;
        }
      }
    }
    // the warp's pool of (lane, child, coordinate) range jobs
    const int nj = 3 * nch;
    int pre = nj;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, pre, off);
      if (lane >= off) pre += y;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    pre -= nj;
    for (int k = 0; k < nj; ++k) sm.jobs[pre + k] = (unsigned short)(lane * 12 + k);
    __syncwarp();
    for (int j = lane; j < total; j += 32) {
      const int code = sm.jobs[j], owner = code / 12, k = code - 12 * owner;
      const double* R = sm.rect[owner][k / 3];
      double mn, mx;
      sub_range(nets + (size_t)sm.patch[owner] * 48, k % 3, R[0], R[1], R[2], R[3], mn, mx);
      sm.range[owner][k][0] = mn;
      sm.range[owner][k][1] = mx;
    }
    __syncwarp();
    for (int ch = 0; ch < nch; ++ch) {
      double lo = 0.0, hi = INFINITY, e = 0.0;
      bool in = true;
      for (int cc = 0; cc < 3 && in; ++cc) {
        const double mn = sm.range[lane][3 * ch + cc][0], mx = sm.range[lane][3 * ch + cc][1];
        if (mx - mn > e) e = mx - mn;
        in = slab(mn, mx, r.o[cc], r.d[cc], r.inv[cc], lo, hi);
      }
      if (in && !(lo > hi) && !(lo >= S.best)) {
        const double* R = sm.rect[lane][ch];
        h.push(Cand{lo, hi, e, R[0], R[1], R[2], R[3], sm.patch[lane]});
      }
    }
    __syncwarp();
  }
  if (h.overflow) {
    S.flags |= SHELL_RAY_OVERFLOW;   // void: reported as a miss
  } else if (S.bp >= 0) {
    S.flags |= SHELL_RAY_HIT;
  }
}

struct RayOut {
  double* tau;
  int* patch;
  double* uv;
  int* flags;
  int* stats;
};

__device__ __forceinline__ void write_hit(const RayOut& out, long long k, const Search& S, const Heap& h) {
  const bool hit = (S.flags & SHELL_RAY_HIT) != 0;
  out.tau[k] = hit ? S.best : INFINITY;
  out.patch[k] = hit ? S.bp : -1;
  out.uv[2 * k] = hit ? S.bu : 0.0;
  out.uv[2 * k + 1] = hit ? S.bv : 0.0;
  out.flags[k] = S.flags;
  if (out.stats) {
    out.stats[4 * k] = S.nexp;
    out.stats[4 * k + 1] = h.peak;
    out.stats[4 * k + 2] = h.boxes;
    out.stats[4 * k + 3] = S.newton_iters;
  }
}

// First pass: one ray per thread, a kHeapCap-entry heap in local memory, the search shared by the
// warp. A ray whose heap overflows stops and is appended to redo_list for the second pass (or,
// when the list is full, reported with SHELL_RAY_OVERFLOW).
__global__ void __launch_bounds__(kRayBlock, 4) k_trace_rays(long long n, const double* __restrict__ origins,
                                                          const double* __restrict__ dirs, int np,
                                                          const double* __restrict__ nets,
                                                          const double* __restrict__ boxes,
                                                          const double* __restrict__ gboxes, int use_newton,
                                                          RayOut out, int* __restrict__ redo_count,
                                                          int* __restrict__ redo_list, Cand* __restrict__ heaps) {
  __shared__ double sbox[kRootChunk * 8];
  __shared__ WarpSmem wsm[kRayBlock / 32];
  const int lane = threadIdx.x & 31;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = k < n;
  Ray r;
  Cand storage[kHeapCap];
  Heap h(storage, kHeapCap);
  h.spill = heaps;
  h.spill_count = redo_count + 1;
  if (active) load_ray(origins, dirs, k, r);
  // every patch's box in patch order, skipping the groups whose box the ray misses (their members
  // would all be missed); the whole CTA stages one chunk of group boxes at a time
  const int ngroups = (np + kGroup - 1) / kGroup;
  for (int base = 0; base < ngroups; base += kRootChunk) {
    const int m = min(kRootChunk, ngroups - base);
    __syncthreads();
    for (int i = threadIdx.x; i < m * 8; i += blockDim.x) sbox[i] = gboxes[(size_t)base * 8 + i];
    __syncthreads();
    if (!active) continue;
    for (int j = 0; j < m; ++j) {
      const double* G = sbox + 8 * j;
      double lo = 0.0, hi = INFINITY;
      bool in = true;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (in) in = slab(G[c], G[3 + c], r.o[c], r.d[c], r.inv[c], lo, hi);
      if (!in || lo > hi) continue;
      const int p0 = (base + j) * kGroup, p1 = min(np, p0 + kGroup);
      for (int p = p0; p < p1; ++p) root_push(h, boxes + 8 * (size_t)p, p, r);
    }
  }
  h.boxes = np;
  Search S;
  S.live = active;
  search(h, r, nets, use_newton, S, wsm[threadIdx.x >> 5], lane);
  if (!active) return;
  if (h.overflow) {
    const int slot = atomicAdd(redo_count, 1);
    if (slot < kRedoList) {
      redo_list[slot] = (int)k;
      return;                                                         // written by the second pass
    }
  }
  write_hit(out, k, S, h);
}

// Second pass over the rays whose first-pass heap overflowed: the same search from the start
// with a kRedoHeap-entry heap per thread in global memory (heaps: kRedoThreads x kRedoHeap).
__global__ void __launch_bounds__(kRedoThreads) k_trace_rays_redo(const double* __restrict__ origins,
                                                                  const double* __restrict__ dirs, int np,
                                                                  const double* __restrict__ nets,
                                                                  const double* __restrict__ boxes, int use_newton,
                                                                  RayOut out, const int* __restrict__ redo_count,
                                                                  const int* __restrict__ redo_list,
                                                                  Cand* __restrict__ heaps) {
  __shared__ WarpSmem wsm[kRedoThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31;
  const int count = min(*redo_count, kRedoList);
  for (int base = 0; base < count; base += kRedoThreads) {   // uniform trip count: the warp stays whole
    const int i = base + tid;
    const bool active = i < count;
    const long long k = active ? redo_list[i] : 0;
    Ray r;
    Heap h(heaps + (size_t)tid * kRedoHeap, kRedoHeap);
    if (active) {
      load_ray(origins, dirs, k, r);
      for (int p = 0; p < np; ++p) root_push(h, boxes + 8 * (size_t)p, p, r);
    }
    h.boxes = np;
    Search S;
    S.live = active;
    search(h, r, nets, use_newton, S, wsm[tid >> 5], lane);
    if (active) write_hit(out, k, S, h);
  }
}

}  // namespace

// One allocation per shell: kRedoThreads x kRedoHeap candidates (at the 256-byte aligned base),
// then two counters (queries sent to the second pass, global heaps claimed) and the redo list.
shell_status search_scratch(Shell& s, void** heaps, int** counters, int** redo_list) {
  if (!s.d_search) {
    const size_t bytes = sizeof(bz::Cand) * (size_t)bz::kRedoThreads * bz::kRedoHeap + sizeof(int) * (4 + bz::kRedoList);
    const cudaError_t e = cudaMalloc(&s.d_search, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s.d_search = nullptr;
      return fail(SHELL_ERR_OOM, std::string("search scratch: ") + cudaGetErrorString(e));
    }
  }
  *heaps = s.d_search;
  *counters = (int*)((bz::Cand*)s.d_search + (size_t)bz::kRedoThreads * bz::kRedoHeap);
  *redo_list = *counters + 4;   // counters: redo count, spill count, query counter, pad
  return SHELL_OK;
}

}  // namespace bhem

using namespace bhem;

extern "C" shell_status shell_trace_rays(shell_t* shell, const double* q, long long n_rays, const double* origins,
                                         const double* dirs, int variant, double* tau, int* patch, double* uv,
                                         int* flags, int* stats) {
  if (!shell) return fail(SHELL_ERR_ARG, "NULL shell");
  if (variant != SHELL_RAY_MIDPOINT && variant != SHELL_RAY_NEWTON) return fail(SHELL_ERR_ARG, "ray variant");
  if (n_rays < 0 || n_rays > INT32_MAX) return fail(SHELL_ERR_ARG, "n_rays outside [0, 2^31 - 1]");
  if (n_rays == 0) return SHELL_OK;
  if (!q || !origins || !dirs || !tau || !patch || !uv || !flags) return fail(SHELL_ERR_ARG, "NULL argument");
  Shell& s = *shell;
  const int np = s.n_patches;
  void* heaps_v = nullptr;
  int *redo_count = nullptr, *redo_list = nullptr;
  BHEM_TRY(search_scratch(s, &heaps_v, &redo_count, &redo_list));
  if (!s.d_ray_nets) {
    const size_t ngroups = ((size_t)np + kGroup - 1) / kGroup;
    const cudaError_t e = cudaMalloc((void**)&s.d_ray_nets, sizeof(double) * (56 * (size_t)np + 8 * ngroups));
    if (e != cudaSuccess) {
      cudaGetLastError();
      s.d_ray_nets = nullptr;
      return fail(SHELL_ERR_OOM, std::string("ray nets: ") + cudaGetErrorString(e));
    }
  }
  Cand* heaps = (Cand*)heaps_v;
  double* nets = s.d_ray_nets;
  double* boxes = nets + 48 * (size_t)np;
  double* gboxes = boxes + 8 * (size_t)np;
  const int ngroups = (np + kGroup - 1) / kGroup;
  RayOut out{tau, patch, uv, flags, stats};
  BHEM_CUDA(cudaMemsetAsync(redo_count, 0, 2 * sizeof(int), s.stream));
  k_ray_nets<<<grid_for(np, kNetBlock), kNetBlock, 0, s.stream>>>(np, s.d_patch_nodes, q, s.grid.dxi1,
                                                                  s.grid.dxi2, nets, boxes);
  k_ray_groups<<<grid_for(ngroups, kNetBlock), kNetBlock, 0, s.stream>>>(np, boxes, gboxes);
  const int use_newton = variant == SHELL_RAY_NEWTON;
  k_trace_rays<<<(unsigned)((n_rays + kRayBlock - 1) / kRayBlock), kRayBlock, 0, s.stream>>>(
      n_rays, origins, dirs, np, nets, boxes, gboxes, use_newton, out, redo_count, redo_list, heaps);
  k_trace_rays_redo<<<1, kRedoThreads, 0, s.stream>>>(origins, dirs, np, nets, boxes, use_newton, out, redo_count,
                                                      redo_list, heaps);
  s.launches += 4;
  BHEM_CUDA(cudaGetLastError());
  return SHELL_OK;
}
