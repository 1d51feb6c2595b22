// Static ray-patch intersection (Sec. 5, Eq. ray, Eq. ineqray): nearest hit of each ray with the
// bicubic Hermite shell by subdivision of the patches' Bezier forms.
//
//   k_ray_nets   one thread per patch: Bezier control net (Hermite data b0 = a, b1 = a + a'/3,
//                b2 = b - b'/3, b3 = b per direction, tensor product) and its box.
//   k_trace_rays one thread per ray, FP64: all patch boxes are tested in patch order (staged
//                through shared memory, one chunk at a time for the whole CTA), hits go into a
//                binary min-heap in local memory keyed by the box's entry time tau_min; the top
//                candidate is refined (box at most kEpsTau on every side: an intersection at the
//                midpoint of its tau interval), or split into four sub-patches, at the parameter
//                midpoint (Fig. submid) or, in the Newton variant, around a Newton root of
//                x(u, v) = o + tau d that is abandoned together with its neighbourhood
//                (Fig. subany). The search ends when the heap's top cannot beat the best tau.
//   k_trace_rays_redo  the rays whose local heap overflowed, traced again from the start with a
//                larger heap in global memory (the search is deterministic, so the result is
//                the one an unbounded heap gives).
//
// Sub-patches are cut from the patch's net by blossoming (each restricted curve's points are
// f(a,a,a), f(a,a,b), f(a,b,b), f(b,b,b), De Casteljau with one parameter per level) and only
// their box is kept: per coordinate the 4 theta1-curves are restricted, then the 4 theta2-curves,
// folded straight into the slab test. This file is compiled without mul-add contraction: each
// product and sum is rounded separately, in the order written, so every decision of the search
// (slab intervals, heap order, refinement, Newton convergence) is that of the same sequence of
// IEEE FP64 operations in any plain sequential program.
#include <cmath>

#include "common.cuh"

namespace bhem {
namespace {

constexpr double kEpsTau = 1e-9;     // refinement size (positions' units; unit directions)
constexpr double kNbhd = 1e-3;       // abandoned neighbourhood, fraction of the parameter extent
constexpr int kNewtonIters = 12;
constexpr int kMaxExpansions = 65536;
constexpr int kHeapCap = SHELL_RAY_HEAP;
constexpr int kNetBlock = 128;
constexpr int kRayBlock = 128;
constexpr int kRootChunk = 256;      // patch boxes staged in shared memory per pass
constexpr int kRedoThreads = 128;    // second pass: threads, each with a kRedoHeap-entry heap
constexpr int kRedoHeap = 8192;
constexpr int kRedoList = 65536;     // rays the second pass can take per call

__device__ __forceinline__ double lerp(double p, double q, double t) { return (1.0 - t) * p + t * q; }

// Bezier points of the cubic with points in[0..3] restricted to [a, b] (blossom values).
__device__ __forceinline__ void curve_restrict(const double in[4], double a, double b, double out[4]) {
  double A1[3], B1[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    A1[i] = lerp(in[i], in[i + 1], a);
    B1[i] = lerp(in[i], in[i + 1], b);
  }
  double AA[2], AB[2], BB[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    AA[i] = lerp(A1[i], A1[i + 1], a);
    AB[i] = lerp(A1[i], A1[i + 1], b);
    BB[i] = lerp(B1[i], B1[i + 1], b);
  }
  out[0] = lerp(AA[0], AA[1], a);
  out[1] = lerp(AA[0], AA[1], b);
  out[2] = lerp(AB[0], AB[1], b);
  out[3] = lerp(BB[0], BB[1], b);
}

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

__global__ void __launch_bounds__(kNetBlock) k_ray_nets(int np, const int4* __restrict__ pnodes,
                                                        const double* __restrict__ q, double dxi1, double dxi2,
                                                        double* __restrict__ nets, double* __restrict__ boxes) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int4 n4 = pnodes[p];
  const int nd[4] = {n4.x, n4.y, n4.z, n4.w};
  double* P = nets + (size_t)p * 48;
  for (int c = 0; c < 3; ++c) {
    double H[4][4];   // H[2 pu + r][2 pv + s]: theta1 end pu, derivative order r; theta2 likewise
#pragma unroll
    for (int pv = 0; pv < 2; ++pv)
#pragma unroll
      for (int pu = 0; pu < 2; ++pu) {
        const double* X = q + 12 * (size_t)nd[pu + 2 * pv];
        H[2 * pu][2 * pv] = X[c];
        H[2 * pu + 1][2 * pv] = X[3 + c] * dxi1;
        H[2 * pu][2 * pv + 1] = X[6 + c] * dxi2;
        H[2 * pu + 1][2 * pv + 1] = X[9 + c] * dxi1 * dxi2;
      }
    double U[4][4];   // along theta1 first, then theta2
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      U[0][b] = H[0][b];
      U[1][b] = H[0][b] + H[1][b] / 3.0;
      U[2][b] = H[2][b] - H[3][b] / 3.0;
      U[3][b] = H[2][b];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      P[16 * c + 4 * i + 0] = U[i][0];
      P[16 * c + 4 * i + 1] = U[i][0] + U[i][1] / 3.0;
      P[16 * c + 4 * i + 2] = U[i][2] - U[i][3] / 3.0;
      P[16 * c + 4 * i + 3] = U[i][2];
    }
  }
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

// Cubic Bernstein polynomials and their derivatives at t.
__device__ __forceinline__ void bernstein(double t, double B[4], double dB[4]) {
  const double s = 1.0 - t;
  B[0] = s * s * s;
  B[1] = 3.0 * t * s * s;
  B[2] = 3.0 * t * t * s;
  B[3] = t * t * t;
  dB[0] = -3.0 * s * s;
  dB[1] = 3.0 * s * (s - 2.0 * t);
  dB[2] = 3.0 * t * (2.0 * s - t);
  dB[3] = 3.0 * t * t;
}

// x(u, v), x_u, x_v of the net P ([c][i][j]): sums over j first, then i.
__device__ void bezier_eval(const double* __restrict__ P, double u, double v, double x[3], double xu[3],
                            double xv[3]) {
  double Bu[4], dBu[4], Bv[4], dBv[4];
  bernstein(u, Bu, dBu);
  bernstein(v, Bv, dBv);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double Q[4], R[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double* row = P + 16 * c + 4 * i;
      const double p0 = __ldg(row), p1 = __ldg(row + 1), p2 = __ldg(row + 2), p3 = __ldg(row + 3);
      Q[i] = ((Bv[0] * p0 + Bv[1] * p1) + Bv[2] * p2) + Bv[3] * p3;
      R[i] = ((dBv[0] * p0 + dBv[1] * p1) + dBv[2] * p2) + dBv[3] * p3;
    }
    x[c] = ((Bu[0] * Q[0] + Bu[1] * Q[1]) + Bu[2] * Q[2]) + Bu[3] * Q[3];
    xu[c] = ((dBu[0] * Q[0] + dBu[1] * Q[1]) + dBu[2] * Q[2]) + dBu[3] * Q[3];
    xv[c] = ((Bu[0] * R[0] + Bu[1] * R[1]) + Bu[2] * R[2]) + Bu[3] * R[3];
  }
}

__device__ __forceinline__ double det3(const double M[3][3]) {
  return (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
          M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])) +
         M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

// Newton's method on F(u, v, tau) = x(u, v) - o - tau d, Jacobian [x_u | x_v | -d] by Cramer's
// rule. True with the root in (u, v, tau) on convergence.
__device__ bool newton_root(const double* __restrict__ P, const double o[3], const double d[3], double on,
                            double& u, double& v, double& tau, int& iters) {
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
  }
  return false;
}

struct Cand {
  double t0, t1, ext, u0, u1, v0, v1;
  int patch;
};

// Binary min-heap on t0 (sift rules of a textbook binary heap) over caller-given storage: a
// local array in the first pass, a slice of library-owned global memory in the second.
struct Heap {
  Cand* a;
  int cap;
  int n = 0, peak = 0;
  int boxes = 0;       // candidate boxes formed (patch roots included)
  bool overflow = false;

  __device__ Heap(Cand* storage, int capacity) : a(storage), cap(capacity) {}

  __device__ void push(const Cand& c) {
    if (n == cap) {
      overflow = true;
      return;
    }
    int i = n++;
    if (n > peak) peak = n;
    while (i > 0) {
      const int parent = (i - 1) / 2;
      if (a[parent].t0 <= c.t0) break;
      a[i] = a[parent];
      i = parent;
    }
    a[i] = c;
  }

  __device__ Cand pop() {
    const Cand top = a[0], last = a[--n];
    int i = 0;
    for (;;) {
      const int l = 2 * i + 1, r = l + 1;
      int m = i;
      double km = last.t0;
      if (l < n && a[l].t0 < km) {
        m = l;
        km = a[l].t0;
      }
      if (r < n && a[r].t0 < km) m = r;
      if (m == i) break;
      a[i] = a[m];
      i = m;
    }
    if (n > 0) a[i] = last;
    return top;
  }
};

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

// Pushes the sub-patch [u0, u1] x [v0, v1] of patch p when the ray enters its box before best.
__device__ void push_sub(Heap& h, const double* __restrict__ P, int p, double u0, double u1, double v0, double v1,
                         const Ray& r, double best) {
  if (!(u1 > u0) || !(v1 > v0)) return;
  ++h.boxes;
  double lo = 0.0, hi = INFINITY, e = 0.0;
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    double mn, mx;
    sub_range(P, c, u0, u1, v0, v1, mn, mx);
    if (mx - mn > e) e = mx - mn;
    if (!slab(mn, mx, r.o[c], r.d[c], r.inv[c], lo, hi)) return;
  }
  if (lo > hi || lo >= best) return;
  h.push(Cand{lo, hi, e, u0, u1, v0, v1, p});
}

struct Hit {
  double tau = INFINITY, u = 0.0, v = 0.0;
  int patch = -1, nexp = 0, flags = 0, newton_iters = 0;
};

// The search over the candidates already in the heap; stops early once the heap overflows.
__device__ Hit search(Heap& h, const Ray& r, const double* __restrict__ nets, int use_newton) {
  Hit res;
  const double on = sqrt((r.o[0] * r.o[0] + r.o[1] * r.o[1]) + r.o[2] * r.o[2]);
  double best = INFINITY, bu = 0.0, bv = 0.0;
  int bp = -1, nexp = 0;
  while (h.n > 0 && !h.overflow) {
    const Cand c = h.pop();
    if (c.t0 >= best - kEpsTau) break;                               // nothing left can be closer
    if (c.ext <= kEpsTau || (c.u1 - c.u0 < 1e-13 && c.v1 - c.v0 < 1e-13)) {   // refined
      const double t = 0.5 * (c.t0 + c.t1);
      if (t < best - kEpsTau) {
        best = t;
        bp = c.patch;
        bu = 0.5 * (c.u0 + c.u1);
        bv = 0.5 * (c.v0 + c.v1);
      }
      continue;
    }
    if (nexp == kMaxExpansions) {
      res.flags |= SHELL_RAY_LIMIT;
      break;
    }
    ++nexp;
    const double* P = nets + (size_t)c.patch * 48;
    const double um = 0.5 * (c.u0 + c.u1), vm = 0.5 * (c.v0 + c.v1);
    if (use_newton) {
      double x[3], xu[3], xv[3];
      bezier_eval(P, um, vm, x, xu, xv);
      double u = um, v = vm;
      double t = ((x[0] - r.o[0]) * r.d[0] + (x[1] - r.o[1]) * r.d[1]) + (x[2] - r.o[2]) * r.d[2];
      if (newton_root(P, r.o, r.d, on, u, v, t, res.newton_iters) && u >= c.u0 && u <= c.u1 && v >= c.v0 && v <= c.v1 &&
          t >= 0.0) {
        if (t < best) {
          best = t;
          bp = c.patch;
          bu = u;
          bv = v;
        }
        // Fig. subany: drop [a1, a2] x [b1, b2] around the root, four rectangles remain
        const double hu = kNbhd * (c.u1 - c.u0), hv = kNbhd * (c.v1 - c.v0);
        const double a1 = fmax(c.u0, u - hu), a2 = fmin(c.u1, u + hu);
        const double b1 = fmax(c.v0, v - hv), b2 = fmin(c.v1, v + hv);
        push_sub(h, P, c.patch, c.u0, a1, b1, c.v1, r, best);
        push_sub(h, P, c.patch, a1, c.u1, b2, c.v1, r, best);
        push_sub(h, P, c.patch, c.u0, a2, c.v0, b1, r, best);
        push_sub(h, P, c.patch, a2, c.u1, c.v0, b2, r, best);
        continue;
      }
    }
    // Fig. submid: four quarters at the parameter midpoint
    push_sub(h, P, c.patch, c.u0, um, vm, c.v1, r, best);
    push_sub(h, P, c.patch, um, c.u1, vm, c.v1, r, best);
    push_sub(h, P, c.patch, c.u0, um, c.v0, vm, r, best);
    push_sub(h, P, c.patch, um, c.u1, c.v0, vm, r, best);
  }
  res.nexp = nexp;
  if (h.overflow) {
    res.flags |= SHELL_RAY_OVERFLOW;   // void: reported as a miss
  } else if (bp >= 0) {
    res.flags |= SHELL_RAY_HIT;
    res.tau = best;
    res.patch = bp;
    res.u = bu;
    res.v = bv;
  }
  return res;
}

struct RayOut {
  double* tau;
  int* patch;
  double* uv;
  int* flags;
  int* stats;
};

__device__ __forceinline__ void write_hit(const RayOut& out, long long k, const Hit& res, const Heap& h) {
  out.tau[k] = res.tau;
  out.patch[k] = res.patch;
  out.uv[2 * k] = res.u;
  out.uv[2 * k + 1] = res.v;
  out.flags[k] = res.flags;
  if (out.stats) {
    out.stats[4 * k] = res.nexp;
    out.stats[4 * k + 1] = h.peak;
    out.stats[4 * k + 2] = h.boxes;
    out.stats[4 * k + 3] = res.newton_iters;
  }
}

// First pass: one ray per thread, a kHeapCap-entry heap in local memory. A ray whose heap
// overflows stops and is appended to redo_list for the second pass (or, when the list is full,
// reported with SHELL_RAY_OVERFLOW).
__global__ void __launch_bounds__(kRayBlock) k_trace_rays(long long n, const double* __restrict__ origins,
                                                          const double* __restrict__ dirs, int np,
                                                          const double* __restrict__ nets,
                                                          const double* __restrict__ boxes, int use_newton,
                                                          RayOut out, int* __restrict__ redo_count,
                                                          int* __restrict__ redo_list) {
  __shared__ double sbox[kRootChunk * 8];
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = k < n;
  Ray r;
  Cand storage[kHeapCap];
  Heap h(storage, kHeapCap);
  if (active) load_ray(origins, dirs, k, r);
  // every patch's box in patch order; the whole CTA stages one chunk at a time
  for (int base = 0; base < np; base += kRootChunk) {
    const int m = min(kRootChunk, np - base);
    __syncthreads();
    for (int i = threadIdx.x; i < m * 8; i += blockDim.x) sbox[i] = boxes[(size_t)base * 8 + i];
    __syncthreads();
    if (!active) continue;
    for (int j = 0; j < m; ++j) root_push(h, sbox + 8 * j, base + j, r);
  }
  if (!active) return;
  h.boxes = np;
  const Hit res = search(h, r, nets, use_newton);
  if (h.overflow) {
    const int slot = atomicAdd(redo_count, 1);
    if (slot < kRedoList) {
      redo_list[slot] = (int)k;
      return;                                                         // written by the second pass
    }
  }
  write_hit(out, k, res, h);
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
  const int tid = threadIdx.x;
  const int count = min(*redo_count, kRedoList);
  for (int i = tid; i < count; i += kRedoThreads) {
    const long long k = redo_list[i];
    Ray r;
    load_ray(origins, dirs, k, r);
    Heap h(heaps + (size_t)tid * kRedoHeap, kRedoHeap);
    for (int p = 0; p < np; ++p) root_push(h, boxes + 8 * (size_t)p, p, r);
    h.boxes = np;
    const Hit res = search(h, r, nets, use_newton);
    write_hit(out, k, res, h);
  }
}

}  // namespace
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
  if (!s.d_ray_nets) {
    const size_t bytes = sizeof(double) * 56 * (size_t)np + sizeof(int) * (1 + kRedoList) +
                         sizeof(Cand) * (size_t)kRedoThreads * kRedoHeap;
    cudaError_t e = cudaMalloc(&s.d_ray_nets, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s.d_ray_nets = nullptr;
      return fail(SHELL_ERR_OOM, std::string("ray scratch: ") + cudaGetErrorString(e));
    }
  }
  // one allocation: second-pass heaps (at the 256-byte aligned base), nets, boxes, redo list
  Cand* heaps = (Cand*)s.d_ray_nets;
  double* nets = (double*)(heaps + (size_t)kRedoThreads * kRedoHeap);
  double* boxes = nets + 48 * (size_t)np;
  int* redo_count = (int*)(boxes + 8 * (size_t)np);
  int* redo_list = redo_count + 1;
  RayOut out{tau, patch, uv, flags, stats};
  BHEM_CUDA(cudaMemsetAsync(redo_count, 0, sizeof(int), s.stream));
  k_ray_nets<<<grid_for(np, kNetBlock), kNetBlock, 0, s.stream>>>(np, s.d_patch_nodes, q, s.grid.dxi1,
                                                                  s.grid.dxi2, nets, boxes);
  const int use_newton = variant == SHELL_RAY_NEWTON;
  k_trace_rays<<<(unsigned)((n_rays + kRayBlock - 1) / kRayBlock), kRayBlock, 0, s.stream>>>(
      n_rays, origins, dirs, np, nets, boxes, use_newton, out, redo_count, redo_list);
  k_trace_rays_redo<<<1, kRedoThreads, 0, s.stream>>>(origins, dirs, np, nets, boxes, use_newton, out, redo_count,
                                                      redo_list, heaps);
  s.launches += 3;
  BHEM_CUDA(cudaGetLastError());
  return SHELL_OK;
}
