// Device building blocks shared by the ray-patch intersection (rays.cu) and the point-patch
// continuous collision detection (ccd.cu) of Sec. 5: the Bezier net of a Hermite patch, cuts of
// a cubic to a parameter range by blossoming, Bezier evaluation, a 3x3 determinant, and the
// candidate heap. Files that include this header are compiled without mul-add contraction, so
// every product and sum here is rounded on its own, in the order written.
#pragma once

#include <cmath>

#include "bhem.h"

namespace bhem {
namespace bz {

constexpr double kNbhd = 1e-3;       // abandoned neighbourhood, fraction of the parameter extent
constexpr int kNewtonIters = 12;
constexpr int kMaxExpansions = 65536;
constexpr int kHeapCap = SHELL_RAY_HEAP;
constexpr int kRedoThreads = 128;    // global heaps: kRedoThreads of kRedoHeap candidates
constexpr int kRedoHeap = 8192;
constexpr int kRedoList = 65536;     // queries the second pass can take per call

// Bezier net P ([c][i][j], i along theta1) of the patch with corner nodes nd (00, 10, 01, 11):
// Hermite data b0 = a, b1 = a + a'/3, b2 = b - b'/3, b3 = b along theta1, then theta2;
// derivative DOFs scaled to the local parameters by dxi1, dxi2.
__device__ __forceinline__ void patch_net(const double* __restrict__ q, const int nd[4], double dxi1, double dxi2,
                                          double* __restrict__ P) {
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
}

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
static __device__ void bezier_eval(const double* __restrict__ P, double u, double v, double x[3], double xu[3],
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

struct Cand {
  double t0, t1, ext, u0, u1, v0, v1;
  int patch;
};

// Binary min-heap on t0 (sift rules of a textbook binary heap) over caller-given storage: a
// local array in the first pass, a slice of library-owned global memory in the second. A full
// first-pass heap moves itself into a free global slice (spill, kRedoThreads slices of kRedoHeap
// entries, claimed through *spill_count) and carries on; only when none is left does it report
// an overflow.
struct Heap {
  Cand* a;
  int cap;
  int n = 0, peak = 0;
  int boxes = 0;       // candidate boxes formed (patch roots included)
  bool overflow = false;
  Cand* spill = nullptr;
  int* spill_count = nullptr;

  __device__ Heap(Cand* storage, int capacity) : a(storage), cap(capacity) {}

  __device__ void push(const Cand& c) {
    if (n == cap) {
      if (spill) {
        const int slot = atomicAdd(spill_count, 1);
        if (slot < kRedoThreads) {
          Cand* g = spill + (size_t)slot * kRedoHeap;
          for (int i = 0; i < n; ++i) g[i] = a[i];
          a = g;
          cap = kRedoHeap;
        }
        spill = nullptr;
      }
      if (n == cap) {
        overflow = true;
        return;
      }
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

}  // namespace bz
}  // namespace bhem
