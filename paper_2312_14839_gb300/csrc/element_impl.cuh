// Device code shared by the element kernels of one shell (element.cu) and of a batch of shells
// (batch.cu): Hermite basis and Gauss rule (App. A), shape tables, 3-vector helpers, the
// Gauss-point matrices of App. B and the per-patch bodies of the element kernels.
#pragma once

#include "common.cuh"

namespace bhem {

// ------------------------------------------------------------------------------------------
// App. A.1 cubic Hermite basis on [0, 1] and its derivatives; App. A.2 Gauss rule.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double herm(int p, int r, double t, int d) {
  // f = 2t^3 - 3t^2 + 1, g = t^3 - 2t^2 + t; w_{0,0} = f(t), w_{1,0} = f(1-t),
  // w_{0,1} = g(t), w_{1,1} = -g(1-t)
  double s = p ? 1.0 - t : t;
  double sg = (p && (d & 1)) ? -1.0 : 1.0;   // chain rule of 1 - t
  double v;
  if (r == 0) v = d == 0 ? (2 * s - 3) * s * s + 1 : d == 1 ? 6 * s * s - 6 * s : 12 * s - 6;
  else        v = d == 0 ? ((s - 2) * s + 1) * s : d == 1 ? (3 * s - 4) * s + 1 : 6 * s - 4;
  if (r == 1 && p == 1) v = -v;
  return sg * v;
}

__device__ __forceinline__ void gauss_unit(double th[4], double wt[4]) {
  const double xi = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
  const double xo = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
  const double wi = (18.0 + sqrt(30.0)) / 72.0, wo = (18.0 - sqrt(30.0)) / 72.0;
  th[0] = 0.5 * (1 - xo); th[1] = 0.5 * (1 - xi); th[2] = 0.5 * (1 + xi); th[3] = 0.5 * (1 + xo);
  wt[0] = wo; wt[1] = wi; wt[2] = wi; wt[3] = wo;
}

// Shape table in shared memory: sphi[I * kPhiStride + k * 16 + g], k = 0..5 for
// Phi, Phi_,1, Phi_,2, Phi_,11, Phi_,22, Phi_,12; g = g2 * 4 + g1. The odd I-stride keeps both
// access patterns (lanes over g, lanes over I) free of bank conflicts.
constexpr int kPhiStride = 97;
constexpr int kPhiSize = 16 * kPhiStride;
constexpr int kPhiTable = kPhiSize + 16;   // + the 16 Gauss weights W_g = dxi1 dxi2 w_g1 w_g2

template <typename R>
__device__ void build_shape_table(R* sphi, double d1, double d2) {
  double th[4], wt[4];
  gauss_unit(th, wt);
  for (int e = threadIdx.x; e < 16 * 96; e += blockDim.x) {
    int I = e / 96, k = (e / 16) % 6, g = e % 16;
    int corner = I >> 2, kind = I & 3;
    int p = corner & 1, q = corner >> 1, r = kind & 1, s = kind >> 1;
    const int dd1[6] = {0, 1, 0, 2, 0, 1}, dd2[6] = {0, 0, 1, 0, 2, 1};
    double t1 = th[g & 3], t2 = th[g >> 2];
    double v = herm(p, r, t1, dd1[k]) * herm(q, s, t2, dd2[k]);
    v *= (r ? d1 : 1.0) * (s ? d2 : 1.0);
    for (int i = 0; i < dd1[k]; ++i) v /= d1;
    for (int i = 0; i < dd2[k]; ++i) v /= d2;
    sphi[I * kPhiStride + k * 16 + g] = (R)v;
  }
}

__device__ __forceinline__ double gauss_weight(int g, double d1, double d2) {
  double th[4], wt[4];
  gauss_unit(th, wt);
  return d1 * d2 * wt[g & 3] * wt[g >> 2];
}

template <typename R>
__device__ __forceinline__ void load_shape_table(R* sphi, const R* __restrict__ table) {
  for (int e = threadIdx.x; e < kPhiTable; e += blockDim.x) sphi[e] = table[e];
}

// ------------------------------------------------------------------------------------------
// 3-vector helpers
// ------------------------------------------------------------------------------------------
template <typename R> struct V3 { R x, y, z; };
template <typename R> __device__ __forceinline__ V3<R> mk(R a, R b, R c) { return {a, b, c}; }
template <typename R> __device__ __forceinline__ V3<R> operator+(V3<R> a, V3<R> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename R> __device__ __forceinline__ V3<R> operator-(V3<R> a, V3<R> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename R> __device__ __forceinline__ V3<R> operator*(R s, V3<R> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename R> __device__ __forceinline__ R dot(V3<R> a, V3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename R> __device__ __forceinline__ V3<R> cross(V3<R> a, V3<R> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename R> __device__ __forceinline__ R comp(V3<R> a, int i) { return i == 0 ? a.x : i == 1 ? a.y : a.z; }

// Interpolate the 5 derivative vectors a_1, a_2, a_{1,1}, a_{2,2}, a_{1,2} at Gauss point g from
// 16 DOF triples (shared memory, [16][3]).
template <typename R, typename S>
__device__ __forceinline__ void interp5(const R* sphi, const S* qv, int g, V3<R> out[5]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) out[k] = mk<R>(0, 0, 0);
#pragma unroll 4
  for (int I = 0; I < 16; ++I) {
    V3<R> v = mk<R>((R)qv[I * 3], (R)qv[I * 3 + 1], (R)qv[I * 3 + 2]);
#pragma unroll
    for (int k = 0; k < 5; ++k) out[k] = out[k] + sphi[I * kPhiStride + (k + 1) * 16 + g] * v;
  }
}

// ------------------------------------------------------------------------------------------
// 1D factors of the bicubic Hermite shape functions (Eq. hermite with the Delta-xi scaling of
// App. A.1): a shape function of corner (p, q) and kind (r, s) is w1[a](theta^1) w2[b](theta^2)
// with a = 2p + r, b = 2q + s, and its (d1, d2) parameter derivative is the product of the d1-th
// and d2-th derivatives of the factors. w[(d * 4 + g) * 4 + a] holds the d-th xi-derivative of
// factor a at Gauss abscissa g (d = 0, 1, 2): herm(p, r, theta_g, d) dxi^r / dxi^d.
// ------------------------------------------------------------------------------------------
constexpr int kHerm1D = 48;

template <typename R>
__device__ __forceinline__ void build_hermite_1d(R* w, double dxi, int tid, int nthreads) {
  double th[4], wt[4];
  gauss_unit(th, wt);
  for (int e = tid; e < kHerm1D; e += nthreads) {
    const int d = e / 16, gi = (e / 4) % 4, a = e % 4;
    const int p = a >> 1, r = a & 1;
    double v = herm(p, r, th[gi], d);
    if (r) v *= dxi;
    for (int i = 0; i < d; ++i) v /= dxi;
    w[e] = (R)v;
  }
}

// FP32 Hessian stage: per Gauss point g and DOF triple J the five derivative values phi_,k and
// the value phi, as sphg[(g * 16 + J) * 8 + l] (l = 0..4: phi_,1 .. phi_,12; 5: phi; 6, 7: 0),
// so that a lane reads them with two 16-byte loads.
constexpr int kPhiGauss = 16 * 16 * 8;

// Elements of the element kernels' shared memory before the per-warp areas: shape table, the two
// 1D factor tables (theta^1, theta^2) and, for FP32, the per-Gauss-point table sphg
template <typename R>
__host__ __device__ constexpr int elem_table_elems() {
  return ((kPhiTable + 3) & ~3) + 2 * kHerm1D + (sizeof(R) == 4 ? kPhiGauss : 0);
}

// Fills sphg from the shape table (FP32 kernels; all threads of the CTA, after sphi is complete).
__device__ __forceinline__ void build_phi_gauss(float* sphg, const float* sphi, int tid, int nthreads) {
  for (int e = tid; e < kPhiGauss; e += nthreads) {
    const int g = e >> 7, J = (e >> 3) & 15, l = e & 7;
    sphg[e] = l < 5 ? sphi[J * kPhiStride + (l + 1) * 16 + g] : (l == 5 ? sphi[J * kPhiStride + g] : 0.f);
  }
}

constexpr int kRestFields = 13;

// ------------------------------------------------------------------------------------------
// Light FP64 energy (and gradient) of one patch, half a warp per patch, lane = Gauss point
// g = 4 g2 + g1. The interpolation to the 4x4 Gauss points and the gradient's transpose are
// sum-factorised over the tensor-product basis: the 48 DOFs are first contracted along theta^1
// (T[d1][g1][b][c], 144 values), then along theta^2 per Gauss point; the gradient runs the two
// contractions in reverse. sq: the half warp's 48 DOFs, sT: its 144-value intermediate, sG: its
// [16][15] gradient vectors (all shared). restgp is SoA over S = (total patches) * 16 entries.
// Returns the patch energy in every lane.
// ------------------------------------------------------------------------------------------
constexpr int kEgPatches = 8;   // patches per CTA (128 threads)

// DOF index (corner * 12 + kind * 3 + c) of the factor pair (a, b), component c
__device__ __forceinline__ int dof_of(int a, int b, int c) {
  return ((a >> 1) + 2 * (b >> 1)) * 12 + ((a & 1) + 2 * (b & 1)) * 3 + c;
}

__device__ __forceinline__ double eg64_patch(const double* w1, const double* w2, double* sq, double* sT,
                                             double (*sG)[15], int p, bool active, int g, const int nd[4],
                                             const double* __restrict__ q,
                                             const double* __restrict__ dir, double step,
                                             const double* __restrict__ restgp, size_t S, double h,
                                             double* __restrict__ grad, int* err) {
  const int g1 = g & 3, g2 = g >> 2;
  if (active) {
    for (int l = g; l < 48; l += 16) {
      size_t a = (size_t)nd[l / 12] * 12 + (l % 12);
      double v = q[a];
      if (dir) v = __fma_rn(step, dir[a], v);
      sq[l] = v;
    }
  }
  __syncwarp();
  // theta^1 contraction: T[((d1 * 4 + gi) * 4 + b) * 3 + c] = sum_a w1[d1][gi][a] Q[a][b][c]
  if (active) {
    for (int e = g; e < 144; e += 16) {
      const int c = e % 3, b = (e / 3) % 4, dg = e / 12;   // dg = d1 * 4 + gi
      double t = 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) t = __fma_rn(w1[dg * 4 + a], sq[dof_of(a, b, c)], t);
      sT[e] = t;
    }
  }
  __syncwarp();
  double e = 0.0;
  if (active) {
    // theta^2 contraction at this Gauss point: (d1, d2) = (1,0), (0,1), (2,0), (0,2), (1,1)
    constexpr int kd1[5] = {1, 0, 2, 0, 1}, kd2[5] = {0, 1, 0, 2, 1};
    V3<double> v[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      double x = 0.0, y = 0.0, z = 0.0;
      const double* T = sT + (kd1[k] * 4 + g1) * 12;
      const double* W = w2 + (kd2[k] * 4 + g2) * 4;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        x = __fma_rn(W[b], T[b * 3 + 0], x);
        y = __fma_rn(W[b], T[b * 3 + 1], y);
        z = __fma_rn(W[b], T[b * 3 + 2], z);
      }
      v[k] = mk<double>(x, y, z);
    }
    const V3<double> a1 = v[0], a2 = v[1];
    const size_t o = (size_t)p * 16 + g;
    const double ab11 = restgp[0 * S + o], ab22 = restgp[1 * S + o], ab12 = restgp[2 * S + o];
    const double bb11 = restgp[3 * S + o], bb22 = restgp[4 * S + o], bb12 = restgp[5 * S + o];
    const double H00 = restgp[6 * S + o], H01 = restgp[7 * S + o], H02 = restgp[8 * S + o];
    const double H11 = restgp[9 * S + o], H12 = restgp[10 * S + o], H22 = restgp[11 * S + o];
    const double wgt = restgp[12 * S + o];
    V3<double> n = cross(a1, a2);
    // 1 / sqrt(a) by one reciprocal square root: no FP64 square root or divide on this path
    const double nn = dot(n, n);
    double isqa = 1.0;
    if (!(nn > 0.0)) atomicOr(err, ERRBIT_DEGENERATE);
    else isqa = rsqrt(nn);
    V3<double> a3 = isqa * n;
    double b11 = dot(v[2], a3), b22 = dot(v[3], a3), b12 = dot(v[4], a3);
    double al[3] = {0.5 * (dot(a1, a1) - ab11), 0.5 * (dot(a2, a2) - ab22), dot(a1, a2) - ab12};
    double be[3] = {b11 - bb11, b22 - bb22, 2.0 * (b12 - bb12)};
    double sg[3] = {H00 * al[0] + H01 * al[1] + H02 * al[2], H01 * al[0] + H11 * al[1] + H12 * al[2],
                    H02 * al[0] + H12 * al[1] + H22 * al[2]};
    double mm[3] = {H00 * be[0] + H01 * be[1] + H02 * be[2], H01 * be[0] + H11 * be[1] + H12 * be[2],
                    H02 * be[0] + H12 * be[1] + H22 * be[2]};
    const double h3 = h * h * h;
    e = wgt * (0.5 * h * (al[0] * sg[0] + al[1] * sg[1] + al[2] * sg[2]) +
               h3 * (1.0 / 24.0) * (be[0] * mm[0] + be[1] * mm[1] + be[2] * mm[2]));
    if (grad) {
      const double s = h3 * (1.0 / 12.0);
      V3<double> ct = mm[0] * v[2] + mm[1] * v[3] + (2.0 * mm[2]) * v[4];
      double bt = dot(ct, a3);
      V3<double> t1 = cross(a2, a3), t2 = cross(a3, a1);
      V3<double> e1 = isqa * (cross(a2, ct) - bt * t1);
      V3<double> e2 = isqa * (cross(ct, a1) - bt * t2);
      V3<double> G[5];
      G[0] = wgt * (h * (sg[0] * a1 + sg[2] * a2) + s * e1);
      G[1] = wgt * (h * (sg[1] * a2 + sg[2] * a1) + s * e2);
      G[2] = (wgt * s * mm[0]) * a3;
      G[3] = (wgt * s * mm[1]) * a3;
      G[4] = (wgt * s * 2.0 * mm[2]) * a3;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        sG[g][k * 3 + 0] = G[k].x;
        sG[g][k * 3 + 1] = G[k].y;
        sG[g][k * 3 + 2] = G[k].z;
      }
    }
  }
  // energy per patch over the 16 lanes of the half warp
  double ep = e;
  for (int o = 8; o > 0; o >>= 1) ep += __shfl_xor_sync(0xffffffffu, ep, o);
  __syncwarp();
  if (active && grad) {
    // transpose of the theta^2 contraction: U[d1][gi][b][c] = sum_g2 sum_{k: d1(k) = d1}
    // w2[d2(k)][g2][b] G_k(gi, g2)[c]; kinds with d1 = 0: (0,1), (0,2); d1 = 1: (1,0), (1,1); d1 = 2: (2,0)
    for (int e2 = g; e2 < 144; e2 += 16) {
      const int c = e2 % 3, b = (e2 / 3) % 4, gi = (e2 / 12) % 4, d1 = e2 / 48;
      const int ka = d1 == 0 ? 1 : d1 == 1 ? 0 : 2, da = d1 == 0 ? 1 : 0;
      const int kb = d1 == 0 ? 3 : 4, db = d1 == 0 ? 2 : 1;
      double u = 0.0;
#pragma unroll
      for (int gj = 0; gj < 4; ++gj) {
        u = __fma_rn(w2[(da * 4 + gj) * 4 + b], sG[gj * 4 + gi][ka * 3 + c], u);
        if (d1 < 2) u = __fma_rn(w2[(db * 4 + gj) * 4 + b], sG[gj * 4 + gi][kb * 3 + c], u);
      }
      sT[e2] = u;
    }
  }
  __syncwarp();
  if (active && grad) {
    // transpose of the theta^1 contraction: dE/dQ[a][b][c] = sum_{d1, gi} w1[d1][gi][a] U[d1][gi][b][c]
    for (int l = g; l < 48; l += 16) {
      const int corner = l / 12, kind = (l / 3) % 4, c = l % 3;
      const int a = 2 * (corner & 1) + (kind & 1), b = 2 * (corner >> 1) + (kind >> 1);
      double s = 0.0;
#pragma unroll
      for (int dg = 0; dg < 12; ++dg) s = __fma_rn(w1[dg * 4 + a], sT[(dg * 4 + b) * 3 + c], s);
      atomicAdd(&grad[(size_t)nd[corner] * 12 + kind * 3 + c], s);
    }
  }
  __syncwarp();
  return ep;
}

// ------------------------------------------------------------------------------------------
// Heavy kernel: one warp per patch computes E, gradient and the 48x48 Hessian.
// ------------------------------------------------------------------------------------------
template <typename R> struct ElemCfg;
template <> struct ElemCfg<float> { static constexpr int kWarps = 4, kJP = 8; };
template <> struct ElemCfg<double> { static constexpr int kWarps = 2, kJP = 4; };

// Packed upper triangle of a symmetric 15x15 matrix (120 entries), row-major.
constexpr int kSym15 = 120;
__device__ __forceinline__ int sym15(int i, int j) {
  if (i > j) { const int t = i; i = j; j = t; }
  return i * 15 - (i * (i - 1)) / 2 + (j - i);
}

// Component-pair block layout of M_g (tensor-core Hessian kernel): for the six pairs c <= d
// (index cd: (0,0) 0, (0,1) 1, (0,2) 2, (1,1) 3, (1,2) 4, (2,2) 5) the 5x5 matrix
// m^{cd}[k][l] = M_g[(k, c), (l, d)] over the derivative kinds, rows of 6 at cd * kBlk + 6 k + l
// (kBlk = 32: rows k, k + 1 of even k start 16-byte aligned). The pairs c > d are the transposes.
constexpr int kBlk = 32;
constexpr int kBlkRow = 6;
// floats per Gauss point: the six blocks (192) padded to 196, so that the 16 lanes that store the
// matrices of 16 Gauss points at once fall in 8 distinct banks
constexpr int kMbG = 6 * kBlk + 4;
__host__ __device__ constexpr int cd_index(int x, int y) { return x * 3 - (x * (x - 1)) / 2 + (y - x); }
struct BlkOff { int a, b; };
// Offsets of the entry M[(K1, x), (L1, y)] in the block layout, and of its mirror in a diagonal
// block (-1: none)
__host__ __device__ constexpr BlkOff blk_off(int K1, int x, int L1, int y) {
  return x < y   ? BlkOff{cd_index(x, y) * kBlk + K1 * kBlkRow + L1, -1}
         : x > y ? BlkOff{cd_index(y, x) * kBlk + L1 * kBlkRow + K1, -1}
                 : BlkOff{cd_index(x, x) * kBlk + K1 * kBlkRow + L1,
                          K1 != L1 ? cd_index(x, x) * kBlk + L1 * kBlkRow + K1 : -1};
}

// Row stride of T: FP32 rows are padded to 52 (16-byte aligned, and the rows that 8 lanes read
// together with 16-byte loads fall in distinct banks).
template <typename R> struct TStride { static constexpr int v = 45; };
template <> struct TStride<float> { static constexpr int v = 52; };

template <typename R>
struct WarpSmem {
  R u[48];        // displacement q - rest
  R qb[48];       // rest DOFs
  R M[16][kSym15];   // M_g per Gauss point (symmetric 15x15, packed upper triangle)
  R T[16 * TStride<R>::v];   // T[I][c*15 + l*3 + c'] of the current Gauss point
  R G[16][15];    // gradient vectors per Gauss point
  R ms[16];       // mass_scale * rho h * W sqrt(a_bar) per Gauss point
  R en[16];       // energy per Gauss point
};

struct ElemArgs {
  int np;
  const void* phi;         // shape table + Gauss weights in the kernel's precision
  const int4* pnodes;
  const int* plist;        // optional patch list (colour order), else identity
  int plist_n;
  const int* pblocks;
  const double* q;
  const double* rest;
  double d1, d2, lam, mu, h, rho_h, mass_scale;
  int pseudo;
  double* energy_p;
  double* grad_p;
  void* hess_p;
  int hess_vec;            // hess_p is 16-byte aligned (FP32 Hessians stored as float4)
  void* bsr;
  int bsr_atomic;
  int* err;
  // FP64 energy and gradient at the same q in the same warps (FP32 kernel only; grad64 null: off):
  // energy64[p] = E_p, grad64 += dE/dq (zeroed by the caller); restgp: rest Gauss-point data [13][np][16]
  const double* restgp;
  double* energy64;
  double* grad64;
};

// Builds M_g (15x15) and the per-point energy, gradient vectors and mass weight for Gauss
// point g of the warp's patch. kSplit = false (FP64 kernel): lanes 0..15, lane = g, every block.
// kSplit = true (FP32 kernel): all 32 lanes, lane g and lane g + 16 share Gauss point g. The
// energy is unchanged when the two parameter directions are exchanged, so its Hessian
// blocks of the exchanged frame are those of the original one with the derivative kinds relabeled
// (xi^1 <-> xi^2: a_1 <-> a_2, x_,11 <-> x_,22, x_,12 fixed; sigma(k) = 1, 0, 3, 2, 4). Half 0 (the
// original frame) computes the blocks (k, l), k <= l, with k in {0, 2, 4}; half 1 runs the same
// instructions in the exchanged frame, which gives the blocks (sigma(k), sigma(l)) with k in
// {1, 3}: together all 15 blocks. Half 1 discards the three blocks that map onto themselves
// ((0, 1), (2, 3), (4, 4)) and the by-products (energy, gradient vectors, mass weight).
template <typename R, bool kSplit, bool kBlocks = false, class WS = WarpSmem<R>>
__device__ __forceinline__ void gauss_point_matrix(const R* sphi, WS& W, int g, int half,
                                                   const ElemArgs& A) {
  V3<R> ub[5], uu[5];   // rest a_bar_1, a_bar_2, x_bar_{,11}, x_bar_{,22}, x_bar_{,12}; displacement derivatives
  if constexpr (kSplit) {
    // both halves need both fields at the same Gauss point: half 0 interpolates the rest DOFs,
    // half 1 the displacement, and they exchange (lane g <-> g + 16)
    V3<R> mine[5];
    interp5<R, R>(sphi, half ? W.u : W.qb, g, mine);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const V3<R> other = mk<R>(__shfl_xor_sync(0xffffffffu, mine[k].x, 16),
                                __shfl_xor_sync(0xffffffffu, mine[k].y, 16),
                                __shfl_xor_sync(0xffffffffu, mine[k].z, 16));
      ub[k] = half ? other : mine[k];
      uu[k] = half ? mine[k] : other;
    }
  } else {
    interp5<R, R>(sphi, W.qb, g, ub);
    interp5<R, R>(sphi, W.u, g, uu);
  }
  {
    // half 1: exchange the parameter directions (selects, no divergent branch)
    const bool x = half != 0;
    const V3<R> b0 = ub[0], b2 = ub[2], d0 = uu[0], d2 = uu[2];
    ub[0] = x ? ub[1] : b0;
    ub[1] = x ? b0 : ub[1];
    ub[2] = x ? ub[3] : b2;
    ub[3] = x ? b2 : ub[3];
    uu[0] = x ? uu[1] : d0;
    uu[1] = x ? d0 : uu[1];
    uu[2] = x ? uu[3] : d2;
    uu[3] = x ? d2 : uu[3];
  }
  const V3<R> ab1 = ub[0], ab2 = ub[1];
  const V3<R> a1 = ab1 + uu[0], a2 = ab2 + uu[1];
  V3<R> c[3] = {ub[2] + uu[2], ub[3] + uu[3], ub[4] + uu[4]};
  // rest metric, contravariant metric, Voigt H (App. B.1)
  R ab11 = dot(ab1, ab1), ab22 = dot(ab2, ab2), ab12 = dot(ab1, ab2);
  R det = ab11 * ab22 - ab12 * ab12;
  if (!(det > (R)0)) { atomicOr(A.err, ERRBIT_DEGENERATE); det = (R)1; }
  R sqab = sqrt(det);
  V3<R> ab3 = ((R)1 / sqab) * cross(ab1, ab2);
  // one reciprocal each for det and sqrt(a), then products (the M_g loop below would otherwise
  // divide by sqrt(a) 54 times)
  const R idet = (R)1 / det;
  R ai11 = ab22 * idet, ai22 = ab11 * idet, ai12 = -ab12 * idet;
  const R lam = (R)A.lam, mu = (R)A.mu, h = (R)A.h;
  R H[3][3];
  H[0][0] = (lam + 2 * mu) * ai11 * ai11;
  H[0][1] = lam * ai11 * ai22 + 2 * mu * ai12 * ai12;
  H[0][2] = (lam + 2 * mu) * ai11 * ai12;
  H[1][1] = (lam + 2 * mu) * ai22 * ai22;
  H[1][2] = (lam + 2 * mu) * ai12 * ai22;
  H[2][2] = (lam + mu) * ai12 * ai12 + mu * ai11 * ai22;
  H[1][0] = H[0][1]; H[2][0] = H[0][2]; H[2][1] = H[1][2];
  // deformed normal
  V3<R> n = cross(a1, a2);
  R sqa = sqrt(dot(n, n));
  if (!(sqa > (R)0)) { atomicOr(A.err, ERRBIT_DEGENERATE); sqa = (R)1; }
  const R isqa = (R)1 / sqa;
  V3<R> a3 = isqa * n;
  // strains from displacements (a_ab - a_bar_ab = a_bar_a.u_b + u_a.a_bar_b + u_a.u_b)
  R al[3] = {dot(ab1, uu[0]) + (R)0.5 * dot(uu[0], uu[0]), dot(ab2, uu[1]) + (R)0.5 * dot(uu[1], uu[1]),
             dot(ab1, uu[1]) + dot(uu[0], ab2) + dot(uu[0], uu[1])};
  V3<R> da3 = a3 - ab3;
  R br[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) br[m] = dot(uu[2 + m], a3) + dot(ub[2 + m], da3);   // b - b_bar
  R be[3] = {br[0], br[1], (R)2 * br[2]};
  R sg[3], mm[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    sg[i] = H[i][0] * al[0] + H[i][1] * al[1] + H[i][2] * al[2];
    mm[i] = H[i][0] * be[0] + H[i][1] * be[1] + H[i][2] * be[2];
  }
  const R wgt = sphi[kPhiSize + g] * sqab;
  const R s = h * h * h * ((R)1 / (R)12);
  if (!half) {
    W.en[g] = wgt * ((R)0.5 * h * (al[0] * sg[0] + al[1] * sg[1] + al[2] * sg[2]) +
                     s * (R)0.5 * (be[0] * mm[0] + be[1] * mm[1] + be[2] * mm[2]));
    W.ms[g] = (R)(A.mass_scale * A.rho_h) * wgt;
  }
  // first derivatives: B matrices (rows = Voigt component, columns = coordinate)
  V3<R> t1 = cross(a2, a3), t2 = cross(a3, a1);
  V3<R> up[3], vp[3];
  R bdef[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    bdef[m] = dot(c[m], a3);
    up[m] = isqa * (cross(a2, c[m]) - bdef[m] * t1);   // coefficient of Phi_,1 in d b_m
    vp[m] = isqa * (cross(c[m], a1) - bdef[m] * t2);   // coefficient of Phi_,2 in d b_m
  }
  V3<R> Ba[2][3] = {{a1, mk<R>(0, 0, 0), a2}, {mk<R>(0, 0, 0), a2, a1}};
  V3<R> Bb[5][3] = {{up[0], up[1], (R)2 * up[2]},
                    {vp[0], vp[1], (R)2 * vp[2]},
                    {a3, mk<R>(0, 0, 0), mk<R>(0, 0, 0)},
                    {mk<R>(0, 0, 0), a3, mk<R>(0, 0, 0)},
                    {mk<R>(0, 0, 0), mk<R>(0, 0, 0), (R)2 * a3}};
  // gradient vectors G_k = W sqrt(a_bar) (h B_alpha,k^T sigma + s B_beta,k^T m)
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    V3<R> gk = mm[0] * Bb[k][0] + mm[1] * Bb[k][1] + mm[2] * Bb[k][2];
    gk = s * gk;
    if (k < 2) gk = gk + h * (sg[0] * Ba[k][0] + sg[1] * Ba[k][1] + sg[2] * Ba[k][2]);
    gk = wgt * gk;
    if (!half) {
      W.G[g][k * 3 + 0] = gk.x;
      W.G[g][k * 3 + 1] = gk.y;
      W.G[g][k * 3 + 2] = gk.z;
    }
  }
  // Q_l = H B_l
  V3<R> Qa[2][3], Qb[5][3];
#pragma unroll
  for (int l = 0; l < 5; ++l)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Qb[l][i] = H[i][0] * Bb[l][0] + H[i][1] * Bb[l][1] + H[i][2] * Bb[l][2];
      if (l < 2) Qa[l][i] = H[i][0] * Ba[l][0] + H[i][1] * Ba[l][1] + H[i][2] * Ba[l][2];
    }
  // exact-Hessian extras: P_1, P_2 (d a3 = (Phi_,1 P_1 + Phi_,2 P_2) dq) and D~^{gamma delta}
  const bool exact = !A.pseudo;
  V3<R> ct = mm[0] * c[0] + mm[1] * c[1] + ((R)2 * mm[2]) * c[2];
  R bt = dot(ct, a3);
  V3<R> s1 = cross(ct, a1), s2 = cross(a2, ct);
  const R ia = isqa * isqa;
  const R a11 = dot(a1, a1), a22 = dot(a2, a2), a12 = dot(a1, a2);
  const R coef[3] = {mm[0], mm[1], (R)2 * mm[2]};
  R* M;
  if constexpr (kBlocks) M = W.Mb[g];
  else M = W.M[g];
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int l = k; l < 5; ++l)
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) {
          if (kSplit && (k == 1 || k == 3)) continue;   // half 1 produces these in the exchanged frame
          if (k == l && y < x) continue;
          R v = s * (comp(Bb[k][0], x) * comp(Qb[l][0], y) + comp(Bb[k][1], x) * comp(Qb[l][1], y) +
                     comp(Bb[k][2], x) * comp(Qb[l][2], y));
          if (k < 2 && l < 2)
            v += h * (comp(Ba[k][0], x) * comp(Qa[l][0], y) + comp(Ba[k][1], x) * comp(Qa[l][1], y) +
                      comp(Ba[k][2], x) * comp(Qa[l][2], y));
          R id = (x == y) ? (R)1 : (R)0;
          // (H alpha)_i d^2 alpha_i
          if (k == 0 && l == 0) v += h * sg[0] * id;
          if (k == 1 && l == 1) v += h * sg[1] * id;
          if (k == 0 && l == 1) v += h * sg[2] * id;
          if (exact) {
            // D~ blocks (App. B.2 with c = c~, beta_{ab} = c~ . a3)
            if (k == 0 && l == 0)
              v += s * ia * (bt * ((R)3 * comp(t1, x) * comp(t1, y) + comp(a2, x) * comp(a2, y) - a22 * id) -
                             comp(s2, x) * comp(t1, y) - comp(t1, x) * comp(s2, y));
            if (k == 1 && l == 1)
              v += s * ia * (bt * ((R)3 * comp(t2, x) * comp(t2, y) + comp(a1, x) * comp(a1, y) - a11 * id) -
                             comp(s1, x) * comp(t2, y) - comp(t2, x) * comp(s1, y));
            if (k == 0 && l == 1) {
              // -sqrt(a) [c~]: [v]_{xy} = eps_{x j y} v_j
              R cx = (x == 0 && y == 1) ? -ct.z : (x == 0 && y == 2) ? ct.y : (x == 1 && y == 0) ? ct.z :
                     (x == 1 && y == 2) ? -ct.x : (x == 2 && y == 0) ? -ct.y : (x == 2 && y == 1) ? ct.x : (R)0;
              v += s * ia * (bt * ((R)3 * comp(t1, x) * comp(t2, y) - (R)2 * comp(a1, x) * comp(a2, y) +
                                   comp(a2, x) * comp(a1, y) + a12 * id) -
                             comp(s2, x) * comp(t2, y) - comp(t1, x) * comp(s1, y) - sqa * cx);
            }
            // Phi~^I d a3/dq_J + Phi~^J (d a3/dq_I)^T, stored in the (l in {1,2}, k' in {11,22,12})
            // upper blocks as the transpose: entry [x][y] = coef_{k'} P_l[y][x]
            if (k < 2 && l >= 2) {
              // P_1 = (-[a2] - a3 (x) t1)/sqrt(a), P_2 = ([a1] - a3 (x) t2)/sqrt(a); need P_k[y][x]
              V3<R> av = (k == 0) ? a2 : a1;
              R sgn = (k == 0) ? (R)-1 : (R)1;
              V3<R> tv = (k == 0) ? t1 : t2;
              R cxm = (y == 0 && x == 1) ? -av.z : (y == 0 && x == 2) ? av.y : (y == 1 && x == 0) ? av.z :
                      (y == 1 && x == 2) ? -av.x : (y == 2 && x == 0) ? -av.y : (y == 2 && x == 1) ? av.x : (R)0;
              R Pyx = (sgn * cxm - comp(a3, y) * comp(tv, x)) * isqa;
              v += s * coef[l - 2] * Pyx;
            }
          }
          v *= wgt;
          // sigma: the kind index in the original frame of a kind of the exchanged frame
          constexpr int kSig[5] = {1, 0, 3, 2, 4};
          const bool self_mirror = (k == 0 && l == 1) || (k == 2 && l == 3) || (k == 4 && l == 4);
          if constexpr (kBlocks) {
            const BlkOff o0 = blk_off(k, x, l, y), o1 = blk_off(kSig[k], x, kSig[l], y);
            if (!half) {
              M[o0.a] = v;
              if (o0.b >= 0) M[o0.b] = v;
            } else if (!self_mirror) {
              M[o1.a] = v;
              if (o1.b >= 0) M[o1.b] = v;
            }
          } else {
            if (!half) M[sym15(k * 3 + x, l * 3 + y)] = v;
            else if (!self_mirror) M[sym15(kSig[k] * 3 + x, kSig[l] * 3 + y)] = v;
          }
        }
}

template <typename R>
__device__ __forceinline__ void atomic_add_row12(R* dst, const R* v);

template <>
__device__ __forceinline__ void atomic_add_row12<float>(float* dst, const float* v) {
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int i = 0; i < 3; ++i) atomicAdd(d4 + i, make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
}
template <>
__device__ __forceinline__ void atomic_add_row12<double>(double* dst, const double* v) {
#pragma unroll
  for (int i = 0; i < 12; ++i) atomicAdd(dst + i, v[i]);
}

template <typename R>
__device__ __forceinline__ void plain_add_row12(R* dst, const R* v) {
#pragma unroll
  for (int i = 0; i < 12; ++i) dst[i] += v[i];
}

// T = Phi_g^T M_g for Gauss point g = 4 g2 + g1: T[I * 45 + c * 15 + l * 3 + c'] =
// sum_k phi_k^I(g) M_g[(k, c), (l, c')] for the 16 DOF triples I. With the tensor-product basis,
// phi_k^I = w1[d1(k)][g1][a] w2[d2(k)][g2][b] (I = corner (p + 2q) * 4 + kind (r + 2s),
// a = 2p + r, b = 2q + s): each lane takes whole (c, l, c') columns, loads the 5 M values of a
// column once, contracts along theta^2 and then theta^1 in registers, and writes 16 T values.
template <typename R>
__device__ __forceinline__ void t_stage(const R* w1d, const R* Mg, R* T, int g, int lane) {
  const int g1 = g & 3, g2 = g >> 2;
  R W1[3][4], W2[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      W1[d][a] = w1d[(d * 4 + g1) * 4 + a];
      W2[d][a] = w1d[kHerm1D + (d * 4 + g2) * 4 + a];
    }
  for (int col = lane; col < 45; col += 32) {
    const int c = col / 15, l = (col / 3) % 5, cp = col % 3;
    R m[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) m[k] = Mg[sym15(k * 3 + c, l * 3 + cp)];
    // kinds k = (d1, d2): 0 (1,0), 1 (0,1), 2 (2,0), 3 (0,2), 4 (1,1); V[d1][b] = sum over the
    // kinds with that d1 of w2[d2][g2][b] M_k
    R V[3][4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      V[0][b] = W2[1][b] * m[1] + W2[2][b] * m[3];
      V[1][b] = W2[0][b] * m[0] + W2[1][b] * m[4];
      V[2][b] = W2[0][b] * m[2];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int I = ((a >> 1) + 2 * (b >> 1)) * 4 + ((a & 1) + 2 * (b & 1));
        T[I * TStride<R>::v + col] = W1[0][a] * V[0][b] + W1[1][a] * V[1][b] + W1[2][a] * V[2][b];
      }
  }
}

// FP32 Hessian K = sum_g Phi_g^T M_g Phi_g of one patch from its upper node-corner blocks. K is
// symmetric, so a lane computes the 3x3 blocks (I, J) of one DOF triple I against the J of its
// own corner and of the later ones only: 136 of the 256 (I, J) pairs in a lane map of at most 6
// J per lane (rows of corner 0: 3 lanes of 6, 6, 4 J; corner 1: 2 lanes of 6; corner 2: 2 lanes
// of 4; corner 3: 1 lane of 4). The blocks, and the transposes of those in a later corner, are
// staged in shared memory over the Gauss-point matrices (no longer needed), from which the
// unassembled Hessian and the BSR rows are written as before.
constexpr int kKStride = 52;   // row stride of the staged 48 x 48 Hessian (16-byte aligned rows)

// Writes one patch's FP32 Hessian, staged in shared memory as K[(I, c) * kKStride + (J, c')], to
// the unassembled output and/or scatters it into the BSR values (one warp).
__device__ __forceinline__ void store_staged_hessian32(const float* K, int p, const ElemArgs& A, int lane) {
  if (A.hess_p && A.hess_vec) {
    // 16-byte pieces: staged rows of 52 floats and output rows of 48 both start 16-byte aligned
    // (the output when its base is, which the host checked)
    float4* Hp = reinterpret_cast<float4*>(reinterpret_cast<float*>(A.hess_p) + (size_t)p * 2304);
    for (int e = lane; e < 576; e += 32)
      Hp[e] = *reinterpret_cast<const float4*>(K + (e / 12) * kKStride + (e % 12) * 4);
  } else if (A.hess_p) {
    float* Hp = reinterpret_cast<float*>(A.hess_p) + (size_t)p * 2304;
    for (int e = lane; e < 2304; e += 32) Hp[e] = K[(e / 48) * kKStride + e % 48];
  }
  if (A.bsr) {
    // lane (I, h): rows (I, c) of the node blocks (I >> 2, b), b = 2h, 2h + 1, 12 entries each
    float* V = reinterpret_cast<float*>(A.bsr);
    const int I = lane >> 1, h = lane & 1, a = I >> 2, r = I & 3;
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
      const int b = 2 * h + bb;
      const int kb = A.pblocks[p * 16 + a * 4 + b];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4* src = reinterpret_cast<const float4*>(K + (I * 3 + c) * kKStride + b * 12);
        float row[12];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float4 v4 = src[q];
          row[4 * q] = v4.x;
          row[4 * q + 1] = v4.y;
          row[4 * q + 2] = v4.z;
          row[4 * q + 3] = v4.w;
        }
        float* dst = V + (size_t)kb * 144 + (r * 3 + c) * 12;
        if (A.bsr_atomic) atomic_add_row12<float>(dst, row);
        else plain_add_row12<float>(dst, row);
      }
    }
  }
  __syncwarp();
}

__device__ __forceinline__ void hessian_sym32(const float* sphi, const float* w1d, const float* sphg,
                                              WarpSmem<float>& W, int p, const ElemArgs& A, int lane) {
  static_assert(sizeof(W.M) + sizeof(W.T) >= sizeof(float) * 48 * kKStride, "staging area");
  constexpr int JS = 6;
  int Is, Js, nJ;
  if (lane < 12) {
    Is = lane / 3;
    Js = 6 * (lane % 3);
    nJ = lane % 3 == 2 ? 4 : 6;
  } else if (lane < 20) {
    Is = 4 + (lane - 12) / 2;
    Js = 4 + 6 * ((lane - 12) % 2);
    nJ = 6;
  } else if (lane < 28) {
    Is = 8 + (lane - 20) / 2;
    Js = 8 + 4 * ((lane - 20) % 2);
    nJ = 4;
  } else {
    Is = 12 + (lane - 28);
    Js = 12;
    nJ = 4;
  }
  float acc[JS][9];
#pragma unroll
  for (int j = 0; j < JS; ++j)
#pragma unroll
    for (int e = 0; e < 9; ++e) acc[j][e] = 0.f;
#pragma unroll 1
  for (int g = 0; g < 16; ++g) {
    t_stage<float>(w1d, W.M[g], W.T, g, lane);
    __syncwarp();
    // row Is of T: 11 16-byte loads and one 4-byte load of the padded row
    float Tr[45];
    const float4* t4 = reinterpret_cast<const float4*>(W.T + Is * TStride<float>::v);
#pragma unroll
    for (int e4 = 0; e4 < 11; ++e4) {
      const float4 v4 = t4[e4];
      Tr[4 * e4] = v4.x;
      Tr[4 * e4 + 1] = v4.y;
      Tr[4 * e4 + 2] = v4.z;
      Tr[4 * e4 + 3] = v4.w;
    }
    Tr[44] = W.T[Is * TStride<float>::v + 44];
    const float mI = W.ms[g] * sphi[Is * kPhiStride + g];
#pragma unroll
    for (int j = 0; j < JS; ++j) {
      if (j >= nJ) break;
      const float4* q4 = reinterpret_cast<const float4*>(sphg + (g * 16 + Js + j) * 8);
      const float4 a4 = q4[0], b4 = q4[1];
      const float pj[5] = {a4.x, a4.y, a4.z, a4.w, b4.x};
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int cp = 0; cp < 3; ++cp) {
          float sacc = acc[j][c * 3 + cp];
#pragma unroll
          for (int l = 0; l < 5; ++l) sacc += Tr[c * 15 + l * 3 + cp] * pj[l];
          acc[j][c * 3 + cp] = sacc;
        }
      const float mm = mI * b4.y;
      acc[j][0] += mm;
      acc[j][4] += mm;
      acc[j][8] += mm;
    }
    __syncwarp();
  }
  // stage: K[(I, c)][(J, c')], row stride kKStride, over M and T
  float* K = &W.M[0][0];
#pragma unroll
  for (int j = 0; j < JS; ++j) {
    if (j >= nJ) break;
    const int J = Js + j;
    const bool mirror = (J >> 2) != (Is >> 2);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int cp = 0; cp < 3; ++cp) {
        const float v = acc[j][c * 3 + cp];
        K[(Is * 3 + c) * kKStride + J * 3 + cp] = v;
        if (mirror) K[(J * 3 + cp) * kKStride + Is * 3 + c] = v;
      }
  }
  __syncwarp();
  store_staged_hessian32(K, p, A, lane);
}

// Gathers the warp's patch: displacement u = q - rest and rest DOFs qb (shared memory).
template <typename R, class WS>
__device__ __forceinline__ void gather_patch(WS& W, int p, const ElemArgs& A, int lane) {
  const int4 pn = A.pnodes[p];
  const int nd[4] = {pn.x, pn.y, pn.z, pn.w};
  // Value DOFs enter only through derivatives, whose value-kind shape functions sum to zero
  // (partition of unity); subtracting corner 00's value in FP64 before rounding removes the
  // O(|x| / dxi) cancellation of the derivative interpolation from the R arithmetic.
  for (int l = lane; l < 48; l += 32) {
    const int kk = l % 12;
    size_t a = (size_t)nd[l / 12] * 12 + kk;
    double qv = A.q[a], rv = A.rest[a];
    if (kk < 3) {
      const size_t a0 = (size_t)nd[0] * 12 + kk;
      const double q0 = A.q[a0], r0 = A.rest[a0];
      W.u[l] = (R)((qv - rv) - (q0 - r0));
      W.qb[l] = (R)(rv - r0);
    } else {
      W.u[l] = (R)(qv - rv);
      W.qb[l] = (R)rv;
    }
  }
}

// Energy and gradient of the patch in the kernel's precision (by-products of the Gauss-point
// matrices: per-point energies W.en and gradient vectors W.G).
template <typename R, class WS>
__device__ __forceinline__ void patch_byproducts(const R* sphi, const WS& W, int p, const ElemArgs& A, int lane) {
  if (A.energy_p) {
    R e = lane < 16 ? W.en[lane] : (R)0;
    for (int o = 8; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) A.energy_p[p] = (double)e;
  }
  if (A.grad_p) {
    for (int l = lane; l < 48; l += 32) {
      int Ig = l / 3, c = l % 3;
      R sacc = 0;
      for (int g = 0; g < 16; ++g)
#pragma unroll
        for (int k = 0; k < 5; ++k) sacc += sphi[Ig * kPhiStride + (k + 1) * 16 + g] * W.G[g][k * 3 + c];
      A.grad_p[(size_t)p * 48 + l] = (double)sacc;
    }
  }
}

// One patch by one warp: gather, Gauss-point matrices M_g, energy/gradient by-products, and the
// Hessian K = sum_g phi_g^T M_g phi_g written unassembled and/or scattered into the BSR.
template <typename R>
__device__ __forceinline__ void element_patch(const R* sphi, const R* w1d, const R* sphg, WarpSmem<R>& W, int p,
                                              const ElemArgs& A, int lane) {
  constexpr int JP = ElemCfg<R>::kJP;          // J columns per pass (16 / 2 / JP passes)
  const int I = lane >> 1, h = lane & 1;
  gather_patch<R>(W, p, A, lane);
  __syncwarp();
  if constexpr (sizeof(R) == 4) gauss_point_matrix<R, true>(sphi, W, lane & 15, lane >> 4, A);
  else if (lane < 16) gauss_point_matrix<R, false>(sphi, W, lane, 0, A);
  __syncwarp();
  patch_byproducts<R>(sphi, W, p, A, lane);

  const bool want_h = A.hess_p || A.bsr;
  if constexpr (sizeof(R) == 4) {
    if (want_h) hessian_sym32(sphi, w1d, sphg, reinterpret_cast<WarpSmem<float>&>(W), p, A, lane);
  } else if (want_h) {
#pragma unroll 1
    for (int pass = 0; pass < 8 / JP; ++pass) {
      R acc[JP][9];
#pragma unroll
      for (int j = 0; j < JP; ++j)
#pragma unroll
        for (int e = 0; e < 9; ++e) acc[j][e] = (R)0;
      const int J0 = 8 * h + pass * JP;
#pragma unroll 1
      for (int g = 0; g < 16; ++g) {
        t_stage<R>(w1d, W.M[g], W.T, g, lane);
        __syncwarp();
        R Tr[45];
        if constexpr (sizeof(R) == 4) {
          // 11 16-byte loads and one 4-byte load of the padded row
          const float4* t4 = reinterpret_cast<const float4*>(W.T + I * TStride<R>::v);
#pragma unroll
          for (int e4 = 0; e4 < 11; ++e4) {
            const float4 v4 = t4[e4];
            Tr[4 * e4] = v4.x;
            Tr[4 * e4 + 1] = v4.y;
            Tr[4 * e4 + 2] = v4.z;
            Tr[4 * e4 + 3] = v4.w;
          }
          Tr[44] = W.T[I * TStride<R>::v + 44];
        } else {
#pragma unroll
          for (int e = 0; e < 45; ++e) Tr[e] = W.T[I * TStride<R>::v + e];
        }
        const R mI = W.ms[g] * sphi[I * kPhiStride + g];
#pragma unroll
        for (int j = 0; j < JP; ++j) {
          const int J = J0 + j;
          R pj[5], phJ;
          if constexpr (sizeof(R) == 4) {
            const float4* q4 = reinterpret_cast<const float4*>(sphg + (g * 16 + J) * 8);
            const float4 a4 = q4[0], b4 = q4[1];
            pj[0] = a4.x;
            pj[1] = a4.y;
            pj[2] = a4.z;
            pj[3] = a4.w;
            pj[4] = b4.x;
            phJ = b4.y;
          } else {
#pragma unroll
            for (int l = 0; l < 5; ++l) pj[l] = sphi[J * kPhiStride + (l + 1) * 16 + g];
            phJ = sphi[J * kPhiStride + g];
          }
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int cp = 0; cp < 3; ++cp) {
              R sacc = acc[j][c * 3 + cp];
#pragma unroll
              for (int l = 0; l < 5; ++l) sacc += Tr[c * 15 + l * 3 + cp] * pj[l];
              acc[j][c * 3 + cp] = sacc;
            }
          const R mm = mI * phJ;
          acc[j][0] += mm;
          acc[j][4] += mm;
          acc[j][8] += mm;
        }
        __syncwarp();
      }
      // outputs of this pass: rows (I, c), columns J0..J0+JP-1
      if (A.hess_p) {
        R* Hp = reinterpret_cast<R*>(A.hess_p) + (size_t)p * 2304;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int j = 0; j < JP; ++j)
#pragma unroll
            for (int cp = 0; cp < 3; ++cp) Hp[(I * 3 + c) * 48 + (J0 + j) * 3 + cp] = acc[j][c * 3 + cp];
      }
      if (A.bsr) {
        // J0..J0+JP-1 covers whole corners (4 kinds each): row segments of 12 in the BSR block
        R* V = reinterpret_cast<R*>(A.bsr);
        const int a = I >> 2, r = I & 3;
#pragma unroll
        for (int bb = 0; bb < JP / 4; ++bb) {
          const int b = (J0 >> 2) + bb;
          const int kb = A.pblocks[p * 16 + a * 4 + b];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            R row[12];
#pragma unroll
            for (int sk = 0; sk < 4; ++sk)
#pragma unroll
              for (int cp = 0; cp < 3; ++cp) row[sk * 3 + cp] = acc[bb * 4 + sk][c * 3 + cp];
            R* dst = V + (size_t)kb * 144 + (r * 3 + c) * 12;
            if (A.bsr_atomic) atomic_add_row12<R>(dst, row);
            else plain_add_row12<R>(dst, row);
          }
        }
      }
    }
  }
  __syncwarp();
}

}  // namespace bhem
