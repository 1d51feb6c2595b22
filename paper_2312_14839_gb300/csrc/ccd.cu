// Point-patch continuous collision detection (Sec. 5, "Dynamic Ray-Patch Intersection",
// Eq. ineqccd): the earliest time in a step at which each moving point meets the moving shell.
//
// Over the step the control points move linearly, p_ij + s dp_ij (s = t / dt in [0, 1]; dp is
// the Bezier net of the nodal displacement over the step), and a point moves as x0 + s dx.
//
//   k_ccd_nets   one thread per patch: start net P, displacement net dP and the swept box (the
//                box of p_ij and p_ij + dp_ij).
//   k_ccd_groups the swept box of every kGroup consecutive patches, to skip groups whole.
//   k_ccd_points one point per thread, FP64. Patches whose swept box misses the point's segment
//                box are skipped; the others enter a binary min-heap keyed by their earliest
//                feasible time s_min. Feasible times of a (sub)net: for each axis and each face
//                of its box, the union over control points of the half-lines a + b s <= 0 is
//                the real line minus one open interval (L, R); [0, 1] minus those six intervals
//                is a sorted list of closed intervals. A candidate whose start-box side plus
//                displacement-box side is at most kEpsX on every axis is refined (contact at
//                s_min); otherwise it is split at its parameter midpoint (Fig. submid) or, in the
//                Newton variant, around a root of x(u, v, s) = x0 + s dx found by Newton's
//                method in (u, v, s), whose neighbourhood is abandoned (Fig. subany). The search
//                ends when the heap's top cannot beat the best s. Feasibility tests, of the
//                patch roots (up to four per lane per round, in patch order) and of the children
//                of every split, are pooled over the warp, one job per (sub)patch and axis; the
//                owner lane then removes the intervals in order. Full local heaps move into
//                global ones as in the ray search.
//   k_ccd_points_redo  points that found no free global heap, searched again from the start.
//
// Compiled without mul-add contraction, like rays.cu: every decision is that of the same IEEE FP64
// operations in the same order as a plain sequential program of these steps.
#include <cmath>

#include "bezier.cuh"
#include "common.cuh"

namespace bhem {
namespace {

using namespace bz;

constexpr double kEpsX = 1e-9;       // refinement size (positions' units)
constexpr double kEpsS = 1e-9;       // stopping test on the normalised time
constexpr int kNetBlock = 128;
constexpr int kCcdBlock = 64;         // 2 warps: the per-warp exchange is 22.7 KB
constexpr int kMaxPieces = 8;        // [0, 1] minus six open intervals has at most 7 pieces
constexpr int kNetStride = 104;      // doubles per patch: P (48), dP (48), swept box (6), unused (2)
constexpr int kGroup = 32;           // consecutive patches per group swept box

__global__ void __launch_bounds__(kNetBlock) k_ccd_nets(int np, const int4* __restrict__ pnodes,
                                                        const double* __restrict__ q, const double* __restrict__ dq,
                                                        double dxi1, double dxi2, double* __restrict__ nets) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int4 n4 = pnodes[p];
  const int nd[4] = {n4.x, n4.y, n4.z, n4.w};
  double* P = nets + (size_t)p * kNetStride;
  double* dP = P + 48;
  double* box = P + 96;
  patch_net(q, nd, dxi1, dxi2, P);
  patch_net(dq, nd, dxi1, dxi2, dP);
  for (int k = 0; k < 3; ++k) {
    double mn = P[16 * k], mx = P[16 * k];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const double a = P[16 * k + 4 * i + j], b = P[16 * k + 4 * i + j] + dP[16 * k + 4 * i + j];
        if (a < mn) mn = a;
        if (a > mx) mx = a;
        if (b < mn) mn = b;
        if (b > mx) mx = b;
      }
    box[k] = mn;
    box[3 + k] = mx;
  }
  box[6] = 0.0;
  box[7] = 0.0;
}

// Swept box of every kGroup consecutive patches (min xyz, max xyz of its members' swept boxes,
// 8 doubles per group after the per-patch data). A segment box that misses it misses every
// member's (comparisons only).
__global__ void k_ccd_groups(int np, const double* __restrict__ nets, double* __restrict__ gboxes) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  const int p0 = gi * kGroup;
  if (p0 >= np) return;
  const int p1 = min(np, p0 + kGroup);
  double mn[3], mx[3];
  for (int c = 0; c < 3; ++c) {
    mn[c] = nets[(size_t)p0 * kNetStride + 96 + c];
    mx[c] = nets[(size_t)p0 * kNetStride + 99 + c];
  }
  for (int p = p0 + 1; p < p1; ++p)
    for (int c = 0; c < 3; ++c) {
      const double a = nets[(size_t)p * kNetStride + 96 + c], b = nets[(size_t)p * kNetStride + 99 + c];
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

// Coordinate k of the sub-net [u0, u1] x [v0, v1] of P ([c][i][j]): S[i][j], theta1-curves cut
// first, then theta2-curves.
__device__ __forceinline__ void cut_coord(const double* __restrict__ P, int k, double u0, double u1, double v0,
                                          double v1, double S[4][4]) {
  const double* Pc = P + 16 * k;
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
  for (int i = 0; i < 4; ++i) curve_restrict(T[i], v0, v1, S[i]);
}

// One axis k of the feasibility test (Eq. ineqccd) of the sub-net [u0, u1] x [v0, v1] of the
// moving net (P, dP) for the point x0 + s dx (x0k = x0[k], dxk = dx[k]): the open intervals
// (L, R) that the lower and upper faces remove from the times (res[0..3] = L_lower, R_lower,
// L_upper, R_upper; *all bit 0 / bit 1 when a face removes nothing because some control point
// has b = 0 on the right side), and the axis's start-box side plus displacement-box side (res[4]).
__device__ void axis_job(const double* __restrict__ P, const double* __restrict__ dP, double u0, double u1,
                         double v0, double v1, int k, double x0k, double dxk, double res[5], int* all) {
  double S[4][4], dS[4][4];
  cut_coord(P, k, u0, u1, v0, v1, S);
  cut_coord(dP, k, u0, u1, v0, v1, dS);
  double Ll = -INFINITY, Rl = INFINITY, Lu = -INFINITY, Ru = INFINITY;   // lower face, upper face
  bool all_l = false, all_u = false;
  double mn = S[0][0], mx = S[0][0], dmn = dS[0][0], dmx = dS[0][0];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // the same updates as a three-way branch on the sign of b, as selects, so that the lanes
      // of a warp do not diverge (r is only used when b != 0)
      const double a = S[i][j] - x0k, b = dS[i][j] - dxk;
      const double r = -a / b;
      const bool pos = b > 0.0, neg = b < 0.0;
      Ll = (pos && r > Ll) ? r : Ll;
      Ru = (pos && r < Ru) ? r : Ru;
      Rl = (neg && r < Rl) ? r : Rl;
      Lu = (neg && r > Lu) ? r : Lu;
      all_l = all_l || (!pos && !neg && a <= 0.0);
      all_u = all_u || (!pos && !neg && a >= 0.0);
      const double sv = S[i][j], dv = dS[i][j];
      if (sv < mn) mn = sv;
      if (sv > mx) mx = sv;
      if (dv < dmn) dmn = dv;
      if (dv > dmx) dmx = dv;
    }
  res[0] = Ll;
  res[1] = Rl;
  res[2] = Lu;
  res[3] = Ru;
  res[4] = (mx - mn) + (dmx - dmn);
  *all = (all_l ? 1 : 0) | (all_u ? 2 : 0);
}

// The feasible times of one (sub)net from its three axis results (ax[k][0..4], all[k]): [0, 1]
// minus the removed intervals, axes in order and the lower face first. False when none is left;
// else the first piece [t0, t1] and the largest per-axis extent (ext).
__device__ bool combine_axes(const double (*ax)[5], const unsigned char* all, double& t0, double& t1,
                             double& ext) {
  double lo[kMaxPieces], hi[kMaxPieces];
  int n = 1;
  lo[0] = 0.0;
  hi[0] = 1.0;
  double e = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double w = ax[k][4];
    if (w > e) e = w;
    for (int side = 0; side < 2; ++side) {
      const double L = ax[k][2 * side], R = ax[k][2 * side + 1];
      if ((all[k] >> side & 1) || !(L < R)) continue;
      // remove the open interval (L, R) from every piece (pieces stay sorted)
      double nlo[kMaxPieces], nhi[kMaxPieces];
      int m = 0;
      for (int p = 0; p < n; ++p) {
        const double a1 = lo[p], b1 = hi[p] < L ? hi[p] : L;
        if (a1 <= b1 && m < kMaxPieces) {
          nlo[m] = a1;
          nhi[m] = b1;
          ++m;
        }
        const double a2 = lo[p] > R ? lo[p] : R, b2 = hi[p];
        if (a2 <= b2 && m < kMaxPieces) {
          nlo[m] = a2;
          nhi[m] = b2;
          ++m;
        }
      }
      n = m;
      for (int p = 0; p < m; ++p) {
        lo[p] = nlo[p];
        hi[p] = nhi[p];
      }
      if (n == 0) return false;
    }
  }
  t0 = lo[0];
  t1 = hi[0];
  ext = e;
  return true;
}

// Newton on F(u, v, s) = X(u, v) + s D(u, v) - x0 - s dx, Jacobian [X_u + s D_u | X_v + s D_v |
// D - dx] by Cramer's rule. True with the root in (u, v, s) on convergence; gives up when (u, v)
// leaves the window win (the candidate's rectangle widened by its extent on each side).
__device__ bool newton_ccd(const double* __restrict__ P, const double* __restrict__ dP, const double x0[3],
                           const double dx[3], double scale, const double win[4], double& u, double& v, double& s,
                           int& iters) {
  double uu = u, vv = v, ss = s;
  for (int it = 0; it < kNewtonIters; ++it) {
    double X[3], Xu[3], Xv[3], D[3], Du[3], Dv[3], F[3], J[3][3];
    ++iters;
    bezier_eval(P, uu, vv, X, Xu, Xv);
    bezier_eval(dP, uu, vv, D, Du, Dv);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      F[c] = (X[c] + ss * D[c]) - (x0[c] + ss * dx[c]);
      J[c][0] = Xu[c] + ss * Du[c];
      J[c][1] = Xv[c] + ss * Dv[c];
      J[c][2] = D[c] - dx[c];
    }
    const double fn = sqrt((F[0] * F[0] + F[1] * F[1]) + F[2] * F[2]);
    if (fn <= 1e-12 * scale) {
      u = uu;
      v = vv;
      s = ss;
      return true;
    }
    const double det = det3(J);
    if (!(fabs(det) > 1e-300)) return false;
    double delta[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double M[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[r][c] = c == k ? -F[r] : J[r][c];
      delta[k] = det3(M) / det;
    }
    uu += delta[0];
    vv += delta[1];
    ss += delta[2];
    if (!isfinite(uu) || !isfinite(vv) || !isfinite(ss)) return false;
    if (uu < win[0] || uu > win[1] || vv < win[2] || vv > win[3]) return false;   // left the window
  }
  return false;
}

struct Query {
  double x0[3], dx[3], seg_lo[3], seg_hi[3], scale;
};

__device__ __forceinline__ void load_query(const double* __restrict__ x0s, const double* __restrict__ dxs,
                                           long long k, Query& Q) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Q.x0[c] = x0s[3 * k + c];
    Q.dx[c] = dxs[3 * k + c];
    const double x1 = Q.x0[c] + Q.dx[c];
    Q.seg_lo[c] = Q.x0[c] < x1 ? Q.x0[c] : x1;
    Q.seg_hi[c] = Q.x0[c] < x1 ? x1 : Q.x0[c];
  }
  Q.scale = (1.0 + sqrt((Q.x0[0] * Q.x0[0] + Q.x0[1] * Q.x0[1]) + Q.x0[2] * Q.x0[2])) +
            sqrt((Q.dx[0] * Q.dx[0] + Q.dx[1] * Q.dx[1]) + Q.dx[2] * Q.dx[2]);
}

struct Search {
  double best = INFINITY, bu = 0.0, bv = 0.0;
  int bp = -1, nexp = 0, flags = 0, newton_iters = 0;
  bool live = false;
};

// Shared-memory exchange of one warp: children listed by each lane in the current split, and
// the axis results computed for them by whichever lanes took the (child, axis) jobs.
struct WarpSmem {
  double rect[32][4][4];
  double ax[32][4][3][5];       // child, axis: L_lower, R_lower, L_upper, R_upper, extent
  double pt[32][6];             // the owner's x0, dx
  int patch[32][4];
  unsigned char all[32][4][3];  // bit 0 / 1: lower / upper face removes nothing
  unsigned short jobs[32 * 12]; // lane * 12 + child * 3 + axis
};

__device__ __forceinline__ void put_rect(WarpSmem& sm, int lane, int& nch, int patch, double u0, double u1,
                                         double v0, double v1) {
  if (!(u1 > u0) || !(v1 > v0)) return;
  sm.patch[lane][nch] = patch;
  double* R = sm.rect[lane][nch++];
  R[0] = u0;
  R[1] = u1;
  R[2] = v0;
  R[3] = v1;
}

// The warp's pool of (lane, child, axis) jobs: every lane lists nch children in sm.rect /
// sm.patch; the 3 axes of every child are spread over the 32 lanes, then each lane combines its
// own children's axes and pushes the feasible ones in order. All 32 lanes call it together.
__device__ void pool_and_push(Heap& h, const double* __restrict__ nets, const Search& S, WarpSmem& sm, int lane,
                              int nch) {
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
    const int code = sm.jobs[j], owner = code / 12, q = code - 12 * owner, ch = q / 3, k = q % 3;
    const double* R = sm.rect[owner][ch];
    const double* P = nets + (size_t)sm.patch[owner][ch] * kNetStride;
    int all = 0;
    axis_job(P, P + 48, R[0], R[1], R[2], R[3], k, sm.pt[owner][k], sm.pt[owner][3 + k], sm.ax[owner][ch][k], &all);
    sm.all[owner][ch][k] = (unsigned char)all;
  }
  __syncwarp();
  for (int ch = 0; ch < nch; ++ch) {
    double t0, t1, e;
    if (combine_axes(sm.ax[lane][ch], sm.all[lane][ch], t0, t1, e) && !(t0 >= S.best)) {
      const double* R = sm.rect[lane][ch];
      h.push(Cand{t0, t1, e, R[0], R[1], R[2], R[3], sm.patch[lane][ch]});
    }
  }
  __syncwarp();
}

// One round of a lane's root scan: the patches from `next` on, in order, whose swept box
// (nets[p * kNetStride + 96 ..]: min xyz, max xyz) meets the query's segment box, up to four;
// true when the scan has passed the last patch.
__device__ __forceinline__ bool root_round(Heap& h, const Query& Q, const double* __restrict__ nets, int np,
                                           WarpSmem& sm, int lane, int& next, int& nch) {
  while (next < np && nch < 4) {
    if (next % kGroup == 0) {   // a group that the segment box misses is skipped whole
      const double* G = nets + (size_t)np * kNetStride + (size_t)(next / kGroup) * 8;
      bool gmiss = false;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (Q.seg_hi[c] < G[c] || Q.seg_lo[c] > G[3 + c]) gmiss = true;
      if (gmiss) {
        next += kGroup;
        continue;
      }
    }
    const double* sw = nets + (size_t)next * kNetStride + 96;
    bool miss = false;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (Q.seg_hi[c] < sw[c] || Q.seg_lo[c] > sw[3 + c]) miss = true;
    if (!miss) put_rect(sm, lane, nch, next, 0.0, 1.0, 0.0, 1.0);
    ++next;
  }
  h.boxes += nch;
  return next >= np;
}

// Root phase, all 32 lanes together: the pooled feasibility tests push each lane's roots in
// patch order.
__device__ void push_roots(Heap& h, const Query& Q, const double* __restrict__ nets, int np, Search& S,
                           WarpSmem& sm, int lane) {
  int next = 0;
  bool more = S.live;
  while (__any_sync(0xffffffffu, more)) {
    int nch = 0;
    if (more && root_round(h, Q, nets, np, sm, lane, next, nch)) more = false;
    pool_and_push(h, nets, S, sm, lane, nch);
  }
}

// One split of a lane's search: pop the earliest candidate and either finish (nothing earlier
// can remain), record a refined contact, or list its 4 children (Newton pinwheel or midpoint
// split) for the warp's pooled feasibility tests.
__device__ __forceinline__ void split_step(Heap& h, const Query& Q, const double* __restrict__ nets, int use_newton,
                                           Search& S, WarpSmem& sm, int lane, int& nch) {
  if (h.n == 0 || h.overflow) {
    S.live = false;
  } else {
    const Cand c = h.pop();
    if (c.t0 >= S.best - kEpsS) {                                      // nothing left can be earlier
      S.live = false;
    } else if (c.ext <= kEpsX || (c.u1 - c.u0 < 1e-13 && c.v1 - c.v0 < 1e-13)) {   // refined
      if (c.t0 < S.best - kEpsS) {
        S.best = c.t0;
        S.bp = c.patch;
        S.bu = 0.5 * (c.u0 + c.u1);
        S.bv = 0.5 * (c.v0 + c.v1);
      }
    } else if (S.nexp == kMaxExpansions) {
      S.flags |= SHELL_RAY_LIMIT;
      S.live = false;
    } else {
      ++S.nexp;
      const double* P = nets + (size_t)c.patch * kNetStride;
      const double um = 0.5 * (c.u0 + c.u1), vm = 0.5 * (c.v0 + c.v1);
      bool pinwheel = false;
      if (use_newton) {
        double u = um, v = vm, s = c.t0;
        const double wu = c.u1 - c.u0, wv = c.v1 - c.v0;
        const double win[4] = {c.u0 - wu, c.u1 + wu, c.v0 - wv, c.v1 + wv};
        if (newton_ccd(P, P + 48, Q.x0, Q.dx, Q.scale, win, u, v, s, S.newton_iters) && u >= c.u0 &&
            u <= c.u1 &&
            v >= c.v0 && v <= c.v1 && s >= 0.0 && s <= 1.0) {
          if (s < S.best) {
            S.best = s;
            S.bp = c.patch;
            S.bu = u;
            S.bv = v;
          }
          const double hu = kNbhd * (c.u1 - c.u0), hv = kNbhd * (c.v1 - c.v0);
          const double a1 = fmax(c.u0, u - hu), a2 = fmin(c.u1, u + hu);
          const double b1 = fmax(c.v0, v - hv), b2 = fmin(c.v1, v + hv);
          put_rect(sm, lane, nch, c.patch, c.u0, a1, b1, c.v1);
          put_rect(sm, lane, nch, c.patch, a1, c.u1, b2, c.v1);
          put_rect(sm, lane, nch, c.patch, c.u0, a2, c.v0, b1);
          put_rect(sm, lane, nch, c.patch, a2, c.u1, c.v0, b2);
          pinwheel = true;
        }
      }
      if (!pinwheel) {
        put_rect(sm, lane, nch, c.patch, c.u0, um, vm, c.v1);
        put_rect(sm, lane, nch, c.patch, um, c.u1, vm, c.v1);
        put_rect(sm, lane, nch, c.patch, c.u0, um, c.v0, vm);
        put_rect(sm, lane, nch, c.patch, um, c.u1, c.v0, vm);
      }
      h.boxes += nch;
    }
  }
}

__device__ __forceinline__ void finish_flags(const Heap& h, Search& S) {
  if (h.overflow) {
    S.flags |= SHELL_RAY_OVERFLOW;
  } else if (S.bp >= 0) {
    S.flags |= SHELL_RAY_HIT;
  }
}

// The search over the candidates in each lane's heap, all 32 lanes of the warp together (lanes
// without a query pass live = false).
__device__ void search(Heap& h, const Query& Q, const double* __restrict__ nets, int np, int use_newton,
                       Search& S, WarpSmem& sm, int lane) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    sm.pt[lane][c] = Q.x0[c];
    sm.pt[lane][3 + c] = Q.dx[c];
  }
  push_roots(h, Q, nets, np, S, sm, lane);
  while (__any_sync(0xffffffffu, S.live)) {
    int nch = 0;
    if (S.live) split_step(h, Q, nets, use_newton, S, sm, lane, nch);
    pool_and_push(h, nets, S, sm, lane, nch);
  }
  finish_flags(h, S);
}

struct CcdOut {
  double* s;
  int* patch;
  double* uv;
  int* flags;
  int* stats;
};

__device__ __forceinline__ void write_result(const CcdOut& out, long long k, const Search& S, const Heap& h) {
  const bool hit = (S.flags & SHELL_RAY_HIT) != 0;
  out.s[k] = hit ? S.best : INFINITY;
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

// Persistent over the queries: every lane starts on query (global lane index) and, when its
// search ends, writes the result and takes the next query from counters[2], while the other lanes
// of its warp go on. A lane's root scan and splits feed the same pooled feasibility tests, so a
// warp keeps all its lanes busy until the queue is empty; each query's heap receives the same
// pushes in the same order as in a one-query-per-lane search.
__global__ void __launch_bounds__(kCcdBlock, 8) k_ccd_points(long long n, const double* __restrict__ x0s,
                                                             const double* __restrict__ dxs, int np,
                                                             const double* __restrict__ nets, int use_newton,
                                                             CcdOut out, int* __restrict__ counters,
                                                             int* __restrict__ redo_list, Cand* __restrict__ heaps) {
  __shared__ WarpSmem wsm[kCcdBlock / 32];
  WarpSmem& sm = wsm[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const long long lanes = (long long)gridDim.x * blockDim.x;
  Cand storage[kHeapCap];
  Heap h(storage, kHeapCap);
  Query Q;
  Search S;
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int phase = 0, next = 0;   // phase 0: no query left, 1: root scan, 2: search
  auto begin = [&]() {
    h.a = storage;
    h.cap = kHeapCap;
    h.n = 0;
    h.peak = 0;
    h.boxes = 0;
    h.overflow = false;
    h.spill = heaps;
    h.spill_count = counters + 1;
    S = Search();
    phase = 0;
    if (k < n) {
      load_query(x0s, dxs, k, Q);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sm.pt[lane][c] = Q.x0[c];
        sm.pt[lane][3 + c] = Q.dx[c];
      }
      S.live = true;
      phase = 1;
      next = 0;
    }
  };
  begin();
  while (__any_sync(0xffffffffu, phase != 0)) {
    int nch = 0;
    if (phase == 1) {
      if (root_round(h, Q, nets, np, sm, lane, next, nch)) phase = 2;
    } else if (phase == 2) {
      split_step(h, Q, nets, use_newton, S, sm, lane, nch);
    }
    pool_and_push(h, nets, S, sm, lane, nch);   // ends with a warp barrier: sm.pt may change below
    if (phase == 2 && !S.live) {
      finish_flags(h, S);
      bool deferred = false;
      if (h.overflow) {
        const int slot = atomicAdd(counters, 1);
        if (slot < kRedoList) {
          redo_list[slot] = (int)k;   // written by the second pass
          deferred = true;
        }
      }
      if (!deferred) write_result(out, k, S, h);
      k = lanes + atomicAdd(counters + 2, 1);
      begin();
    }
  }
}

__global__ void __launch_bounds__(kCcdBlock) k_ccd_points_redo(const double* __restrict__ x0s,
                                                                  const double* __restrict__ dxs, int np,
                                                                  const double* __restrict__ nets, int use_newton,
                                                                  CcdOut out, const int* __restrict__ counters,
                                                                  const int* __restrict__ redo_list,
                                                                  Cand* __restrict__ heaps) {
  __shared__ WarpSmem wsm[kCcdBlock / 32];
  const int tid = blockIdx.x * kCcdBlock + threadIdx.x, lane = threadIdx.x & 31;
  const int count = min(counters[0], kRedoList);
  for (int base = 0; base < count; base += kRedoThreads) {   // uniform trip count: the warp stays whole
    const int i = base + tid;
    const bool active = i < count;
    const long long k = active ? redo_list[i] : 0;
    Query Q;
    Heap h(heaps + (size_t)tid * kRedoHeap, kRedoHeap);
    if (active) load_query(x0s, dxs, k, Q);
    Search S;
    S.live = active;
    search(h, Q, nets, np, use_newton, S, wsm[threadIdx.x >> 5], lane);
    if (active) write_result(out, k, S, h);
  }
}

}  // namespace
}  // namespace bhem

using namespace bhem;

extern "C" shell_status shell_ccd_points(shell_t* shell, const double* q, const double* dq, long long n_points,
                                         const double* x0, const double* dx, int variant, double* s, int* patch,
                                         double* uv, int* flags, int* stats) {
  if (!shell) return fail(SHELL_ERR_ARG, "NULL shell");
  if (variant != SHELL_RAY_MIDPOINT && variant != SHELL_RAY_NEWTON) return fail(SHELL_ERR_ARG, "split variant");
  if (n_points < 0 || n_points > INT32_MAX) return fail(SHELL_ERR_ARG, "n_points outside [0, 2^31 - 1]");
  if (n_points == 0) return SHELL_OK;
  if (!q || !dq || !x0 || !dx || !s || !patch || !uv || !flags) return fail(SHELL_ERR_ARG, "NULL argument");
  Shell& sh = *shell;
  const int np = sh.n_patches;
  void* heaps_v = nullptr;
  int *counters = nullptr, *redo_list = nullptr;
  BHEM_TRY(search_scratch(sh, &heaps_v, &counters, &redo_list));
  if (!sh.d_ccd_nets) {
    const size_t ngroups = ((size_t)np + kGroup - 1) / kGroup;
    const cudaError_t e = cudaMalloc((void**)&sh.d_ccd_nets, sizeof(double) * (kNetStride * (size_t)np + 8 * ngroups));
    if (e != cudaSuccess) {
      cudaGetLastError();
      sh.d_ccd_nets = nullptr;
      return fail(SHELL_ERR_OOM, std::string("collision nets: ") + cudaGetErrorString(e));
    }
  }
  Cand* heaps = (Cand*)heaps_v;
  CcdOut out{s, patch, uv, flags, stats};
  BHEM_CUDA(cudaMemsetAsync(counters, 0, 4 * sizeof(int), sh.stream));
  k_ccd_nets<<<grid_for(np, kNetBlock), kNetBlock, 0, sh.stream>>>(np, sh.d_patch_nodes, q, dq, sh.grid.dxi1,
                                                                   sh.grid.dxi2, sh.d_ccd_nets);
  k_ccd_groups<<<grid_for((np + kGroup - 1) / kGroup, kNetBlock), kNetBlock, 0, sh.stream>>>(
      np, sh.d_ccd_nets, sh.d_ccd_nets + (size_t)kNetStride * np);
  const int use_newton = variant == SHELL_RAY_NEWTON;
  // persistent: exactly the CTAs that can be resident at once (a CTA that waits for a free SM would
  // start only after the queue is empty), lanes refill from the query counter
  if (sh.num_sms <= 0) BHEM_CUDA(cudaDeviceGetAttribute(&sh.num_sms, cudaDevAttrMultiProcessorCount, sh.device));
  int occ = 0;
  BHEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ccd_points, kCcdBlock, 0));
  const long long ctas = std::min<long long>((n_points + kCcdBlock - 1) / kCcdBlock,
                                             (long long)std::max(1, occ) * sh.num_sms);
  k_ccd_points<<<(unsigned)ctas, kCcdBlock, 0, sh.stream>>>(n_points, x0, dx, np, sh.d_ccd_nets, use_newton, out,
                                                          counters, redo_list, heaps);
  k_ccd_points_redo<<<kRedoThreads / kCcdBlock, kCcdBlock, 0, sh.stream>>>(x0, dx, np, sh.d_ccd_nets, use_newton, out, counters,
                                                       redo_list, heaps);
  sh.launches += 4;
  BHEM_CUDA(cudaGetLastError());
  return SHELL_OK;
}
