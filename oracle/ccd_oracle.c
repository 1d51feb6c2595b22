/*
 * Plain FP64 CPU oracle of the point-patch continuous collision detection of Sec. 5 ("Dynamic
 * Ray-Patch Intersection", Eq. ineqccd) for bicubic Hermite shells moving over one time step.
 *
 * TEST INFRASTRUCTURE. Only the tests and the bench's CPU-baseline leg use this code. The CUDA
 * library never calls, links or includes it, and it shares no code with the CUDA path. It uses
 * the Bezier form, De Casteljau cuts and Bezier evaluation of ray_oracle.c.
 *
 * Problem. Over a step the control points move linearly, p_ij + s dp_ij with s = t / dt in
 * [0, 1] (dp = the Bezier form of the nodal displacement over the step, since the Hermite-to-
 * Bezier map is linear), and a point moves as x0 + s dx. Wanted: the earliest s at which the
 * point lies on a patch, that patch and the local (u, v) there.
 *
 * Steps, in the order of Sec. 5:
 *   1. Feasible times of a (sub)patch (Eq. ineqccd). For axis k the point is above the box's
 *      lower face at time s when some control point satisfies a + b s <= 0 with
 *      a = (p_ij - x0)_k, b = (dp_ij - dx)_k; the union over ij of these half-lines is the real
 *      line minus one open interval (L, R), L = max over b > 0 of -a/b, R = min over b < 0 of
 *      -a/b (nothing is removed when some b = 0 has a <= 0, or when L >= R). The upper face gives
 *      the same with a, b negated. The feasible set is [0, 1] minus the six removed intervals:
 *      a sorted list of closed intervals.
 *   2. Candidates (patch, parameter rectangle) go into a binary min-heap keyed by their earliest
 *      feasible time s_min; the top is taken next. A candidate whose control-point box is at most
 *      EPS_X on every axis at every time of the step (start box side + displacement box side
 *      <= EPS_X per axis) is refined: s_min is a contact time within that tolerance. The search
 *      ends when the top cannot beat the best s found.
 *   3. Otherwise the candidate is split as in the static case: at its parameter midpoint
 *      (Fig. submid) or, in the Newton variant, Newton's method on
 *      x(u, v, s) - x0 - s dx = 0 in (u, v, s) runs from the candidate's centre at s_min; a root
 *      inside the candidate with s in [0, 1] updates the best s, its neighbourhood (NBHD of the
 *      candidate's parameter extent) is abandoned and the rest is split as in Fig. subany.
 *
 * Readings where the paper gives no numbers or leaves a choice:
 *   - Time is normalised to the step (s in [0, 1]); EPS_X = 1e-9 (position units), EPS_S =
 *     1e-9 for the stopping test, NBHD = 1e-3, at most 12 Newton iterations, converged when
 *     |F| <= 1e-12 (1 + |x0| + |dx|); as in the static search, Newton gives up once (u, v)
 *     leaves the candidate's rectangle widened by its own extent on each side.
 *   - The refinement box is bounded over the whole step by the start box plus the displacement
 *     box per axis, so a refined candidate is small at every time, not only at s_min. A
 *     candidate below 1e-13 in both parameter extents also counts as refined.
 *   - The removed intervals are subtracted from [0, 1] one at a time (axes in order, lower face
 *     before upper face); the result is the same set in any order.
 *   - A patch is first compared by its swept box (the box of p_ij and p_ij + dp_ij) against the
 *     point's segment box; a patch whose swept box misses it can have no feasible time and is
 *     not pushed (a cheap rejection before step 1; the GPU applies the same test).
 *   - Patches are pushed in patch order, children in the order of the figures. At most
 *     MAX_EXPANSIONS splits per query.
 *
 * Parity pins: tests/test_ccd_oracle.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int nu, nv, periodic_u, periodic_v; double dxi1, dxi2; } og_grid;
void og_bezier_patch(const og_grid* g, const double* q, int p, double P[4][4][3]);
void og_bezier_eval(const double P[4][4][3], double u, double v, double x[3], double xu[3], double xv[3]);
void og_bezier_sub(const double P[4][4][3], double u0, double u1, double v0, double v1, double S[4][4][3]);

#define EPS_X 1e-9
#define EPS_S 1e-9
#define NBHD 1e-3
#define NEWTON_ITERS 12
#define MAX_EXPANSIONS 65536
#define MAX_PIECES 8

/* 1. Feasible times in [0, 1] of the moving net (S, dS) for the point x0 + s dx: up to
   MAX_PIECES sorted closed intervals lo[i] <= hi[i]; returns their number (0: never). */
int og_ccd_feasible(const double S[4][4][3], const double dS[4][4][3], const double x0[3], const double dx[3],
                    double lo[MAX_PIECES], double hi[MAX_PIECES]) {
  int n = 1;
  lo[0] = 0.0;
  hi[0] = 1.0;
  for (int k = 0; k < 3; ++k) {
    double Ll = -INFINITY, Rl = INFINITY, Lu = -INFINITY, Ru = INFINITY;   /* lower face, upper face */
    int all_l = 0, all_u = 0;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const double a = S[i][j][k] - x0[k], b = dS[i][j][k] - dx[k];
        if (b > 0.0) {
          const double r = -a / b;
          if (r > Ll) Ll = r;           /* lower face: a + b s <= 0 for s <= r */
          if (r < Ru) Ru = r;           /* upper face: -a - b s <= 0 for s >= r */
        } else if (b < 0.0) {
          const double r = -a / b;
          if (r < Rl) Rl = r;
          if (r > Lu) Lu = r;
        } else {
          if (a <= 0.0) all_l = 1;
          if (a >= 0.0) all_u = 1;
        }
      }
    const double cut[2][2] = {{Ll, Rl}, {Lu, Ru}};
    const int all[2] = {all_l, all_u};
    for (int side = 0; side < 2; ++side) {
      const double L = cut[side][0], R = cut[side][1];
      if (all[side] || !(L < R)) continue;
      /* remove the open interval (L, R) from every piece */
      double nlo[MAX_PIECES], nhi[MAX_PIECES];
      int m = 0;
      for (int p = 0; p < n; ++p) {
        const double a1 = lo[p], b1 = hi[p] < L ? hi[p] : L;
        if (a1 <= b1 && m < MAX_PIECES) { nlo[m] = a1; nhi[m] = b1; ++m; }
        const double a2 = lo[p] > R ? lo[p] : R, b2 = hi[p];
        if (a2 <= b2 && m < MAX_PIECES) { nlo[m] = a2; nhi[m] = b2; ++m; }
      }
      n = m;
      memcpy(lo, nlo, sizeof(double) * (size_t)m);
      memcpy(hi, nhi, sizeof(double) * (size_t)m);
      if (n == 0) return 0;
    }
  }
  return n;
}

/* Largest per-axis (start box side + displacement box side) of the moving net. */
static double moving_extent(const double S[4][4][3], const double dS[4][4][3]) {
  double e = 0.0;
  for (int k = 0; k < 3; ++k) {
    double mn = S[0][0][k], mx = S[0][0][k], dmn = dS[0][0][k], dmx = dS[0][0][k];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const double s = S[i][j][k], d = dS[i][j][k];
        if (s < mn) mn = s;
        if (s > mx) mx = s;
        if (d < dmn) dmn = d;
        if (d > dmx) dmx = d;
      }
    const double w = (mx - mn) + (dmx - dmn);
    if (w > e) e = w;
  }
  return e;
}

static double det3(const double M[3][3]) {
  return (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
          M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])) +
         M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* Newton on F(u, v, s) = X(u, v) + s D(u, v) - x0 - s dx, Jacobian [X_u + s D_u | X_v + s D_v |
   D - dx] by Cramer's rule, from (*u, *v, *s). Returns 1 with the root on convergence. */
static int newton_root(const double P[4][4][3], const double dP[4][4][3], const double x0[3], const double dx[3],
                       double scale, const double win[4], double* u, double* v, double* s, int* iters) {
  double uu = *u, vv = *v, ss = *s;
  for (int it = 0; it < NEWTON_ITERS; ++it) {
    double X[3], Xu[3], Xv[3], D[3], Du[3], Dv[3], F[3], J[3][3];
    ++*iters;
    og_bezier_eval(P, uu, vv, X, Xu, Xv);
    og_bezier_eval(dP, uu, vv, D, Du, Dv);
    for (int c = 0; c < 3; ++c) {
      F[c] = (X[c] + ss * D[c]) - (x0[c] + ss * dx[c]);
      J[c][0] = Xu[c] + ss * Du[c];
      J[c][1] = Xv[c] + ss * Dv[c];
      J[c][2] = D[c] - dx[c];
    }
    const double fn = sqrt((F[0] * F[0] + F[1] * F[1]) + F[2] * F[2]);
    if (fn <= 1e-12 * scale) {
      *u = uu; *v = vv; *s = ss;
      return 1;
    }
    const double det = det3(J);
    if (!(fabs(det) > 1e-300)) return 0;
    double delta[3];
    for (int k = 0; k < 3; ++k) {
      double M[3][3];
      memcpy(M, J, sizeof(M));
      for (int r = 0; r < 3; ++r) M[r][k] = -F[r];
      delta[k] = det3(M) / det;
    }
    uu += delta[0]; vv += delta[1]; ss += delta[2];
    if (!isfinite(uu) || !isfinite(vv) || !isfinite(ss)) return 0;
    if (uu < win[0] || uu > win[1] || vv < win[2] || vv > win[3]) return 0;   /* left the window */
  }
  return 0;
}

/* 2. Binary min-heap keyed by s_min. */
typedef struct { double t0, t1, ext, u0, u1, v0, v1; int patch; } oc_cand;
typedef struct { oc_cand* a; int n, cap, peak, boxes; } oc_heap;

static void heap_push(oc_heap* h, oc_cand c) {
  if (h->n == h->cap) {
    h->cap = h->cap ? 2 * h->cap : 64;
    h->a = (oc_cand*)realloc(h->a, sizeof(oc_cand) * (size_t)h->cap);
  }
  int i = h->n++;
  if (h->n > h->peak) h->peak = h->n;
  while (i > 0) {
    const int parent = (i - 1) / 2;
    if (h->a[parent].t0 <= c.t0) break;
    h->a[i] = h->a[parent];
    i = parent;
  }
  h->a[i] = c;
}

static oc_cand heap_pop(oc_heap* h) {
  const oc_cand top = h->a[0], last = h->a[--h->n];
  int i = 0;
  for (;;) {
    const int l = 2 * i + 1, r = l + 1;
    int m = i;
    double km = last.t0;
    if (l < h->n && h->a[l].t0 < km) { m = l; km = h->a[l].t0; }
    if (r < h->n && h->a[r].t0 < km) m = r;
    if (m == i) break;
    h->a[i] = h->a[m];
    i = m;
  }
  if (h->n > 0) h->a[i] = last;
  return top;
}

/* Pushes the sub-patch [u0, u1] x [v0, v1] of patch p when it has a feasible time before best. */
static void push_sub(oc_heap* h, const double P[4][4][3], const double dP[4][4][3], int p, double u0, double u1,
                     double v0, double v1, const double x0[3], const double dx[3], double best) {
  if (!(u1 > u0) || !(v1 > v0)) return;
  double S[4][4][3], dS[4][4][3], lo[MAX_PIECES], hi[MAX_PIECES];
  ++h->boxes;
  og_bezier_sub(P, u0, u1, v0, v1, S);
  og_bezier_sub(dP, u0, u1, v0, v1, dS);
  if (og_ccd_feasible(S, dS, x0, dx, lo, hi) == 0 || lo[0] >= best) return;
  const oc_cand c = {lo[0], hi[0], moving_extent(S, dS), u0, u1, v0, v1, p};
  heap_push(h, c);
}

/* One query point against all patches. P, dP: start nets and displacement nets; swept[p]:
   min xyz, max xyz of patch p's swept box. Returns flags: bit 0 contact (s, patch, u, v
   written), bit 1 MAX_EXPANSIONS reached. stats (may be NULL): splits, largest heap, candidate
   feasibility tests (patch roots that passed the swept-box test included), Newton iterations. */
static int query_one(const double (*P)[4][4][3], const double (*dP)[4][4][3], const double (*swept)[6], int np,
                     const double x0[3], const double dx[3], int use_newton, double* s_out, int* patch_out,
                     double* u_out, double* v_out, int stats[4]) {
  double seg_lo[3], seg_hi[3];
  for (int c = 0; c < 3; ++c) {
    const double x1 = x0[c] + dx[c];
    seg_lo[c] = x0[c] < x1 ? x0[c] : x1;
    seg_hi[c] = x0[c] < x1 ? x1 : x0[c];
  }
  const double scale = (1.0 + sqrt((x0[0] * x0[0] + x0[1] * x0[1]) + x0[2] * x0[2])) +
                       sqrt((dx[0] * dx[0] + dx[1] * dx[1]) + dx[2] * dx[2]);
  oc_heap h = {NULL, 0, 0, 0, 0};
  double best = INFINITY, bu = 0.0, bv = 0.0;
  int bp = -1, nexp = 0, flags = 0, newton_iters = 0;
  for (int p = 0; p < np; ++p) {
    int miss = 0;
    for (int c = 0; c < 3; ++c)
      if (seg_hi[c] < swept[p][c] || seg_lo[c] > swept[p][3 + c]) miss = 1;
    if (!miss) push_sub(&h, P[p], dP[p], p, 0.0, 1.0, 0.0, 1.0, x0, dx, best);
  }
  while (h.n > 0) {
    const oc_cand c = heap_pop(&h);
    if (c.t0 >= best - EPS_S) break;                            /* nothing left can be earlier */
    if (c.ext <= EPS_X || (c.u1 - c.u0 < 1e-13 && c.v1 - c.v0 < 1e-13)) {   /* refined */
      if (c.t0 < best - EPS_S) {
        best = c.t0; bp = c.patch; bu = 0.5 * (c.u0 + c.u1); bv = 0.5 * (c.v0 + c.v1);
      }
      continue;
    }
    if (nexp == MAX_EXPANSIONS) { flags |= 2; break; }
    ++nexp;
    const double (*Pp)[4][3] = P[c.patch];
    const double (*dPp)[4][3] = dP[c.patch];
    const double um = 0.5 * (c.u0 + c.u1), vm = 0.5 * (c.v0 + c.v1);
    if (use_newton) {
      double u = um, v = vm, s = c.t0;
      const double wu = c.u1 - c.u0, wv = c.v1 - c.v0;
      const double win[4] = {c.u0 - wu, c.u1 + wu, c.v0 - wv, c.v1 + wv};
      if (newton_root(Pp, dPp, x0, dx, scale, win, &u, &v, &s, &newton_iters) && u >= c.u0 && u <= c.u1 &&
          v >= c.v0 && v <= c.v1 && s >= 0.0 && s <= 1.0) {
        if (s < best) { best = s; bp = c.patch; bu = u; bv = v; }
        const double hu = NBHD * (c.u1 - c.u0), hv = NBHD * (c.v1 - c.v0);
        const double a1 = fmax(c.u0, u - hu), a2 = fmin(c.u1, u + hu);
        const double b1 = fmax(c.v0, v - hv), b2 = fmin(c.v1, v + hv);
        push_sub(&h, Pp, dPp, c.patch, c.u0, a1, b1, c.v1, x0, dx, best);
        push_sub(&h, Pp, dPp, c.patch, a1, c.u1, b2, c.v1, x0, dx, best);
        push_sub(&h, Pp, dPp, c.patch, c.u0, a2, c.v0, b1, x0, dx, best);
        push_sub(&h, Pp, dPp, c.patch, a2, c.u1, c.v0, b2, x0, dx, best);
        continue;
      }
    }
    push_sub(&h, Pp, dPp, c.patch, c.u0, um, vm, c.v1, x0, dx, best);
    push_sub(&h, Pp, dPp, c.patch, um, c.u1, vm, c.v1, x0, dx, best);
    push_sub(&h, Pp, dPp, c.patch, c.u0, um, c.v0, vm, x0, dx, best);
    push_sub(&h, Pp, dPp, c.patch, um, c.u1, c.v0, vm, x0, dx, best);
  }
  free(h.a);
  if (stats) { stats[0] = nexp; stats[1] = h.peak; stats[2] = h.boxes; stats[3] = newton_iters; }
  if (bp >= 0) {
    flags |= 1;
    *s_out = best; *patch_out = bp; *u_out = bu; *v_out = bv;
  }
  return flags;
}

/* Swept box of a patch over the step: min xyz, max xyz of its start and end control points. */
static void swept_box(const double P[4][4][3], const double dP[4][4][3], double box[6]) {
  for (int k = 0; k < 3; ++k) {
    double mn = P[0][0][k], mx = P[0][0][k];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const double a = P[i][j][k], b = P[i][j][k] + dP[i][j][k];
        if (a < mn) mn = a;
        if (a > mx) mx = a;
        if (b < mn) mn = b;
        if (b > mx) mx = b;
      }
    box[k] = mn;
    box[3 + k] = mx;
  }
}

/* Many points: x0, dx [n][3]; shell DOFs q (start of step) and dq (displacement over the step).
   Outputs s [n] (INFINITY when no contact), patch [n] (-1), uv [n][2], flags [n], stats [n][4]
   (may be NULL). */
void og_ccd_points(const og_grid* g, const double* q, const double* dq, int n, const double* x0s, const double* dxs,
                   int use_newton, double* s, int* patch, double* uv, int* flags, int* stats) {
  const int np = g->nu * g->nv;
  double (*P)[4][4][3] = (double(*)[4][4][3])malloc(sizeof(double) * 48 * (size_t)np);
  double (*dP)[4][4][3] = (double(*)[4][4][3])malloc(sizeof(double) * 48 * (size_t)np);
  double (*sw)[6] = (double(*)[6])malloc(sizeof(double) * 6 * (size_t)np);
  for (int p = 0; p < np; ++p) {
    og_bezier_patch(g, q, p, P[p]);
    og_bezier_patch(g, dq, p, dP[p]);
    swept_box(P[p], dP[p], sw[p]);
  }
  /* queries are independent (each keeps its own heap): all host cores with OpenMP */
#pragma omp parallel for schedule(dynamic, 16) if (n >= 256)
  for (int k = 0; k < n; ++k) {
    double t = INFINITY, u = 0.0, v = 0.0;
    int p = -1;
    const int f = query_one((const double(*)[4][4][3])P, (const double(*)[4][4][3])dP, (const double(*)[6])sw, np,
                            x0s + 3 * (size_t)k, dxs + 3 * (size_t)k, use_newton, &t, &p, &u, &v,
                            stats ? stats + 4 * (size_t)k : NULL);
    if (f & 1) {
      s[k] = t; patch[k] = p; uv[2 * k] = u; uv[2 * k + 1] = v;
    } else {
      s[k] = INFINITY; patch[k] = -1; uv[2 * k] = uv[2 * k + 1] = 0.0;
    }
    flags[k] = f;
  }
  free(P);
  free(dP);
  free(sw);
}
