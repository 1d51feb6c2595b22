/*
 * Plain FP64 CPU oracle of the static ray-patch intersection of Sec. 5 ("Static Ray-Patch
 * Intersection", Eq. ray and Eq. ineqray) for bicubic Hermite shells.
 *
 * TEST INFRASTRUCTURE. Only the tests and the bench's CPU-baseline leg use this code. The CUDA
 * library never calls, links or includes it, and it shares no code with the CUDA path.
 *
 * Steps, in the order of Sec. 5:
 *   1. Each patch is rewritten in the Bernstein basis (the Bezier form at the start of Sec. 5):
 *      the cubic Hermite data of one parameter direction, value a, b and derivatives a', b' with
 *      respect to the local parameter theta in [0, 1], become the Bezier points
 *      b0 = a, b1 = a + a'/3, b2 = b - b'/3, b3 = b; the patch is their tensor product.
 *   2. Ray-AABB test (Eq. ineqray): the box of a (sub)patch's control points gives the interval
 *      [tau_min, tau_max] of ray times tau >= 0 inside the box, or no interval.
 *   3. Candidate (sub)patches go into a binary min-heap keyed by tau_min; the top is taken next.
 *      A candidate whose box is at most EPS_TAU in every axis is refined: the midpoint of its
 *      tau interval is an intersection. The search ends when the top of the heap cannot beat
 *      the best tau found.
 *   4. Otherwise the candidate is split into four sub-patches (De Casteljau): at its parameter
 *      midpoint (Fig. submid) or, in the Newton variant, Newton's method is first run on
 *      x(theta1, theta2) = o + tau d from the candidate's centre; a root inside the candidate
 *      updates the best tau, its neighbourhood (half-width NBHD times the candidate's parameter
 *      extent) is abandoned and the rest is split into the four rectangles of Fig. subany.
 *
 * Readings where the paper gives no numbers or leaves a choice:
 *   - EPS_TAU = 1e-9 (absolute, in the units of the positions; directions are unit vectors),
 *     NBHD = 1e-3, at most 12 Newton iterations, Newton converged when
 *     |F| <= 1e-12 (1 + |o| + |tau|), Newton starts with tau = (x(centre) - o) . d.
 *   - Newton gives up as soon as an iterate leaves the candidate's parameter rectangle widened by
 *     its own extent on each side: only a root inside the candidate is used, and Newton is an
 *     accelerator; a region where it gives up is subdivided as usual.
 *   - "Refined" means the box is small, not only the ray's tau interval through it: a ray that
 *     clips the corner of a large box gets a tiny tau interval although the surface need not
 *     cross the ray there. A box no larger than EPS_TAU in every axis also gives a tau interval
 *     of at most EPS_TAU for a unit direction, so the paper's condition holds at termination.
 *     A candidate whose parameter extent is below 1e-13 in both directions also counts as
 *     refined (degenerate geometry).
 *   - Every sub-patch is cut out of its patch's control net directly (its parameter rectangle
 *     within the patch), rather than by splitting the parent's net again, which is the same
 *     polynomial without repeated rounding. The four cut points of a curve restricted to
 *     [a, b] are its blossom values f(a,a,a), f(a,a,b), f(a,b,b), f(b,b,b), each a
 *     De Casteljau evaluation with one parameter per level.
 *   - Slab test with the reciprocal direction 1/d_k per axis; an axis with d_k = 0 keeps the
 *     ray only when o_k lies inside the slab.
 *   - At most MAX_EXPANSIONS candidates are split per ray; a ray that reaches it is reported.
 *   - Patches are pushed in patch order; children in the order given in og_trace_ray.
 *
 * Parity pins: tests/test_ray_oracle.py (Bezier form against the Hermite shape functions, the
 * plane closed form, De Casteljau pieces against direct evaluation, an independent multi-start
 * Newton on curved scenes, both variants against each other).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int nu, nv, periodic_u, periodic_v; double dxi1, dxi2; } og_grid;
void og_patch_nodes(const og_grid* g, int patch, int nodes[4]);

#define EPS_TAU 1e-9
#define NBHD 1e-3
#define NEWTON_ITERS 12
#define MAX_EXPANSIONS 65536

/* Hermite data -> Bezier points of one cubic (h0 = a, h1 = a', h2 = b, h3 = b'). */
static void hermite_to_bezier(const double h[4], double b[4]) {
  b[0] = h[0];
  b[1] = h[0] + h[1] / 3.0;
  b[2] = h[2] - h[3] / 3.0;
  b[3] = h[2];
}

/* 1. Control points P[i][j][c] (i along theta1, j along theta2) of patch p from the nodal DOFs
   q (12 per node: x, x_,1, x_,2, x_,12; derivatives with respect to the global xi). The local
   derivatives are d/dtheta1 = dxi1 d/dxi1, d/dtheta2 = dxi2 d/dxi2. */
void og_bezier_patch(const og_grid* g, const double* q, int p, double P[4][4][3]) {
  int nd[4];
  og_patch_nodes(g, p, nd);
  for (int c = 0; c < 3; ++c) {
    /* H[a][b]: a = 2 pu + r (theta1 end, derivative order), b = 2 pv + s */
    double H[4][4];
    for (int pv = 0; pv < 2; ++pv)
      for (int pu = 0; pu < 2; ++pu) {
        const double* X = q + 12 * (size_t)nd[pu + 2 * pv];
        H[2 * pu][2 * pv] = X[c];
        H[2 * pu + 1][2 * pv] = X[3 + c] * g->dxi1;
        H[2 * pu][2 * pv + 1] = X[6 + c] * g->dxi2;
        H[2 * pu + 1][2 * pv + 1] = X[9 + c] * g->dxi1 * g->dxi2;
      }
    /* along theta1 first (for each Hermite index b), then along theta2 */
    double U[4][4];
    for (int b = 0; b < 4; ++b) {
      double h[4] = {H[0][b], H[1][b], H[2][b], H[3][b]}, o[4];
      hermite_to_bezier(h, o);
      for (int i = 0; i < 4; ++i) U[i][b] = o[i];
    }
    for (int i = 0; i < 4; ++i) {
      double o[4];
      hermite_to_bezier(U[i], o);
      for (int j = 0; j < 4; ++j) P[i][j][c] = o[j];
    }
  }
}

/* Cubic Bernstein polynomials and their derivatives at t. */
static void bernstein(double t, double B[4], double dB[4]) {
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

/* x(u, v) and its local derivatives x_u, x_v of a Bezier patch: sums over j first, then i. */
void og_bezier_eval(const double P[4][4][3], double u, double v, double x[3], double xu[3], double xv[3]) {
  double Bu[4], dBu[4], Bv[4], dBv[4];
  bernstein(u, Bu, dBu);
  bernstein(v, Bv, dBv);
  for (int c = 0; c < 3; ++c) {
    double Q[4], R[4];
    for (int i = 0; i < 4; ++i) {
      Q[i] = ((Bv[0] * P[i][0][c] + Bv[1] * P[i][1][c]) + Bv[2] * P[i][2][c]) + Bv[3] * P[i][3][c];
      R[i] = ((dBv[0] * P[i][0][c] + dBv[1] * P[i][1][c]) + dBv[2] * P[i][2][c]) + dBv[3] * P[i][3][c];
    }
    x[c] = ((Bu[0] * Q[0] + Bu[1] * Q[1]) + Bu[2] * Q[2]) + Bu[3] * Q[3];
    xu[c] = ((dBu[0] * Q[0] + dBu[1] * Q[1]) + dBu[2] * Q[2]) + dBu[3] * Q[3];
    xv[c] = ((Bu[0] * R[0] + Bu[1] * R[1]) + Bu[2] * R[2]) + Bu[3] * R[3];
  }
}

static double lerp(double p, double q, double t) { return (1.0 - t) * p + t * q; }

/* Bezier points of the cubic with points in[0..3] restricted to [a, b]: blossom values
   f(a,a,a), f(a,a,b), f(a,b,b), f(b,b,b) by De Casteljau with one parameter per level. */
static void curve_restrict(const double in[4], double a, double b, double out[4]) {
  double A1[3], B1[3];
  for (int i = 0; i < 3; ++i) {
    A1[i] = lerp(in[i], in[i + 1], a);
    B1[i] = lerp(in[i], in[i + 1], b);
  }
  double AA[2], AB[2], BB[2];
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

/* Control points of the sub-patch [u0, u1] x [v0, v1] of P: each theta1-curve (fixed j) is
   restricted first, then each theta2-curve (fixed i). */
void og_bezier_sub(const double P[4][4][3], double u0, double u1, double v0, double v1, double S[4][4][3]) {
  for (int c = 0; c < 3; ++c) {
    double T[4][4];
    for (int j = 0; j < 4; ++j) {
      double in[4] = {P[0][j][c], P[1][j][c], P[2][j][c], P[3][j][c]}, o[4];
      curve_restrict(in, u0, u1, o);
      for (int i = 0; i < 4; ++i) T[i][j] = o[i];
    }
    for (int i = 0; i < 4; ++i) {
      double o[4];
      curve_restrict(T[i], v0, v1, o);
      for (int j = 0; j < 4; ++j) S[i][j][c] = o[j];
    }
  }
}

/* 2. Eq. ineqray for control points S: the interval [*t0, *t1] of tau >= 0 inside their box.
   inv[k] = 1 / d[k] (unused where d[k] = 0). *ext receives the box's largest side. Returns 0
   when no tau >= 0 is inside. */
int og_ray_box(const double S[4][4][3], const double o[3], const double d[3], const double inv[3],
               double* t0, double* t1, double* ext) {
  double lo = 0.0, hi = INFINITY, e = 0.0;
  for (int c = 0; c < 3; ++c) {
    double mn = S[0][0][c], mx = S[0][0][c];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const double s = S[i][j][c];
        if (s < mn) mn = s;
        if (s > mx) mx = s;
      }
    if (mx - mn > e) e = mx - mn;
    if (d[c] == 0.0) {
      if (o[c] < mn || o[c] > mx) return 0;
      continue;
    }
    double a = (mn - o[c]) * inv[c], b = (mx - o[c]) * inv[c];
    if (a > b) { const double t = a; a = b; b = t; }
    if (a > lo) lo = a;
    if (b < hi) hi = b;
  }
  if (lo > hi) return 0;
  *t0 = lo;
  *t1 = hi;
  *ext = e;
  return 1;
}

static double det3(const double M[3][3]) {
  return (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
          M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])) +
         M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* Newton's method on F(u, v, tau) = x(u, v) - o - tau d from (*u, *v, *tau), Jacobian
   [x_u | x_v | -d] solved by Cramer's rule. Returns 1 with the root on convergence; gives up when
   an iterate leaves the window win (u_min, u_max, v_min, v_max). */
static int newton_root(const double P[4][4][3], const double o[3], const double d[3], const double win[4],
                       double* u, double* v, double* tau, int* iters) {
  double uu = *u, vv = *v, tt = *tau;
  const double on = sqrt((o[0] * o[0] + o[1] * o[1]) + o[2] * o[2]);
  for (int it = 0; it < NEWTON_ITERS; ++it) {
    double x[3], xu[3], xv[3], F[3];
    ++*iters;
    og_bezier_eval(P, uu, vv, x, xu, xv);
    for (int c = 0; c < 3; ++c) F[c] = (x[c] - o[c]) - tt * d[c];
    const double fn = sqrt((F[0] * F[0] + F[1] * F[1]) + F[2] * F[2]);
    if (fn <= 1e-12 * ((1.0 + on) + fabs(tt))) {
      *u = uu; *v = vv; *tau = tt;
      return 1;
    }
    const double J[3][3] = {{xu[0], xv[0], -d[0]}, {xu[1], xv[1], -d[1]}, {xu[2], xv[2], -d[2]}};
    const double det = det3(J);
    if (!(fabs(det) > 1e-300)) return 0;
    double delta[3];
    for (int k = 0; k < 3; ++k) {
      double M[3][3];
      memcpy(M, J, sizeof(M));
      for (int r = 0; r < 3; ++r) M[r][k] = -F[r];
      delta[k] = det3(M) / det;
    }
    uu += delta[0]; vv += delta[1]; tt += delta[2];
    if (!isfinite(uu) || !isfinite(vv) || !isfinite(tt)) return 0;
    if (uu < win[0] || uu > win[1] || vv < win[2] || vv > win[3]) return 0;   /* left the window */
  }
  return 0;
}

/* 3. Binary min-heap of candidate sub-patches keyed by tau_min. */
typedef struct { double t0, t1, ext, u0, u1, v0, v1; int patch; } og_cand;
typedef struct { og_cand* a; int n, cap, peak, boxes; } og_heap;

static void heap_push(og_heap* h, og_cand c) {
  if (h->n == h->cap) {
    h->cap = h->cap ? 2 * h->cap : 64;
    h->a = (og_cand*)realloc(h->a, sizeof(og_cand) * (size_t)h->cap);
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

static og_cand heap_pop(og_heap* h) {
  const og_cand top = h->a[0], last = h->a[--h->n];
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

/* Pushes the sub-patch [u0, u1] x [v0, v1] of patch p when the ray enters its box before best. */
static void push_sub(og_heap* h, const double P[4][4][3], int p, double u0, double u1, double v0, double v1,
                     const double o[3], const double d[3], const double inv[3], double best) {
  if (!(u1 > u0) || !(v1 > v0)) return;
  double S[4][4][3], t0, t1, ext;
  ++h->boxes;
  og_bezier_sub(P, u0, u1, v0, v1, S);
  if (!og_ray_box(S, o, d, inv, &t0, &t1, &ext) || t0 >= best) return;
  const og_cand c = {t0, t1, ext, u0, u1, v0, v1, p};
  heap_push(h, c);
}

/* One ray o + tau d (unit d) against the control nets P[np] of all patches. Returns flags:
   bit 0 set on a hit (tau, patch, local (u, v) written), bit 1 set when MAX_EXPANSIONS was
   reached. stats (may be NULL): [0] candidates split, [1] largest heap size, [2] sub-patch boxes
   formed (patch roots included), [3] Newton iterations run. */
static int trace_one(const double (*P)[4][4][3], int np, const double o[3], const double d[3], int use_newton,
                     double* tau_out, int* patch_out, double* u_out, double* v_out, int stats[4]) {
  double inv[3];
  for (int c = 0; c < 3; ++c) inv[c] = d[c] != 0.0 ? 1.0 / d[c] : 0.0;
  og_heap h = {NULL, 0, 0, 0, 0};
  double best = INFINITY, bu = 0.0, bv = 0.0;
  int bp = -1, nexp = 0, flags = 0, newton_iters = 0;
  for (int p = 0; p < np; ++p) push_sub(&h, P[p], p, 0.0, 1.0, 0.0, 1.0, o, d, inv, best);
  while (h.n > 0) {
    const og_cand c = heap_pop(&h);
    if (c.t0 >= best - EPS_TAU) break;                         /* nothing left can be closer */
    if (c.ext <= EPS_TAU || (c.u1 - c.u0 < 1e-13 && c.v1 - c.v0 < 1e-13)) {   /* refined */
      const double t = 0.5 * (c.t0 + c.t1);
      if (t < best - EPS_TAU) {
        best = t; bp = c.patch; bu = 0.5 * (c.u0 + c.u1); bv = 0.5 * (c.v0 + c.v1);
      }
      continue;
    }
    if (nexp == MAX_EXPANSIONS) { flags |= 2; break; }
    ++nexp;
    const double (*Pp)[4][3] = P[c.patch];
    const double um = 0.5 * (c.u0 + c.u1), vm = 0.5 * (c.v0 + c.v1);
    if (use_newton) {
      double x[3], xu[3], xv[3];
      og_bezier_eval(Pp, um, vm, x, xu, xv);
      double u = um, v = vm, t = ((x[0] - o[0]) * d[0] + (x[1] - o[1]) * d[1]) + (x[2] - o[2]) * d[2];
      const double wu = c.u1 - c.u0, wv = c.v1 - c.v0;
      const double win[4] = {c.u0 - wu, c.u1 + wu, c.v0 - wv, c.v1 + wv};
      if (newton_root(Pp, o, d, win, &u, &v, &t, &newton_iters) && u >= c.u0 && u <= c.u1 && v >= c.v0 && v <= c.v1 && t >= 0.0) {
        if (t < best) { best = t; bp = c.patch; bu = u; bv = v; }
        /* Fig. subany: drop [a1, a2] x [b1, b2] around the root, four rectangles remain */
        const double hu = NBHD * (c.u1 - c.u0), hv = NBHD * (c.v1 - c.v0);
        const double a1 = fmax(c.u0, u - hu), a2 = fmin(c.u1, u + hu);
        const double b1 = fmax(c.v0, v - hv), b2 = fmin(c.v1, v + hv);
        push_sub(&h, Pp, c.patch, c.u0, a1, b1, c.v1, o, d, inv, best);
        push_sub(&h, Pp, c.patch, a1, c.u1, b2, c.v1, o, d, inv, best);
        push_sub(&h, Pp, c.patch, c.u0, a2, c.v0, b1, o, d, inv, best);
        push_sub(&h, Pp, c.patch, a2, c.u1, c.v0, b2, o, d, inv, best);
        continue;
      }
    }
    /* Fig. submid: four quarters at the parameter midpoint */
    push_sub(&h, Pp, c.patch, c.u0, um, vm, c.v1, o, d, inv, best);
    push_sub(&h, Pp, c.patch, um, c.u1, vm, c.v1, o, d, inv, best);
    push_sub(&h, Pp, c.patch, c.u0, um, c.v0, vm, o, d, inv, best);
    push_sub(&h, Pp, c.patch, um, c.u1, c.v0, vm, o, d, inv, best);
  }
  free(h.a);
  if (stats) { stats[0] = nexp; stats[1] = h.peak; stats[2] = h.boxes; stats[3] = newton_iters; }
  if (bp >= 0) {
    flags |= 1;
    *tau_out = best; *patch_out = bp; *u_out = bu; *v_out = bv;
  }
  return flags;
}

/* Many rays: origins, dirs [n][3]. Outputs: tau [n] (INFINITY on a miss), patch [n] (-1 on a
   miss), uv [n][2] (local parameters, 0 on a miss), flags [n] (as trace_one), stats [n][4]
   (may be NULL). Control nets are formed once for all rays. */
void og_trace_rays(const og_grid* g, const double* q, int n, const double* origins, const double* dirs,
                   int use_newton, double* tau, int* patch, double* uv, int* flags, int* stats) {
  const int np = g->nu * g->nv;
  double (*P)[4][4][3] = (double(*)[4][4][3])malloc(sizeof(double) * 48 * (size_t)np);
  for (int p = 0; p < np; ++p) og_bezier_patch(g, q, p, P[p]);
  /* queries are independent (each keeps its own heap): all host cores with OpenMP */
#pragma omp parallel for schedule(dynamic, 16) if (n >= 256)
  for (int k = 0; k < n; ++k) {
    double t = INFINITY, u = 0.0, v = 0.0;
    int p = -1;
    const int f = trace_one((const double(*)[4][4][3])P, np, origins + 3 * (size_t)k, dirs + 3 * (size_t)k,
                            use_newton, &t, &p, &u, &v, stats ? stats + 4 * (size_t)k : NULL);
    if (f & 1) {
      tau[k] = t; patch[k] = p; uv[2 * k] = u; uv[2 * k + 1] = v;
    } else {
      tau[k] = INFINITY; patch[k] = -1; uv[2 * k] = uv[2 * k + 1] = 0.0;
    }
    flags[k] = f;
  }
  free(P);
}
