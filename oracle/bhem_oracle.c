/*
 * Plain FP64 CPU oracle of the BHEM hot path (bicubic Hermite elements for Kirchhoff-Love
 * shells, arXiv 2312.14839).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the bench's CPU-baseline leg use this
 * code. The CUDA library never calls, links or includes it, and it shares no code, header or
 * table with the CUDA path.
 *
 * Each routine follows the paper's definitions in the paper's order, without blocking, fusion
 * or reordering, so that it can be checked against the paper by eye:
 *   - Hermite basis w_{p,r} and first derivatives: App. A.1. Second derivatives are the
 *     derivatives of the same cubics (the paper does not print them).
 *   - 4x4 Gauss-Legendre rule: App. A.2 (nodes and weights given in closed form there).
 *   - Midsurface geometry, 1st/2nd fundamental forms: Sec. 3.1-3.2.
 *   - Energy density (St. Venant-Kirchhoff, thickness-integrated): Sec. 3.3 (areal density
 *     V_e = (A A h + B B h^3/3) H^{abgd}, H^{abgd} = lambda/2 a^{ab} a^{gd} + mu a^{bg} a^{ad}).
 *   - Gradient: App. B.1 (Voigt form, Eq. matrix with Eq. paabpqi and Eq. pbabpqi).
 *   - Hessian: App. B.2 (G1, G2, second derivatives of alpha and of b, D^{gamma delta}); the
 *     pseudo Hessian ("The pseudo Hessian", App. B) drops the d^2 beta / dq dq term.
 *   - Mass matrix: Eq. mass; gravity: Sec. 4.3 ("External Forces").
 *   - Time step: implicit Euler (Eq. implicit) solved by Newton with a line search (Sec. 6.1);
 *     the linear solve is block-Jacobi PCG with the diagonal regulariser of Sec. 6.1.
 *
 * Readings of the paper used here (where it is silent or ambiguous):
 *   - Derivative DOFs are derivatives w.r.t. the global parameters; a shape function is
 *     (dxi1)^r (dxi2)^s w_{p,r}(theta1) w_{q,s}(theta2).
 *   - "tau" in App. B is the thickness h; the "beta_{alpha beta}" inside D^{gamma delta} is the
 *     deformed b_{alpha beta}.
 *   - Line search: Armijo (c1 = 1e-4) from alpha = 1, then a quadratic and afterwards cubic
 *     interpolation (Nocedal-Wright Sec. 3.5), each clamped to [0.1, 0.5] of the last step, at
 *     most 20 trials; alpha = 1 is accepted without a test once |g| <= 1e-6 |g_ref|.
 *   - Regulariser (Sec. 6.1 adds "a diagonal regularizer" to make the matrix positive definite,
 *     with no form or magnitude), in two parts. D is diagonal: for each DOF kind (x, x_,1, x_,2,
 *     x_,12) the mean of |A_ii| over the free DOFs of that kind (positive, and scaled like each
 *     kind's stiffness). Local part: every free diagonal entry A_ii <= 0 is replaced by
 *     max(-A_ii, 1e-8 D_k), its magnitude, so that the diagonal is positive without shifting the
 *     entries that already are. Global part: PCG solves (A + tau D) d = -g; tau starts at a tenth
 *     of the previous Newton iteration's accepted tau (at the first iteration, of the level the
 *     caller carries in, 0 by default; 0 when a tenth is below 1e-8), each time PCG meets
 *     p^T A p <= 0 the solve restarts with
 *     tau = max(10 tau, 1e-8), and beyond tau = 1e4 the step gives up. A 12x12 block that is not
 *     SPD is replaced by the inverse of its diagonal in the block-Jacobi preconditioner.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------------ */
/* Types shared with the Python wrapper (plain structs of ints and doubles).                   */
/* ------------------------------------------------------------------------------------------ */
typedef struct { int nu, nv, periodic_u, periodic_v; double dxi1, dxi2; } og_grid;
typedef struct { double young, poisson, thickness, density; } og_material;
typedef struct {
  double dt, gravity[3], newton_rtol;
  int newton_max;
  double pcg_rtol;
  int pcg_max, pcg_fixed_iters;
  int pseudo_hessian;   /* 1: Newton matrix with the pseudo Hessian (App. B, "The pseudo Hessian") */
  double tau_carry;     /* regulariser level carried in: the first iteration starts at a tenth */
} og_step_params;
typedef struct {
  int newton_iters, pcg_iters_total, ls_backtracks, regularizations, status;
  int diag_fixes;   /* free diagonal entries replaced by the local part of the regulariser */
  double res0, res_final;
  double tau_final; /* tau of the last accepted solve */
} og_step_stats;

enum { OG_OK = 0, OG_ERR_ARG = 1, OG_ERR_NOT_CONVERGED = 6, OG_ERR_LINESEARCH = 7,
       OG_ERR_INDEFINITE = 8, OG_PCG_NEG_CURV = 100 };

/* Host threads of the independent per-patch and per-row loops (OpenMP builds; 1 otherwise).
   Results do not depend on the count: sums over patches and dot products stay serial. */
int og_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Small vector helpers                                                                       */
/* ------------------------------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1]*b[2] - a[2]*b[1];
  c[1] = a[2]*b[0] - a[0]*b[2];
  c[2] = a[0]*b[1] - a[1]*b[0];
}
/* [v]: the cross-product matrix of v (App. B.2), [v] w = v x w. */
static void crossmat(const double* v, double m[3][3]) {
  m[0][0] = 0.0;   m[0][1] = -v[2]; m[0][2] = v[1];
  m[1][0] = v[2];  m[1][1] = 0.0;   m[1][2] = -v[0];
  m[2][0] = -v[1]; m[2][1] = v[0];  m[2][2] = 0.0;
}
/* u (x) v = u v^T */
static void outer3(const double* u, const double* v, double m[3][3]) {
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) m[i][j] = u[i] * v[j];
}

/* ------------------------------------------------------------------------------------------ */
/* App. A.1: cubic Hermite basis                                                              */
/* ------------------------------------------------------------------------------------------ */
static double f0(double t) { return 2*t*t*t - 3*t*t + 1; }
static double g0(double t) { return t*t*t - 2*t*t + t; }
static double f1(double t) { return 6*t*t - 6*t; }          /* f' */
static double g1(double t) { return 3*t*t - 4*t + 1; }      /* g' */
static double f2(double t) { return 12*t - 6; }             /* f'' */
static double g2(double t) { return 6*t - 4; }              /* g'' */

/* d-th derivative (d = 0, 1, 2) of w_{p,r}(theta) with respect to theta. */
double og_hermite_w(int p, int r, double t, int d) {
  if (p == 0 && r == 0) return d == 0 ? f0(t) : d == 1 ? f1(t) : f2(t);
  if (p == 1 && r == 0) return d == 0 ? f0(1 - t) : d == 1 ? -f1(1 - t) : f2(1 - t);
  if (p == 0 && r == 1) return d == 0 ? g0(t) : d == 1 ? g1(t) : g2(t);
  /* p == 1 && r == 1 */ return d == 0 ? -g0(1 - t) : d == 1 ? g1(1 - t) : -g2(1 - t);
}

/* App. A.2: 4-point Gauss-Legendre nodes and weights on [-1, 1], ascending nodes.
   Inner nodes +-sqrt(3/7 - 2/7 sqrt(6/5)) carry (18 + sqrt 30)/36, outer ones (18 - sqrt 30)/36
   (the paper's per-line factors (18 +- sqrt 30) dxi / 72 are these times dxi / 2). */
void og_gauss4(double x[4], double w[4]) {
  double xi = sqrt(3.0/7.0 - 2.0/7.0 * sqrt(6.0/5.0));
  double xo = sqrt(3.0/7.0 + 2.0/7.0 * sqrt(6.0/5.0));
  double wi = (18.0 + sqrt(30.0)) / 36.0, wo = (18.0 - sqrt(30.0)) / 36.0;
  x[0] = -xo; x[1] = -xi; x[2] = xi; x[3] = xo;
  w[0] = wo;  w[1] = wi;  w[2] = wi; w[3] = wo;
}

/* Shape functions of one patch (Eq. hermite, Eq. hermite_weight, Eq. shape) at (theta1, theta2).
   Local index I = corner * 4 + kind, corner = p + 2 q, kind = r + 2 s.
   phi[I][0..5] = Phi, Phi_,1, Phi_,2, Phi_,11, Phi_,22, Phi_,12 (derivatives w.r.t. xi). */
void og_shape(double d1, double d2, double t1, double t2, double phi[16][6]) {
  for (int q = 0; q < 2; ++q) for (int p = 0; p < 2; ++p)
    for (int s = 0; s < 2; ++s) for (int r = 0; r < 2; ++r) {
      int I = (p + 2*q) * 4 + (r + 2*s);
      double sc = (r ? d1 : 1.0) * (s ? d2 : 1.0);
      double u0 = og_hermite_w(p, r, t1, 0), u1 = og_hermite_w(p, r, t1, 1), u2 = og_hermite_w(p, r, t1, 2);
      double v0 = og_hermite_w(q, s, t2, 0), v1 = og_hermite_w(q, s, t2, 1), v2 = og_hermite_w(q, s, t2, 2);
      phi[I][0] = sc * u0 * v0;
      phi[I][1] = sc * u1 * v0 / d1;
      phi[I][2] = sc * u0 * v1 / d2;
      phi[I][3] = sc * u2 * v0 / (d1 * d1);
      phi[I][4] = sc * u0 * v2 / (d2 * d2);
      phi[I][5] = sc * u1 * v1 / (d1 * d2);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Grid topology (Sec. 4.1 regular grid embedding, Sec. 4.2 periodic boundary conditions)      */
/* ------------------------------------------------------------------------------------------ */
static int n1_of(const og_grid* g) { return g->periodic_u ? g->nu : g->nu + 1; }
static int n2_of(const og_grid* g) { return g->periodic_v ? g->nv : g->nv + 1; }
int og_n_nodes(const og_grid* g) { return n1_of(g) * n2_of(g); }

/* Node ids of the corners 00, 10, 01, 11 of patch (pu, pv); periodic wrap merges nodes. */
void og_patch_nodes(const og_grid* g, int patch, int nodes[4]) {
  int n1 = n1_of(g), n2 = n2_of(g);
  int pu = patch % g->nu, pv = patch / g->nu;
  for (int q = 0; q < 2; ++q) for (int p = 0; p < 2; ++p) {
    int i = (pu + p) % n1, j = (pv + q) % n2;
    nodes[p + 2*q] = j * n1 + i;
  }
}

static void gather48(const og_grid* g, const double* nodal, int patch, double out[48]) {
  int nd[4];
  og_patch_nodes(g, patch, nd);
  for (int c = 0; c < 4; ++c) for (int k = 0; k < 12; ++k) out[c*12 + k] = nodal[nd[c]*12 + k];
}

/* ------------------------------------------------------------------------------------------ */
/* Geometry at one Gauss point (Sec. 3.1-3.2)                                                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  double x[3], a1[3], a2[3], c[3][3];  /* c[0] = a_{1,1}, c[1] = a_{2,2}, c[2] = a_{1,2} */
  double n[3], sqa, a3[3];
  double a11, a22, a12, b[3];          /* b[0] = b_11, b[1] = b_22, b[2] = b_12 */
} og_geo;

static void geometry(const double q[48], double phi[16][6], og_geo* G) {
  memset(G, 0, sizeof(*G));
  for (int I = 0; I < 16; ++I) for (int k = 0; k < 3; ++k) {
    double v = q[I*3 + k];
    G->x[k]    += phi[I][0] * v;
    G->a1[k]   += phi[I][1] * v;
    G->a2[k]   += phi[I][2] * v;
    G->c[0][k] += phi[I][3] * v;
    G->c[1][k] += phi[I][4] * v;
    G->c[2][k] += phi[I][5] * v;
  }
  cross3(G->a1, G->a2, G->n);
  G->sqa = sqrt(dot3(G->n, G->n));
  for (int k = 0; k < 3; ++k) G->a3[k] = G->n[k] / G->sqa;
  G->a11 = dot3(G->a1, G->a1);
  G->a22 = dot3(G->a2, G->a2);
  G->a12 = dot3(G->a1, G->a2);
  for (int m = 0; m < 3; ++m) G->b[m] = dot3(G->c[m], G->a3);
}

static void lame(const og_material* m, double* lam, double* mu) {
  *lam = m->young * m->poisson / (1.0 - m->poisson * m->poisson);
  *mu = m->young / (2.0 * (1.0 + m->poisson));
}

/* ------------------------------------------------------------------------------------------ */
/* Element energy: the plain definition (Sec. 3.3), integrated with the 4x4 Gauss rule.        */
/* ------------------------------------------------------------------------------------------ */
double og_element_energy(const double q[48], const double qb[48], double d1, double d2,
                         const og_material* mat) {
  double lam, mu, h = mat->thickness, gx[4], gw[4], E = 0.0;
  lame(mat, &lam, &mu);
  og_gauss4(gx, gw);
  for (int j = 0; j < 4; ++j) for (int i = 0; i < 4; ++i) {
    double phi[16][6];
    og_shape(d1, d2, 0.5 * (1 + gx[i]), 0.5 * (1 + gx[j]), phi);
    double W = (0.5 * d1 * gw[i]) * (0.5 * d2 * gw[j]);
    og_geo G, R;
    geometry(q, phi, &G);
    geometry(qb, phi, &R);
    /* a_{ab}, b_{ab}, rest contravariant metric a^{ab} = (a_{ab})^{-1} */
    double a[2][2] = {{G.a11, G.a12}, {G.a12, G.a22}};
    double ab[2][2] = {{R.a11, R.a12}, {R.a12, R.a22}};
    double b[2][2] = {{G.b[0], G.b[2]}, {G.b[2], G.b[1]}};
    double bb[2][2] = {{R.b[0], R.b[2]}, {R.b[2], R.b[1]}};
    double det = ab[0][0]*ab[1][1] - ab[0][1]*ab[1][0];
    double ai[2][2] = {{ab[1][1]/det, -ab[0][1]/det}, {-ab[1][0]/det, ab[0][0]/det}};
    double A[2][2], B[2][2];
    for (int x = 0; x < 2; ++x) for (int y = 0; y < 2; ++y) {
      A[x][y] = 0.5 * (a[x][y] - ab[x][y]);
      B[x][y] = 0.5 * (b[x][y] - bb[x][y]);
    }
    double V = 0.0;
    for (int al = 0; al < 2; ++al) for (int be = 0; be < 2; ++be)
      for (int ga = 0; ga < 2; ++ga) for (int de = 0; de < 2; ++de) {
        double H = 0.5 * lam * ai[al][be] * ai[ga][de] + mu * ai[be][ga] * ai[al][de];
        V += (A[al][be] * A[ga][de] * h + B[al][be] * B[ga][de] * h * h * h / 3.0) * H;
      }
    E += W * sqrt(det) * V;  /* d(Omega bar) = sqrt(a bar) dxi1 dxi2 */
  }
  return E;
}

/* Voigt matrix H of App. B.1 from the rest contravariant metric. */
static void voigt_H(double lam, double mu, double ai11, double ai22, double ai12, double H[3][3]) {
  H[0][0] = (lam + 2*mu) * ai11 * ai11;
  H[0][1] = lam * ai11 * ai22 + 2*mu * ai12 * ai12;
  H[0][2] = (lam + 2*mu) * ai11 * ai12;
  H[1][1] = (lam + 2*mu) * ai22 * ai22;
  H[1][2] = (lam + 2*mu) * ai12 * ai22;
  H[2][2] = (lam + mu) * ai12 * ai12 + mu * ai11 * ai22;
  H[1][0] = H[0][1]; H[2][0] = H[0][2]; H[2][1] = H[1][2];
}

/* ------------------------------------------------------------------------------------------ */
/* Element energy, gradient (App. B.1) and exact Hessian (App. B.2), or with pseudo != 0 the     */
/* pseudo Hessian of App. B: the same without the d^2 beta_i / dq_J dq_I term.                  */
/* grad[I*3+c], hess[(I*3+c)*48 + (J*3+d)], local I = corner*4 + kind.                          */
/* ------------------------------------------------------------------------------------------ */
void og_element_egh(const double q[48], const double qb[48], double d1, double d2,
                    const og_material* mat, double* E_out, double* grad, double* hess, int pseudo) {
  double lam, mu, h = mat->thickness, gx[4], gw[4];
  double h3 = h * h * h;
  lame(mat, &lam, &mu);
  og_gauss4(gx, gw);
  if (grad) memset(grad, 0, 48 * sizeof(double));
  if (hess) memset(hess, 0, 48 * 48 * sizeof(double));
  if (E_out) *E_out = og_element_energy(q, qb, d1, d2, mat);
  if (!grad && !hess) return;

  for (int j = 0; j < 4; ++j) for (int i = 0; i < 4; ++i) {
    double phi[16][6];
    og_shape(d1, d2, 0.5 * (1 + gx[i]), 0.5 * (1 + gx[j]), phi);
    double W = (0.5 * d1 * gw[i]) * (0.5 * d2 * gw[j]);
    og_geo G, R;
    geometry(q, phi, &G);
    geometry(qb, phi, &R);
    double det = R.a11 * R.a22 - R.a12 * R.a12;      /* a bar */
    double sqab = sqrt(det);
    double ai11 = R.a22 / det, ai22 = R.a11 / det, ai12 = -R.a12 / det;
    double Hv[3][3];
    voigt_H(lam, mu, ai11, ai22, ai12, Hv);
    /* alpha = (A11, A22, 2 A12), beta = 2 (B11, B22, 2 B12) */
    double alpha[3] = {0.5 * (G.a11 - R.a11), 0.5 * (G.a22 - R.a22), (G.a12 - R.a12)};
    double beta[3] = {G.b[0] - R.b[0], G.b[1] - R.b[1], 2.0 * (G.b[2] - R.b[2])};
    double Ha[3], Hb[3];
    for (int r = 0; r < 3; ++r) {
      Ha[r] = Hv[r][0]*alpha[0] + Hv[r][1]*alpha[1] + Hv[r][2]*alpha[2];
      Hb[r] = Hv[r][0]*beta[0] + Hv[r][1]*beta[1] + Hv[r][2]*beta[2];
    }
    double wgt = W * sqab;

    /* First derivatives per generalised coordinate (Eq. paabpqi, Eq. pbabpqi):
       da[I][row][c]: row 0..2 = d alpha_i / d q_I; db[I][row][c] = d beta_i / d q_I. */
    double da[16][3][3], db[16][3][3], a2xa3[3], a3xa1[3];
    cross3(G.a2, G.a3, a2xa3);
    cross3(G.a3, G.a1, a3xa1);
    for (int I = 0; I < 16; ++I) {
      double P1 = phi[I][1], P2 = phi[I][2];
      for (int c = 0; c < 3; ++c) {
        /* d alpha / d q_I = 1/2 (d a11, d a22, 2 d a12), d a_ab = Phi_a a_b + Phi_b a_a */
        da[I][0][c] = 0.5 * (2.0 * P1 * G.a1[c]);
        da[I][1][c] = 0.5 * (2.0 * P2 * G.a2[c]);
        da[I][2][c] = 0.5 * 2.0 * (P1 * G.a2[c] + P2 * G.a1[c]);
      }
      double dbab[3][3];
      for (int m = 0; m < 3; ++m) {   /* m = 11, 22, 12 */
        const double* cm = G.c[m];
        double a2xc[3], cxa1[3];
        cross3(G.a2, cm, a2xc);
        cross3(cm, G.a1, cxa1);
        double cdota3 = dot3(cm, G.a3);
        double Pab = phi[I][3 + m];
        for (int c = 0; c < 3; ++c)
          dbab[m][c] = Pab * G.a3[c] +
                       (P1 * a2xc[c] + P2 * cxa1[c] - cdota3 * (P1 * a2xa3[c] + P2 * a3xa1[c])) / G.sqa;
      }
      for (int c = 0; c < 3; ++c) {
        db[I][0][c] = dbab[0][c];
        db[I][1][c] = dbab[1][c];
        db[I][2][c] = 2.0 * dbab[2][c];
      }
    }

    if (grad) {   /* Eq. matrix */
      for (int I = 0; I < 16; ++I) for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int r = 0; r < 3; ++r) s += h * da[I][r][c] * Ha[r] + h3 / 12.0 * db[I][r][c] * Hb[r];
        grad[I*3 + c] += wgt * s;
      }
    }
    if (!hess) continue;

    /* Second-order pieces (App. B.2). t1 = a2 x a3, t2 = a3 x a1; per m: s1 = c x a1, s2 = a2 x c */
    double t1[3], t2[3], D11[3][3][3], D22[3][3][3], D12[3][3][3], D21[3][3][3];
    cross3(G.a2, G.a3, t1);
    cross3(G.a3, G.a1, t2);
    double a = G.sqa * G.sqa;
    for (int m = 0; m < 3; ++m) {
      const double* cm = G.c[m];
      double s1[3], s2[3], bm = G.b[m], C[3][3];
      cross3(cm, G.a1, s1);
      cross3(G.a2, cm, s2);
      crossmat(cm, C);
      for (int x = 0; x < 3; ++x) for (int y = 0; y < 3; ++y) {
        double id = (x == y) ? 1.0 : 0.0;
        D11[m][x][y] = (bm * (3*t1[x]*t1[y] + G.a2[x]*G.a2[y] - G.a22*id) - s2[x]*t1[y] - t1[x]*s2[y]) / a;
        D22[m][x][y] = (bm * (3*t2[x]*t2[y] + G.a1[x]*G.a1[y] - G.a11*id) - s1[x]*t2[y] - t2[x]*s1[y]) / a;
        D12[m][x][y] = (bm * (3*t1[x]*t2[y] - 2*G.a1[x]*G.a2[y] + G.a2[x]*G.a1[y] + G.a12*id)
                        - s2[x]*t2[y] - t1[x]*s1[y] - G.sqa * C[x][y]) / a;
        D21[m][x][y] = (bm * (3*t2[x]*t1[y] - 2*G.a2[x]*G.a1[y] + G.a1[x]*G.a2[y] + G.a12*id)
                        - s1[x]*t1[y] - t2[x]*s2[y] + G.sqa * C[x][y]) / a;
      }
    }
    /* d a3 / d q_I = 1/sqrt(a) (-Phi_1 [a2] + Phi_2 [a1] - a3 (x) (Phi_1 t1 + Phi_2 t2)) */
    double da3[16][3][3], A1x[3][3], A2x[3][3];
    crossmat(G.a1, A1x);
    crossmat(G.a2, A2x);
    for (int I = 0; I < 16; ++I) {
      double P1 = phi[I][1], P2 = phi[I][2], v[3], o[3][3];
      for (int c = 0; c < 3; ++c) v[c] = P1 * t1[c] + P2 * t2[c];
      outer3(G.a3, v, o);
      for (int x = 0; x < 3; ++x) for (int y = 0; y < 3; ++y)
        da3[I][x][y] = (-P1 * A2x[x][y] + P2 * A1x[x][y] - o[x][y]) / G.sqa;
    }

    for (int I = 0; I < 16; ++I) for (int J = 0; J < 16; ++J) {
      double P1I = phi[I][1], P2I = phi[I][2], P1J = phi[J][1], P2J = phi[J][2];
      double G1[3][3], G2[3][3];
      for (int x = 0; x < 3; ++x) for (int y = 0; y < 3; ++y) {
        double s1v = 0.0, s2v = 0.0;
        for (int r = 0; r < 3; ++r) for (int t = 0; t < 3; ++t) {
          s1v += da[I][r][x] * Hv[r][t] * da[J][t][y];
          s2v += db[I][r][x] * Hv[r][t] * db[J][t][y];
        }
        G1[x][y] = s1v;
        G2[x][y] = s2v;
      }
      /* sum_i H^{ij} alpha_j d^2 alpha_i = (H alpha)_i d^2 alpha_i */
      double d2a0 = P1I * P1J, d2a1 = P2I * P2J, d2a2 = P1I * P2J + P2I * P1J;
      for (int x = 0; x < 3; ++x) G1[x][x] += Ha[0] * d2a0 + Ha[1] * d2a1 + Ha[2] * d2a2;
      /* d^2 b_{ab} / dq_J dq_I, then d^2 beta = (d^2 b11, d^2 b22, 2 d^2 b12); the pseudo
         Hessian leaves this term out */
      for (int m = 0; m < 3 && !pseudo; ++m) {
        double wm = (m == 2) ? 2.0 * Hb[2] : Hb[m];
        double PabI = phi[I][3 + m], PabJ = phi[J][3 + m];
        for (int x = 0; x < 3; ++x) for (int y = 0; y < 3; ++y) {
          double d2b = PabI * da3[J][x][y] + PabJ * da3[I][y][x]
                     + P1I * P1J * D11[m][x][y] + P2I * P2J * D22[m][x][y]
                     + P1I * P2J * D12[m][x][y] + P2I * P1J * D21[m][x][y];
          G2[x][y] += wm * d2b;
        }
      }
      for (int x = 0; x < 3; ++x) for (int y = 0; y < 3; ++y)
        hess[(I*3 + x) * 48 + (J*3 + y)] += wgt * (h * G1[x][y] + h3 / 12.0 * G2[x][y]);
    }
  }
}

/* Consistent mass (Eq. mass) and gravity load factors of one patch with the same 4x4 rule:
   m[I*16+J] = int rho h Phi^I Phi^J sqrt(a bar), f[I] = int rho h Phi^I sqrt(a bar). */
void og_element_mass(const double qb[48], double d1, double d2, const og_material* mat,
                     double* m, double* f) {
  double gx[4], gw[4], rh = mat->density * mat->thickness;
  og_gauss4(gx, gw);
  memset(m, 0, 256 * sizeof(double));
  memset(f, 0, 16 * sizeof(double));
  for (int j = 0; j < 4; ++j) for (int i = 0; i < 4; ++i) {
    double phi[16][6];
    og_shape(d1, d2, 0.5 * (1 + gx[i]), 0.5 * (1 + gx[j]), phi);
    double W = (0.5 * d1 * gw[i]) * (0.5 * d2 * gw[j]);
    og_geo R;
    geometry(qb, phi, &R);
    double sqab = sqrt(R.a11 * R.a22 - R.a12 * R.a12);
    for (int I = 0; I < 16; ++I) {
      f[I] += W * rh * phi[I][0] * sqab;
      for (int J = 0; J < 16; ++J) m[I*16 + J] += W * rh * phi[I][0] * phi[J][0] * sqab;
    }
  }
}

/* Per-patch outputs over a patch range (for element-by-element comparison). */
void og_elements(const og_grid* g, const og_material* mat, const double* rest, const double* q,
                 int p0, int p1, double* E, double* grad, double* hess, int pseudo) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int p = p0; p < p1; ++p) {
    double ql[48], qbl[48];
    gather48(g, q, p, ql);
    gather48(g, rest, p, qbl);
    og_element_egh(ql, qbl, g->dxi1, g->dxi2, mat, E ? &E[p - p0] : NULL,
                   grad ? &grad[(size_t)(p - p0) * 48] : NULL,
                   hess ? &hess[(size_t)(p - p0) * 2304] : NULL, pseudo);
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Block sparse (12x12 BSR) pattern and assembly (Sec. 4.3 "Properties of the mass matrix":     */
/* two generalised coordinates couple iff their nodes share a patch).                          */
/* ------------------------------------------------------------------------------------------ */
/* Returns the number of blocks; fills row_ptr[n+1] and col[] (sorted per row) when non-NULL. */
int og_bsr_pattern(const og_grid* g, int* row_ptr, int* col) {
  int n = og_n_nodes(g), np = g->nu * g->nv;
  int cap = 16;
  int* nb = (int*)calloc((size_t)n * cap, sizeof(int));
  int* cnt = (int*)calloc((size_t)n, sizeof(int));
  for (int p = 0; p < np; ++p) {
    int nd[4];
    og_patch_nodes(g, p, nd);
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) {
      int r = nd[a], c = nd[b], seen = 0;
      for (int k = 0; k < cnt[r]; ++k) if (nb[r*cap + k] == c) { seen = 1; break; }
      if (!seen) nb[r*cap + cnt[r]++] = c;
    }
  }
  int total = 0;
  for (int r = 0; r < n; ++r) {
    for (int x = 1; x < cnt[r]; ++x)   /* insertion sort of the row */
      for (int y = x; y > 0 && nb[r*cap + y - 1] > nb[r*cap + y]; --y) {
        int t = nb[r*cap + y]; nb[r*cap + y] = nb[r*cap + y - 1]; nb[r*cap + y - 1] = t;
      }
    if (row_ptr) row_ptr[r] = total;
    if (col) for (int k = 0; k < cnt[r]; ++k) col[total + k] = nb[r*cap + k];
    total += cnt[r];
  }
  if (row_ptr) row_ptr[n] = total;
  free(nb);
  free(cnt);
  return total;
}

static int find_block(const int* row_ptr, const int* col, int r, int c) {
  for (int k = row_ptr[r]; k < row_ptr[r + 1]; ++k) if (col[k] == c) return k;
  return -1;
}

/* Assembled elastic energy, gradient [n*12] and K + mass_scale * M into val[nblocks*144]
   (any output may be NULL); K is the pseudo Hessian when pseudo != 0. */
void og_assemble(const og_grid* g, const og_material* mat, const double* rest, const double* q,
                 const int* row_ptr, const int* col, double mass_scale,
                 double* energy, double* grad, double* val, int pseudo) {
  int n = og_n_nodes(g), np = g->nu * g->nv;
  if (energy) *energy = 0.0;
  if (grad) memset(grad, 0, (size_t)n * 12 * sizeof(double));
  if (val) memset(val, 0, (size_t)row_ptr[n] * 144 * sizeof(double));
  /* The patches' element terms are independent: a chunk of them is evaluated (on all host cores
     when built with OpenMP), then added in patch order, so the sums do not depend on the threads. */
  enum { CHUNK = 64 };
  double* Ec = (double*)malloc(CHUNK * sizeof(double));
  double* Gc = (double*)malloc((size_t)CHUNK * 48 * sizeof(double));
  double* Hc = val ? (double*)malloc((size_t)CHUNK * 2304 * sizeof(double)) : NULL;
  for (int p0 = 0; p0 < np; p0 += CHUNK) {
    int p1 = p0 + CHUNK < np ? p0 + CHUNK : np;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = p0; p < p1; ++p) {
      double ql[48], qbl[48], m[256], f[16];
      double* H = val ? &Hc[(size_t)(p - p0) * 2304] : NULL;
      gather48(g, q, p, ql);
      gather48(g, rest, p, qbl);
      og_element_egh(ql, qbl, g->dxi1, g->dxi2, mat, energy ? &Ec[p - p0] : NULL,
                     grad ? &Gc[(size_t)(p - p0) * 48] : NULL, H, pseudo);
      if (val && mass_scale != 0.0) {
        og_element_mass(qbl, g->dxi1, g->dxi2, mat, m, f);
        for (int I = 0; I < 16; ++I) for (int J = 0; J < 16; ++J)
          for (int c = 0; c < 3; ++c) H[(I*3 + c)*48 + J*3 + c] += mass_scale * m[I*16 + J];
      }
    }
    for (int p = p0; p < p1; ++p) {
      int nd[4];
      og_patch_nodes(g, p, nd);
      const double* ge = &Gc[(size_t)(p - p0) * 48];
      if (energy) *energy += Ec[p - p0];
      if (grad) for (int c = 0; c < 4; ++c) for (int k = 0; k < 12; ++k) grad[nd[c]*12 + k] += ge[c*12 + k];
      if (!val) continue;
      const double* H = &Hc[(size_t)(p - p0) * 2304];
      for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) {
        int k = find_block(row_ptr, col, nd[a], nd[b]);
        for (int x = 0; x < 12; ++x) for (int y = 0; y < 12; ++y)
          val[(size_t)k*144 + x*12 + y] += H[(a*12 + x)*48 + b*12 + y];
      }
    }
  }
  free(Ec); free(Gc); free(Hc);
}

/* Nodal mass in the same pattern as 4x4 scalar blocks mval[nblocks*16] (M = mval (x) I3), and
   gravity load factors fs[n*4] (F = fs (x) g). */
void og_mass(const og_grid* g, const og_material* mat, const double* rest,
             const int* row_ptr, const int* col, double* mval, double* fs) {
  int n = og_n_nodes(g), np = g->nu * g->nv;
  memset(mval, 0, (size_t)row_ptr[n] * 16 * sizeof(double));
  memset(fs, 0, (size_t)n * 4 * sizeof(double));
  for (int p = 0; p < np; ++p) {
    double qbl[48], m[256], f[16];
    int nd[4];
    og_patch_nodes(g, p, nd);
    gather48(g, rest, p, qbl);
    og_element_mass(qbl, g->dxi1, g->dxi2, mat, m, f);
    for (int a = 0; a < 4; ++a) {
      for (int r = 0; r < 4; ++r) fs[nd[a]*4 + r] += f[a*4 + r];
      for (int b = 0; b < 4; ++b) {
        int k = find_block(row_ptr, col, nd[a], nd[b]);
        for (int r = 0; r < 4; ++r) for (int s = 0; s < 4; ++s)
          mval[(size_t)k*16 + r*4 + s] += m[(a*4 + r)*16 + b*4 + s];
      }
    }
  }
}

/* y = M x with the 4x4-block scalar mass. */
static void mass_mult(int n, const int* row_ptr, const int* col, const double* mval,
                      const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double acc[12] = {0};
    for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      int j = col[k];
      for (int r = 0; r < 4; ++r) for (int s = 0; s < 4; ++s) for (int c = 0; c < 3; ++c)
        acc[r*3 + c] += mval[(size_t)k*16 + r*4 + s] * x[j*12 + s*3 + c];
    }
    memcpy(&y[i*12], acc, sizeof(acc));
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Block-Jacobi PCG (replaces the direct LDL^T solve of Sec. 6.1).                              */
/* A is the 12x12 BSR; fixed DOFs (mask != 0) get identity rows and columns. tau adds           */
/* tau * dbar[kind] to the free diagonal (the regulariser; dbar[k] = mean |A_ii| of kind k).    */
/* ------------------------------------------------------------------------------------------ */
static void bsr_mult(int n, const int* row_ptr, const int* col, const double* val,
                     const unsigned char* mask, double tau, const double* dbar,
                     const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    for (int r = 0; r < 12; ++r) {
      int gi = i*12 + r;
      if (mask && mask[gi]) { y[gi] = x[gi]; continue; }
      double acc = 0.0;
      for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
        int j = col[k];
        for (int s = 0; s < 12; ++s) {
          int gj = j*12 + s;
          if (mask && mask[gj]) continue;
          acc += val[(size_t)k*144 + r*12 + s] * x[gj];
        }
      }
      y[gi] = acc + (tau != 0.0 ? tau * dbar[r / 3] * x[gi] : 0.0);
    }
  }
}

/* Inverse of one 12x12 SPD block by Cholesky; returns 0 when a pivot is not positive. */
static int chol_inverse12(const double* A, double* Ainv) {
  double L[12][12] = {{0}};
  for (int j = 0; j < 12; ++j) {
    double s = A[j*12 + j];
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0.0)) return 0;
    L[j][j] = sqrt(s);
    for (int i = j + 1; i < 12; ++i) {
      double t = A[i*12 + j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / L[j][j];
    }
  }
  for (int c = 0; c < 12; ++c) {   /* solve L L^T x = e_c */
    double y[12], x[12];
    for (int i = 0; i < 12; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
      y[i] = t / L[i][i];
    }
    for (int i = 11; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < 12; ++k) t -= L[k][i] * x[k];
      x[i] = t / L[i][i];
    }
    for (int i = 0; i < 12; ++i) Ainv[i*12 + c] = x[i];
  }
  return 1;
}

/* Block-Jacobi inverses D[n*144] of the masked, regularised diagonal blocks. */
static void block_jacobi(int n, const int* row_ptr, const int* col, const double* val,
                         const unsigned char* mask, double tau, const double* dbar, double* D) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    int k = find_block(row_ptr, col, i, i);
    double A[144];
    for (int r = 0; r < 12; ++r) for (int s = 0; s < 12; ++s) {
      int fr = mask && mask[i*12 + r], fs = mask && mask[i*12 + s];
      double v = val[(size_t)k*144 + r*12 + s];
      if (fr || fs) v = (r == s) ? 1.0 : 0.0;
      else if (r == s && tau != 0.0) v += tau * dbar[r / 3];
      A[r*12 + s] = v;
    }
    if (!chol_inverse12(A, &D[(size_t)i*144])) {
      memset(&D[(size_t)i*144], 0, 144 * sizeof(double));
      for (int r = 0; r < 12; ++r) D[(size_t)i*144 + r*13] = A[r*13] > 0.0 ? 1.0 / A[r*13] : 1.0;
    }
  }
}

static double vdot(int m, const double* a, const double* b) {
  double s = 0.0;
  for (int i = 0; i < m; ++i) s += a[i] * b[i];
  return s;
}

/* Solves A x = b from x = 0. Stops when |r| <= rtol |b| (or after exactly fixed_iters
   iterations when fixed_iters > 0), or after max_iter. Returns OG_OK, or OG_PCG_NEG_CURV when
   p^T A p <= 0. *iters receives the iterations done. */
/* Per-kind regulariser scale: dbar[k] = mean over free DOFs of kind k of |A_ii| (1 if none). */
void og_kind_scale(int n, const int* row_ptr, const int* col, const double* val,
                   const unsigned char* mask, double dbar[4]) {
  double sum[4] = {0, 0, 0, 0};
  long cnt[4] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i) {
    int k = find_block(row_ptr, col, i, i);
    for (int a = 0; a < 12; ++a) {
      if (mask && mask[i*12 + a]) continue;
      sum[a / 3] += fabs(val[(size_t)k*144 + a*13]);
      cnt[a / 3] += 1;
    }
  }
  for (int q = 0; q < 4; ++q) dbar[q] = cnt[q] ? sum[q] / (double)cnt[q] : 1.0;
}

int og_pcg(int n, const int* row_ptr, const int* col, const double* val,
           const unsigned char* mask, double tau, const double* dbar, const double* b,
           double rtol, int max_iter, int fixed_iters, double* x, int* iters) {
  int m = n * 12;
  double* D = (double*)malloc((size_t)n * 144 * sizeof(double));
  double *r = (double*)malloc(m * sizeof(double)), *z = (double*)malloc(m * sizeof(double));
  double *p = (double*)malloc(m * sizeof(double)), *Ap = (double*)malloc(m * sizeof(double));
  block_jacobi(n, row_ptr, col, val, mask, tau, dbar, D);
  for (int i = 0; i < m; ++i) { x[i] = 0.0; r[i] = (mask && mask[i]) ? 0.0 : b[i]; }
  double bnorm = sqrt(vdot(m, r, r));
  int status = OG_OK, it = 0;
  int limit = fixed_iters > 0 ? fixed_iters : max_iter;
  if (bnorm == 0.0) goto done;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) for (int a = 0; a < 12; ++a) {
    double s = 0.0;
    for (int c = 0; c < 12; ++c) s += D[(size_t)i*144 + a*12 + c] * r[i*12 + c];
    z[i*12 + a] = s;
  }
  memcpy(p, z, m * sizeof(double));
  double rz = vdot(m, r, z);
  while (it < limit) {
    bsr_mult(n, row_ptr, col, val, mask, tau, dbar, p, Ap);
    for (int i = 0; i < m; ++i) if (mask && mask[i]) Ap[i] = 0.0;
    double pAp = vdot(m, p, Ap);
    if (!(pAp > 0.0)) { status = OG_PCG_NEG_CURV; break; }
    double al = rz / pAp;
    for (int i = 0; i < m; ++i) { x[i] += al * p[i]; r[i] -= al * Ap[i]; }
    ++it;
    double rn = sqrt(vdot(m, r, r));
    if (fixed_iters <= 0 && rn <= rtol * bnorm) break;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) for (int a = 0; a < 12; ++a) {
      double s = 0.0;
      for (int c = 0; c < 12; ++c) s += D[(size_t)i*144 + a*12 + c] * r[i*12 + c];
      z[i*12 + a] = (mask && mask[i*12 + a]) ? 0.0 : s;
    }
    double rz_new = vdot(m, r, z);
    if (rz_new == 0.0) break;
    double be = rz_new / rz;
    rz = rz_new;
    for (int i = 0; i < m; ++i) p[i] = z[i] + be * p[i];
  }
done:
  *iters = it;
  free(D); free(r); free(z); free(p); free(Ap);
  return status;
}

/* ------------------------------------------------------------------------------------------ */
/* The regularised Newton direction (Sec. 6.1 "a diagonal regularizer is added").               */
/* ------------------------------------------------------------------------------------------ */
/* Local part of the regulariser: every free diagonal entry A_ii <= 0 (i of kind k) is replaced by
   max(-A_ii, 1e-8 D_k). val is changed in place; returns the number of entries replaced. */
int og_fix_diagonal(int n, const int* row_ptr, const int* col, double* val,
                    const unsigned char* mask, const double* dbar) {
  int fixed = 0;
  for (int i = 0; i < n; ++i) {
    int k = find_block(row_ptr, col, i, i);
    for (int a = 0; a < 12; ++a) {
      if (mask && mask[i*12 + a]) continue;
      double* v = &val[(size_t)k*144 + a*13];
      if (*v <= 0.0) {
        double floor = 1e-8 * dbar[a / 3];
        *v = -*v > floor ? -*v : floor;
        ++fixed;
      }
    }
  }
  return fixed;
}

/* Solves (A' + tau D) d = rhs by block-Jacobi PCG, A' = A with its diagonal fixed by
   og_fix_diagonal and D from A (og_kind_scale). tau starts at *tau_carry / 10, or at 0 when that
   is below 1e-8; each negative curvature met by PCG restarts the solve with tau = max(10 tau,
   1e-8); a tau beyond 1e4 ends it with OG_ERR_INDEFINITE. On success *tau_carry receives the tau of
   the accepted solve. Counters (added to): PCG iterations, solves run with tau > 0, diagonal
   entries replaced. */
int og_newton_direction(int n, const int* row_ptr, const int* col, const double* val,
                        const unsigned char* mask, const double* rhs, double rtol, int max_iter,
                        int fixed_iters, double* tau_carry, double* d, int* pcg_iters,
                        int* regularizations, int* diag_fixes) {
  size_t nb = (size_t)row_ptr[n];
  double* A = (double*)malloc(nb * 144 * sizeof(double));
  memcpy(A, val, nb * 144 * sizeof(double));
  double dbar[4];
  og_kind_scale(n, row_ptr, col, val, mask, dbar);
  *diag_fixes += og_fix_diagonal(n, row_ptr, col, A, mask, dbar);
  double tau = *tau_carry / 10.0;
  if (tau < 1e-8) tau = 0.0;
  int status = OG_OK;
  for (;;) {
    if (tau > 1e4) { status = OG_ERR_INDEFINITE; break; }
    int it = 0;
    int ps = og_pcg(n, row_ptr, col, A, mask, tau, dbar, rhs, rtol, max_iter, fixed_iters, d, &it);
    *pcg_iters += it;
    if (tau > 0.0) *regularizations += 1;
    if (ps != OG_PCG_NEG_CURV) break;
    tau = 10.0 * tau > 1e-8 ? 10.0 * tau : 1e-8;
  }
  if (status == OG_OK) *tau_carry = tau;
  free(A);
  return status;
}

/* ------------------------------------------------------------------------------------------ */
/* Backtracking line search on phi(alpha) = Pi(q + alpha d) - Pi(q), phi'(0) = gd < 0 (Sec. 6.1  */
/* "quadratic and cubic line searches"; interpolation formulas of Nocedal-Wright Sec. 3.5).     */
/* ------------------------------------------------------------------------------------------ */
/* The trial after a failed trial number `trial` (0-based) at alpha with value phi; a_prev, f_prev
   are the trial before it (used from the second backtrack on). */
double og_ls_next_alpha(int trial, double alpha, double phi, double gd, double a_prev, double f_prev) {
  double a_new;
  if (!isfinite(phi)) {
    a_new = 0.5 * alpha;
  } else if (trial == 0) {
    /* minimiser of the quadratic with phi(0) = 0, phi'(0) = gd, phi(alpha) = phi */
    a_new = -gd * alpha * alpha / (2.0 * (phi - gd * alpha));
  } else {
    /* minimiser of the cubic c a^3 + b a^2 + gd a through phi(a_prev) and phi(alpha) */
    double a0 = a_prev, a1 = alpha;
    double r1 = phi - gd * a1, r0 = f_prev - gd * a0;
    double den = a0 * a0 * a1 * a1 * (a1 - a0);
    double c = (a0 * a0 * r1 - a1 * a1 * r0) / den;
    double b = (-a0 * a0 * a0 * r1 + a1 * a1 * a1 * r0) / den;
    double disc = b * b - 3.0 * c * gd;
    if (c == 0.0 || disc < 0.0) a_new = 0.5 * alpha;
    else a_new = (-b + sqrt(disc)) / (3.0 * c);
  }
  if (!(a_new >= 0.1 * alpha)) a_new = 0.1 * alpha;
  if (a_new > 0.5 * alpha) a_new = 0.5 * alpha;
  return a_new;
}

typedef double (*og_phi_fn)(double alpha, void* ctx);

/* Armijo backtracking from alpha = 1: accepts the first trial with a finite phi(alpha) <= 1e-4
   alpha gd, at most 20 trials. Returns OG_OK with *alpha, or OG_ERR_LINESEARCH; *backtracks is
   incremented once per rejected trial. */
int og_line_search(double gd, og_phi_fn phi_of, void* ctx, double* alpha_out, int* backtracks) {
  double alpha = 1.0, a_prev = 0.0, f_prev = 0.0;
  for (int trial = 0; trial < 20; ++trial) {
    double phi = phi_of(alpha, ctx);
    if (isfinite(phi) && phi <= 1e-4 * alpha * gd) { *alpha_out = alpha; return OG_OK; }
    *backtracks += 1;
    double a_new = og_ls_next_alpha(trial, alpha, phi, gd, a_prev, f_prev);
    a_prev = alpha;
    f_prev = phi;
    alpha = a_new;
  }
  return OG_ERR_LINESEARCH;
}

/* ------------------------------------------------------------------------------------------ */
/* One implicit-Euler step (Eq. implicit) by Newton's method with a line search (Sec. 6.1).     */
/* Incremental potential Pi(q) = 1/(2 dt^2) (q-y)^T M (q-y) + V_e(q) - F^T q, y = q^n + dt v^n; */
/* its stationarity is Eq. implicit. Fixed DOFs take prescribed values (Sec. 4.2).             */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  const og_grid* g; const og_material* mat; const double* rest;
  int n, m, nb; const int* row_ptr; const int* col; const double* mval; const double* fs;
  const unsigned char* mask; double dt; double grav[3];
} og_ctx;

/* g = grad V_e + M (q - y) / dt^2 - F on free DOFs (0 on fixed); returns |g|. ginert receives
   M (q - y)/dt^2 - F when non-NULL. */
static double full_gradient(const og_ctx* C, const double* q, const double* y, double* gout,
                            double* ginert, double* work) {
  og_assemble(C->g, C->mat, C->rest, q, C->row_ptr, C->col, 0.0, NULL, gout, NULL, 0);
  for (int i = 0; i < C->m; ++i) work[i] = q[i] - y[i];
  double* Mw = (double*)malloc(C->m * sizeof(double));
  mass_mult(C->n, C->row_ptr, C->col, C->mval, work, Mw);
  double s = 0.0;
  for (int i = 0; i < C->n; ++i) for (int k = 0; k < 4; ++k) for (int c = 0; c < 3; ++c) {
    int gi = i*12 + k*3 + c;
    double gin = Mw[gi] / (C->dt * C->dt) - C->fs[i*4 + k] * C->grav[c];
    if (ginert) ginert[gi] = (C->mask && C->mask[gi]) ? 0.0 : gin;
    gout[gi] += gin;
    if (C->mask && C->mask[gi]) gout[gi] = 0.0;
    s += gout[gi] * gout[gi];
  }
  free(Mw);
  return sqrt(s);
}

/* Per-patch elastic energies. */
static void patch_energies(const og_ctx* C, const double* q, double* Ep) {
  int np = C->g->nu * C->g->nv;
#pragma omp parallel for schedule(static)
  for (int p = 0; p < np; ++p) {
    double ql[48], qbl[48];
    gather48(C->g, q, p, ql);
    gather48(C->g, C->rest, p, qbl);
    Ep[p] = og_element_energy(ql, qbl, C->g->dxi1, C->g->dxi2, C->mat);
  }
}

/* phi(alpha) = Pi(q + alpha d) - Pi(q): the elastic part as a sum of per-patch energy differences,
   the inertial and load parts exactly (alpha d.g_inert + alpha^2/2 d^T M d / dt^2). */
typedef struct {
  const og_ctx* C; const double* q; const double* d; double* qt; const double* Ep; double* Et;
  double dMd, dgin;
} og_phi_ctx;

static double phi_of_alpha(double alpha, void* ctx) {
  og_phi_ctx* L = (og_phi_ctx*)ctx;
  int m = L->C->m, np = L->C->g->nu * L->C->g->nv;
  for (int i = 0; i < m; ++i) L->qt[i] = L->q[i] + alpha * L->d[i];
  patch_energies(L->C, L->qt, L->Et);
  double dV = 0.0;
  for (int p = 0; p < np; ++p) dV += L->Et[p] - L->Ep[p];
  return dV + alpha * L->dgin + 0.5 * alpha * alpha * L->dMd;
}

int og_newton_step(const og_grid* g, const og_material* mat, const double* rest,
                   const og_step_params* P, const unsigned char* mask, const double* qfix,
                   double* q, double* v, const double* warm, og_step_stats* st) {
  og_ctx C;
  C.g = g; C.mat = mat; C.rest = rest; C.n = og_n_nodes(g); C.m = C.n * 12;
  C.mask = mask; C.dt = P->dt;
  C.grav[0] = P->gravity[0]; C.grav[1] = P->gravity[1]; C.grav[2] = P->gravity[2];
  int n = C.n, m = C.m, np = g->nu * g->nv;
  memset(st, 0, sizeof(*st));
  int* row_ptr = (int*)malloc((n + 1) * sizeof(int));
  C.nb = og_bsr_pattern(g, row_ptr, NULL);
  int* col = (int*)malloc(C.nb * sizeof(int));
  og_bsr_pattern(g, row_ptr, col);
  C.row_ptr = row_ptr; C.col = col;
  double* mval = (double*)malloc((size_t)C.nb * 16 * sizeof(double));
  double* fs = (double*)malloc((size_t)n * 4 * sizeof(double));
  og_mass(g, mat, rest, row_ptr, col, mval, fs);
  C.mval = mval; C.fs = fs;

  double *qn = malloc(m * sizeof(double)), *y = malloc(m * sizeof(double));
  double *gr = malloc(m * sizeof(double)), *gin = malloc(m * sizeof(double));
  double *d = malloc(m * sizeof(double)), *work = malloc(m * sizeof(double));
  double *qt = malloc(m * sizeof(double)), *rhs = malloc(m * sizeof(double));
  double *Md = malloc(m * sizeof(double));
  double *Ep = malloc(np * sizeof(double)), *Et = malloc(np * sizeof(double));
  double* val = (double*)malloc((size_t)C.nb * 144 * sizeof(double));
  memcpy(qn, q, m * sizeof(double));
  for (int i = 0; i < m; ++i) y[i] = qn[i] + P->dt * v[i];

  /* zero guess: q^n with the prescribed DOFs overwritten; its residual is the reference */
  for (int i = 0; i < m; ++i) q[i] = (mask && mask[i]) ? qfix[i] : qn[i];
  double gref = full_gradient(&C, q, y, gr, NULL, work);
  st->res0 = gref;
  if (warm) for (int i = 0; i < m; ++i) q[i] = (mask && mask[i]) ? qfix[i] : warm[i];
  int status = OG_OK;
  double gn = 0.0, tau_carry = P->tau_carry;
  for (int it = 0;; ++it) {
    gn = full_gradient(&C, q, y, gr, gin, work);
    if (gn <= P->newton_rtol * gref) break;
    if (it >= P->newton_max) { status = OG_ERR_NOT_CONVERGED; break; }
    og_assemble(g, mat, rest, q, row_ptr, col, 1.0 / (P->dt * P->dt), NULL, NULL, val, P->pseudo_hessian);
    for (int i = 0; i < m; ++i) rhs[i] = -gr[i];
    status = og_newton_direction(n, row_ptr, col, val, mask, rhs, P->pcg_rtol, P->pcg_max,
                                 P->pcg_fixed_iters, &tau_carry, d, &st->pcg_iters_total,
                                 &st->regularizations, &st->diag_fixes);
    if (status != OG_OK) break;

    /* line search on phi(alpha) = Pi(q + alpha d) - Pi(q) */
    double gd = vdot(m, gr, d);
    double alpha = 1.0;
    if (gn > 1e-6 * gref) {
      if (!(gd < 0.0)) { status = OG_ERR_LINESEARCH; break; }
      mass_mult(n, row_ptr, col, mval, d, Md);
      og_phi_ctx L;
      L.C = &C; L.q = q; L.d = d; L.qt = qt; L.Ep = Ep; L.Et = Et;
      L.dMd = vdot(m, d, Md) / (P->dt * P->dt);
      L.dgin = vdot(m, d, gin);
      patch_energies(&C, q, Ep);
      status = og_line_search(gd, phi_of_alpha, &L, &alpha, &st->ls_backtracks);
      if (status != OG_OK) break;
    }
    for (int i = 0; i < m; ++i) q[i] += alpha * d[i];
    st->newton_iters++;
  }
  st->res_final = gn;
  st->tau_final = tau_carry;
  for (int i = 0; i < m; ++i) v[i] = (q[i] - qn[i]) / P->dt;
  st->status = status;
  free(row_ptr); free(col); free(mval); free(fs); free(qn); free(y); free(gr); free(gin);
  free(d); free(work); free(qt); free(rhs); free(Md); free(Ep); free(Et); free(val);
  return status;
}
