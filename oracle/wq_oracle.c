/*
 * wq_oracle.c -- plain, slow, FP64 CPU oracle for row-wise mass and stiffness
 * assembly with weighted Gaussian quadrature (Barton, Puzyrev, Deng, Calo,
 * "Efficient mass and stiffness matrix assembly via weighted Gaussian
 * quadrature rules for B-splines").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * What it computes, in the paper's order:
 *   - open uniform knot vectors of maximal continuity (Sec. 2.2, Eq. 3);
 *   - B-splines and their derivatives by the Cox-de Boor recursion;
 *   - the univariate weighted Gaussian rules as roots of the exactness
 *     systems (Sec. 3.1, Eq. GaussQuadSys; Sec. 3.2, Eq. GaussQuadSysStiff),
 *     with the symmetric parametrisation and the free-parameter choices the
 *     paper makes (Sec. 3.1.1, 3.1.2, 3.2.1, 3.2.2), solved by Newton's method;
 *   - Gauss-Legendre rules on every element of the support for rows whose
 *     weight function touches the boundary (Remark at the end of Sec. 3);
 *   - the matrices M (Eq. Mass) and K (Eq. Stiffness) row by row: each row r
 *     is integrated by the tensor product of its own 1D rules, the
 *     geometry factor c*|det J| (mass) or c*|det J|*(J^-1 J^-T)_aa (stiffness
 *     term a) being evaluated at every rule point from the full Jacobian of
 *     the tensor control net (Eq. Gmap1, Gmap2), with no sum factorisation:
 *     nested loops over rows x rule points x band columns.
 *
 * Only the diagonal metric terms have a weighted rule in the paper (Sec. 3.2);
 * wqo_assemble reports the largest off-diagonal metric entry relative to the
 * diagonal ones so tests can confirm the map is separable.  For a map given
 * by its full control net, wqo_assemble_general adds the off-diagonal terms,
 * integrated with mixed-derivative rules (wqo_cross_rule) whose construction
 * the paper leaves open; the reading taken is stated there.
 *
 * Band layout of a row r = r1 + n1*(r2 + n2*r3): entry
 *   (d3+p)*(2p+1)^2 + (d2+p)*(2p+1) + (d1+p),  column s_a = r_a + d_a,
 * zero where a column index falls outside [0, n_a).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXP 3
#define MAXL ((MAXP + 1) * (MAXP + 1)) /* most rule points of one row in one direction (RULE_GL) */
#define MAXKNOTS 4096

/* ------------------------------------------------------------------ */
/* Knot vectors and B-splines                                          */
/* ------------------------------------------------------------------ */

/* Eq. 3: p+1 copies of 0, the single interior knots i/N, p+1 copies of 1. */
static int open_uniform_knots(int p, int N, double *t) {
  int m = N + 2 * p + 1;
  for (int i = 0; i < m; i++) {
    if (i <= p)
      t[i] = 0.0;
    else if (i >= N + p)
      t[i] = 1.0;
    else
      t[i] = (double)(i - p) / (double)N;
  }
  return m;
}

/* Cox-de Boor recursion for B_{i,k} on knots t[0..nt-1].  Spans are half
 * open; the last non-empty span also owns the right end point. */
static double cox_de_boor(const double *t, int nt, int i, int k, double x) {
  if (k == 0) {
    if (t[i] < t[i + 1]) {
      if (t[i] <= x && x < t[i + 1]) return 1.0;
      if (x == t[nt - 1] && t[i + 1] == t[nt - 1]) return 1.0;
    }
    return 0.0;
  }
  double v = 0.0;
  double d1 = t[i + k] - t[i];
  double d2 = t[i + k + 1] - t[i + 1];
  if (d1 > 0.0) v += (x - t[i]) / d1 * cox_de_boor(t, nt, i, k - 1, x);
  if (d2 > 0.0) v += (t[i + k + 1] - x) / d2 * cox_de_boor(t, nt, i + 1, k - 1, x);
  return v;
}

/* Derivative of B_{i,k}: k/(t_{i+k}-t_i) B_{i,k-1} - k/(t_{i+k+1}-t_{i+1}) B_{i+1,k-1}. */
static double cox_de_boor_deriv(const double *t, int nt, int i, int k, double x) {
  double v = 0.0;
  double d1 = t[i + k] - t[i];
  double d2 = t[i + k + 1] - t[i + 1];
  if (d1 > 0.0) v += (double)k / d1 * cox_de_boor(t, nt, i, k - 1, x);
  if (d2 > 0.0) v -= (double)k / d2 * cox_de_boor(t, nt, i + 1, k - 1, x);
  return v;
}

/* Value (nu = 0) or derivative (nu = 1) of B_i of degree k. */
static double bspl(const double *t, int nt, int i, int k, int nu, double x) {
  return nu ? cox_de_boor_deriv(t, nt, i, k, x) : cox_de_boor(t, nt, i, k, x);
}

/* Cardinal B-spline N_p on the integer knots 0..p+1 (Sec. 3.1 works on this
 * domain), value or derivative, at y. */
static double cardinal(int p, int nu, double y) {
  double t[MAXP + 2];
  for (int i = 0; i <= p + 1; i++) t[i] = (double)i;
  if (y < 0.0 || y > (double)(p + 1)) return 0.0;
  return bspl(t, p + 2, 0, p, nu, y);
}

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rules: Newton on P_n from the three-term recurrence   */
/* ------------------------------------------------------------------ */

static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; i++) {
    double z = cos(M_PI * ((double)(n - i) - 0.25) / ((double)n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / (double)k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p0 = 1.0; p1 = z; }
      dp = (double)n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    /* recompute P_n' at the converged root for the weight */
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; k++) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / (double)k;
      p0 = p1;
      p1 = p2;
    }
    dp = (double)n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

int wqo_gauss_legendre(int n, double *x, double *w) {
  if (n < 1 || n > 64) return 1;
  gauss_legendre(n, x, w);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Moments of the weight function (right-hand sides of the systems)    */
/* ------------------------------------------------------------------ */

/* int_0^{p+1} N_p^(nu)(y) N_p^(nu)(y - d) dy, element by element with a
 * Gauss-Legendre rule exact for the piecewise polynomial integrand. */
static double moment(int p, int nu, int d) {
  double gx[8], gw[8];
  int ng = p + 2;
  gauss_legendre(ng, gx, gw);
  double s = 0.0;
  for (int u = 0; u <= p; u++)
    for (int g = 0; g < ng; g++) {
      double y = (double)u + 0.5 * (gx[g] + 1.0);
      s += 0.5 * gw[g] * cardinal(p, nu, y) * cardinal(p, nu, y - (double)d);
    }
  return s;
}

double wqo_moment(int p, int nu, int d) { return moment(p, nu, d); }

double wqo_bspline(int p, int N, int i, int nu, double x) {
  double t[MAXKNOTS];
  if (N + 2 * p + 1 > MAXKNOTS) return NAN;
  int nt = open_uniform_knots(p, N, t);
  return bspl(t, nt, i, p, nu, x);
}

double wqo_cardinal(int p, int nu, double y) { return cardinal(p, nu, y); }

/* ------------------------------------------------------------------ */
/* Univariate weighted Gaussian rules (Sec. 3)                          */
/* ------------------------------------------------------------------ */

/* The symmetric rules of Sec. 3: tau_{p+2-k} = (p+1) - tau_k, omega_{p+2-k} =
 * omega_k.  The unknown vector u and the free-parameter choices are:
 *   mass p=2      (Eq. QuadraticQuadrature): tau_2 = 3/2; u = (tau_1, omega_1, omega_2)
 *   mass p=3      (Eq. CubicQuadrature):     u = (tau_1, tau_2, omega_1, omega_2)
 *   stiffness p=2 (Eq. QuadraticQuadratureStiff): tau_2 = 3/2, omega_2 = 8/9 as
 *                 printed (B'_j vanishes there, so omega_2 is free); u = (tau_1, omega_1)
 *   stiffness p=3 (Eq. CubicQuadratureStiff, CubicStiffTau1W): omega_1 = 1;
 *                 u = (tau_1, tau_2, omega_2), smaller tau_1 root. */
static void expand_rule(int p, int nu, const double *u, double *tau, double *om) {
  if (p == 2 && nu == 0) {
    tau[0] = u[0]; tau[1] = 1.5; tau[2] = 3.0 - u[0];
    om[0] = u[1]; om[1] = u[2]; om[2] = u[1];
  } else if (p == 3 && nu == 0) {
    tau[0] = u[0]; tau[1] = u[1]; tau[2] = 4.0 - u[1]; tau[3] = 4.0 - u[0];
    om[0] = u[2]; om[1] = u[3]; om[2] = u[3]; om[3] = u[2];
  } else if (p == 2 && nu == 1) {
    tau[0] = u[0]; tau[1] = 1.5; tau[2] = 3.0 - u[0];
    om[0] = u[1]; om[1] = 8.0 / 9.0; om[2] = u[1];
  } else { /* p == 3, nu == 1 */
    tau[0] = u[0]; tau[1] = u[1]; tau[2] = 4.0 - u[1]; tau[3] = 4.0 - u[0];
    om[0] = 1.0; om[1] = u[2]; om[2] = u[2]; om[3] = 1.0;
  }
}

/* Residual of one exactness condition, Eq. GaussQuadSys (nu = 0) or
 * GaussQuadSysStiff (nu = 1): sum_k omega_k N(tau_k) N(tau_k - d) - moment(d). */
static double exactness_residual(int p, int nu, const double *tau, const double *om, int d) {
  double s = 0.0;
  for (int k = 0; k <= p; k++) s += om[k] * cardinal(p, nu, tau[k]) * cardinal(p, nu, tau[k] - (double)d);
  return s - moment(p, nu, d);
}

/* Which shifts d form the square Newton system for each rule (by symmetry
 * the shifts -d and d give the same condition; for the stiffness rules one
 * condition is dependent on the others because the translates' derivatives
 * sum to zero, Sec. 3.2). */
static int newton_equations(int p, int nu, int *ds) {
  if (p == 2 && nu == 0) { ds[0] = 0; ds[1] = 1; ds[2] = 2; return 3; }
  if (p == 3 && nu == 0) { ds[0] = 0; ds[1] = 1; ds[2] = 2; ds[3] = 3; return 4; }
  if (p == 2 && nu == 1) { ds[0] = 1; ds[1] = 2; return 2; }
  ds[0] = 0; ds[1] = 2; ds[2] = 3; return 3;
}

/* Dense Gaussian elimination with partial pivoting; A is n x n row major. */
static int solve_dense(int n, double *A, double *b) {
  for (int c = 0; c < n; c++) {
    int piv = c;
    for (int r = c + 1; r < n; r++)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return 1;
    if (piv != c) {
      for (int k = 0; k < n; k++) { double tmp = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = tmp; }
      double tmp = b[c]; b[c] = b[piv]; b[piv] = tmp;
    }
    for (int r = c + 1; r < n; r++) {
      double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; k++) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; r--) {
    double s = b[r];
    for (int k = r + 1; k < n; k++) s -= A[r * n + k] * b[k];
    b[r] = s / A[r * n + r];
  }
  return 0;
}

/* Exactness check of a rule against all 2p+1 conditions d = -p..p, plus the
 * one-node-per-element property (Sec. 3.1.2 and 3.2) and, for the mass rules,
 * positive weights.  Returns 0 if the rule passes; *max_resid receives the
 * largest residual. */
int wqo_rule_check(int p, int nu, const double *tau, const double *om, double tol, double *max_resid) {
  if (p < 2 || p > MAXP || (nu != 0 && nu != 1)) return 2;
  double mr = 0.0;
  for (int d = -p; d <= p; d++) {
    double r = fabs(exactness_residual(p, nu, tau, om, d));
    if (!(r <= mr)) mr = r; /* also propagates NaN */
  }
  if (max_resid) *max_resid = mr;
  int bad = !(mr <= tol);
  for (int k = 0; k <= p; k++) {
    if (!(tau[k] > (double)k && tau[k] < (double)(k + 1))) bad = 1;
    if (nu == 0 && !(om[k] > 0.0)) bad = 1;
  }
  return bad;
}

int wqo_rule_newton(int p, int nu, double *u, int n, const int *ds, double *tau, double *om, double *max_resid);

/* Solves the rule by Newton's method with a central-difference Jacobian.
 * Initial guesses: element midpoints for the nodes and unit weights, except
 * the smaller-root branch of the p=3 stiffness rule, started in [0, 1/2].
 * Returns 0 on success (converged and passing wqo_rule_check at 1e-14). */
int wqo_rule(int p, int nu, double *tau, double *om, double *max_resid) {
  if (p < 2 || p > MAXP || (nu != 0 && nu != 1)) return 2;
  double u[4];
  int n;
  if (p == 2 && nu == 0) { u[0] = 0.5; u[1] = 1.0; u[2] = 1.0; n = 3; }
  else if (p == 3 && nu == 0) { u[0] = 0.5; u[1] = 1.5; u[2] = 1.0; u[3] = 1.0; n = 4; }
  else if (p == 2 && nu == 1) { u[0] = 0.5; u[1] = 1.0; n = 2; }
  else { u[0] = 0.25; u[1] = 1.5; u[2] = 1.0; n = 3; }
  int ds[4];
  newton_equations(p, nu, ds);
  return wqo_rule_newton(p, nu, u, n, ds, tau, om, max_resid);
}

/* Newton iteration from a caller-supplied start u (length n). */
int wqo_rule_newton(int p, int nu, double *u, int n, const int *ds, double *tau, double *om, double *max_resid) {
  for (int it = 0; it < 200; it++) {
    double F[4], A[16];
    expand_rule(p, nu, u, tau, om);
    double fmax = 0.0;
    for (int e = 0; e < n; e++) {
      F[e] = exactness_residual(p, nu, tau, om, ds[e]);
      if (fabs(F[e]) > fmax) fmax = fabs(F[e]);
    }
    if (!(fmax < 1e3)) return 3; /* diverged */
    for (int j = 0; j < n; j++) {
      double h = 1e-6 * (fabs(u[j]) > 1.0 ? fabs(u[j]) : 1.0);
      double up[4], um[4], tp[4], op[4], tm[4], omm[4];
      memcpy(up, u, sizeof(double) * n);
      memcpy(um, u, sizeof(double) * n);
      up[j] += h;
      um[j] -= h;
      expand_rule(p, nu, up, tp, op);
      expand_rule(p, nu, um, tm, omm);
      for (int e = 0; e < n; e++)
        A[e * n + j] = (exactness_residual(p, nu, tp, op, ds[e]) - exactness_residual(p, nu, tm, omm, ds[e])) / (2.0 * h);
    }
    double step[4];
    for (int e = 0; e < n; e++) step[e] = -F[e];
    if (solve_dense(n, A, step)) return 3;
    /* Step halving keeps node k inside element k (one node per element,
     * Sec. 3.1.2 and Sec. 3.2); a start outside that region is left as is. */
    double ttry[4], otry[4], ustart[4];
    expand_rule(p, nu, u, ttry, otry);
    int inside0 = 1;
    for (int k = 0; k <= p; k++)
      if (!(ttry[k] > (double)k && ttry[k] < (double)(k + 1))) inside0 = 0;
    memcpy(ustart, u, sizeof(double) * n);
    double scale = 1.0;
    for (int halv = 0; halv < 60; halv++) {
      for (int j = 0; j < n; j++) u[j] = ustart[j] + scale * step[j];
      if (!inside0) break;
      expand_rule(p, nu, u, ttry, otry);
      int inside = 1;
      for (int k = 0; k <= p; k++)
        if (!(ttry[k] > (double)k && ttry[k] < (double)(k + 1))) inside = 0;
      if (inside) break;
      scale *= 0.5;
    }
    double smax = 0.0;
    for (int j = 0; j < n; j++)
      if (fabs(scale * step[j]) > smax) smax = fabs(scale * step[j]);
    if (smax < 1e-16 && it > 3) break;
  }
  expand_rule(p, nu, u, tau, om);
  return wqo_rule_check(p, nu, tau, om, 1e-14, max_resid) ? 3 : 0;
}

/* ------------------------------------------------------------------ */
/* Newton-Cotes-type weighted rules (the comparison rules of Sec. 1, 4) */
/* ------------------------------------------------------------------ */

/* The row-wise weighted rules of Newton-Cotes type that Sec. 1 and Sec. 4
 * compare against: on the cardinal support [0, p+1], nodes at the interior
 * knots and the element midpoints, y_k = (k+1)/2 for k = 0..2p, and weights
 * v_k with the weight function's value folded in, such that
 *   sum_k v_k N^(nu)(y_k - d) = int N^(nu)(y) N^(nu)(y - d) dy,  d = -p..p
 * (one node per interacting function, so the system is square and linear).
 * Stiffness: N'(y) vanishes at the centre y = (p+1)/2, so that node gets
 * weight 0 and the other 2p weights solve the conditions d = -p..p-1; the
 * last one then holds because the translates' derivatives sum to zero.
 * Returns 0 when all 2p+1 conditions hold to 1e-14 (*max_resid). */
int wqo_rule_nc(int p, int nu, double *y, double *v, double *max_resid) {
  if (p < 2 || p > MAXP || (nu != 0 && nu != 1)) return 2;
  int nn = 2 * p + 1, centre = p;
  for (int k = 0; k < nn; k++) { y[k] = 0.5 * (double)(k + 1); v[k] = 0.0; }
  int cols[2 * MAXP + 1], nu_k = 0;
  for (int k = 0; k < nn; k++)
    if (!(nu == 1 && k == centre)) cols[nu_k++] = k;
  double A[(2 * MAXP + 1) * (2 * MAXP + 1)], b[2 * MAXP + 1];
  for (int e = 0; e < nu_k; e++) {
    int d = -p + e;
    for (int j = 0; j < nu_k; j++) A[e * nu_k + j] = cardinal(p, nu, y[cols[j]] - (double)d);
    b[e] = moment(p, nu, d);
  }
  if (solve_dense(nu_k, A, b)) return 3;
  for (int j = 0; j < nu_k; j++) v[cols[j]] = b[j];
  double mr = 0.0;
  for (int d = -p; d <= p; d++) {
    double sres = -moment(p, nu, d);
    for (int k = 0; k < nn; k++) sres += v[k] * cardinal(p, nu, y[k] - (double)d);
    if (!(fabs(sres) <= mr)) mr = fabs(sres);
  }
  if (max_resid) *max_resid = mr;
  return mr <= 1e-14 ? 0 : 3;
}

/* ------------------------------------------------------------------ */
/* Per-row 1D rules                                                    */
/* ------------------------------------------------------------------ */

typedef struct {
  int p, N, n, nt;
  double h;
  double t[MAXKNOTS];   /* degree-p knots */
  double tc[MAXKNOTS];  /* degree-3 knots of the coefficient spline */
  int ntc;
} dir1d;

static int dir_init(dir1d *D, int p, int N) {
  if (N < 1 || N + 2 * p + 1 > MAXKNOTS || N + 7 > MAXKNOTS) return 1;
  D->p = p; D->N = N; D->n = N + p; D->h = 1.0 / (double)N;
  D->nt = open_uniform_knots(p, N, D->t);
  D->ntc = open_uniform_knots(3, N, D->tc);
  return 0;
}

/* Which rule the interior rows use: the weighted Gaussian rules of Sec. 3
 * (the method), Gauss-Legendre on every element of supp B_r for every row
 * (the element-wise Gauss point set), or the Newton-Cotes-type weighted
 * rules (wqo_rule_nc).  Rows touching the boundary use Gauss-Legendre in
 * these three.  RULE_WQB is the method with weighted Gaussian rules for the
 * boundary rows too (wqo_boundary_rule), where such a rule is defined. */
enum { RULE_WQ = 0, RULE_GL = 1, RULE_NC = 2, RULE_WQB = 3 };

typedef struct {
  int mode;
  double tau[2][2 * MAXP + 1], om[2][2 * MAXP + 1];  /* WQ: nodes and weights; NC: nodes and folded weights */
  /* RULE_WQB: the low-side boundary rules of rows r < p, in units of h:
   * nodes t_k = x_k / h, weights Wl_k = W_k / h^(1 - nu) (W = omega B_r^(nu)
   * with omega ~ h and B_r' ~ 1/h); nb = 0: none */
  int nb[2][MAXP];
  double bt[2][MAXP][MAXP + 1], bw[2][MAXP][MAXP + 1];
} rule_set;

int wqo_boundary_rule(int p, int nu, int r, double *t, double *Wl, int *npts, double *max_resid);

static int rule_set_init(rule_set *S, int p, int mode) {
  double res;
  S->mode = mode;
  memset(S->nb, 0, sizeof(S->nb));
  if (mode == RULE_WQB)
    for (int nu = 0; nu < 2; nu++)
      for (int r = 0; r < p; r++) {
        int st = wqo_boundary_rule(p, nu, r, S->bt[nu][r], S->bw[nu][r], &S->nb[nu][r], &res);
        if (st == 1) return 3; /* a rule that should exist was not found */
      }
  for (int nu = 0; nu < 2; nu++) {
    if (mode == RULE_NC) {
      if (wqo_rule_nc(p, nu, S->tau[nu], S->om[nu], &res)) return 3;
    } else if (wqo_rule(p, nu, S->tau[nu], S->om[nu], &res)) {
      return 3;
    }
  }
  return 0;
}

/* Quadrature points and weights of row r in one direction.  Interior rows
 * (all knots of B_r distinct: p <= r <= N-1) use, in RULE_WQ, the weighted
 * Gaussian rule mapped to supp B_r: x_k = (r - p + tau_k) h, W_k = h omega_k
 * B_r^(nu)(x_k) (the weight function is not folded into omega, Eq.
 * GaussQuadSys); in RULE_NC the nodes y_k of wqo_rule_nc, W_k = h^(1-nu) v_k
 * (v_k carries N^(nu)(y_k); B_r^(nu)(x) = h^-nu N^(nu)(y)).  Other rows, and
 * every row in RULE_GL, use (p+1)-point Gauss-Legendre on each element of
 * supp B_r, W = (h/2) w_g B_r^(nu)(x) (Remark on boundary functions, Sec. 3). */
static int row_rule(const dir1d *D, const rule_set *S, int nu, int r, double *x, double *W) {
  int p = D->p;
  double h = D->h;
  if (S->mode != RULE_GL && r >= p && r <= D->N - 1) {
    if (S->mode == RULE_NC) {
      for (int k = 0; k <= 2 * p; k++) {
        x[k] = ((double)(r - p) + S->tau[nu][k]) * h;
        W[k] = (nu ? 1.0 : h) * S->om[nu][k];
      }
      return 2 * p + 1;
    }
    for (int k = 0; k <= p; k++) {
      x[k] = ((double)(r - p) + S->tau[nu][k]) * h;
      W[k] = h * S->om[nu][k] * bspl(D->t, D->nt, r, p, nu, x[k]);
    }
    return p + 1;
  }
  if (S->mode == RULE_WQB && D->N >= 2 * p + 1) {
    /* low-side row r < p, or the mirror image x -> 1 - x of low-side row
     * n-1-r (B_{n-1-j}(1-x) = B_j(x), so derivatives change sign) */
    int low = r < p, rm = low ? r : D->n - 1 - r;
    if (rm < p && S->nb[nu][rm] > 0) {
      double scale = nu ? 1.0 : h;
      double sgn = (low || !nu) ? 1.0 : -1.0;
      for (int k = 0; k < S->nb[nu][rm]; k++) {
        x[k] = low ? S->bt[nu][rm][k] * h : 1.0 - S->bt[nu][rm][k] * h;
        W[k] = sgn * S->bw[nu][rm][k] * scale;
      }
      return S->nb[nu][rm];
    }
  }
  double gx[MAXP + 1], gw[MAXP + 1];
  gauss_legendre(p + 1, gx, gw);
  int L = 0;
  int elo = r - p < 0 ? 0 : r - p;
  int ehi = r > D->N - 1 ? D->N - 1 : r;
  for (int e = elo; e <= ehi; e++)
    for (int g = 0; g <= p; g++) {
      x[L] = ((double)e + 0.5 * (gx[g] + 1.0)) * h;
      W[L] = 0.5 * h * gw[g] * bspl(D->t, D->nt, r, p, nu, x[L]);
      L++;
    }
  return L;
}

/* The element holding x.  A point on a knot (the Newton-Cotes-type nodes)
 * may land in either neighbour; the splines evaluated there are continuous. */
static int element_of(const dir1d *D, double x) {
  int e = (int)floor(x * (double)D->N);
  if (e < 0) e = 0;
  if (e > D->N - 1) e = D->N - 1;
  return e;
}

/* ------------------------------------------------------------------ */
/* Weighted Gaussian rules for the boundary rows                        */
/* ------------------------------------------------------------------ */

/* The Remark closing Sec. 3 leaves the boundary rows to systems "modified
 * accordingly".  Reading taken here (open uniform knots, a mesh of at least
 * 2p+1 elements, so the low-side rows do not see the other boundary): the
 * rule of row r < p and kind nu is exact for the products B_r^(nu) B_s^(nu)
 * with every interacting s = 0 .. r+p, and has n = ceil(rank/2) nodes, rank
 * being the dimension of the span of the B_s^(nu) on supp B_r (m = r+p+1 for
 * the mass kind; m-1 for the stiffness kind, whose derivatives sum to zero,
 * so the condition of s = r+p is dropped).  When rank is odd one more
 * condition fixes the free parameter: exactness for B_r^(nu) times the
 * monomial (x/h)^(p-nu+1), the next degree above the span on one element
 * (for a one-element support this makes the rule the classical Gauss rule
 * of the weight B_r^(nu)).  The rows that have such a rule with every node
 * strictly inside supp B_r: every mass row, the stiffness rows 0 and 1 for
 * p = 2, and the stiffness rows 0 and 2 for p = 3 (for p = 3, row 1 the
 * system has no real solution inside the support; that row keeps
 * Gauss-Legendre).  Unknowns are the nodes x_k and the combined weights
 * W_k = omega_k B_r^(nu)(x_k); moments by Gauss-Legendre on each element of
 * the support (exact for these piecewise polynomials); solved by damped
 * Gauss-Newton (Levenberg-Marquardt) with a central-difference Jacobian from
 * a fixed list of starts, keeping the nodes inside the support. */
static int brule_defined(int p, int nu, int r) {
  if (r < 0 || r >= p) return 0;
  if (nu == 0) return 1;
  return p == 2 ? 1 : (r != 1);
}

typedef struct {
  dir1d D;
  int p, nu, r, nf, n, extra;
  double mu[2 * MAXP + 2];
} brule_sys;

static double brule_f(const brule_sys *B, int j, double x) {
  if (B->extra && j == B->nf - 1) return pow(x / B->D.h, (double)(B->p - B->nu + 1));
  return bspl(B->D.t, B->D.nt, j, B->p, B->nu, x); /* s = j */
}

static void brule_residual(const brule_sys *B, const double *u, double *F) {
  for (int j = 0; j < B->nf; j++) {
    double s = -B->mu[j];
    for (int k = 0; k < B->n; k++) s += u[B->n + k] * brule_f(B, j, u[k]);
    F[j] = s;
  }
}

int wqo_boundary_rule(int p, int nu, int r, double *t, double *Wl, int *npts, double *max_resid) {
  *npts = 0;
  *max_resid = 0.0;
  if (p < 2 || p > MAXP || nu < 0 || nu > 1 || r < 0 || r >= p) return 2;
  if (!brule_defined(p, nu, r)) return 2;
  brule_sys B;
  if (dir_init(&B.D, p, 2 * p + 1)) return 2;
  B.p = p; B.nu = nu; B.r = r;
  int m = r + p + 1;
  int rank = nu ? m - 1 : m;
  B.n = (rank + 1) / 2;
  B.extra = rank % 2;
  B.nf = rank + B.extra;
  double h = B.D.h, a = 0.0, b = (double)(r + 1) * h;
  /* moments: 8-point Gauss-Legendre on each element of [a, b] */
  double gx[8], gw[8];
  gauss_legendre(8, gx, gw);
  for (int j = 0; j < B.nf; j++) {
    double s = 0.0;
    for (int e = 0; e <= r; e++)
      for (int g = 0; g < 8; g++) {
        double x = ((double)e + 0.5 * (gx[g] + 1.0)) * h;
        s += 0.5 * h * gw[g] * bspl(B.D.t, B.D.nt, r, p, nu, x) * brule_f(&B, j, x);
      }
    B.mu[j] = s;
  }
  double mumax = 1.0;
  for (int j = 0; j < B.nf; j++) if (fabs(B.mu[j]) > mumax) mumax = fabs(B.mu[j]);
  const int n = B.n, nn = 2 * B.n;
  double lg[MAXP + 1], lw[MAXP + 1];
  gauss_legendre(n, lg, lw);
  for (int start = 0; start < 4; start++) {
    double u[2 * MAXP + 2], F[2 * MAXP + 2];
    for (int k = 0; k < n; k++) {
      double f = (double)(k + 1) / (double)(n + 1);
      if (start == 0) f = 0.5 * (lg[k] + 1.0);
      if (start == 2) f = ((k + 0.5) / n) * ((k + 0.5) / n);
      if (start == 3) f = 1.0 - (1.0 - (k + 0.5) / n) * (1.0 - (k + 0.5) / n);
      u[k] = a + f * (b - a);
    }
    /* weights for the start nodes: least squares on the conditions */
    {
      double A[2 * MAXP + 2][MAXP + 1], N[(MAXP + 1) * (MAXP + 1)], rhs[MAXP + 1];
      for (int j = 0; j < B.nf; j++)
        for (int k = 0; k < n; k++) A[j][k] = brule_f(&B, j, u[k]);
      for (int k = 0; k < n; k++) {
        rhs[k] = 0.0;
        for (int j = 0; j < B.nf; j++) rhs[k] += A[j][k] * B.mu[j];
        for (int l = 0; l < n; l++) {
          double s = 0.0;
          for (int j = 0; j < B.nf; j++) s += A[j][k] * A[j][l];
          N[k * n + l] = s;
        }
      }
      if (solve_dense(n, N, rhs)) continue;
      for (int k = 0; k < n; k++) u[n + k] = rhs[k];
    }
    brule_residual(&B, u, F);
    double lam = 1e-3;
    for (int it = 0; it < 300; it++) {
      double fn = 0.0, fmax = 0.0;
      for (int j = 0; j < B.nf; j++) { fn += F[j] * F[j]; if (fabs(F[j]) > fmax) fmax = fabs(F[j]); }
      if (fmax <= 1e-15 * mumax) break;
      double J[2 * MAXP + 2][2 * MAXP + 2];
      for (int c = 0; c < nn; c++) {
        double up[2 * MAXP + 2], um[2 * MAXP + 2], Fp[2 * MAXP + 2], Fm[2 * MAXP + 2];
        double dstep = c < n ? 1e-7 * h : 1e-7 * (fabs(u[c]) > 1.0 ? fabs(u[c]) : 1.0);
        memcpy(up, u, sizeof(double) * nn);
        memcpy(um, u, sizeof(double) * nn);
        up[c] += dstep;
        um[c] -= dstep;
        brule_residual(&B, up, Fp);
        brule_residual(&B, um, Fm);
        for (int j = 0; j < B.nf; j++) J[j][c] = (Fp[j] - Fm[j]) / (2.0 * dstep);
      }
      int moved = 0;
      while (lam <= 1e12) {
        double A[(2 * MAXP + 2) * (2 * MAXP + 2)], g[2 * MAXP + 2];
        for (int c = 0; c < nn; c++) {
          g[c] = 0.0;
          for (int j = 0; j < B.nf; j++) g[c] -= J[j][c] * F[j];
          for (int d = 0; d < nn; d++) {
            double s = 0.0;
            for (int j = 0; j < B.nf; j++) s += J[j][c] * J[j][d];
            A[c * nn + d] = s;
          }
        }
        for (int c = 0; c < nn; c++) A[c * nn + c] *= 1.0 + lam;
        if (solve_dense(nn, A, g)) { lam *= 10.0; continue; }
        double v[2 * MAXP + 2], Fv[2 * MAXP + 2];
        int inside = 1;
        for (int c = 0; c < nn; c++) v[c] = u[c] + g[c];
        for (int k = 0; k < n; k++) if (!(v[k] > a && v[k] < b)) inside = 0;
        if (inside) {
          brule_residual(&B, v, Fv);
          double fv = 0.0;
          for (int j = 0; j < B.nf; j++) fv += Fv[j] * Fv[j];
          if (fv < fn) {
            memcpy(u, v, sizeof(double) * nn);
            memcpy(F, Fv, sizeof(double) * B.nf);
            lam = lam / 10.0 > 1e-12 ? lam / 10.0 : 1e-12;
            moved = 1;
            break;
          }
        }
        lam *= 10.0;
      }
      if (!moved) break;
    }
    double fmax = 0.0;
    for (int j = 0; j < B.nf; j++) if (fabs(F[j]) > fmax) fmax = fabs(F[j]);
    if (fmax <= 1e-14 * mumax) {
      /* ascending nodes, in units of h */
      for (int k = 0; k < n; k++)
        for (int l = k + 1; l < n; l++)
          if (u[l] < u[k]) {
            double tx = u[k]; u[k] = u[l]; u[l] = tx;
            double tw = u[n + k]; u[n + k] = u[n + l]; u[n + l] = tw;
          }
      double wscale = nu ? 1.0 : 1.0 / h; /* W = Wl h^(1-nu) */
      for (int k = 0; k < n; k++) {
        t[k] = u[k] / h;
        Wl[k] = u[n + k] * wscale;
      }
      *npts = n;
      *max_resid = fmax / mumax;
      return 0;
    }
  }
  return 1;
}

/* ------------------------------------------------------------------ */
/* Mixed-derivative rules for non-separable maps                        */
/* ------------------------------------------------------------------ */

/* A map whose Jacobian is not diagonal adds to Eq. Stiffness the terms
 * dB_r/dxhat_a C_ab dB_s/dxhat_b with a != b.  Their direction-a factor
 * pairs the weight B_r' with the test functions B_s ("kind 2") and their
 * direction-b factor the weight B_r with the test functions B_s' ("kind 3");
 * Sec. 3.2 gives rules for the (B', B') pair only.  Reading taken here (the
 * paper is silent on these pairs): one node set per interior row serves both
 * mixed kinds, on the cardinal support [0, p+1],
 *   kind 2: sum_k w_k N(y_k - d)  = int N'(y) N(y - d) dy,
 *   kind 3: sum_k v_k N'(y_k - d) = int N(y) N'(y - d) dy,   d = -p..p,
 * with nodes symmetric about (p+1)/2, w antisymmetric (as the weight N' is)
 * and v symmetric.  Under these symmetries the conditions of d and -d
 * coincide and d = 0 holds identically, so each kind keeps the p conditions
 * d = 1..p.  p = 3: two node pairs, unknowns (y1, y2, w1, w2, v1, v2), six
 * conditions; p = 2: one pair and the centre node (where the antisymmetric
 * kind has weight 0), unknowns (y1, w1, v1, vc), four conditions.  One node
 * per element, as the rules of Sec. 3.  Solved by Newton's method with a
 * central-difference Jacobian, started from the element midpoints. */

/* int_0^{p+1} N^(nuw)(y) N^(nut)(y - d) dy, element by element with a
 * Gauss-Legendre rule exact for the piecewise polynomial integrand. */
static double mixed_moment(int p, int nuw, int nut, int d) {
  double gx[8], gw[8];
  int ng = p + 2;
  gauss_legendre(ng, gx, gw);
  double s = 0.0;
  for (int u = 0; u <= p; u++)
    for (int g = 0; g < ng; g++) {
      double y = (double)u + 0.5 * (gx[g] + 1.0);
      s += 0.5 * gw[g] * cardinal(p, nuw, y) * cardinal(p, nut, y - (double)d);
    }
  return s;
}

static void expand_cross(int p, const double *u, double *y, double *w, double *v) {
  if (p == 2) {
    y[0] = u[0]; y[1] = 1.5; y[2] = 3.0 - u[0];
    w[0] = u[1]; w[1] = 0.0; w[2] = -u[1];
    v[0] = u[2]; v[1] = u[3]; v[2] = u[2];
  } else {
    y[0] = u[0]; y[1] = u[1]; y[2] = 4.0 - u[1]; y[3] = 4.0 - u[0];
    w[0] = u[2]; w[1] = u[3]; w[2] = -u[3]; w[3] = -u[2];
    v[0] = u[4]; v[1] = u[5]; v[2] = u[5]; v[3] = u[4];
  }
}

/* Residual of condition d of kind 2 or 3 (see above). */
static double cross_residual(int p, int kind, const double *y, const double *w, const double *v, int d) {
  double s = 0.0;
  for (int k = 0; k <= p; k++)
    s += kind == 2 ? w[k] * cardinal(p, 0, y[k] - (double)d) : v[k] * cardinal(p, 1, y[k] - (double)d);
  return s - (kind == 2 ? mixed_moment(p, 1, 0, d) : mixed_moment(p, 0, 1, d));
}

static void cross_system(int p, const double *u, double *F) {
  double y[MAXP + 1], w[MAXP + 1], v[MAXP + 1];
  expand_cross(p, u, y, w, v);
  for (int d = 1; d <= p; d++) {
    F[d - 1] = cross_residual(p, 2, y, w, v, d);
    F[p + d - 1] = cross_residual(p, 3, y, w, v, d);
  }
}

/* The mixed rules (y, w, v), p + 1 nodes each.  Returns 0 when Newton
 * converged and both kinds meet all 2p+1 conditions to 1e-14 with node k in
 * element k; *max_resid receives the largest residual. */
int wqo_cross_rule(int p, double *y, double *w, double *v, double *max_resid) {
  if (p < 2 || p > MAXP) return 2;
  int n = 2 * p;
  double u[6];
  if (p == 2) { u[0] = 0.5; u[1] = 1.0; u[2] = 0.25; u[3] = 0.5; }
  else { u[0] = 0.5; u[1] = 1.5; u[2] = 1.0; u[3] = 1.0; u[4] = 0.25; u[5] = 0.25; }
  for (int it = 0; it < 100; it++) {
    double F[6], A[36], step[6];
    cross_system(p, u, F);
    double fmax = 0.0;
    for (int e = 0; e < n; e++) if (fabs(F[e]) > fmax) fmax = fabs(F[e]);
    if (!(fmax < 1e3)) return 3;
    for (int j = 0; j < n; j++) {
      double hj = 1e-6 * (fabs(u[j]) > 1.0 ? fabs(u[j]) : 1.0);
      double up[6], um[6], Fp[6], Fm[6];
      memcpy(up, u, sizeof(up));
      memcpy(um, u, sizeof(um));
      up[j] += hj;
      um[j] -= hj;
      cross_system(p, up, Fp);
      cross_system(p, um, Fm);
      for (int e = 0; e < n; e++) A[e * n + j] = (Fp[e] - Fm[e]) / (2.0 * hj);
    }
    for (int e = 0; e < n; e++) step[e] = -F[e];
    if (solve_dense(n, A, step)) return 3;
    double smax = 0.0;
    for (int j = 0; j < n; j++) {
      u[j] += step[j];
      if (fabs(step[j]) > smax) smax = fabs(step[j]);
    }
    if (smax < 1e-16 && it > 3) break;
  }
  expand_cross(p, u, y, w, v);
  double mr = 0.0;
  for (int kind = 2; kind <= 3; kind++)
    for (int d = -p; d <= p; d++) {
      double r = fabs(cross_residual(p, kind, y, w, v, d));
      if (!(r <= mr)) mr = r;
    }
  if (max_resid) *max_resid = mr;
  int bad = !(mr <= 1e-14);
  for (int k = 0; k <= p; k++)
    if (!(y[k] > (double)k && y[k] < (double)(k + 1))) bad = 1;
  return bad ? 3 : 0;
}

/* Points and weights of row r in one direction for kind 2 (weight B_r', test
 * functions B_s) or kind 3 (weight B_r, test functions B_s').  Interior rows
 * (p <= r <= N-1): the mixed rule mapped to supp B_r, x_k = (r - p + y_k) h,
 * W_k = w_k (kind 2: int B_r' B_s dx = int N' N dy) or W_k = h v_k (kind 3:
 * B_s' = N'/h).  Other rows: (p+1)-point Gauss-Legendre on each element of
 * supp B_r with the weight function folded in, as for the other kinds. */
static int cross_row_rule(const dir1d *D, const double *cy, const double *cw, const double *cv, int kind, int r,
                          double *x, double *W) {
  int p = D->p;
  double h = D->h;
  if (r >= p && r <= D->N - 1) {
    for (int k = 0; k <= p; k++) {
      x[k] = ((double)(r - p) + cy[k]) * h;
      W[k] = kind == 2 ? cw[k] : h * cv[k];
    }
    return p + 1;
  }
  double gx[MAXP + 1], gw[MAXP + 1];
  gauss_legendre(p + 1, gx, gw);
  int L = 0;
  int elo = r - p < 0 ? 0 : r - p;
  int ehi = r > D->N - 1 ? D->N - 1 : r;
  for (int e = elo; e <= ehi; e++)
    for (int g = 0; g <= p; g++) {
      x[L] = ((double)e + 0.5 * (gx[g] + 1.0)) * h;
      W[L] = 0.5 * h * gw[g] * bspl(D->t, D->nt, r, p, kind == 2 ? 1 : 0, x[L]);
      L++;
    }
  return L;
}

/* ------------------------------------------------------------------ */
/* Geometry and coefficient at a parameter point                       */
/* ------------------------------------------------------------------ */

typedef struct {
  int dim, p;
  dir1d dir[3];
  const double *g[3];  /* 1D control values; control point i = (g1[i1], g2[i2], g3[i3]) */
  /* or, when not NULL, the full control net (Eq. Gmap1): component a of
   * control point (i1, i2, i3) at net[a * nctrl + i1 + n1 * (i2 + n2 * i3)] */
  const double *net;
  long long nctrl;
  const double *coef;  /* degree-3 coefficient spline, x fastest, or NULL for c = 1 */
} problem;

/* c(x) = sum_l c_l B3_l1(x1) B3_l2(x2) B3_l3(x3) over the 4^dim non-zero terms. */
static double coef_at(const problem *P, const double *x) {
  if (!P->coef) return 1.0;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, nc[3] = {1, 1, 1};
  double b[3][4] = {{1, 0, 0, 0}, {1, 0, 0, 0}, {1, 0, 0, 0}};
  for (int a = 0; a < P->dim; a++) {
    const dir1d *D = &P->dir[a];
    nc[a] = D->N + 3;
    lo[a] = element_of(D, x[a]);
    hi[a] = lo[a] + 3;
    for (int l = lo[a]; l <= hi[a]; l++) b[a][l - lo[a]] = cox_de_boor(D->tc, D->ntc, l, 3, x[a]);
  }
  double s = 0.0;
  for (int l3 = lo[2]; l3 <= hi[2]; l3++)
    for (int l2 = lo[1]; l2 <= hi[1]; l2++)
      for (int l1 = lo[0]; l1 <= hi[0]; l1++)
        s += P->coef[l1 + nc[0] * ((long long)l2 + nc[1] * (long long)l3)] * b[0][l1 - lo[0]] * b[1][l2 - lo[1]] * b[2][l3 - lo[2]];
  return s;
}

/* Full Jacobian J_ab = d x_a / d xhat_b of the tensor-product map (Eq. Gmap1,
 * Gmap2), summed over the (p+1)^dim control points that act at x.  Rows and
 * columns beyond dim are the identity. */
static void jacobian_at(const problem *P, const double *x, double J[3][3]) {
  int p = P->p, dim = P->dim;
  int lo[3] = {0, 0, 0}, cnt[3] = {1, 1, 1};
  double B[3][MAXP + 1], dB[3][MAXP + 1];
  for (int a = 0; a < 3; a++) { B[a][0] = 1.0; dB[a][0] = 0.0; }
  for (int a = 0; a < dim; a++) {
    const dir1d *D = &P->dir[a];
    lo[a] = element_of(D, x[a]);
    cnt[a] = p + 1;
    for (int i = 0; i <= p; i++) {
      B[a][i] = cox_de_boor(D->t, D->nt, lo[a] + i, p, x[a]);
      dB[a][i] = cox_de_boor_deriv(D->t, D->nt, lo[a] + i, p, x[a]);
    }
  }
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) J[a][b] = (a == b && a >= dim) ? 1.0 : 0.0;
  for (int i3 = 0; i3 < cnt[2]; i3++)
    for (int i2 = 0; i2 < cnt[1]; i2++)
      for (int i1 = 0; i1 < cnt[0]; i1++) {
        int idx[3] = {lo[0] + i1, lo[1] + i2, lo[2] + i3};
        int ii[3] = {i1, i2, i3};
        long long lin = idx[0] + (long long)P->dir[0].n * (idx[1] + (long long)P->dir[1].n * idx[2]);
        for (int b = 0; b < dim; b++) {
          double db = 1.0;
          for (int c = 0; c < dim; c++) db *= (c == b) ? dB[c][ii[c]] : B[c][ii[c]];
          for (int a = 0; a < dim; a++) J[a][b] += (P->net ? P->net[a * P->nctrl + lin] : P->g[a][idx[a]]) * db;
        }
      }
}

static double det3(double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

/* Inverse by the adjugate. */
static void inv3(double J[3][3], double det, double I[3][3]) {
  I[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  I[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  I[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  I[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  I[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  I[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  I[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  I[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  I[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
}

/* Geometry factors at x: out[0] = |det J| (the c-free mass factor) and
 * out[1+a] = |det J| (J^-1 J^-T)_aa; *offd = largest |(J^-1 J^-T)_ab|, a != b,
 * over the largest diagonal entry. */
static void geometry_factors(const problem *P, const double *x, double out[4], double *offd) {
  double J[3][3], I[3][3];
  jacobian_at(P, x, J);
  double det = det3(J);
  inv3(J, det, I);
  double G[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      G[a][b] = 0.0;
      for (int m = 0; m < 3; m++) G[a][b] += I[a][m] * I[b][m];
    }
  double ad = fabs(det);
  out[0] = ad;
  double dmax = 0.0, omax = 0.0;
  for (int a = 0; a < P->dim; a++) {
    out[1 + a] = ad * G[a][a];
    if (fabs(G[a][a]) > dmax) dmax = fabs(G[a][a]);
    for (int b = 0; b < P->dim; b++)
      if (a != b && fabs(G[a][b]) > omax) omax = fabs(G[a][b]);
  }
  *offd = dmax > 0.0 ? omax / dmax : omax;
}

/* ------------------------------------------------------------------ */
/* Row-wise weighted-quadrature assembly                               */
/* ------------------------------------------------------------------ */

static int setup_problem(problem *P, int dim, int p, const int *nel, const double *g1, const double *g2,
                         const double *g3, const double *coef) {
  if (dim < 1 || dim > 3 || p < 2 || p > MAXP) return 2;
  P->dim = dim;
  P->p = p;
  const double *gs[3] = {g1, g2, g3};
  for (int a = 0; a < 3; a++) {
    int N = a < dim ? nel[a] : 1;
    if (dir_init(&P->dir[a], p, N)) return 2;
    P->g[a] = a < dim ? gs[a] : NULL;
    if (a < dim && !gs[a]) return 2;
  }
  P->net = NULL;
  P->nctrl = 1;
  for (int a = 0; a < dim; a++) P->nctrl *= P->dir[a].n;
  P->coef = coef;
  return 0;
}

/* The same for a full control net (dim components of prod n_a values). */
static int setup_problem_net(problem *P, int dim, int p, const int *nel, const double *net, const double *coef) {
  if (!net) return 2;
  const double *gs[3] = {net, net, net}; /* placeholders, unused with a net */
  int st = setup_problem(P, dim, p, nel, gs[0], gs[1], gs[2], coef);
  if (st) return st;
  for (int a = 0; a < 3; a++) P->g[a] = NULL;
  P->net = net;
  return 0;
}

/* Assembles rows [row_begin, row_end) of M and/or K in band layout, each row
 * with its own rule (mode: RULE_WQ, the weighted Gaussian rules; RULE_GL or
 * RULE_NC, the comparison rules).  g1..g3: 1D control values of the
 * separable map (n_a = nel_a + p each); coef: degree-3 coefficient spline on
 * the same mesh (prod (nel_a + 3) values, x fastest) or NULL for c = 1.
 * Returns 0, 2 for bad arguments, 3 if a rule fails its check. */
static int assemble_mode(int mode, int dim, int p, const int *nel, const double *g1, const double *g2,
                         const double *g3, const double *coef, long long row_begin, long long row_end, double *M,
                         double *K, double *offdiag_max, int nthreads) {
  problem P;
  int st = setup_problem(&P, dim, p, nel, g1, g2, g3, coef);
  if (st) return st;
  rule_set RS;
  if (rule_set_init(&RS, p, mode)) return 3;
  int nb = 2 * p + 1;
  int band = 1;
  long long nrows = 1;
  int n[3] = {1, 1, 1};
  for (int a = 0; a < dim; a++) { band *= nb; n[a] = P.dir[a].n; nrows *= n[a]; }
  if (row_begin < 0 || row_end > nrows || row_begin > row_end) return 2;
  double offd_all = 0.0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 4) reduction(max : offd_all)
  for (long long r = row_begin; r < row_end; r++) {
    int ri[3] = {(int)(r % n[0]), (int)((r / n[0]) % n[1]), (int)(r / ((long long)n[0] * n[1]))};
    /* each direction's rule points for both kinds, and the band columns' basis
     * values (or derivatives) at those points */
    double x[3][2][MAXL], W[3][2][MAXL], bv[3][2][MAXL][2 * MAXP + 1];
    int L[3][2];
    for (int a = 0; a < 3; a++)
      for (int nu = 0; nu < 2; nu++) {
        if (a >= dim) {
          L[a][nu] = 1; x[a][nu][0] = 0.0; W[a][nu][0] = 1.0;
          for (int d = 0; d < nb; d++) bv[a][nu][0][d] = (d == p) ? 1.0 : 0.0;
          continue;
        }
        const dir1d *D = &P.dir[a];
        L[a][nu] = row_rule(D, &RS, nu, ri[a], x[a][nu], W[a][nu]);
        for (int k = 0; k < L[a][nu]; k++)
          for (int d = -p; d <= p; d++) {
            int s = ri[a] + d;
            bv[a][nu][k][d + p] = (s >= 0 && s < D->n) ? bspl(D->t, D->nt, s, p, nu, x[a][nu][k]) : 0.0;
          }
      }
    double *Mr = M ? M + (r - row_begin) * band : NULL;
    double *Kr = K ? K + (r - row_begin) * band : NULL;
    if (Mr) memset(Mr, 0, sizeof(double) * band);
    if (Kr) memset(Kr, 0, sizeof(double) * band);
    int dlo[3], dhi[3];
    for (int a = 0; a < 3; a++) { dlo[a] = a < dim ? -p : 0; dhi[a] = a < dim ? p : 0; }
    /* term 0: mass; term 1+a: stiffness, derivative direction a */
    for (int term = 0; term <= dim; term++) {
      if (term == 0 && !Mr) continue;
      if (term > 0 && !Kr) continue;
      int kind[3];
      for (int a = 0; a < 3; a++) kind[a] = (term == a + 1) ? 1 : 0;
      double *out = term == 0 ? Mr : Kr;
      for (int k3 = 0; k3 < L[2][kind[2]]; k3++)
        for (int k2 = 0; k2 < L[1][kind[1]]; k2++)
          for (int k1 = 0; k1 < L[0][kind[0]]; k1++) {
            double xp[3] = {x[0][kind[0]][k1], x[1][kind[1]][k2], x[2][kind[2]][k3]};
            double wprod = W[0][kind[0]][k1] * W[1][kind[1]][k2] * W[2][kind[2]][k3];
            double gf[4], offd;
            geometry_factors(&P, xp, gf, &offd);
            if (offd > offd_all) offd_all = offd;
            double C = coef_at(&P, xp) * gf[term];
            double wc = wprod * C;
            for (int d3 = dlo[2]; d3 <= dhi[2]; d3++)
              for (int d2 = dlo[1]; d2 <= dhi[1]; d2++)
                for (int d1 = dlo[0]; d1 <= dhi[0]; d1++) {
                  double v = wc * bv[0][kind[0]][k1][d1 + p] * bv[1][kind[1]][k2][d2 + p] * bv[2][kind[2]][k3][d3 + p];
                  int bi = 0, mul = 1;
                  int dd[3] = {d1, d2, d3};
                  for (int a = 0; a < dim; a++) { bi += (dd[a] + p) * mul; mul *= nb; }
                  out[bi] += v;
                }
          }
    }
  }
  if (offdiag_max) *offdiag_max = offd_all;
  return 0;
}

int wqo_assemble(int dim, int p, const int *nel, const double *g1, const double *g2, const double *g3,
                 const double *coef, long long row_begin, long long row_end, double *M, double *K,
                 double *offdiag_max, int nthreads) {
  return assemble_mode(RULE_WQ, dim, p, nel, g1, g2, g3, coef, row_begin, row_end, M, K, offdiag_max, nthreads);
}

/* The same assembly with the comparison rules: mode 1 = Gauss-Legendre on
 * every element of supp B_r for every row, mode 2 = Newton-Cotes-type
 * weighted rules on the interior rows; or mode 3, the weighted Gaussian
 * rules with boundary rows on their own weighted rules (wqo_boundary_rule,
 * Gauss-Legendre where none is defined or the mesh is below 2p+1 elements). */
int wqo_assemble_rule(int mode, int dim, int p, const int *nel, const double *g1, const double *g2,
                      const double *g3, const double *coef, long long row_begin, long long row_end, double *M,
                      double *K, int nthreads) {
  if (mode != RULE_GL && mode != RULE_NC && mode != RULE_WQB) return 2;
  return assemble_mode(mode, dim, p, nel, g1, g2, g3, coef, row_begin, row_end, M, K, NULL, nthreads);
}

/* ------------------------------------------------------------------ */
/* Element-wise Gauss-Legendre assembly of the exact integrals           */
/* ------------------------------------------------------------------ */

/* Rows [row_begin, row_end) of M_rs = int c |det J| B_r B_s and K_rs =
 * int c |det J| grad B_r^T J^-1 J^-T grad B_s (Eq. Mass, Eq. Stiffness, with
 * the full metric) by ng-point Gauss-Legendre on every element of supp B_r:
 * the classical element-wise assembly, exact when the integrand is a
 * piecewise polynomial of degree <= 2 ng - 1 per direction. */
static int assemble_gl_problem(problem *PP, int ng, long long row_begin, long long row_end, double *M, double *K,
                               int nthreads);

int wqo_assemble_gl(int dim, int p, const int *nel, const double *g1, const double *g2, const double *g3,
                    const double *coef, int ng, long long row_begin, long long row_end, double *M, double *K,
                    int nthreads) {
  problem P;
  int st = setup_problem(&P, dim, p, nel, g1, g2, g3, coef);
  if (st) return st;
  return assemble_gl_problem(&P, ng, row_begin, row_end, M, K, nthreads);
}

/* The same with the map given by its full control net (layout of problem.net). */
int wqo_assemble_gl_net(int dim, int p, const int *nel, const double *net, const double *coef, int ng,
                        long long row_begin, long long row_end, double *M, double *K, int nthreads) {
  problem P;
  int st = setup_problem_net(&P, dim, p, nel, net, coef);
  if (st) return st;
  return assemble_gl_problem(&P, ng, row_begin, row_end, M, K, nthreads);
}

static int assemble_gl_problem(problem *PP, int ng, long long row_begin, long long row_end, double *M, double *K,
                               int nthreads) {
  const problem P = *PP;
  const int dim = P.dim, p = P.p;
  if (ng < 1 || ng > 16) return 2;
  double gx[16], gw[16];
  gauss_legendre(ng, gx, gw);
  int nb = 2 * p + 1, band = 1;
  long long nrows = 1;
  int n[3] = {1, 1, 1};
  for (int a = 0; a < dim; a++) { band *= nb; n[a] = P.dir[a].n; nrows *= n[a]; }
  if (row_begin < 0 || row_end > nrows || row_begin > row_end) return 2;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 4)
  for (long long r = row_begin; r < row_end; r++) {
    int ri[3] = {(int)(r % n[0]), (int)((r / n[0]) % n[1]), (int)(r / ((long long)n[0] * n[1]))};
    double *Mr = M ? M + (r - row_begin) * band : NULL;
    double *Kr = K ? K + (r - row_begin) * band : NULL;
    if (Mr) memset(Mr, 0, sizeof(double) * band);
    if (Kr) memset(Kr, 0, sizeof(double) * band);
    int elo[3] = {0, 0, 0}, ehi[3] = {0, 0, 0};
    for (int a = 0; a < dim; a++) {
      elo[a] = ri[a] - p < 0 ? 0 : ri[a] - p;
      ehi[a] = ri[a] > P.dir[a].N - 1 ? P.dir[a].N - 1 : ri[a];
    }
    int nq[3] = {1, 1, 1};
    for (int a = 0; a < dim; a++) nq[a] = ng;
    for (int e3 = elo[2]; e3 <= ehi[2]; e3++)
      for (int e2 = elo[1]; e2 <= ehi[1]; e2++)
        for (int e1 = elo[0]; e1 <= ehi[0]; e1++)
          for (int g3 = 0; g3 < nq[2]; g3++)
            for (int g2 = 0; g2 < nq[1]; g2++)
              for (int g1 = 0; g1 < nq[0]; g1++) {
                int ee[3] = {e1, e2, e3}, gg[3] = {g1, g2, g3};
                double xp[3] = {0, 0, 0}, w = 1.0;
                for (int a = 0; a < dim; a++) {
                  double h = P.dir[a].h;
                  xp[a] = ((double)ee[a] + 0.5 * (gx[gg[a]] + 1.0)) * h;
                  w *= 0.5 * h * gw[gg[a]];
                }
                double J[3][3], I[3][3];
                jacobian_at(&P, xp, J);
                double det = det3(J);
                inv3(J, det, I);
                double c = coef_at(&P, xp);
                double Br[3] = {1, 1, 1}, dBr[3] = {0, 0, 0};
                for (int a = 0; a < dim; a++) {
                  Br[a] = bspl(P.dir[a].t, P.dir[a].nt, ri[a], p, 0, xp[a]);
                  dBr[a] = bspl(P.dir[a].t, P.dir[a].nt, ri[a], p, 1, xp[a]);
                }
                double gradr[3] = {0, 0, 0};
                for (int a = 0; a < dim; a++) {
                  gradr[a] = dBr[a];
                  for (int b = 0; b < dim; b++)
                    if (b != a) gradr[a] *= Br[b];
                }
                /* physical gradient of B_r: J^-T grad_hat */
                double pr[3] = {0, 0, 0};
                for (int m = 0; m < dim; m++)
                  for (int a = 0; a < dim; a++) pr[m] += I[a][m] * gradr[a];
                int dlo[3], dhi[3];
                for (int a = 0; a < 3; a++) { dlo[a] = a < dim ? -p : 0; dhi[a] = a < dim ? p : 0; }
                /* the band columns' basis values and derivatives at this point */
                double cB[3][2 * MAXP + 1], cdB[3][2 * MAXP + 1];
                int cok[3][2 * MAXP + 1];
                for (int a = 0; a < 3; a++)
                  for (int d = dlo[a]; d <= dhi[a]; d++) {
                    int j = d - dlo[a];
                    if (a >= dim) { cB[a][j] = 1.0; cdB[a][j] = 0.0; cok[a][j] = 1; continue; }
                    int s = ri[a] + d;
                    cok[a][j] = (s >= 0 && s < n[a]);
                    cB[a][j] = cok[a][j] ? bspl(P.dir[a].t, P.dir[a].nt, s, p, 0, xp[a]) : 0.0;
                    cdB[a][j] = cok[a][j] ? bspl(P.dir[a].t, P.dir[a].nt, s, p, 1, xp[a]) : 0.0;
                  }
                double wdc = w * fabs(det) * c;
                for (int d3 = dlo[2]; d3 <= dhi[2]; d3++)
                  for (int d2 = dlo[1]; d2 <= dhi[1]; d2++)
                    for (int d1 = dlo[0]; d1 <= dhi[0]; d1++) {
                      int dd[3] = {d1, d2, d3};
                      int jj[3] = {d1 - dlo[0], d2 - dlo[1], d3 - dlo[2]};
                      if (!cok[0][jj[0]] || !cok[1][jj[1]] || !cok[2][jj[2]]) continue;
                      double Bs[3], dBs[3];
                      for (int a = 0; a < 3; a++) { Bs[a] = cB[a][jj[a]]; dBs[a] = cdB[a][jj[a]]; }
                      int bi = 0, mul = 1;
                      for (int a = 0; a < dim; a++) { bi += (dd[a] + p) * mul; mul *= nb; }
                      if (Mr) Mr[bi] += wdc * Br[0] * Br[1] * Br[2] * Bs[0] * Bs[1] * Bs[2];
                      if (Kr) {
                        double grads[3] = {0, 0, 0}, ps[3] = {0, 0, 0};
                        for (int a = 0; a < dim; a++) {
                          grads[a] = dBs[a];
                          for (int b = 0; b < dim; b++)
                            if (b != a) grads[a] *= Bs[b];
                        }
                        for (int m = 0; m < dim; m++)
                          for (int a = 0; a < dim; a++) ps[m] += I[a][m] * grads[a];
                        double dot = 0.0;
                        for (int m = 0; m < dim; m++) dot += pr[m] * ps[m];
                        Kr[bi] += wdc * dot;
                      }
                    }
              }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Weighted-quadrature assembly for a non-separable map                 */
/* ------------------------------------------------------------------ */

/* |det J| and the metric G = J^-1 J^-T at x (full Jacobian, Eq. Gmap2). */
static double metric_at(const problem *P, const double *x, double G[3][3]) {
  double J[3][3], I[3][3];
  jacobian_at(P, x, J);
  double det = det3(J);
  inv3(J, det, I);
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      G[a][b] = 0.0;
      for (int m = 0; m < 3; m++) G[a][b] += I[a][m] * I[b][m];
    }
  return fabs(det);
}

/* Rows [row_begin, row_end) of M (Eq. Mass) and K (Eq. Stiffness with the
 * full metric) for the map given by its full control net, each row with its
 * own rules: M = the mass term; K = sum over a, b of the terms
 *   int dB_r/dxhat_a  c |det J| (J^-1 J^-T)_ab  dB_s/dxhat_b,
 * each integrated by the tensor product of one 1D rule per direction d:
 *   d = a = b: the stiffness rule (kind 1, Eq. GaussQuadSysStiff);
 *   d = a != b: the mixed rule of kind 2 (weight B_r', tests B_s);
 *   d = b != a: the mixed rule of kind 3 (weight B_r, tests B_s');
 *   otherwise: the mass rule (kind 0, Eq. GaussQuadSys);
 * the factor c |det J| (J^-1 J^-T)_ab (c |det J| for M) evaluated at every
 * point of that tensor grid.  Boundary rows use Gauss-Legendre in every kind
 * (Remark closing Sec. 3).  net: dim components of prod(nel_a + p) values
 * (layout of problem.net); coef as in wqo_assemble.  For a separable net the
 * off-diagonal metric is exactly zero and this equals wqo_assemble.
 * Returns 0, 2 for bad arguments, 3 if a rule fails its check. */
int wqo_assemble_general(int dim, int p, const int *nel, const double *net, const double *coef,
                         long long row_begin, long long row_end, double *M, double *K, int nthreads) {
  problem P;
  int st = setup_problem_net(&P, dim, p, nel, net, coef);
  if (st) return st;
  rule_set RS;
  if (rule_set_init(&RS, p, RULE_WQ)) return 3;
  double cy[MAXP + 1], cw[MAXP + 1], cv[MAXP + 1], cres;
  if (wqo_cross_rule(p, cy, cw, cv, &cres)) return 3;
  int nb = 2 * p + 1;
  int band = 1;
  long long nrows = 1;
  int n[3] = {1, 1, 1};
  for (int a = 0; a < dim; a++) { band *= nb; n[a] = P.dir[a].n; nrows *= n[a]; }
  if (row_begin < 0 || row_end > nrows || row_begin > row_end) return 2;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 4)
  for (long long r = row_begin; r < row_end; r++) {
    int ri[3] = {(int)(r % n[0]), (int)((r / n[0]) % n[1]), (int)(r / ((long long)n[0] * n[1]))};
    /* each direction's points and weights for the four kinds, and the band
     * columns' test values there: B_s for kinds 0 and 2, B_s' for 1 and 3 */
    double x[3][4][MAXL], W[3][4][MAXL], bv[3][4][MAXL][2 * MAXP + 1];
    int L[3][4];
    for (int a = 0; a < 3; a++)
      for (int kind = 0; kind < 4; kind++) {
        if (a >= dim) {
          L[a][kind] = 1; x[a][kind][0] = 0.0; W[a][kind][0] = 1.0;
          for (int d = 0; d < nb; d++) bv[a][kind][0][d] = (d == p) ? 1.0 : 0.0;
          continue;
        }
        const dir1d *D = &P.dir[a];
        L[a][kind] = kind < 2 ? row_rule(D, &RS, kind, ri[a], x[a][kind], W[a][kind])
                              : cross_row_rule(D, cy, cw, cv, kind, ri[a], x[a][kind], W[a][kind]);
        int nut = (kind == 1 || kind == 3);
        for (int k = 0; k < L[a][kind]; k++)
          for (int d = -p; d <= p; d++) {
            int s = ri[a] + d;
            bv[a][kind][k][d + p] = (s >= 0 && s < D->n) ? bspl(D->t, D->nt, s, p, nut, x[a][kind][k]) : 0.0;
          }
      }
    double *Mr = M ? M + (r - row_begin) * band : NULL;
    double *Kr = K ? K + (r - row_begin) * band : NULL;
    if (Mr) memset(Mr, 0, sizeof(double) * band);
    if (Kr) memset(Kr, 0, sizeof(double) * band);
    int dlo[3], dhi[3];
    for (int a = 0; a < 3; a++) { dlo[a] = a < dim ? -p : 0; dhi[a] = a < dim ? p : 0; }
    /* term -1: mass; term (a, b) = a * dim + b: stiffness */
    for (int term = -1; term < dim * dim; term++) {
      if (term < 0 && !Mr) continue;
      if (term >= 0 && !Kr) continue;
      int ta = term < 0 ? -1 : term / dim, tb = term < 0 ? -1 : term % dim;
      int kind[3];
      for (int d = 0; d < 3; d++) {
        if (term < 0 || d >= dim) kind[d] = 0;
        else if (d == ta && d == tb) kind[d] = 1;
        else if (d == ta) kind[d] = 2;
        else if (d == tb) kind[d] = 3;
        else kind[d] = 0;
      }
      double *out = term < 0 ? Mr : Kr;
      for (int k3 = 0; k3 < L[2][kind[2]]; k3++)
        for (int k2 = 0; k2 < L[1][kind[1]]; k2++)
          for (int k1 = 0; k1 < L[0][kind[0]]; k1++) {
            double xp[3] = {x[0][kind[0]][k1], x[1][kind[1]][k2], x[2][kind[2]][k3]};
            double wprod = W[0][kind[0]][k1] * W[1][kind[1]][k2] * W[2][kind[2]][k3];
            double G[3][3];
            double adet = metric_at(&P, xp, G);
            double C = coef_at(&P, xp) * adet * (term < 0 ? 1.0 : G[ta][tb]);
            double wc = wprod * C;
            for (int d3 = dlo[2]; d3 <= dhi[2]; d3++)
              for (int d2 = dlo[1]; d2 <= dhi[1]; d2++)
                for (int d1 = dlo[0]; d1 <= dhi[0]; d1++) {
                  double v = wc * bv[0][kind[0]][k1][d1 + p] * bv[1][kind[1]][k2][d2 + p] *
                             bv[2][kind[2]][k3][d3 + p];
                  int bi = 0, mul = 1;
                  int dd[3] = {d1, d2, d3};
                  for (int a = 0; a < dim; a++) { bi += (dd[a] + p) * mul; mul *= nb; }
                  out[bi] += v;
                }
          }
    }
  }
  return 0;
}

/* Points and weights of row r in one direction for kind 2 or 3 (for pins). */
int wqo_row_points_cross(int p, int N, int kind, int r, double *x, double *W) {
  dir1d D;
  if (kind != 2 && kind != 3) return -1;
  if (dir_init(&D, p, N)) return -1;
  double cy[MAXP + 1], cw[MAXP + 1], cv[MAXP + 1], res;
  if (wqo_cross_rule(p, cy, cw, cv, &res)) return -1;
  if (r < 0 || r >= D.n) return -1;
  return cross_row_rule(&D, cy, cw, cv, kind, r, x, W);
}

/* ------------------------------------------------------------------ */
/* Gradient of J(c) = sum G.*K(c) + sum H.*M(c) w.r.t. the coefficients  */
/* ------------------------------------------------------------------ */

/* grad[l] = dJ/dc_l, with K and M assembled by wqo_assemble.  Since every
 * band entry is linear in c, the derivative of entry (r, s) w.r.t. c_l is
 * the same weighted sum with c(x_k) replaced by B3_l(x_k).  G (for K) and H
 * (for M) are band arrays over all rows; either may be NULL.  grad has
 * prod(nel_a + 3) entries and is overwritten.  Runs on one thread. */
int wqo_gradient(int dim, int p, const int *nel, const double *g1, const double *g2, const double *g3,
                 const double *G, const double *H, double *grad) {
  problem P;
  int st = setup_problem(&P, dim, p, nel, g1, g2, g3, NULL);
  if (st) return st;
  rule_set RS;
  if (rule_set_init(&RS, p, RULE_WQ)) return 3;
  int nb = 2 * p + 1, band = 1;
  long long nrows = 1, ncoef = 1;
  int n[3] = {1, 1, 1}, nc[3] = {1, 1, 1};
  for (int a = 0; a < dim; a++) {
    band *= nb; n[a] = P.dir[a].n; nrows *= n[a];
    nc[a] = P.dir[a].N + 3; ncoef *= nc[a];
  }
  for (long long l = 0; l < ncoef; l++) grad[l] = 0.0;
  for (long long r = 0; r < nrows; r++) {
    int ri[3] = {(int)(r % n[0]), (int)((r / n[0]) % n[1]), (int)(r / ((long long)n[0] * n[1]))};
    double x[3][2][MAXL], W[3][2][MAXL], bv[3][2][MAXL][2 * MAXP + 1];
    int L[3][2];
    for (int a = 0; a < 3; a++)
      for (int nu = 0; nu < 2; nu++) {
        if (a >= dim) {
          L[a][nu] = 1; x[a][nu][0] = 0.0; W[a][nu][0] = 1.0;
          for (int d = 0; d < nb; d++) bv[a][nu][0][d] = (d == p) ? 1.0 : 0.0;
          continue;
        }
        const dir1d *D = &P.dir[a];
        L[a][nu] = row_rule(D, &RS, nu, ri[a], x[a][nu], W[a][nu]);
        for (int k = 0; k < L[a][nu]; k++)
          for (int d = -p; d <= p; d++) {
            int s = ri[a] + d;
            bv[a][nu][k][d + p] = (s >= 0 && s < D->n) ? bspl(D->t, D->nt, s, p, nu, x[a][nu][k]) : 0.0;
          }
      }
    int dlo[3], dhi[3];
    for (int a = 0; a < 3; a++) { dlo[a] = a < dim ? -p : 0; dhi[a] = a < dim ? p : 0; }
    for (int term = 0; term <= dim; term++) {
      const double *S = term == 0 ? H : G;
      if (!S) continue;
      const double *Sr = S + r * band;
      int kind[3];
      for (int a = 0; a < 3; a++) kind[a] = (term == a + 1) ? 1 : 0;
      for (int k3 = 0; k3 < L[2][kind[2]]; k3++)
        for (int k2 = 0; k2 < L[1][kind[1]]; k2++)
          for (int k1 = 0; k1 < L[0][kind[0]]; k1++) {
            double xp[3] = {x[0][kind[0]][k1], x[1][kind[1]][k2], x[2][kind[2]][k3]};
            double wprod = W[0][kind[0]][k1] * W[1][kind[1]][k2] * W[2][kind[2]][k3];
            double gf[4], offd;
            geometry_factors(&P, xp, gf, &offd);
            /* sum over the band of S_rs * prod_a basis values */
            double acc = 0.0;
            for (int d3 = dlo[2]; d3 <= dhi[2]; d3++)
              for (int d2 = dlo[1]; d2 <= dhi[1]; d2++)
                for (int d1 = dlo[0]; d1 <= dhi[0]; d1++) {
                  int dd[3] = {d1, d2, d3};
                  int bi = 0, mul = 1;
                  for (int a = 0; a < dim; a++) { bi += (dd[a] + p) * mul; mul *= nb; }
                  acc += Sr[bi] * bv[0][kind[0]][k1][d1 + p] * bv[1][kind[1]][k2][d2 + p] * bv[2][kind[2]][k3][d3 + p];
                }
            double f = wprod * gf[term] * acc;
            /* scatter into the coefficients acting at xp */
            int lo[3] = {0, 0, 0}, cnt[3] = {1, 1, 1};
            double b[3][4] = {{1, 0, 0, 0}, {1, 0, 0, 0}, {1, 0, 0, 0}};
            for (int a = 0; a < dim; a++) {
              const dir1d *D = &P.dir[a];
              lo[a] = element_of(D, xp[a]);
              cnt[a] = 4;
              for (int i = 0; i < 4; i++) b[a][i] = cox_de_boor(D->tc, D->ntc, lo[a] + i, 3, xp[a]);
            }
            for (int i3 = 0; i3 < cnt[2]; i3++)
              for (int i2 = 0; i2 < cnt[1]; i2++)
                for (int i1 = 0; i1 < cnt[0]; i1++)
                  grad[(lo[0] + i1) + nc[0] * ((long long)(lo[1] + i2) + nc[1] * (long long)(lo[2] + i3))] +=
                      f * b[0][i1] * b[1][i2] * b[2][i3];
          }
    }
  }
  return 0;
}

/* Number of rule points of row r in one direction (for point-count pins). */
int wqo_row_points(int p, int N, int nu, int r, double *x, double *W) {
  dir1d D;
  if (dir_init(&D, p, N)) return -1;
  rule_set RS;
  if (rule_set_init(&RS, p, RULE_WQ)) return -1;
  if (r < 0 || r >= D.n) return -1;
  return row_rule(&D, &RS, nu, r, x, W);
}

/* The same in a given rule mode (RULE_WQ .. RULE_WQB). */
int wqo_row_points_mode(int mode, int p, int N, int nu, int r, double *x, double *W) {
  dir1d D;
  if (mode < RULE_WQ || mode > RULE_WQB) return -1;
  if (dir_init(&D, p, N)) return -1;
  rule_set RS;
  if (rule_set_init(&RS, p, mode)) return -1;
  if (r < 0 || r >= D.n) return -1;
  return row_rule(&D, &RS, nu, r, x, W);
}
