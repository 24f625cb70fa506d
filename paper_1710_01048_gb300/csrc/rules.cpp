// Host FP64 construction of the univariate weighted Gaussian rules and of the
// per-direction row tables consumed by the assembly kernels.
//
// Rules (Sec. 3): a symmetric (p+1)-point rule on the cardinal support
// [0, p+1] that is exact for the products N(y) N(y-d) (mass, Eq. GaussQuadSys)
// or N'(y) N'(y-d) (stiffness, Eq. GaussQuadSysStiff), d = -p..p.  The right
// hand sides are exact rationals: int N_p(y) N_p(y-d) dy = N_{2p+1}(p+1+d) and
// int N_p'(y) N_p'(y-d) dy = -N''_{2p+1}(p+1+d).  The unknowns of the symmetric
// rule are found by Gauss-Newton with an analytic Jacobian over the p+1
// independent conditions d = 0..p, steps halved whenever a node would leave
// its element (one node per element, Sec. 3.1.2 and Sec. 3.2), then checked
// against all 2p+1 conditions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "wq_internal.h"

namespace wq {
namespace {

long long binom(int n, int k) {
  long long r = 1;
  for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
  return r;
}

long long factorial(int n) {
  long long r = 1;
  for (int i = 2; i <= n; i++) r *= i;
  return r;
}

// m-th derivative of the cardinal B-spline of degree n at an integer x, as an
// exact integer numerator over (n-m)!: sum_j (-1)^j C(n+1, j) (x-j)_+^(n-m).
long long cardinal_at_integer_num(int n, int m, int x) {
  long long s = 0;
  for (int j = 0; j <= n + 1; j++) {
    int t = x - j;
    if (t <= 0) continue;
    long long pw = 1;
    for (int k = 0; k < n - m; k++) pw *= t;
    s += ((j & 1) ? -1 : 1) * binom(n + 1, j) * pw;
  }
  return s;
}

// Exact moment of the weight function: mass m(d) = N_{2p+1}(p+1+d),
// stiffness k(d) = -N''_{2p+1}(p+1+d).
double exact_moment(int p, int kind, int d) {
  int n = 2 * p + 1;
  d = std::abs(d);
  if (d > p) return 0.0;
  if (kind == WQ_KIND_MASS) return (double)cardinal_at_integer_num(n, 0, p + 1 + d) / (double)factorial(n);
  return -(double)cardinal_at_integer_num(n, 2, p + 1 + d) / (double)factorial(n - 2);
}

// m-th derivative of the degree-p cardinal B-spline at real y by the
// truncated-power form, evaluated on the nearer half of the support
// (N^(m)(y) = (-1)^m N^(m)(p+1-y)) to limit cancellation.
double cardinal(int p, int m, double y) {
  if (!(y > 0.0 && y < (double)(p + 1))) return 0.0;
  double sign = 1.0;
  if (y > 0.5 * (p + 1)) {
    y = (double)(p + 1) - y;
    if (m & 1) sign = -1.0;
  }
  double s = 0.0;
  for (int j = 0; j <= p + 1; j++) {
    double t = y - (double)j;
    if (t <= 0.0) break;
    double pw = 1.0;
    for (int k = 0; k < p - m; k++) pw *= t;
    s += ((j & 1) ? -1.0 : 1.0) * (double)binom(p + 1, j) * pw;
  }
  return sign * s / (double)factorial(p - m);
}

// Affine parametrisation of the symmetric rule: tau = At*u + bt, omega = Aw*u + bw.
struct Param {
  int nu;  // unknowns
  double At[4][4], bt[4], Aw[4][4], bw[4];
};

Param make_param(int p, int kind) {
  Param P;
  std::memset(&P, 0, sizeof(P));
  int L = p + 1;
  if (p == 2 && kind == WQ_KIND_MASS) {  // u = (tau1, omega1, omega2), tau2 = 3/2
    P.nu = 3;
    P.At[0][0] = 1; P.bt[1] = 1.5; P.At[2][0] = -1; P.bt[2] = 3;
    P.Aw[0][1] = 1; P.Aw[1][2] = 1; P.Aw[2][1] = 1;
  } else if (p == 3 && kind == WQ_KIND_MASS) {  // u = (tau1, tau2, omega1, omega2)
    P.nu = 4;
    P.At[0][0] = 1; P.At[1][1] = 1; P.At[2][1] = -1; P.bt[2] = 4; P.At[3][0] = -1; P.bt[3] = 4;
    P.Aw[0][2] = 1; P.Aw[1][3] = 1; P.Aw[2][3] = 1; P.Aw[3][2] = 1;
  } else if (p == 2) {  // stiffness: u = (tau1, omega1), tau2 = 3/2, omega2 = 8/9
    P.nu = 2;
    P.At[0][0] = 1; P.bt[1] = 1.5; P.At[2][0] = -1; P.bt[2] = 3;
    P.Aw[0][1] = 1; P.bw[1] = 8.0 / 9.0; P.Aw[2][1] = 1;
  } else {  // p = 3 stiffness: u = (tau1, tau2, omega2), omega1 = 1
    P.nu = 3;
    P.At[0][0] = 1; P.At[1][1] = 1; P.At[2][1] = -1; P.bt[2] = 4; P.At[3][0] = -1; P.bt[3] = 4;
    P.bw[0] = 1; P.Aw[1][2] = 1; P.Aw[2][2] = 1; P.bw[3] = 1;
  }
  (void)L;
  return P;
}

void expand(const Param &P, int L, const double *u, double *tau, double *om) {
  for (int k = 0; k < L; k++) {
    tau[k] = P.bt[k];
    om[k] = P.bw[k];
    for (int j = 0; j < P.nu; j++) {
      tau[k] += P.At[k][j] * u[j];
      om[k] += P.Aw[k][j] * u[j];
    }
  }
}

double residual(int p, int kind, const double *tau, const double *om, int d) {
  int m = kind;  // the weight function's derivative order
  double s = 0.0;
  for (int k = 0; k <= p; k++) s += om[k] * cardinal(p, m, tau[k]) * cardinal(p, m, tau[k] - d);
  return s - exact_moment(p, kind, d);
}

bool nodes_in_elements(int p, const double *tau) {
  for (int k = 0; k <= p; k++)
    if (!(tau[k] > (double)k && tau[k] < (double)(k + 1))) return false;
  return true;
}

// Solves the small symmetric positive system (J^T J) x = r by Gaussian elimination.
bool solve_small(int n, double A[4][4], double *b) {
  for (int c = 0; c < n; c++) {
    int piv = c;
    for (int r = c + 1; r < n; r++)
      if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
    if (A[piv][c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < n; k++) std::swap(A[c][k], A[piv][k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; r++) {
      double f = A[r][c] / A[c][c];
      for (int k = c; k < n; k++) A[r][k] -= f * A[c][k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; r--) {
    double s = b[r];
    for (int k = r + 1; k < n; k++) s -= A[r][k] * b[k];
    b[r] = s / A[r][r];
  }
  return true;
}

}  // namespace

wq_status solve_rule(int p, int kind, const double *start, double *tau, double *omega) {
  if (p < 2 || p > kMaxP || (kind != WQ_KIND_MASS && kind != WQ_KIND_STIFFNESS)) return WQ_ERR_UNSUPPORTED;
  int L = p + 1;
  Param P = make_param(p, kind);
  double u[4];
  for (int j = 0; j < P.nu; j++) u[j] = start[j];
  int neq = p + 1;  // conditions d = 0..p
  int m = kind;
  for (int it = 0; it < 100; it++) {
    double t[4], w[4];
    expand(P, L, u, t, w);
    double F[4], Jm[4][4];
    for (int e = 0; e < neq; e++) {
      int d = e;
      F[e] = residual(p, kind, t, w, d);
      double dFt[4], dFw[4];
      for (int k = 0; k < L; k++) {
        double a = cardinal(p, m, t[k]), b = cardinal(p, m, t[k] - d);
        double da = cardinal(p, m + 1, t[k]), db = cardinal(p, m + 1, t[k] - d);
        dFt[k] = w[k] * (da * b + a * db);
        dFw[k] = a * b;
      }
      for (int j = 0; j < P.nu; j++) {
        double s = 0.0;
        for (int k = 0; k < L; k++) s += dFt[k] * P.At[k][j] + dFw[k] * P.Aw[k][j];
        Jm[e][j] = s;
      }
    }
    double N[4][4], g[4];
    for (int i = 0; i < P.nu; i++) {
      g[i] = 0.0;
      for (int e = 0; e < neq; e++) g[i] -= Jm[e][i] * F[e];
      for (int j = 0; j < P.nu; j++) {
        N[i][j] = 0.0;
        for (int e = 0; e < neq; e++) N[i][j] += Jm[e][i] * Jm[e][j];
      }
    }
    if (!solve_small(P.nu, N, g)) return WQ_ERR_NO_CONVERGENCE;
    bool inside0 = nodes_in_elements(p, t);
    double scale = 1.0, unew[4];
    for (int h = 0; h < 60; h++) {
      for (int j = 0; j < P.nu; j++) unew[j] = u[j] + scale * g[j];
      if (!inside0) break;
      double tt[4], ww[4];
      expand(P, L, unew, tt, ww);
      if (nodes_in_elements(p, tt)) break;
      scale *= 0.5;
    }
    double smax = 0.0;
    for (int j = 0; j < P.nu; j++) {
      smax = std::max(smax, std::fabs(unew[j] - u[j]));
      u[j] = unew[j];
      if (!std::isfinite(u[j]) || std::fabs(u[j]) > 1e6) return WQ_ERR_NO_CONVERGENCE;
    }
    if (smax < 1e-16 && it >= 3) break;
  }
  expand(P, L, u, tau, omega);
  if (!nodes_in_elements(p, tau)) return WQ_ERR_NO_CONVERGENCE;
  for (int d = -p; d <= p; d++)
    if (!(std::fabs(residual(p, kind, tau, omega, d)) <= 1e-14)) return WQ_ERR_NO_CONVERGENCE;
  if (kind == WQ_KIND_MASS)
    for (int k = 0; k < L; k++)
      if (!(omega[k] > 0.0)) return WQ_ERR_NO_CONVERGENCE;
  return WQ_OK;
}

// Default rules.  p=2 stiffness has the closed form tau = (3/4, 3/2, 9/4),
// omega = 8/9 (Sec. 3.2.1); the others start from element midpoints (the
// p=3 stiffness tau_1 from the midpoint of [0, 1/2], on the branch of the
// smaller root, Sec. 3.2.2).
wq_status default_rule(int p, int kind, double *tau, double *omega) {
  if (p < 2 || p > kMaxP || (kind != WQ_KIND_MASS && kind != WQ_KIND_STIFFNESS)) return WQ_ERR_UNSUPPORTED;
  if (p == 2 && kind == WQ_KIND_STIFFNESS) {
    tau[0] = 0.75; tau[1] = 1.5; tau[2] = 2.25;
    omega[0] = omega[1] = omega[2] = 8.0 / 9.0;
    for (int d = -p; d <= p; d++)
      if (!(std::fabs(residual(p, kind, tau, omega, d)) <= 1e-14)) return WQ_ERR_NO_CONVERGENCE;
    return WQ_OK;
  }
  double start[4];
  if (p == 2) { start[0] = 0.5; start[1] = 1.0; start[2] = 1.0; }
  else if (kind == WQ_KIND_MASS) { start[0] = 0.5; start[1] = 1.5; start[2] = 1.0; start[3] = 1.0; }
  else { start[0] = 0.25; start[1] = 1.5; start[2] = 1.0; }
  return solve_rule(p, kind, start, tau, omega);
}

namespace {

// Gauss-Legendre on [-1, 1] for n = 3, 4 in closed form.
void gauss_legendre(int n, double *x, double *w) {
  if (n == 3) {
    double a = std::sqrt(0.6);
    x[0] = -a; x[1] = 0.0; x[2] = a;
    w[0] = 5.0 / 9.0; w[1] = 8.0 / 9.0; w[2] = 5.0 / 9.0;
  } else {  // n == 4
    double s = 2.0 / 7.0 * std::sqrt(1.2);
    double xi = std::sqrt(3.0 / 7.0 - s), xo = std::sqrt(3.0 / 7.0 + s);
    double wi = (18.0 + std::sqrt(30.0)) / 36.0, wo = (18.0 - std::sqrt(30.0)) / 36.0;
    x[0] = -xo; x[1] = -xi; x[2] = xi; x[3] = xo;
    w[0] = wo; w[1] = wi; w[2] = wi; w[3] = wo;
  }
}

std::vector<double> knots(int q, int N) {
  std::vector<double> t(N + 2 * q + 1);
  for (int i = 0; i < (int)t.size(); i++) {
    int k = i - q;
    t[i] = k <= 0 ? 0.0 : (k >= N ? 1.0 : (double)k / (double)N);
  }
  return t;
}

// Values and first derivatives of the q+1 degree-q B-splines B_e..B_{e+q}
// acting on element e, at x, by the triangular (de Boor) recurrence.
void basis(const std::vector<double> &t, int q, int e, double x, double *val, double *der, double *low = nullptr) {
  int i = e + q;
  double left[8], right[8], Nt[8][8];
  Nt[0][0] = 1.0;
  for (int d = 1; d <= q; d++) {
    left[d] = x - t[i + 1 - d];
    right[d] = t[i + d] - x;
    double saved = 0.0;
    for (int r = 0; r < d; r++) {
      double temp = Nt[d - 1][r] / (right[r + 1] + left[d - r]);
      Nt[d][r] = saved + right[r + 1] * temp;
      saved = left[d - r] * temp;
    }
    Nt[d][d] = saved;
  }
  for (int j = 0; j <= q; j++) {
    val[j] = Nt[q][j];
    double a = 0.0, b = 0.0;
    if (j >= 1) {
      double den = t[i + j] - t[i - q + j];
      if (den > 0.0) a = Nt[q - 1][j - 1] / den;
    }
    if (j <= q - 1) {
      double den = t[i + j + 1] - t[i - q + j + 1];
      if (den > 0.0) b = Nt[q - 1][j] / den;
    }
    der[j] = (double)q * (a - b);
  }
  // degree q-1 on the same knots: B_{e+1+j, q-1}(x), j = 0..q-1
  if (low)
    for (int j = 0; j < q; j++) low[j] = Nt[q - 1][j];
}

// ------------------------------------------------------------------ boundary rows
// Weighted Gaussian rules for the rows whose weight function touches the
// boundary (the Remark closing Sec. 3 leaves them to the systems "modified
// accordingly").  Row r < p of kind nu: ceil(rank/2) nodes exact for the
// products B_r^(nu) B_s^(nu), s = 0 .. r+p (rank r+p+1 for the mass kind;
// r+p for the stiffness kind, whose derivatives sum to zero, so s = r+p is
// dropped), and, when the rank is odd, for B_r^(nu) (x/h)^(p-nu+1).  Defined
// for every mass row, the stiffness rows of p = 2 and rows 0 and 2 of p = 3
// stiffness (row 1 has no such rule inside its support).  The rule is found
// by variable projection: for given nodes the combined weights W_k solve the
// linear least-squares problem of the conditions, and the nodes follow
// damped Gauss-Newton steps on the remaining residual (central-difference
// Jacobian), from a fixed list of starting nodes, on a reference mesh of
// 2p+1 elements; results in units of h (t = x/h, Wl = W / h^(1-nu)).

bool boundary_rule_defined(int p, int kind, int r) {
  if (r < 0 || r >= p) return false;
  return kind == WQ_KIND_MASS || p == 2 || r != 1;
}

struct BoundarySystem {
  int p, kind, r, nf, n;
  bool extra;
  double h, a, b;
  std::vector<double> t;  // degree-p knots of the reference mesh
  double mu[2 * kMaxP + 2];
  // condition function j at x: B_j^(kind)(x) (j < rank), else (x/h)^(p-kind+1)
  double f(int j, double x) const {
    if (extra && j == nf - 1) return std::pow(x / h, (double)(p - kind + 1));
    const int N = (int)std::lround(1.0 / h);
    int e = (int)std::floor(x / h);
    e = std::max(0, std::min(N - 1, e));
    const int i = j - e;
    if (i < 0 || i > p) return 0.0;
    double v[8], dv[8];
    basis(t, p, e, x, v, dv);
    return kind == WQ_KIND_MASS ? v[i] : dv[i];
  }
};

// Weights minimising |A(x) W - mu| for nodes x (normal equations), and the
// residual A W - mu; false if the normal matrix is singular.
bool project_weights(const BoundarySystem &S, const double *x, double *W, double *res) {
  const int n = S.n, nf = S.nf;
  double A[2 * kMaxP + 2][kMaxP + 1];
  for (int j = 0; j < nf; j++)
    for (int k = 0; k < n; k++) A[j][k] = S.f(j, x[k]);
  double G[kMaxP + 1][kMaxP + 2];
  for (int k = 0; k < n; k++) {
    for (int l = 0; l < n; l++) {
      double acc = 0.0;
      for (int j = 0; j < nf; j++) acc += A[j][k] * A[j][l];
      G[k][l] = acc;
    }
    double acc = 0.0;
    for (int j = 0; j < nf; j++) acc += A[j][k] * S.mu[j];
    G[k][n] = acc;
  }
  for (int c = 0; c < n; c++) {
    int piv = c;
    for (int r = c + 1; r < n; r++)
      if (std::fabs(G[r][c]) > std::fabs(G[piv][c])) piv = r;
    if (!(std::fabs(G[piv][c]) > 0.0)) return false;
    for (int k = 0; k <= n; k++) std::swap(G[c][k], G[piv][k]);
    for (int r = 0; r < n; r++) {
      if (r == c) continue;
      const double m = G[r][c] / G[c][c];
      for (int k = c; k <= n; k++) G[r][k] -= m * G[c][k];
    }
  }
  for (int k = 0; k < n; k++) W[k] = G[k][n] / G[k][k];
  for (int j = 0; j < nf; j++) {
    double acc = -S.mu[j];
    for (int k = 0; k < n; k++) acc += A[j][k] * W[k];
    res[j] = acc;
  }
  return true;
}

double sumsq(const double *v, int n) {
  double s = 0.0;
  for (int i = 0; i < n; i++) s += v[i] * v[i];
  return s;
}

wq_status boundary_rule_impl(int p, int kind, int r, double *tl, double *wl, int *npts) {
  *npts = 0;
  if (!boundary_rule_defined(p, kind, r)) return WQ_ERR_UNSUPPORTED;
  BoundarySystem S;
  const int Nref = 2 * p + 1;
  S.p = p;
  S.kind = kind;
  S.r = r;
  S.h = 1.0 / (double)Nref;
  S.t = knots(p, Nref);
  const int m = r + p + 1, rank = kind == WQ_KIND_MASS ? m : m - 1;
  S.n = (rank + 1) / 2;
  S.extra = (rank % 2) == 1;
  S.nf = rank + (S.extra ? 1 : 0);
  S.a = 0.0;
  S.b = (double)(r + 1) * S.h;
  // moments: 4-point Gauss-Legendre on each element of the support (exact
  // for the products, of degree <= 2p+1)
  double gx[4], gw[4];
  gauss_legendre(4, gx, gw);
  for (int j = 0; j < S.nf; j++) {
    double acc = 0.0;
    for (int e = 0; e <= r; e++)
      for (int g = 0; g < 4; g++) {
        const double x = ((double)e + 0.5 * (gx[g] + 1.0)) * S.h;
        double v[8], dv[8];
        basis(S.t, p, e, x, v, dv);
        const double wr = kind == WQ_KIND_MASS ? v[r - e] : dv[r - e];
        acc += 0.5 * S.h * gw[g] * wr * S.f(j, x);
      }
    S.mu[j] = acc;
  }
  double scale = 1.0;
  for (int j = 0; j < S.nf; j++) scale = std::max(scale, std::fabs(S.mu[j]));
  const int n = S.n, nf = S.nf;
  for (int start = 0; start < 4; start++) {
    double x[kMaxP + 1], W[kMaxP + 1], res[2 * kMaxP + 2];
    for (int k = 0; k < n; k++) {
      const double u = (k + 0.5) / (double)n;
      const double f = start == 0 ? (k + 1.0) / (n + 1.0) : start == 1 ? u * u : start == 2 ? 1.0 - (1.0 - u) * (1.0 - u) : u;
      x[k] = S.a + f * (S.b - S.a);
    }
    if (!project_weights(S, x, W, res)) continue;
    double lam = 1e-3;
    for (int it = 0; it < 400 && std::sqrt(sumsq(res, nf)) > 1e-16 * scale; it++) {
      // Jacobian of the projected residual with respect to the nodes
      double J[2 * kMaxP + 2][kMaxP + 1];
      for (int k = 0; k < n; k++) {
        double xp[kMaxP + 1], xm[kMaxP + 1], Wt[kMaxP + 1], rp[2 * kMaxP + 2], rm[2 * kMaxP + 2];
        std::copy(x, x + n, xp);
        std::copy(x, x + n, xm);
        const double d = 1e-7 * S.h;
        xp[k] += d;
        xm[k] -= d;
        if (!project_weights(S, xp, Wt, rp) || !project_weights(S, xm, Wt, rm)) return WQ_ERR_NO_CONVERGENCE;
        for (int j = 0; j < nf; j++) J[j][k] = (rp[j] - rm[j]) / (2.0 * d);
      }
      bool moved = false;
      while (lam < 1e14 && !moved) {
        double G[kMaxP + 1][kMaxP + 2];
        for (int k = 0; k < n; k++) {
          for (int l = 0; l < n; l++) {
            double acc = 0.0;
            for (int j = 0; j < nf; j++) acc += J[j][k] * J[j][l];
            G[k][l] = acc * (k == l ? 1.0 + lam : 1.0);
          }
          double acc = 0.0;
          for (int j = 0; j < nf; j++) acc -= J[j][k] * res[j];
          G[k][n] = acc;
        }
        bool ok = true;
        for (int c = 0; c < n && ok; c++) {
          int piv = c;
          for (int r2 = c + 1; r2 < n; r2++)
            if (std::fabs(G[r2][c]) > std::fabs(G[piv][c])) piv = r2;
          if (!(std::fabs(G[piv][c]) > 0.0)) ok = false;
          else {
            for (int k = 0; k <= n; k++) std::swap(G[c][k], G[piv][k]);
            for (int r2 = 0; r2 < n; r2++) {
              if (r2 == c) continue;
              const double mm = G[r2][c] / G[c][c];
              for (int k = c; k <= n; k++) G[r2][k] -= mm * G[c][k];
            }
          }
        }
        if (ok) {
          double xn[kMaxP + 1], Wn[kMaxP + 1], rn[2 * kMaxP + 2];
          bool inside = true;
          for (int k = 0; k < n; k++) {
            xn[k] = x[k] + G[k][n] / G[k][k];
            if (!(xn[k] > S.a && xn[k] < S.b)) inside = false;
          }
          if (inside && project_weights(S, xn, Wn, rn) && sumsq(rn, nf) < sumsq(res, nf)) {
            std::copy(xn, xn + n, x);
            std::copy(Wn, Wn + n, W);
            std::copy(rn, rn + nf, res);
            lam = std::max(lam * 0.1, 1e-12);
            moved = true;
            break;
          }
        }
        lam *= 10.0;
      }
      if (!moved) break;
    }
    double worst = 0.0;
    for (int j = 0; j < nf; j++) worst = std::max(worst, std::fabs(res[j]));
    if (worst <= 1e-14 * scale) {
      // ascending nodes in units of h
      for (int k = 0; k < n; k++)
        for (int l = k + 1; l < n; l++)
          if (x[l] < x[k]) {
            std::swap(x[k], x[l]);
            std::swap(W[k], W[l]);
          }
      for (int k = 0; k < n; k++) {
        tl[k] = x[k] / S.h;
        wl[k] = kind == WQ_KIND_MASS ? W[k] / S.h : W[k];
      }
      *npts = n;
      return WQ_OK;
    }
  }
  return WQ_ERR_NO_CONVERGENCE;
}

}  // namespace

// Newton-Cotes-type weighted rule on the cardinal support [0, p+1] (the
// comparison rules of Sec. 1 and Sec. 4): nodes at the interior knots and the
// element midpoints, y_k = (k+1)/2, k = 0..2p, one per interacting function;
// weights v_k (the weight function's value folded in) from the square linear
// system sum_k v_k N^(nu)(y_k - d) = exact moment(d), d = -p..p.  For the
// stiffness kind N' vanishes at the centre y = (p+1)/2: its weight is 0 and
// the other 2p weights solve d = -p..p-1 (the translates' derivatives sum to
// zero, so d = p follows).  All 2p+1 conditions are checked to 1e-14.
wq_status nc_rule(int p, int kind, double *y, double *v) {
  const int nn = 2 * p + 1, centre = p;
  int cols[2 * kMaxP + 1], m = 0;
  for (int k = 0; k < nn; k++) {
    y[k] = 0.5 * (double)(k + 1);
    v[k] = 0.0;
    if (!(kind == WQ_KIND_STIFFNESS && k == centre)) cols[m++] = k;
  }
  // Gaussian elimination with partial pivoting on the m x m system
  double A[2 * kMaxP + 1][2 * kMaxP + 1], b[2 * kMaxP + 1];
  for (int e = 0; e < m; e++) {
    const int d = -p + e;
    for (int j = 0; j < m; j++) A[e][j] = cardinal(p, kind, y[cols[j]] - (double)d);
    b[e] = exact_moment(p, kind, d);
  }
  for (int c = 0; c < m; c++) {
    int piv = c;
    for (int r = c + 1; r < m; r++)
      if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
    if (A[piv][c] == 0.0) return WQ_ERR_NO_CONVERGENCE;
    for (int k = 0; k < m; k++) std::swap(A[c][k], A[piv][k]);
    std::swap(b[c], b[piv]);
    for (int r = c + 1; r < m; r++) {
      const double f = A[r][c] / A[c][c];
      for (int k = c; k < m; k++) A[r][k] -= f * A[c][k];
      b[r] -= f * b[c];
    }
  }
  for (int r = m - 1; r >= 0; r--) {
    double acc = b[r];
    for (int k = r + 1; k < m; k++) acc -= A[r][k] * b[k];
    b[r] = acc / A[r][r];
  }
  for (int j = 0; j < m; j++) v[cols[j]] = b[j];
  for (int d = -p; d <= p; d++) {
    double res = -exact_moment(p, kind, d);
    for (int k = 0; k < nn; k++) res += v[k] * cardinal(p, kind, y[k] - (double)d);
    if (!(std::fabs(res) <= 1e-14)) return WQ_ERR_NO_CONVERGENCE;
  }
  return WQ_OK;
}

// ------------------------------------------------------------------ mixed-derivative rules
// A non-separable map adds to Eq. Stiffness the terms dB_r/dxhat_a C_ab
// dB_s/dxhat_b, a != b.  In direction a they pair the weight B_r' with the
// tests B_s (kind 2), in direction b the weight B_r with the tests B_s'
// (kind 3); Sec. 3.2 covers the (B', B') pair only.  One node set per
// interior row serves both kinds: on the cardinal support [0, p+1], nodes y
// symmetric about the centre, kind 2 weights w antisymmetric, kind 3 weights
// v symmetric, so that each kind keeps the p conditions d = 1..p
//   sum_k w_k N(y_k - d) = int N' N(. - d) =  N'_{2p+1}(p+1+d),
//   sum_k v_k N'(y_k - d) = int N N'(. - d) = -N'_{2p+1}(p+1+d)
// (derivatives of the convolution identity int N N(. - d) = N_{2p+1}(p+1+d)).
// p = 3: two node pairs, six unknowns; p = 2: one pair and the centre node
// (antisymmetric weight 0 there), four unknowns.  Newton's method with the
// analytic Jacobian from the element midpoints; the result must meet all
// 2p+1 conditions of both kinds and keep one node per element.
namespace {

struct MixedParam {
  int nu;
  double Ay[4][6], by[4], Aw[4][6], Av[4][6];
};

MixedParam mixed_param(int p) {
  MixedParam P;
  std::memset(&P, 0, sizeof(P));
  if (p == 2) {  // u = (y1, w1, v1, vc)
    P.nu = 4;
    P.Ay[0][0] = 1; P.by[1] = 1.5; P.Ay[2][0] = -1; P.by[2] = 3;
    P.Aw[0][1] = 1; P.Aw[2][1] = -1;
    P.Av[0][2] = 1; P.Av[1][3] = 1; P.Av[2][2] = 1;
  } else {  // u = (y1, y2, w1, w2, v1, v2)
    P.nu = 6;
    P.Ay[0][0] = 1; P.Ay[1][1] = 1; P.Ay[2][1] = -1; P.by[2] = 4; P.Ay[3][0] = -1; P.by[3] = 4;
    P.Aw[0][2] = 1; P.Aw[1][3] = 1; P.Aw[2][3] = -1; P.Aw[3][2] = -1;
    P.Av[0][4] = 1; P.Av[1][5] = 1; P.Av[2][5] = 1; P.Av[3][4] = 1;
  }
  return P;
}

void mixed_expand(const MixedParam &P, int L, const double *u, double *y, double *w, double *v) {
  for (int k = 0; k < L; k++) {
    y[k] = P.by[k];
    w[k] = 0.0;
    v[k] = 0.0;
    for (int j = 0; j < P.nu; j++) {
      y[k] += P.Ay[k][j] * u[j];
      w[k] += P.Aw[k][j] * u[j];
      v[k] += P.Av[k][j] * u[j];
    }
  }
}

// int N'(y) N(y - d) dy = N'_{2p+1}(p+1+d) (kind 2; kind 3 is its negative).
double mixed_moment(int p, int d) {
  if (d < -p || d > p) return 0.0;
  const int n = 2 * p + 1;
  return (double)cardinal_at_integer_num(n, 1, p + 1 + d) / (double)factorial(n - 1);
}

double mixed_residual(int p, int kind, const double *y, const double *w, const double *v, int d) {
  double s = 0.0;
  for (int k = 0; k <= p; k++)
    s += kind == 2 ? w[k] * cardinal(p, 0, y[k] - d) : v[k] * cardinal(p, 1, y[k] - d);
  return s - (kind == 2 ? mixed_moment(p, d) : -mixed_moment(p, d));
}

bool solve_n(int n, double A[6][6], double *b) {
  for (int c = 0; c < n; c++) {
    int piv = c;
    for (int r = c + 1; r < n; r++)
      if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
    if (A[piv][c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < n; k++) std::swap(A[c][k], A[piv][k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; r++) {
      const double f = A[r][c] / A[c][c];
      for (int k = c; k < n; k++) A[r][k] -= f * A[c][k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; r--) {
    double t = b[r];
    for (int k = r + 1; k < n; k++) t -= A[r][k] * b[k];
    b[r] = t / A[r][r];
  }
  return true;
}

}  // namespace

wq_status mixed_rule(int p, double *y, double *w, double *v) {
  if (p < 2 || p > kMaxP) return WQ_ERR_UNSUPPORTED;
  const int L = p + 1;
  const MixedParam P = mixed_param(p);
  double u[6];
  if (p == 2) { u[0] = 0.5; u[1] = 1.0; u[2] = 0.25; u[3] = 0.5; }
  else { u[0] = 0.5; u[1] = 1.5; u[2] = 1.0; u[3] = 1.0; u[4] = 0.25; u[5] = 0.25; }
  for (int it = 0; it < 100; it++) {
    double yy[4], ww[4], vv[4];
    mixed_expand(P, L, u, yy, ww, vv);
    double F[6], Jm[6][6];
    for (int e = 0; e < 2 * p; e++) {
      const int kind = e < p ? 2 : 3, d = e % p + 1;
      F[e] = -mixed_residual(p, kind, yy, ww, vv, d);
      for (int j = 0; j < P.nu; j++) {
        double t = 0.0;
        for (int k = 0; k < L; k++) {
          if (kind == 2)
            t += ww[k] * cardinal(p, 1, yy[k] - d) * P.Ay[k][j] + cardinal(p, 0, yy[k] - d) * P.Aw[k][j];
          else
            t += vv[k] * cardinal(p, 2, yy[k] - d) * P.Ay[k][j] + cardinal(p, 1, yy[k] - d) * P.Av[k][j];
        }
        Jm[e][j] = t;
      }
    }
    if (!solve_n(P.nu, Jm, F)) return WQ_ERR_NO_CONVERGENCE;
    double smax = 0.0;
    for (int j = 0; j < P.nu; j++) {
      u[j] += F[j];
      smax = std::max(smax, std::fabs(F[j]));
      if (!std::isfinite(u[j]) || std::fabs(u[j]) > 1e6) return WQ_ERR_NO_CONVERGENCE;
    }
    if (smax < 1e-16 && it >= 3) break;
  }
  mixed_expand(P, L, u, y, w, v);
  for (int k = 0; k < L; k++)
    if (!(y[k] > (double)k && y[k] < (double)(k + 1))) return WQ_ERR_NO_CONVERGENCE;
  for (int kind = 2; kind <= 3; kind++)
    for (int d = -p; d <= p; d++)
      if (!(std::fabs(mixed_residual(p, kind, y, w, v, d)) <= 1e-14)) return WQ_ERR_NO_CONVERGENCE;
  return WQ_OK;
}

wq_status boundary_rule(int p, int kind, int r, double *t, double *Wl, int *npts) {
  return boundary_rule_impl(p, kind, r, t, Wl, npts);
}

wq_status build_host_tables(wq_rules *R) {
  int p = R->p;
  // boundary weighted rules of the low-side rows, both kinds (units of h)
  double bt[2][kMaxP][kMaxP + 1] = {}, bw[2][kMaxP][kMaxP + 1] = {};
  int bn[2][kMaxP] = {};
  if (R->bnd_weighted)
    for (int kind = 0; kind < 2; kind++)
      for (int r = 0; r < p; r++) {
        if (!boundary_rule_defined(p, kind, r)) continue;
        wq_status st = boundary_rule_impl(p, kind, r, bt[kind][r], bw[kind][r], &bn[kind][r]);
        if (st != WQ_OK) return st;
      }
  for (int kind = 0; kind < 2; kind++) {
    wq_status st = default_rule(p, kind, R->tau[kind], R->omega[kind]);
    if (st != WQ_OK) return st;
  }
  double ncy[2][2 * kMaxP + 1], ncv[2][2 * kMaxP + 1];
  if (R->mode == kModeNC)
    for (int kind = 0; kind < 2; kind++) {
      wq_status st = nc_rule(p, kind, ncy[kind], ncv[kind]);
      if (st != WQ_OK) return st;
    }
  double gx[4], gw[4];
  gauss_legendre(p + 1, gx, gw);
  for (int a = 0; a < R->dim; a++) {
    int N = R->nel[a], n = R->n[a];
    double h = 1.0 / (double)N;
    std::vector<double> tp = knots(p, N), tc = knots(kCoefDeg, N);
    for (int kind = 0; kind < 2; kind++) {
      HostDirKind &H = R->host[a][kind];
      H = HostDirKind();
      H.off.assign(n + 1, 0);
      for (int r = 0; r < n; r++) {
        H.off[r] = (int)H.elem.size();
        // points of row r: (element, x, weight factor before B_r)
        std::vector<int> pe;
        std::vector<double> px, pf;
        bool folded = false;  // pf already holds the combined weight W
        const bool bnd_row = r < p || r > N - 1;
        if (R->bnd_weighted && bnd_row && N >= 2 * p + 1) {
          // both kinds' points (weighted rule, or Gauss-Legendre where none
          // is defined) with combined weights, then per element the larger
          // of the two counts, the shorter list padded with zero weights at
          // the element's midpoint
          folded = true;
          const int low = r < p, rm = low ? r : n - 1 - r;
          const int elo = std::max(0, r - p), ehi = std::min(N - 1, r);
          std::vector<int> ke[2];
          std::vector<double> kx[2], kw[2];
          for (int k = 0; k < 2; k++) {
            if (bn[k][rm] > 0) {
              for (int q = 0; q < bn[k][rm]; q++) {
                const double x = low ? bt[k][rm][q] * h : 1.0 - bt[k][rm][q] * h;
                const double sgn = (low || k == WQ_KIND_MASS) ? 1.0 : -1.0;
                ke[k].push_back(std::max(0, std::min(N - 1, (int)std::floor(x / h))));
                kx[k].push_back(x);
                kw[k].push_back(sgn * bw[k][rm][q] * (k == WQ_KIND_MASS ? h : 1.0));
              }
            } else {
              for (int e = elo; e <= ehi; e++)
                for (int g = 0; g <= p; g++) {
                  const double x = ((double)e + 0.5 * (gx[g] + 1.0)) * h;
                  double v[8], dv[8];
                  basis(tp, p, e, x, v, dv);
                  ke[k].push_back(e);
                  kx[k].push_back(x);
                  kw[k].push_back(0.5 * h * gw[g] * (k == WQ_KIND_MASS ? v[r - e] : dv[r - e]));
                }
            }
          }
          for (int e = elo; e <= ehi; e++) {
            int cnt[2] = {0, 0};
            for (int k = 0; k < 2; k++)
              for (size_t q = 0; q < ke[k].size(); q++) cnt[k] += ke[k][q] == e;
            std::vector<std::pair<double, double>> own;  // (x, W) of this kind in element e
            for (size_t q = 0; q < ke[kind].size(); q++)
              if (ke[kind][q] == e) own.push_back({kx[kind][q], kw[kind][q]});
            std::sort(own.begin(), own.end());
            while ((int)own.size() < std::max(cnt[0], cnt[1])) own.push_back({((double)e + 0.5) * h, 0.0});
            for (const auto &pt : own) {
              pe.push_back(e);
              px.push_back(pt.first);
              pf.push_back(pt.second);
            }
          }
        } else if (R->mode == kModeWQ && r >= p && r <= N - 1) {
          for (int k = 0; k <= p; k++) {
            pe.push_back(r - p + k);
            px.push_back(((double)(r - p) + R->tau[kind][k]) * h);
            pf.push_back(h * R->omega[kind][k]);
          }
        } else if (R->mode == kModeNC && r >= p && r <= N - 1) {
          // W = h v (mass) or v (stiffness): B_r^(nu)(x) = h^-nu N^(nu)(y)
          folded = true;
          for (int k = 0; k <= 2 * p; k++) {
            pe.push_back(r - p + (int)std::floor(ncy[kind][k]));
            px.push_back(((double)(r - p) + ncy[kind][k]) * h);
            pf.push_back(kind == WQ_KIND_MASS ? h * ncv[kind][k] : ncv[kind][k]);
          }
        } else {
          int elo = std::max(0, r - p), ehi = std::min(N - 1, r);
          for (int e = elo; e <= ehi; e++)
            for (int g = 0; g <= p; g++) {
              pe.push_back(e);
              px.push_back(((double)e + 0.5 * (gx[g] + 1.0)) * h);
              pf.push_back(0.5 * h * gw[g]);
            }
        }
        for (size_t q = 0; q < pe.size(); q++) {
          int e = pe[q];
          double x = px[q];
          double v[8], dv[8], cv[8], cd[8], lo[8];
          basis(tp, p, e, x, v, dv, lo);
          for (int i = 0; i < p; i++) H.tl.push_back(lo[i]);
          basis(tc, kCoefDeg, e, x, cv, cd);
          int j = r - e;  // B_r among B_e..B_{e+p}
          double br = folded ? 1.0 : (kind == WQ_KIND_MASS ? v[j] : dv[j]);
          H.elem.push_back(e);
          H.x.push_back(x);
          H.w.push_back(pf[q] * br);
          for (int i = 0; i <= p; i++) {
            H.t0.push_back(v[i]);
            H.t1.push_back(dv[i]);
          }
          for (int i = 0; i <= kCoefDeg; i++) H.beta.push_back(cv[i]);
        }
      }
      H.off[n] = (int)H.elem.size();
    }
  }
  // mixed-derivative kinds (maps given by a full control net): the mixed
  // rules on interior rows, Gauss-Legendre with B_r' (kind 2) or B_r (kind
  // 3) folded in on boundary rows; same point counts and elements per row as
  // the mass kind
  for (int a = 0; a < 3; a++) R->hostx[a] = HostCross();
  if (R->mode == kModeWQ && !R->bnd_weighted) {
    double my[kMaxP + 1], mw[kMaxP + 1], mv[kMaxP + 1];
    wq_status st = mixed_rule(p, my, mw, mv);
    if (st != WQ_OK) return st;
    for (int a = 0; a < R->dim; a++) {
      const int N = R->nel[a], n = R->n[a];
      const double h = 1.0 / (double)N;
      std::vector<double> tp = knots(p, N), tc = knots(kCoefDeg, N);
      HostCross &X = R->hostx[a];
      X.off.assign(n + 1, 0);
      for (int r = 0; r < n; r++) {
        X.off[r] = (int)X.elem.size();
        std::vector<int> pe;
        std::vector<double> px, pw2, pw3;
        if (r >= p && r <= N - 1) {
          for (int k = 0; k <= p; k++) {
            pe.push_back(r - p + k);
            px.push_back(((double)(r - p) + my[k]) * h);
            pw2.push_back(mw[k]);      // int B_r' B_s dx = int N' N dy
            pw3.push_back(h * mv[k]);  // B_s' = N' / h
          }
        } else {
          const int elo = std::max(0, r - p), ehi = std::min(N - 1, r);
          for (int e = elo; e <= ehi; e++)
            for (int g = 0; g <= p; g++) {
              const double x = ((double)e + 0.5 * (gx[g] + 1.0)) * h;
              double v[8], dv[8];
              basis(tp, p, e, x, v, dv);
              pe.push_back(e);
              px.push_back(x);
              pw2.push_back(0.5 * h * gw[g] * dv[r - e]);
              pw3.push_back(0.5 * h * gw[g] * v[r - e]);
            }
        }
        for (size_t q = 0; q < pe.size(); q++) {
          double v[8], dv[8], cv[8], cd[8], lo[8];
          basis(tp, p, pe[q], px[q], v, dv, lo);
          for (int i = 0; i < p; i++) X.tl.push_back(lo[i]);
          basis(tc, kCoefDeg, pe[q], px[q], cv, cd);
          X.elem.push_back(pe[q]);
          X.x.push_back(px[q]);
          X.w2.push_back(pw2[q]);
          X.w3.push_back(pw3[q]);
          for (int i = 0; i <= p; i++) {
            X.t0.push_back(v[i]);
            X.t1.push_back(dv[i]);
          }
          for (int i = 0; i <= kCoefDeg; i++) X.beta.push_back(cv[i]);
        }
      }
      X.off[n] = (int)X.elem.size();
    }
  }
  // lines: D=3 -> (r2, r3), D=2 -> r2; interior when dirs 2..D are interior rows
  R->lines = Lines();
  int nl = R->dim == 3 ? R->n[1] * R->n[2] : R->n[1];
  for (int l = 0; l < nl; l++) {
    int r2 = l % R->n[1];
    int r3 = R->dim == 3 ? l / R->n[1] : 0;
    bool in2 = r2 >= p && r2 <= R->nel[1] - 1;
    bool in3 = R->dim == 3 ? (r3 >= p && r3 <= R->nel[2] - 1) : true;
    (in2 && in3 ? R->lines.interior : R->lines.boundary).push_back(l);
  }
  return WQ_OK;
}

// Flops of the sum-factorised contractions over the band's non-zero
// structure: per row and per direction, L_a points each touching p+1 band
// entries, and an active band width A_a (the union of the touched entries).
// Mass uses one point grid; stiffness uses d grids whose first two stages
// are separate and whose last stage runs over the mass- and stiffness-kind
// points of direction 1 (the terms with mass kind in direction 1 are summed
// before it).  Coefficient evaluation: the cubic spline of c on each grid,
// sum-factorised over the coefficients of each line of rows.
int chunk_length(const wq_rules *R, int tmax) {
  const int n1 = R->n[0], nch = (n1 + tmax - 1) / tmax;
  return (n1 + nch - 1) / nch;
}

int max_chunk_points(const wq_rules *R, int T) {
  const std::vector<int> &off = R->host[0][0].off;
  const int n1 = R->n[0];
  int mx = 0;
  for (int c = 0; c * T < n1; c++) mx = std::max(mx, off[std::min(n1, (c + 1) * T)] - off[c * T]);
  return mx;
}

double flop_count(const wq_rules *R, int want_m, int want_k, int64_t row_begin, int64_t row_end,
                  double *coef_flops) {
  int p = R->p, D = R->dim, NP = p + 1;
  auto pts = [&](int a, int r) { return R->host[a][0].off[r + 1] - R->host[a][0].off[r]; };
  auto active = [&](int a, int r) {
    int lo = std::max(0, r - p), hi = std::min(R->n[a] - 1, r + p);
    return hi - lo + 1;
  };
  double fl = 0.0, cf = 0.0;
  int ng = (want_m ? 1 : 0) + (want_k ? D : 0);
  for (int64_t row = row_begin; row < row_end; row++) {
    int r1 = (int)(row % R->n[0]);
    int64_t rest = row / R->n[0];
    int r2 = (int)(rest % R->n[1]);
    int r3 = D == 3 ? (int)(rest / R->n[1]) : 0;
    double L1 = pts(0, r1), L2 = pts(1, r2), L3 = D == 3 ? pts(2, r3) : 1;
    double A2 = active(1, r2), A3 = D == 3 ? active(2, r3) : 1;
    double fma = 0.0;
    if (D == 3) {
      double xy = L1 * L2 * L3 * NP + L1 * A3 * L2 * NP;  // per grid: dir-3 then dir-2 stage
      if (want_m) fma += xy + A2 * A3 * L1 * NP;
      if (want_k) fma += 3 * xy + A2 * A3 * 2 * L1 * NP + 0.5 * A2 * A3 * L1;  // + the (K2+K3) adds
    } else {
      double y = L1 * L2 * NP;
      if (want_m) fma += y + A2 * L1 * NP;
      if (want_k) fma += 2 * y + A2 * 2 * L1 * NP;
    }
    fl += 2.0 * fma;
    cf += 2.0 * ng * L1 * L2 * L3 * (kCoefDeg + 1);
  }
  if (coef_flops) {
    // per line of rows: dir-3 then dir-2 contraction of the coefficient block
    // (one pass over the n1 + 3 coefficient columns), shared by its rows
    double lines_part = 0.0;
    int64_t first_line = row_begin / R->n[0], last_line = row_end > row_begin ? (row_end - 1) / R->n[0] : -1;
    for (int64_t l = first_line; l <= last_line; l++) {
      int r2 = (int)(l % R->n[1]);
      int r3 = D == 3 ? (int)(l / R->n[1]) : 0;
      double L2 = pts(1, r2), L3 = D == 3 ? pts(2, r3) : 1;
      double nl2 = std::min(R->nel[1] - 1, r2) - std::max(0, r2 - p) + 1 + kCoefDeg;
      double ncomb = want_k ? D : 1;
      if (D == 3) {
        double nl3kinds = want_k ? 2 : 1;
        lines_part += 2.0 * R->nc[0] * (nl3kinds * nl2 * L3 * 4 + ncomb * L2 * L3 * 4);
      } else {
        lines_part += 2.0 * R->nc[0] * (want_k ? 2 : 1) * L2 * 4;
      }
    }
    *coef_flops = cf + lines_part;
  }
  return fl;
}

}  // namespace wq
