/*
 * oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Written for readability against the paper (arXiv 2211.05458), not speed:
 * direct sums instead of sum factorisation, Bezier subdivision instead of a
 * Newton face solve, Newton from xi = 0 instead of a tuned initial guess.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXG 6   /* geometry nodes per direction, NGeo <= 5 */
#define MAXN 10  /* solution nodes per direction, N <= 9    */

struct or_ctx {
  int nelem, ngeo, g;
  double* xgeo;
  int32_t *nbr, *nbf, *bc;
  double* shift;
  int nmortar;
  int32_t* mortar; /* [nmortar][9] non-conforming faces, layout in oracle.h */
  double* ctrl; /* [nelem][6][g*g][3] Bezier control points of every face */
  double* bbox; /* [nelem][6][6]    lo xyz, hi xyz of those control points */
  double geo_nodes[MAXG];
  int N, n, node_type;
  double nodes[MAXN];
  double* U;
};

/* ------------------------------------------------------------------------ */
/* 1-D nodes and Lagrange polynomials (Sec. 3.1, Eq. dgsem_interpolation)    */
/* ------------------------------------------------------------------------ */

/* Legendre polynomial P_n(x) by Bonnet's recurrence; *dp receives P_n'(x). */
static double legendre(int n, double x, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    if (dp) *dp = 0.0;
    return 1.0;
  }
  for (int k = 2; k <= n; ++k) {
    double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = pk;
  }
  /* (x^2-1) P_n' = n (x P_n - P_{n-1}) */
  if (dp) *dp = n * (x * p1 - p0) / (x * x - 1.0);
  return p1;
}

/* kind 0: n Legendre-Gauss nodes (roots of P_n);
 * kind 1: n Legendre-Gauss-Lobatto nodes (+-1 and the roots of P_{n-1}');
 * kind 2: n equidistant nodes.  Ascending order. */
void or_nodes(int kind, int n, double* out) {
  const double pi = 3.14159265358979323846;
  if (n == 1) {
    out[0] = 0.0;
    return;
  }
  if (kind == 2) {
    for (int i = 0; i < n; ++i) out[i] = -1.0 + 2.0 * i / (n - 1);
    return;
  }
  if (kind == 0) {
    for (int i = 0; i < n; ++i) {
      double x = -cos(pi * (i + 0.75) / (n + 0.5));
      for (int it = 0; it < 100; ++it) {
        double dp, p = legendre(n, x, &dp);
        double dx = p / dp;
        x -= dx;
        if (fabs(dx) < 1e-16) break;
      }
      out[i] = x;
    }
    return;
  }
  /* GLL: interior points are the roots of P_N', N = n-1.  Newton on P_N' with
   * P_N'' from Legendre's equation (1-x^2) P'' - 2x P' + N(N+1) P = 0. */
  int N = n - 1;
  out[0] = -1.0;
  out[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double x = -cos(pi * i / N);
    for (int it = 0; it < 100; ++it) {
      double dp, p = legendre(N, x, &dp);
      double d2p = (2.0 * x * dp - N * (N + 1.0) * p) / (1.0 - x * x);
      double dx = dp / d2p;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    out[i] = x;
  }
}

/* l_i(x) = prod_{m != i} (x - x_m) / (x_i - x_m) */
double or_lagrange(int n, const double* xn, int i, double x) {
  double r = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != i) r *= (x - xn[m]) / (xn[i] - xn[m]);
  return r;
}

/* l_i'(x) = sum_{k != i} 1/(x_i - x_k) prod_{m != i,k} (x - x_m)/(x_i - x_m) */
double or_lagrange_deriv(int n, const double* xn, int i, double x) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    if (k == i) continue;
    double r = 1.0 / (xn[i] - xn[k]);
    for (int m = 0; m < n; ++m)
      if (m != i && m != k) r *= (x - xn[m]) / (xn[i] - xn[m]);
    s += r;
  }
  return s;
}

/* ------------------------------------------------------------------------ */
/* small dense linear algebra                                                 */
/* ------------------------------------------------------------------------ */

/* Solve A x = b (n x n, row-major, copied) by Gaussian elimination with
 * partial pivoting.  Returns 0 if A is singular. */
static int gauss_solve(int n, const double* Ain, const double* b, double* x) {
  double A[MAXG * MAXG + 16], r[MAXG + 4];
  memcpy(A, Ain, sizeof(double) * n * n);
  memcpy(r, b, sizeof(double) * n);
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > fabs(A[piv * n + k])) piv = i;
    if (A[piv * n + k] == 0.0) return 0;
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[k * n + j];
        A[k * n + j] = A[piv * n + j];
        A[piv * n + j] = t;
      }
      double t = r[k];
      r[k] = r[piv];
      r[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      r[i] -= f * r[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = r[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
    x[i] = s / A[i * n + i];
  }
  return 1;
}

static double maxabs3(const double* a) {
  double m = fabs(a[0]);
  if (fabs(a[1]) > m) m = fabs(a[1]);
  if (fabs(a[2]) > m) m = fabs(a[2]);
  return m;
}

static double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------ */
/* element geometry: x = chi(xi) (Sec. 3.1, Eq. dgsem_curvedfaces)            */
/* ------------------------------------------------------------------------ */

/* node index of face node (m, k) on local face f; the face parameter s runs
 * along the first free reference direction, t along the second. */
static int face_node(int f, int g, int m, int k) {
  int last = g - 1, a, b, c;
  switch (f) {
    case 0: a = 0; b = m; c = k; break;
    case 1: a = last; b = m; c = k; break;
    case 2: a = m; b = 0; c = k; break;
    case 3: a = m; b = last; c = k; break;
    case 4: a = m; b = k; c = 0; break;
    default: a = m; b = k; c = last; break;
  }
  return a + g * (b + g * c);
}

static void face_to_xi(int f, double s, double t, double* xi) {
  double side = (f & 1) ? 1.0 : -1.0;
  switch (f / 2) {
    case 0: xi[0] = side; xi[1] = s; xi[2] = t; break;
    case 1: xi[0] = s; xi[1] = side; xi[2] = t; break;
    default: xi[0] = s; xi[1] = t; xi[2] = side; break;
  }
}

/* chi(xi) = sum_abc X_abc l_a(xi1) l_b(xi2) l_c(xi3) and its Jacobian
 * J[r][q] = d chi_r / d xi_q, as a direct triple sum. */
void or_elem_map(const or_ctx* c, int e, const double xi[3], double x[3], double J[9]) {
  int g = c->g;
  const double* X = c->xgeo + (size_t)e * g * g * g * 3;
  double l[3][MAXG], dl[3][MAXG];
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < g; ++a) {
      l[d][a] = or_lagrange(g, c->geo_nodes, a, xi[d]);
      dl[d][a] = or_lagrange_deriv(g, c->geo_nodes, a, xi[d]);
    }
  for (int r = 0; r < 3; ++r) {
    x[r] = 0.0;
    for (int q = 0; q < 3; ++q) J[r * 3 + q] = 0.0;
  }
  for (int cc = 0; cc < g; ++cc)
    for (int b = 0; b < g; ++b)
      for (int a = 0; a < g; ++a) {
        const double* P = X + 3 * (a + g * (b + g * cc));
        double w = l[0][a] * l[1][b] * l[2][cc];
        double w0 = dl[0][a] * l[1][b] * l[2][cc];
        double w1 = l[0][a] * dl[1][b] * l[2][cc];
        double w2 = l[0][a] * l[1][b] * dl[2][cc];
        for (int r = 0; r < 3; ++r) {
          x[r] += P[r] * w;
          J[r * 3 + 0] += P[r] * w0;
          J[r * 3 + 1] += P[r] * w1;
          J[r * 3 + 2] += P[r] * w2;
        }
      }
}

/* Newton's method for chi(xi) - x = 0 from xi = 0 (Sec. 3.2.1).  Stops when
 * |dxi|_inf < newton_tol; fails after max_newton iterations, on a singular
 * Jacobian, or if an iterate leaves [-4, 4]^3 (divergence: from xi = 0 the
 * first step may overshoot the element on curved meshes, so the bound is loose). */
int or_newton(const or_ctx* c, const or_params* p, int e, const double x[3], double xi[3],
              int* iters) {
  xi[0] = xi[1] = xi[2] = 0.0;
  for (int it = 1; it <= p->max_newton; ++it) {
    double chi[3], J[9], r[3], dxi[3];
    or_elem_map(c, e, xi, chi, J);
    for (int d = 0; d < 3; ++d) r[d] = chi[d] - x[d];
    if (!gauss_solve(3, J, r, dxi)) return 0;
    for (int d = 0; d < 3; ++d) xi[d] -= dxi[d];
    if (iters) *iters = it;
    if (maxabs3(dxi) < p->newton_tol) return 1;
    if (maxabs3(xi) > 4.0) return 0;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* interpolation of the nodal state (Sec. 3.2.1, Eq. part_interpolation)      */
/* ------------------------------------------------------------------------ */

void or_interp(const or_ctx* c, int e, const double xi[3], double U[5]) {
  int n = c->n;
  double l[3][MAXN];
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < n; ++i) l[d][i] = or_lagrange(n, c->nodes, i, xi[d]);
  const double* Ue = c->U + (size_t)e * 5 * n * n * n;
  for (int v = 0; v < 5; ++v) {
    double s = 0.0;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
          s += Ue[(size_t)v * n * n * n + i + n * (j + n * k)] * l[0][i] * l[1][j] * l[2][k];
    U[v] = s;
  }
}

/* U and its reference-space derivatives dU[v][q] = dU_v / dxi_q, by
 * differentiating the same Lagrange interpolant. */
void or_interp_grad(const or_ctx* c, int e, const double xi[3], double U[5], double dU[15]) {
  int n = c->n;
  double l[3][MAXN], dl[3][MAXN];
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < n; ++i) {
      l[d][i] = or_lagrange(n, c->nodes, i, xi[d]);
      dl[d][i] = or_lagrange_deriv(n, c->nodes, i, xi[d]);
    }
  const double* Ue = c->U + (size_t)e * 5 * n * n * n;
  for (int v = 0; v < 5; ++v) {
    double s = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          double u = Ue[(size_t)v * n * n * n + i + n * (j + n * k)];
          s += u * l[0][i] * l[1][j] * l[2][k];
          s0 += u * dl[0][i] * l[1][j] * l[2][k];
          s1 += u * l[0][i] * dl[1][j] * l[2][k];
          s2 += u * l[0][i] * l[1][j] * dl[2][k];
        }
    U[v] = s;
    dU[3 * v] = s0;
    dU[3 * v + 1] = s1;
    dU[3 * v + 2] = s2;
  }
}

/* Physical velocity gradient G[i][j] = du_i/dx_j of u = (rho u)/rho:
 * du_i/dxi_q = (d(rho u_i)/dxi_q - u_i drho/dxi_q) / rho, and by the chain
 * rule du_i/dx_j = sum_q du_i/dxi_q dxi_q/dx_j with dxi/dx = J^{-1}. */
void or_velocity_gradient(const or_ctx* c, int e, const double xi[3], double G[9]) {
  double U[5], dU[15], chi[3], J[9];
  or_interp_grad(c, e, xi, U, dU);
  or_elem_map(c, e, xi, chi, J);
  double Dxi[9]; /* Dxi[i][q] = du_i/dxi_q */
  for (int i = 0; i < 3; ++i) {
    double ui = U[1 + i] / U[0];
    for (int q = 0; q < 3; ++q) Dxi[3 * i + q] = (dU[3 * (1 + i) + q] - ui * dU[q]) / U[0];
  }
  /* row i of G solves G_i J = Dxi_i, i.e. J^T G_i^T = Dxi_i^T */
  double JT[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) JT[3 * a + b] = J[3 * b + a];
  for (int i = 0; i < 3; ++i) {
    double row[3];
    gauss_solve(3, JT, Dxi + 3 * i, row);
    for (int j = 0; j < 3; ++j) G[3 * i + j] = row[j];
  }
}

/* ------------------------------------------------------------------------ */
/* face representation: Bezier control points (Sec. 3.2.4)                   */
/* ------------------------------------------------------------------------ */

static double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

/* Bernstein basis of degree p on u in [0,1] */
static double bernstein(int p, int k, double u) {
  return binom(p, k) * pow(u, k) * pow(1.0 - u, p - k);
}

/* Vinv such that Bezier control points B = Vinv * (nodal values at the
 * equidistant geometry nodes), i.e. the inverse of V_jk = B_k(u_j). */
static void lagrange_to_bezier(int g, const double* nodes, double* Vinv) {
  double V[MAXG * MAXG], e[MAXG], col[MAXG];
  int p = g - 1;
  for (int j = 0; j < g; ++j)
    for (int k = 0; k < g; ++k) V[j * g + k] = bernstein(p, k, 0.5 * (nodes[j] + 1.0));
  for (int k = 0; k < g; ++k) {
    for (int j = 0; j < g; ++j) e[j] = (j == k) ? 1.0 : 0.0;
    gauss_solve(g, V, e, col);
    for (int j = 0; j < g; ++j) Vinv[j * g + k] = col[j];
  }
}

static void build_faces(or_ctx* c) {
  int g = c->g;
  double Vinv[MAXG * MAXG];
  lagrange_to_bezier(g, c->geo_nodes, Vinv);
  c->ctrl = (double*)malloc(sizeof(double) * (size_t)c->nelem * 6 * g * g * 3);
  c->bbox = (double*)malloc(sizeof(double) * (size_t)c->nelem * 6 * 6);
  for (int e = 0; e < c->nelem; ++e) {
    const double* X = c->xgeo + (size_t)e * g * g * g * 3;
    for (int f = 0; f < 6; ++f) {
      double* C = c->ctrl + ((size_t)e * 6 + f) * g * g * 3;
      double* bb = c->bbox + ((size_t)e * 6 + f) * 6;
      for (int km = 0; km < g; ++km)
        for (int kk = 0; kk < g; ++kk)
          for (int r = 0; r < 3; ++r) {
            double s = 0.0;
            for (int m = 0; m < g; ++m)
              for (int k = 0; k < g; ++k)
                s += Vinv[km * g + m] * Vinv[kk * g + k] * X[3 * face_node(f, g, m, k) + r];
            C[3 * (km + g * kk) + r] = s;
          }
      for (int r = 0; r < 3; ++r) {
        bb[r] = INFINITY;
        bb[3 + r] = -INFINITY;
      }
      for (int q = 0; q < g * g; ++q)
        for (int r = 0; r < 3; ++r) {
          if (C[3 * q + r] < bb[r]) bb[r] = C[3 * q + r];
          if (C[3 * q + r] > bb[3 + r]) bb[3 + r] = C[3 * q + r];
        }
    }
  }
}

void or_face_ctrl(const or_ctx* c, int e, int f, double* out) {
  int g = c->g;
  memcpy(out, c->ctrl + ((size_t)e * 6 + f) * g * g * 3, sizeof(double) * g * g * 3);
}

/* ------------------------------------------------------------------------ */
/* ray / face intersection by Bezier subdivision (Sec. 3.2.4, Eq. intersection)
 * The face is projected onto two planes that contain the ray (normals n1, n2);
 * a root of the intersection problem is a common zero of the two projected
 * scalar Bezier patches.  Sub-patches whose projected control values do not
 * straddle zero are clipped (convex-hull property); survivors are split by de
 * Casteljau at the midpoints until the control net is bilinear to rounding,
 * where the bilinear system is solved in closed form.                         */
/* ------------------------------------------------------------------------ */

typedef struct {
  double alpha, s, t;
} hit_t;

typedef struct {
  hit_t h[16];
  int n;
} hitlist;

static void add_hit(hitlist* hl, double alpha, double s, double t) {
  for (int i = 0; i < hl->n; ++i)
    if (fabs(hl->h[i].s - s) < 1e-9 && fabs(hl->h[i].t - t) < 1e-9) return;
  if (hl->n < 16) {
    hl->h[hl->n].alpha = alpha;
    hl->h[hl->n].s = s;
    hl->h[hl->n].t = t;
    hl->n++;
  }
}

/* real roots of a2 u^2 + a1 u + a0 = 0 (stable form) */
static int quad_roots(double a2, double a1, double a0, double* r, double scale) {
  if (fabs(a2) <= 1e-14 * scale) {
    if (fabs(a1) <= 1e-300) return 0;
    r[0] = -a0 / a1;
    return 1;
  }
  double disc = a1 * a1 - 4.0 * a2 * a0;
  if (disc < 0.0) return 0;
  double sq = sqrt(disc);
  double q = -0.5 * (a1 + (a1 >= 0.0 ? sq : -sq));
  if (q == 0.0) {
    r[0] = 0.0;
    return 1;
  }
  r[0] = q / a2;
  r[1] = a0 / q;
  return 2;
}

/* Solve the bilinear system f_k(u,w) = 0, k = 1,2, where f_k interpolates the
 * corner values q_k[0..3] = (00, 10, 01, 11); returns roots in (u,w). */
static int bilinear_roots(const double* q1, const double* q2, double* uu, double* ww) {
  double D1 = q1[0], B1 = q1[1] - q1[0], C1 = q1[2] - q1[0], A1 = q1[3] - q1[1] - q1[2] + q1[0];
  double D2 = q2[0], B2 = q2[1] - q2[0], C2 = q2[2] - q2[0], A2 = q2[3] - q2[1] - q2[2] + q2[0];
  double scale = fabs(A1) + fabs(B1) + fabs(C1) + fabs(D1) + fabs(A2) + fabs(B2) + fabs(C2) +
                 fabs(D2);
  if (scale == 0.0) return 0;
  int nr = 0;
  /* eliminate w: (B1 u + D1)(A2 u + C2) - (B2 u + D2)(A1 u + C1) = 0 */
  double r[2];
  int k = quad_roots(B1 * A2 - B2 * A1, B1 * C2 + D1 * A2 - B2 * C1 - D2 * A1,
                     D1 * C2 - D2 * C1, r, scale * scale);
  for (int i = 0; i < k; ++i) {
    double u = r[i];
    double den1 = A1 * u + C1, den2 = A2 * u + C2, w;
    if (fabs(den1) >= fabs(den2)) {
      if (fabs(den1) <= 1e-14 * scale) continue;
      w = -(B1 * u + D1) / den1;
    } else {
      if (fabs(den2) <= 1e-14 * scale) continue;
      w = -(B2 * u + D2) / den2;
    }
    uu[nr] = u;
    ww[nr] = w;
    nr++;
  }
  if (nr > 0) return nr;
  /* eliminate u instead: (C1 w + D1)(A2 w + B2) - (C2 w + D2)(A1 w + B1) = 0 */
  k = quad_roots(C1 * A2 - C2 * A1, C1 * B2 + D1 * A2 - C2 * B1 - D2 * A1, D1 * B2 - D2 * B1, r,
                 scale * scale);
  for (int i = 0; i < k; ++i) {
    double w = r[i];
    double den1 = A1 * w + B1, den2 = A2 * w + B2, u;
    if (fabs(den1) >= fabs(den2)) {
      if (fabs(den1) <= 1e-14 * scale) continue;
      u = -(C1 * w + D1) / den1;
    } else {
      if (fabs(den2) <= 1e-14 * scale) continue;
      u = -(C2 * w + D2) / den2;
    }
    uu[nr] = u;
    ww[nr] = w;
    nr++;
  }
  return nr;
}

typedef struct {
  int g;
  double L, band, tol;
  hitlist* out;
} subdiv_job;

static void minmax(const double* a, int n, double* lo, double* hi) {
  *lo = *hi = a[0];
  for (int i = 1; i < n; ++i) {
    if (a[i] < *lo) *lo = a[i];
    if (a[i] > *hi) *hi = a[i];
  }
}

/* de Casteljau split of a row of g values at the midpoint */
static void split_half(int g, const double* in, int stride, double* left, double* right,
                       int ostride) {
  double w[MAXG];
  for (int i = 0; i < g; ++i) w[i] = in[i * stride];
  left[0] = w[0];
  right[(g - 1) * ostride] = w[g - 1];
  for (int r = 1; r < g; ++r) {
    for (int i = 0; i < g - r; ++i) w[i] = 0.5 * (w[i] + w[i + 1]);
    left[r * ostride] = w[0];
    right[(g - 1 - r) * ostride] = w[g - 1 - r];
  }
}

/* split a g x g net (index m + g*k) in s (m) or t (k) */
static void split_net(int g, const double* P, int dir, double* Pa, double* Pb) {
  for (int j = 0; j < g; ++j) {
    if (dir == 0)
      split_half(g, P + g * j, 1, Pa + g * j, Pb + g * j, 1);
    else
      split_half(g, P + j, g, Pa + j, Pb + j, g);
  }
}

static int is_bilinear(int g, const double* P, double tol) {
  int p = g - 1;
  for (int k = 0; k < g; ++k)
    for (int m = 0; m < g; ++m) {
      double u = (double)m / p, w = (double)k / p;
      double b = (1 - u) * (1 - w) * P[0] + u * (1 - w) * P[p] + (1 - u) * w * P[g * p] +
                 u * w * P[p + g * p];
      if (fabs(P[m + g * k] - b) > tol) return 0;
    }
  return 1;
}

static void subdiv(const subdiv_job* J, const double* A, const double* D1, const double* D2,
                   double s0, double s1, double t0, double t1, int depth) {
  int g = J->g, n = g * g, p = g - 1;
  double lo, hi;
  minmax(D1, n, &lo, &hi);
  if (lo > J->tol || hi < -J->tol) return;
  minmax(D2, n, &lo, &hi);
  if (lo > J->tol || hi < -J->tol) return;
  minmax(A, n, &lo, &hi);
  if (hi < -J->band || lo > J->L + J->band) return;
  if (depth >= 60 || (is_bilinear(g, D1, J->tol) && is_bilinear(g, D2, J->tol) &&
                      is_bilinear(g, A, J->tol))) {
    double q1[4] = {D1[0], D1[p], D1[g * p], D1[p + g * p]};
    double q2[4] = {D2[0], D2[p], D2[g * p], D2[p + g * p]};
    double qa[4] = {A[0], A[p], A[g * p], A[p + g * p]};
    double uu[4], ww[4];
    int k = bilinear_roots(q1, q2, uu, ww);
    for (int i = 0; i < k; ++i) {
      double u = uu[i], w = ww[i];
      if (u < -1e-9 || u > 1 + 1e-9 || w < -1e-9 || w > 1 + 1e-9) continue;
      double alpha = (1 - u) * (1 - w) * qa[0] + u * (1 - w) * qa[1] + (1 - u) * w * qa[2] +
                     u * w * qa[3];
      double s = s0 + u * (s1 - s0), t = t0 + w * (t1 - t0);
      add_hit(J->out, alpha, 2.0 * s - 1.0, 2.0 * t - 1.0);
    }
    return;
  }
  /* split along both directions into four children */
  double Aa[MAXG * MAXG], Ab[MAXG * MAXG], D1a[MAXG * MAXG], D1b[MAXG * MAXG];
  double D2a[MAXG * MAXG], D2b[MAXG * MAXG];
  split_net(g, A, 0, Aa, Ab);
  split_net(g, D1, 0, D1a, D1b);
  split_net(g, D2, 0, D2a, D2b);
  double sm = 0.5 * (s0 + s1), tm = 0.5 * (t0 + t1);
  const double* halves[2][3] = {{Aa, D1a, D2a}, {Ab, D1b, D2b}};
  for (int hs = 0; hs < 2; ++hs) {
    double Ac[MAXG * MAXG], Ad[MAXG * MAXG], D1c[MAXG * MAXG], D1d[MAXG * MAXG];
    double D2c[MAXG * MAXG], D2d[MAXG * MAXG];
    split_net(g, halves[hs][0], 1, Ac, Ad);
    split_net(g, halves[hs][1], 1, D1c, D1d);
    split_net(g, halves[hs][2], 1, D2c, D2d);
    double sa = hs ? sm : s0, sb = hs ? s1 : sm;
    subdiv(J, Ac, D1c, D2c, sa, sb, t0, tm, depth + 1);
    subdiv(J, Ad, D1d, D2d, sa, sb, tm, t1, depth + 1);
  }
}

/* All crossings of the segment x0 -> x1 with face f of element e, each as
 * (alpha, s, t): alpha is the distance from x0 along the segment, (s,t) in
 * [-1,1]^2 the face parameters.  Crossings with alpha in [-band, L+band] are
 * reported.  Returns the number written to out[3*k]. */
static int face_hits_ray(const or_ctx* c, int e, int f, const double x0[3], const double td[3],
                         double L, double band, hitlist* hl) {
  int g = c->g;
  const double* C = c->ctrl + ((size_t)e * 6 + f) * g * g * 3;
  const double* bb = c->bbox + ((size_t)e * 6 + f) * 6;
  hl->n = 0;
  /* bounding-box rejection (Sec. 3.2.4): the segment's box against the box of
   * the control points, both widened by the band */
  for (int r = 0; r < 3; ++r) {
    double a = x0[r], b = x0[r] + L * td[r];
    double slo = (a < b ? a : b) - band - fabs(td[r]) * band;
    double shi = (a > b ? a : b) + band + fabs(td[r]) * band;
    double pad = 1e-12 * (fabs(bb[r]) + fabs(bb[3 + r]) + 1.0);
    if (shi < bb[r] - pad || slo > bb[3 + r] + pad) return 0;
  }
  /* orthonormal frame (td, n1, n2) */
  double n1[3], n2[3], ax[3] = {0, 0, 0};
  int imin = 0;
  if (fabs(td[1]) < fabs(td[imin])) imin = 1;
  if (fabs(td[2]) < fabs(td[imin])) imin = 2;
  ax[imin] = 1.0;
  cross3(td, ax, n1);
  double nn = sqrt(dot3(n1, n1));
  for (int r = 0; r < 3; ++r) n1[r] /= nn;
  cross3(td, n1, n2);
  double A[MAXG * MAXG], D1[MAXG * MAXG], D2[MAXG * MAXG], scale = 0.0;
  for (int q = 0; q < g * g; ++q) {
    double dlt[3] = {C[3 * q] - x0[0], C[3 * q + 1] - x0[1], C[3 * q + 2] - x0[2]};
    A[q] = dot3(td, dlt);
    D1[q] = dot3(n1, dlt);
    D2[q] = dot3(n2, dlt);
    double m = maxabs3(dlt);
    if (m > scale) scale = m;
  }
  subdiv_job J = {g, L, band, 1e-13 * (scale + 1e-300), hl};
  subdiv(&J, A, D1, D2, 0.0, 1.0, 0.0, 1.0, 0);
  return hl->n;
}

int or_face_hits(const or_ctx* c, int e, int f, const double x0[3], const double x1[3],
                 double band, double* out, int maxout) {
  double td[3] = {x1[0] - x0[0], x1[1] - x0[1], x1[2] - x0[2]};
  double L = sqrt(dot3(td, td));
  if (L == 0.0) return 0;
  for (int r = 0; r < 3; ++r) td[r] /= L;
  hitlist hl;
  int n = face_hits_ray(c, e, f, x0, td, L, band, &hl);
  if (n > maxout) n = maxout;
  for (int i = 0; i < n; ++i) {
    out[3 * i] = hl.h[i].alpha;
    out[3 * i + 1] = hl.h[i].s;
    out[3 * i + 2] = hl.h[i].t;
  }
  return n;
}

/* unit normal of face f at face parameters (s,t), from the tangents of the
 * element map there */
static void face_normal(const or_ctx* c, int e, int f, double s, double t, double nrm[3]) {
  double xi[3], x[3], J[9], t1[3], t2[3];
  face_to_xi(f, s, t, xi);
  or_elem_map(c, e, xi, x, J);
  int q1 = (f / 2 == 0) ? 1 : 0, q2 = (f / 2 == 2) ? 1 : 2;
  for (int r = 0; r < 3; ++r) {
    t1[r] = J[r * 3 + q1];
    t2[r] = J[r * 3 + q2];
  }
  cross3(t1, t2, nrm);
  double nn = sqrt(dot3(nrm, nrm));
  for (int r = 0; r < 3; ++r) nrm[r] /= nn;
}

/* ------------------------------------------------------------------------ */
/* tracking of one RK-stage segment (Sec. 3.2.3) with the wall model of       */
/* Sec. 2.4 and periodic / open boundaries                                   */
/* ------------------------------------------------------------------------ */

static void reflect(double* a, const double* n) {
  double s = 2.0 * dot3(a, n);
  for (int r = 0; r < 3; ++r) a[r] -= s * n[r];
}

/* 1 if local face f of element e is a wall or an open boundary: a near-face
 * event there can change the wall-hit count or the particle's fate, while one
 * on an internal or periodic face changes only the stage at which the owner
 * changes (Sec. 3.2.3 follows the same straight segment either way). */
static int is_wall_or_open(const or_ctx* c, int e, int f) {
  int b = c->bc[e * 6 + f];
  return b == 1 || b == 3;
}

/* Near-face band at a stage start (R8): max |xi_d| > 1 - band_ref sets the
 * near-face bit; when the face of such a component (2d + (xi_d > 0)) is a wall
 * or open face the near-wall bit as well. */
static uint32_t near_bits(const or_ctx* c, const or_params* p, int e, const double xi[3]) {
  uint32_t b = 0;
  for (int d = 0; d < 3; ++d) {
    if (fabs(xi[d]) > 1.0 - p->band_ref) {
      b |= OR_ST_NEAR_FACE;
      if (is_wall_or_open(c, e, 2 * d + (xi[d] > 0.0))) b |= OR_ST_NEAR_WALL;
    }
  }
  return b;
}

/* Moves the particle along x -> xe.  The ray x(alpha) = xs + alpha*td,
 * alpha in (a0, L] (Eq. parttrajectory) is tested against every face of the
 * current element except the one it came in by; the smallest accepted alpha
 * wins (lowest face index on ties).  Internal face: continue in the neighbour
 * on the same ray.  Periodic face: continue in the neighbour on the ray
 * translated by the period.  Wall: restart the ray at the hit point with the
 * remaining length and direction, velocity and RK registers mirrored by
 * I - 2 n n^T.  Open: the particle leaves (frozen at the hit point). */
static void track(const or_ctx* c, const or_params* p, int32_t* elem, double x[3],
                  const double xe_in[3], double v[3], double kx[3], double kv[3], int32_t* hits,
                  uint32_t* status) {
  double xs[3] = {x[0], x[1], x[2]}, xe[3] = {xe_in[0], xe_in[1], xe_in[2]};
  double td[3] = {xe[0] - xs[0], xe[1] - xs[1], xe[2] - xs[2]};
  double L = sqrt(dot3(td, td));
  if (L == 0.0) return;
  for (int r = 0; r < 3; ++r) td[r] /= L;
  int e = *elem, fin = -1;
  double a0 = 0.0;
  int n;
  for (n = 0; n < p->max_cross; ++n) {
    double best = INFINITY, bs = 0, bt = 0;
    int bf = -1;
    for (int f = 0; f < 6; ++f) {
      if (f == fin) continue;
      hitlist hl;
      face_hits_ray(c, e, f, xs, td, L, p->band_x, &hl);
      for (int i = 0; i < hl.n; ++i) {
        double al = hl.h[i].alpha, s = hl.h[i].s, t = hl.h[i].t;
        double m = fabs(s) > fabs(t) ? fabs(s) : fabs(t);
        if (al < a0 - p->band_x || al > L + p->band_x) continue;
        if (fabs(m - 1.0) < p->band_ref || fabs(al - a0) < p->band_x || fabs(L - al) < p->band_x) {
          *status |= OR_ST_NEAR_FACE;
          if (is_wall_or_open(c, e, f)) *status |= OR_ST_NEAR_WALL;
        }
        if (m <= 1.0 && al > a0 && al <= L && al < best) {
          best = al;
          bf = f;
          bs = s;
          bt = t;
        }
      }
    }
    if (bf < 0) break;
    int kind = c->bc[e * 6 + bf];
    if (kind == 4) {
      /* big side of a mortar (Sec. 3.2.3): the crossing is searched again on
       * the small faces matched to it; the one whose crossing lies closest to
       * the big face's (lowest index on ties) is the face the particle enters
       * by.  The ray is the same, only its entry and exit roles swap, so
       * the search needs no inversion here: face_hits_ray reports both. */
      const int32_t* mt = c->mortar + 9 * (size_t)c->nbr[e * 6 + bf];
      int ns = mt[0] == 1 ? 4 : 2, kb = -1;
      double dbest = INFINITY, ka = best, km = 0.0;
      for (int k = 0; k < ns; ++k) {
        hitlist hl;
        face_hits_ray(c, mt[1 + k], mt[5 + k], xs, td, L, p->band_x, &hl);
        for (int i = 0; i < hl.n; ++i) {
          double al = hl.h[i].alpha, s = hl.h[i].s, t = hl.h[i].t;
          double m = fabs(s) > fabs(t) ? fabs(s) : fabs(t);
          if (m > 1.0 + p->band_ref) continue;
          if (al < a0 - p->band_x || al > L + p->band_x) continue;
          if (fabs(al - best) < dbest) {
            dbest = fabs(al - best);
            kb = k;
            ka = al;
            km = m;
          }
        }
      }
      if (kb < 0) {
        /* no small face reports the crossing (a gap of rounding size at their
         * shared edges): take the small face whose part of the big face holds
         * the big face's crossing parameters */
        int is = bs > 0.0, it = bt > 0.0;
        kb = mt[0] == 1 ? is + 2 * it : (mt[0] == 2 ? is : it);
        ka = best;
        km = 1.0;
      }
      if (fabs(km - 1.0) < p->band_ref) *status |= OR_ST_NEAR_FACE;
      e = mt[1 + kb];
      fin = mt[5 + kb];
      a0 = ka;
    } else if (kind == 0 || kind == 2) {
      if (kind == 2) {
        const double* sh = c->shift + ((size_t)e * 6 + bf) * 3;
        for (int r = 0; r < 3; ++r) {
          xs[r] += sh[r];
          xe[r] += sh[r];
        }
      }
      int en = c->nbr[e * 6 + bf];
      fin = c->nbf[e * 6 + bf];
      e = en;
      a0 = best;
    } else if (kind == 1) {
      double nrm[3], xh[3];
      face_normal(c, e, bf, bs, bt, nrm);
      for (int r = 0; r < 3; ++r) xh[r] = xs[r] + best * td[r];
      double Lr = L - best;
      reflect(td, nrm);
      reflect(v, nrm);
      reflect(kx, nrm);
      reflect(kv, nrm);
      for (int r = 0; r < 3; ++r) {
        xs[r] = xh[r];
        xe[r] = xs[r] + Lr * td[r];
      }
      L = Lr;
      a0 = 0.0;
      fin = bf;
      (*hits)++;
    } else {
      for (int r = 0; r < 3; ++r) x[r] = xs[r] + best * td[r];
      *elem = e;
      *status |= OR_ST_OPEN;
      return;
    }
  }
  if (n >= p->max_cross) *status |= OR_ST_CROSS_CAP;
  *elem = e;
  for (int r = 0; r < 3; ++r) x[r] = xe[r];
}

/* ------------------------------------------------------------------------ */
/* drag (Sec. 2.2) and the 5-stage low-storage RK scheme (Sec. 3.1)           */
/* ------------------------------------------------------------------------ */

/* Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage scheme:
 * du <- A_i du + dt F(u);  u <- u + B_i du;  stage time t + C_i dt. */
void or_lserk_coeffs(double* A, double* B, double* C) {
  const double a[5] = {0.0, -567301805773.0 / 1357537059087.0,
                       -2404267990393.0 / 2016746695238.0, -3550918686646.0 / 2091501179385.0,
                       -1275806237668.0 / 842570457699.0};
  const double b[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                       1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                       2277821191437.0 / 14882151754819.0};
  const double cc[5] = {0.0, 1432997174477.0 / 9575080441755.0,
                        2526269341429.0 / 6820363962896.0, 2006345519317.0 / 3224310063776.0,
                        2802321613138.0 / 2924317926251.0};
  for (int i = 0; i < 5; ++i) {
    A[i] = a[i];
    B[i] = b[i];
    C[i] = cc[i];
  }
}

/* tau_p = d^2 rho_p / (18 mu) (Eq. stokesnumber); Re_p = rho |u - v| d / mu;
 * F_D = 3 pi mu d f_D (u - v) (Eq. dragforce) => dv/dt = f_D (u - v) / tau_p;
 * f_D = 1 (Stokes), 1 + 0.15 Re_p^0.687 (Schiller-Naumann, Eq. dragfactor) or
 * the four-parameter correlation 1 + A Re^B + (Re/24) C / (1 + D/Re) of
 * Haider & Levenspiel (1989, Powder Technol. 58), whose parameters are their
 * published fits in the sphericity phi:
 *   A = exp(2.3288 - 6.4581 phi + 2.4486 phi^2),  B = 0.0964 + 0.5565 phi,
 *   C = exp(4.905 - 13.8944 phi + 18.4222 phi^2 - 10.2599 phi^3),
 *   D = exp(1.4681 + 12.2584 phi - 20.7322 phi^2 + 15.8855 phi^3). */
double or_drag_factor(const or_params* p, double re) {
  if (p->drag_law == 0) return 1.0;
  if (p->drag_law == 1) return 1.0 + 0.15 * pow(re, 0.687);
  double f = p->sphericity;
  double A = exp(2.3288 - 6.4581 * f + 2.4486 * f * f);
  double B = 0.0964 + 0.5565 * f;
  double C = exp(4.905 - 13.8944 * f + 18.4222 * f * f - 10.2599 * f * f * f);
  double D = exp(1.4681 + 12.2584 * f - 20.7322 * f * f + 15.8855 * f * f * f);
  if (!(re > 0.0)) return 1.0;
  return 1.0 + A * pow(re, B) + re / 24.0 * C / (1.0 + D / re);
}

static double drag_factor(const or_params* p, double rho, const double rel[3], double d,
                          uint32_t* status) {
  if (p->drag_law == 0) return 1.0;
  double re = rho * sqrt(dot3(rel, rel)) * d / p->mu;
  if (p->drag_law == 1 && re >= 800.0 && status) *status |= OR_ST_REP800;
  return or_drag_factor(p, re);
}

/* Saffman lift (Sec. 2.2): F_S = 6.46/4 C_S d^2 sqrt(rho mu / |w|) (w x (v - u)),
 * w = curl u (the relative velocity in the printed cross product is read as
 * particle minus fluid: a particle lagging in a shear flow then drifts toward
 * the faster fluid, as in Saffman 1965), with Mei's correction C_S = (1 - 0.3314 sqrt(th)) exp(-Re_p/10)
 * + 0.3314 sqrt(th) for Re_p <= 40 and 0.0524 sqrt(th Re_p) above, where
 * th = d |w| / (2 |u - v|) is held within [0.005, 0.4] (the range the paper
 * states for it).  Zero when w or u - v vanishes. */
void or_saffman_force(const or_params* p, double rho, const double rel[3],
                      const double omega[3], double d, double F[3]) {
  double wn = sqrt(dot3(omega, omega)), rn = sqrt(dot3(rel, rel));
  F[0] = F[1] = F[2] = 0.0;
  if (!(wn > 0.0) || !(rn > 0.0)) return;
  double re = rho * rn * d / p->mu;
  double th = d * wn / (2.0 * rn);
  if (th < 0.005) th = 0.005;
  if (th > 0.4) th = 0.4;
  double cs = re <= 40.0 ? (1.0 - 0.3314 * sqrt(th)) * exp(-0.1 * re) + 0.3314 * sqrt(th)
                         : 0.0524 * sqrt(th * re);
  double k = 6.46 / 4.0 * cs * d * d * sqrt(rho * p->mu / wn);
  double rxw[3]; /* w x (v - u) = (u - v) x w */
  cross3(rel, omega, rxw);
  for (int r = 0; r < 3; ++r) F[r] = k * rxw[r];
}

/* Acceleration of the particle: f_D (u - v) / tau_p (+ F_S / m_p) + g; F gets
 * the fluid force on the particle, F_D (+ F_S). */
static void particle_accel(const or_ctx* c, const or_params* p, int e, const double xi[3],
                           const double vp[3], double d, uint32_t* status, double acc[3],
                           double F[3]) {
  const double pi = 3.14159265358979323846;
  double U[5], rel[3];
  or_interp(c, e, xi, U);
  for (int r = 0; r < 3; ++r) rel[r] = U[1 + r] / U[0] - vp[r];
  double tau = p->rho_p * d * d / (18.0 * p->mu);
  double mp = p->rho_p * pi * d * d * d / 6.0;
  double fD = drag_factor(p, U[0], rel, d, status);
  for (int r = 0; r < 3; ++r) {
    /* gravity on m_p - m_f with buoyancy (Eq. theory:maxey), else on m_p */
    acc[r] = p->mask[r] * fD * rel[r] / tau + p->g[r] * (p->buoyancy ? 1.0 - U[0] / p->rho_p : 1.0);
    F[r] = mp * fD * rel[r] / tau;
  }
  if (p->lift) {
    double G[9], w[3], FS[3];
    or_velocity_gradient(c, e, xi, G);
    w[0] = G[7] - G[5]; /* du_z/dy - du_y/dz */
    w[1] = G[2] - G[6]; /* du_x/dz - du_z/dx */
    w[2] = G[3] - G[1]; /* du_y/dx - du_x/dy */
    or_saffman_force(p, U[0], rel, w, d, FS);
    for (int r = 0; r < 3; ++r) {
      acc[r] += FS[r] / mp;
      F[r] += FS[r];
    }
  }
}

/* First RK stage of one particle without tracking (Sec. 3.2.1, Eq.
 * part_interpolation, Sec. 2.2, Sec. 3.1): xi of x in e by Newton, the fluid
 * state U(xi), the particle's acceleration, and the stage's increments of
 * position and velocity, B_1 k_x and B_1 k_v with k_x = dt v and k_v = dt a
 * (A_1 = 0).  out = [xi (3), U (5), a (3), dx (3), dv (3)]; returns 0 if the
 * inverse map fails. */
int or_stage1(const or_ctx* c, const or_params* p, int e, const double x[3], const double v[3],
              double d, double dt, double out[17]) {
  double A[5], B[5], C[5], xi[3], U[5], acc[3], F[3];
  int it;
  or_lserk_coeffs(A, B, C);
  if (!or_newton(c, p, e, x, xi, &it)) return 0;
  or_interp(c, e, xi, U);
  particle_accel(c, p, e, xi, v, d, NULL, acc, F);
  for (int r = 0; r < 3; ++r) out[r] = xi[r];
  for (int q = 0; q < 5; ++q) out[3 + q] = U[q];
  for (int r = 0; r < 3; ++r) {
    double kx = dt * v[r], kv = dt * acc[r]; /* registers start at 0 in a step */
    out[8 + r] = acc[r];
    out[11 + r] = B[0] * kx;
    out[14 + r] = B[0] * kv;
  }
  return 1;
}

void or_push(const or_ctx* c, const or_params* p, int64_t np, double* x, double* v,
             const double* d, int32_t* elem, int32_t* hits, uint32_t* status, int nsteps,
             double dt) {
  double A[5], B[5], C[5];
  or_lserk_coeffs(A, B, C);
  for (int64_t ip = 0; ip < np; ++ip) {
    double* xp = x + 3 * ip;
    double* vp = v + 3 * ip;
    for (int step = 0; step < nsteps && !(status[ip] & OR_ST_FROZEN); ++step) {
      double kx[3] = {0, 0, 0}, kv[3] = {0, 0, 0};
      for (int st = 0; st < 5; ++st) {
        double xi[3], acc[3], Ff[3], xe[3];
        int it;
        int e = elem[ip];
        if (!or_newton(c, p, e, xp, xi, &it)) {
          status[ip] |= OR_ST_NEWTON_FAIL;
          break;
        }
        double m = maxabs3(xi);
        if (m > 1.0 + p->lost_tol) {
          status[ip] |= OR_ST_LOST;
          break;
        }
        status[ip] |= near_bits(c, p, e, xi);
        particle_accel(c, p, e, xi, vp, d[ip], &status[ip], acc, Ff);
        for (int r = 0; r < 3; ++r) {
          kx[r] = A[st] * kx[r] + dt * vp[r];
          kv[r] = A[st] * kv[r] + dt * acc[r];
          xe[r] = xp[r] + B[st] * kx[r];
          vp[r] = vp[r] + B[st] * kv[r];
        }
        track(c, p, &elem[ip], xp, xe, vp, kx, kv, &hits[ip], &status[ip]);
        if (status[ip] & OR_ST_FROZEN) break;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* two-way coupling source (Sec. 2.3, Eq. theory:source), Lagrange weights    */
/* ------------------------------------------------------------------------ */

/* For every live particle: F = m_p f_D (u - v) / tau_p, m_p = rho_p pi d^3 / 6
 * (plus the Saffman lift when enabled).
 * Momentum source -F and energy source -F.v_p are spread over the nodes of the
 * owning element with weights l_i(xi1) l_j(xi2) l_k(xi3), so the nodal sums of
 * an element equal the particle's source (partition of unity).
 * S[nelem][4][n^3] is accumulated into (not cleared). */
void or_deposit(const or_ctx* c, const or_params* p, int64_t np, const double* x,
                const double* v, const double* d, const int32_t* elem, const uint32_t* status,
                double* S) {
  int n = c->n, n3 = n * n * n;
  for (int64_t ip = 0; ip < np; ++ip) {
    if (status[ip] & OR_ST_FROZEN) continue;
    int e = elem[ip], it;
    double xi[3], acc[3], Fp[3], F[4];
    if (!or_newton(c, p, e, x + 3 * ip, xi, &it)) continue;
    particle_accel(c, p, e, xi, v + 3 * ip, d[ip], NULL, acc, Fp);
    F[3] = 0.0;
    for (int r = 0; r < 3; ++r) {
      F[r] = -Fp[r];
      F[3] -= Fp[r] * v[3 * ip + r];
    }
    double l[3][MAXN];
    for (int dd = 0; dd < 3; ++dd)
      for (int i = 0; i < n; ++i) l[dd][i] = or_lagrange(n, c->nodes, i, xi[dd]);
    double* Se = S + (size_t)e * 4 * n3;
    for (int q = 0; q < 4; ++q)
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i)
            Se[(size_t)q * n3 + i + n * (j + n * k)] += F[q] * l[0][i] * l[1][j] * l[2][k];
  }
}

/* Quadrature weights of the solution nodes (kind 0 Gauss, 1 GLL):
 * Gauss w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2); GLL w_i = 2 / (N (N+1) P_N(x_i)^2). */
void or_quad_weights(int kind, int n, const double* x, double* w) {
  if (n == 1) {
    w[0] = 2.0;
    return;
  }
  for (int i = 0; i < n; ++i) {
    if (kind == 0) {
      double dp;
      legendre(n, x[i], &dp);
      w[i] = 2.0 / ((1.0 - x[i] * x[i]) * dp * dp);
    } else {
      int N = n - 1;
      double p = legendre(N, x[i], NULL);
      w[i] = 2.0 / (N * (N + 1.0) * p * p);
    }
  }
}

/* Nearest-DoF projection (Sec. 2.3): the whole source of a particle goes to
 * the node nearest to it, as the density a / V_ijk, V_ijk = w_i w_j w_k |det J|
 * at that node (the node's share of the element volume).  "Nearest" is taken
 * per reference direction.  S[nelem][4][n^3] is accumulated into. */
void or_deposit_nearest(const or_ctx* c, const or_params* p, int64_t np, const double* x,
                        const double* v, const double* d, const int32_t* elem,
                        const uint32_t* status, double* S) {
  int n = c->n, n3 = n * n * n;
  double w[MAXN];
  or_quad_weights(c->node_type, n, c->nodes, w);
  for (int64_t ip = 0; ip < np; ++ip) {
    if (status[ip] & OR_ST_FROZEN) continue;
    int e = elem[ip], it;
    double xi[3], acc[3], Fp[3], F[4];
    if (!or_newton(c, p, e, x + 3 * ip, xi, &it)) continue;
    particle_accel(c, p, e, xi, v + 3 * ip, d[ip], NULL, acc, Fp);
    F[3] = 0.0;
    for (int r = 0; r < 3; ++r) {
      F[r] = -Fp[r];
      F[3] -= Fp[r] * v[3 * ip + r];
    }
    int idx[3];
    for (int dd = 0; dd < 3; ++dd) {
      idx[dd] = 0;
      for (int i = 1; i < n; ++i)
        if (fabs(xi[dd] - c->nodes[i]) < fabs(xi[dd] - c->nodes[idx[dd]])) idx[dd] = i;
    }
    double xn[3] = {c->nodes[idx[0]], c->nodes[idx[1]], c->nodes[idx[2]]}, xx[3], J[9];
    or_elem_map(c, e, xn, xx, J);
    double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                 J[2] * (J[3] * J[7] - J[4] * J[6]);
    double V = w[idx[0]] * w[idx[1]] * w[idx[2]] * fabs(det);
    double* Se = S + (size_t)e * 4 * n3;
    int node = idx[0] + n * (idx[1] + n * idx[2]);
    for (int q = 0; q < 4; ++q) Se[(size_t)q * n3 + node] += F[q] / V;
  }
}

/* Two-way time-step restriction (Sec. 2.3): with f_D = 1 the source term's
 * eigenvalue is 1/tau_p; a fourth-order RK scheme allows dt <= 2.75 tau_p.
 * Returns the number of particles that violate it. */
int64_t or_dt_violations(const or_params* p, int64_t np, const double* d, double dt) {
  int64_t bad = 0;
  for (int64_t ip = 0; ip < np; ++ip) {
    double tau = p->rho_p * d[ip] * d[ip] / (18.0 * p->mu);
    if (dt > 2.75 * tau) ++bad;
  }
  return bad;
}

/* ------------------------------------------------------------------------ */
/* brute-force point location: every element whose Newton solution lies in   */
/* [-1-tol, 1+tol]^3 (Sec. 3.2.3, localisation in reference space)           */
/* ------------------------------------------------------------------------ */

int or_locate_bruteforce(const or_ctx* c, const or_params* p, const double x[3], double tol,
                         int32_t* elems, int maxout) {
  int k = 0;
  for (int e = 0; e < c->nelem; ++e) {
    double xi[3];
    int it;
    if (!or_newton(c, p, e, x, xi, &it)) continue;
    if (maxabs3(xi) <= 1.0 + tol && k < maxout) elems[k++] = e;
  }
  return k;
}

/* ------------------------------------------------------------------------ */
/* learned initial guess: features and an FP64 MLP (no counterpart in the     */
/* paper; checks the network that predicts the Newton start)                  */
/* ------------------------------------------------------------------------ */

/* Features of x in element e (NGeo = 3 only): the trilinear guess
 * xi_tri = Jc^{-1} (x - xc), with xc and Jc the value and Jacobian at xi = 0 of
 * the trilinear map through the 8 corner nodes, followed by the 48 deviations
 * (y of the node minus y of the trilinear map at that node) / h_y of the edge-
 * and face-interior geometry nodes in node-index order; h_y is the mean length
 * of the four xi2-edges measured in y. */
void or_mlp_features(const or_ctx* c, int e, const double x[3], double feat[51]) {
  int g = c->g, last = g - 1;
  const double* X = c->xgeo + (size_t)e * g * g * g * 3;
  double corner[8][3];
  for (int q = 0; q < 8; ++q) {
    int a = (q & 1) ? last : 0, b = (q & 2) ? last : 0, cc = (q & 4) ? last : 0;
    for (int r = 0; r < 3; ++r) corner[q][r] = X[3 * (a + g * (b + g * cc)) + r];
  }
  double xc[3] = {0, 0, 0}, Jc[9] = {0};
  for (int q = 0; q < 8; ++q)
    for (int r = 0; r < 3; ++r) {
      xc[r] += corner[q][r] / 8.0;
      for (int dd = 0; dd < 3; ++dd) {
        double sgn = (q & (1 << dd)) ? 1.0 : -1.0;
        Jc[r * 3 + dd] += sgn * corner[q][r] / 8.0;
      }
    }
  double rhs[3] = {x[0] - xc[0], x[1] - xc[1], x[2] - xc[2]}, xt[3];
  gauss_solve(3, Jc, rhs, xt);
  feat[0] = xt[0];
  feat[1] = xt[1];
  feat[2] = xt[2];
  double hy = 0.0;
  for (int q = 0; q < 8; ++q)
    if (q & 2) hy += fabs(corner[q][1] - corner[q & ~2][1]) / 4.0;
  int k = 3;
  for (int cc = 0; cc < g; ++cc)
    for (int b = 0; b < g; ++b)
      for (int a = 0; a < g; ++a) {
        int nb = (a == 0 || a == last) + (b == 0 || b == last) + (cc == 0 || cc == last);
        if (nb != 1 && nb != 2) continue;
        double xi[3] = {c->geo_nodes[a], c->geo_nodes[b], c->geo_nodes[cc]}, yt = 0.0;
        for (int q = 0; q < 8; ++q) {
          double w = 1.0;
          for (int dd = 0; dd < 3; ++dd)
            w *= 0.5 * (1.0 + ((q & (1 << dd)) ? 1.0 : -1.0) * xi[dd]);
          yt += w * corner[q][1];
        }
        if (k < 51) feat[k] = (X[3 * (a + g * (b + g * cc)) + 1] - yt) / hy;
        k++;
      }
  for (; k < 51; ++k) feat[k] = 0.0;
}

#define MLP_IN 51
#define MLP_H 64
#define MLP_OUT 3
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + MLP_H * MLP_IN)
#define OFF_W2 (OFF_B1 + MLP_H)
#define OFF_B2 (OFF_W2 + MLP_H * MLP_H)
#define OFF_W3 (OFF_B2 + MLP_H)
#define OFF_B3 (OFF_W3 + MLP_H * MLP_H)
#define OFF_W4 (OFF_B3 + MLP_H)
#define OFF_B4 (OFF_W4 + MLP_OUT * MLP_H)
#define MLP_NP (OFF_B4 + MLP_OUT)

int or_mlp_nparams(void) { return MLP_NP; }

/* GELU, erf form: 0.5 z (1 + erf(z / sqrt 2)) and its derivative */
static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }
static double gelu_d(double z) {
  const double pi = 3.14159265358979323846;
  return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * pi);
}

/* dense layer y = W x + b, W[nout][nin] row-major */
static void dense(const double* W, const double* b, int nout, int nin, const double* x,
                  double* y) {
  for (int o = 0; o < nout; ++o) {
    double s = b[o];
    for (int i = 0; i < nin; ++i) s += W[o * nin + i] * x[i];
    y[o] = s;
  }
}

/* 51 -> 64 -> 64 -> 64 -> 3, GELU after each hidden layer */
static void mlp_one(const double* th, const double* in, double z[3][MLP_H], double h[3][MLP_H],
                    double* out) {
  dense(th + OFF_W1, th + OFF_B1, MLP_H, MLP_IN, in, z[0]);
  for (int i = 0; i < MLP_H; ++i) h[0][i] = gelu(z[0][i]);
  dense(th + OFF_W2, th + OFF_B2, MLP_H, MLP_H, h[0], z[1]);
  for (int i = 0; i < MLP_H; ++i) h[1][i] = gelu(z[1][i]);
  dense(th + OFF_W3, th + OFF_B3, MLP_H, MLP_H, h[1], z[2]);
  for (int i = 0; i < MLP_H; ++i) h[2][i] = gelu(z[2][i]);
  dense(th + OFF_W4, th + OFF_B4, MLP_OUT, MLP_H, h[2], out);
}

void or_mlp_forward(const double* theta, int B, const double* in, double* out) {
  double z[3][MLP_H], h[3][MLP_H];
  for (int b = 0; b < B; ++b) mlp_one(theta, in + (size_t)b * MLP_IN, z, h, out + 3 * b);
}

/* loss = mean over the batch and the 3 outputs of (y - target)^2; grad is
 * overwritten with d loss / d theta (backpropagation by the chain rule). */
double or_mlp_loss_grad(const double* theta, int B, const double* in, const double* target,
                        double* grad) {
  double loss = 0.0;
  memset(grad, 0, sizeof(double) * MLP_NP);
  for (int b = 0; b < B; ++b) {
    const double* xin = in + (size_t)b * MLP_IN;
    double z[3][MLP_H], h[3][MLP_H], y[3], dy[3], dh[MLP_H], dz[MLP_H];
    mlp_one(theta, xin, z, h, y);
    for (int o = 0; o < 3; ++o) {
      double r = y[o] - target[3 * b + o];
      loss += r * r / (3.0 * B);
      dy[o] = 2.0 * r / (3.0 * B);
    }
    /* output layer */
    for (int o = 0; o < 3; ++o) {
      grad[OFF_B4 + o] += dy[o];
      for (int i = 0; i < MLP_H; ++i) grad[OFF_W4 + o * MLP_H + i] += dy[o] * h[2][i];
    }
    for (int i = 0; i < MLP_H; ++i) {
      double s = 0.0;
      for (int o = 0; o < 3; ++o) s += theta[OFF_W4 + o * MLP_H + i] * dy[o];
      dh[i] = s;
    }
    /* hidden layers 3, 2, 1 */
    const int offW[3] = {OFF_W1, OFF_W2, OFF_W3}, offB[3] = {OFF_B1, OFF_B2, OFF_B3};
    for (int l = 2; l >= 0; --l) {
      int nin = (l == 0) ? MLP_IN : MLP_H;
      const double* xl = (l == 0) ? xin : h[l - 1];
      for (int o = 0; o < MLP_H; ++o) dz[o] = dh[o] * gelu_d(z[l][o]);
      for (int o = 0; o < MLP_H; ++o) {
        grad[offB[l] + o] += dz[o];
        for (int i = 0; i < nin; ++i) grad[offW[l] + o * nin + i] += dz[o] * xl[i];
      }
      if (l > 0)
        for (int i = 0; i < MLP_H; ++i) {
          double s = 0.0;
          for (int o = 0; o < MLP_H; ++o) s += theta[offW[l] + o * MLP_H + i] * dz[o];
          dh[i] = s;
        }
    }
  }
  return loss;
}

/* Adam (Kingma & Ba 2015) with bias correction; t counts from 1 */
void or_adam(int n, double* theta, const double* g, double* m, double* v, int t, double lr,
             double b1, double b2, double eps) {
  for (int i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    double mh = m[i] / (1.0 - pow(b1, t));
    double vh = v[i] / (1.0 - pow(b2, t));
    theta[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* ------------------------------------------------------------------------ */
/* context                                                                    */
/* ------------------------------------------------------------------------ */

or_ctx* or_create(int nelem, int ngeo, const double* xgeo, const int32_t* neighbor,
                  const int32_t* nbr_face, const int32_t* bc, const double* shift) {
  if (nelem <= 0 || ngeo < 1 || ngeo + 1 > MAXG) return NULL;
  or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
  c->nelem = nelem;
  c->ngeo = ngeo;
  c->g = ngeo + 1;
  size_t nx = (size_t)nelem * c->g * c->g * c->g * 3;
  c->xgeo = (double*)malloc(sizeof(double) * nx);
  memcpy(c->xgeo, xgeo, sizeof(double) * nx);
  c->nbr = (int32_t*)malloc(sizeof(int32_t) * nelem * 6);
  c->nbf = (int32_t*)malloc(sizeof(int32_t) * nelem * 6);
  c->bc = (int32_t*)malloc(sizeof(int32_t) * nelem * 6);
  c->shift = (double*)malloc(sizeof(double) * nelem * 18);
  memcpy(c->nbr, neighbor, sizeof(int32_t) * nelem * 6);
  memcpy(c->nbf, nbr_face, sizeof(int32_t) * nelem * 6);
  memcpy(c->bc, bc, sizeof(int32_t) * nelem * 6);
  memcpy(c->shift, shift, sizeof(double) * nelem * 18);
  or_nodes(2, c->g, c->geo_nodes);
  build_faces(c);
  return c;
}

int or_set_mortars(or_ctx* c, int nmortar, const int32_t* mortar) {
  if (nmortar < 0) return 0;
  for (int m = 0; m < nmortar; ++m) {
    const int32_t* mt = mortar + 9 * (size_t)m;
    int ns = mt[0] == 1 ? 4 : 2;
    if (mt[0] < 1 || mt[0] > 3) return 0;
    for (int k = 0; k < ns; ++k)
      if (mt[1 + k] < 0 || mt[1 + k] >= c->nelem || mt[5 + k] < 0 || mt[5 + k] > 5) return 0;
  }
  free(c->mortar);
  c->mortar = (int32_t*)malloc(sizeof(int32_t) * 9 * (size_t)(nmortar > 0 ? nmortar : 1));
  if (nmortar > 0) memcpy(c->mortar, mortar, sizeof(int32_t) * 9 * (size_t)nmortar);
  c->nmortar = nmortar;
  return 1;
}

int or_set_fluid(or_ctx* c, int N, int node_type, const double* U) {
  if (N < 0 || N + 1 > MAXN || (node_type != 0 && node_type != 1)) return 0;
  c->N = N;
  c->n = N + 1;
  c->node_type = node_type;
  or_nodes(node_type, c->n, c->nodes);
  size_t nu = (size_t)c->nelem * 5 * c->n * c->n * c->n;
  free(c->U);
  c->U = (double*)malloc(sizeof(double) * nu);
  memcpy(c->U, U, sizeof(double) * nu);
  return 1;
}

void or_destroy(or_ctx* c) {
  if (!c) return;
  free(c->xgeo);
  free(c->nbr);
  free(c->nbf);
  free(c->bc);
  free(c->shift);
  free(c->mortar);
  free(c->ctrl);
  free(c->bbox);
  free(c->U);
  free(c);
}
