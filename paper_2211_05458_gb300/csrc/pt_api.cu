// pt_api.cu -- the C ABI of libpt (include/pt.h): context life cycle, mesh
// preprocessing on the host, and the launch sequences of push / locate /
// deposit.  Host-side preprocessing follows Sec. 3.2.4 of arXiv 2211.05458
// (face kind by bounding-box flatness, Bezier control points for bounds).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pt.h"
#include "pt_bin.h"
#include "pt_ctx.h"
#include "pt_internal.h"

namespace pt {
int fam_g2_fp64_push(int, const PushArgs&, int, int, void*);
int fam_g2_fp32_push(int, const PushArgs&, int, int, void*);
int fam_g3_fp64_push(int, const PushArgs&, int, int, void*);
int fam_g3_fp32_push(int, const PushArgs&, int, int, void*);
int fam_g4_fp64_push(int, const PushArgs&, int, int, void*);
int fam_g4_fp32_push(int, const PushArgs&, int, int, void*);
int fam_g5_fp64_push(int, const PushArgs&, int, int, void*);
int fam_g5_fp32_push(int, const PushArgs&, int, int, void*);
int fam_g2_fp64_dep(int, int, const DepositArgs&, int, int, void*);
int fam_g2_fp32_dep(int, int, const DepositArgs&, int, int, void*);
int fam_g3_fp64_dep(int, int, const DepositArgs&, int, int, void*);
int fam_g3_fp32_dep(int, int, const DepositArgs&, int, int, void*);
int fam_g4_fp64_dep(int, int, const DepositArgs&, int, int, void*);
int fam_g4_fp32_dep(int, int, const DepositArgs&, int, int, void*);
int fam_g5_fp64_dep(int, int, const DepositArgs&, int, int, void*);
int fam_g5_fp32_dep(int, int, const DepositArgs&, int, int, void*);
int fam_g2_fp64_occ(int, int);
int fam_g2_fp32_occ(int, int);
int fam_g3_fp64_occ(int, int);
int fam_g3_fp32_occ(int, int);
int fam_g4_fp64_occ(int, int);
int fam_g4_fp32_occ(int, int);
int fam_g5_fp64_occ(int, int);
int fam_g5_fp32_occ(int, int);
int fam_g2_fp64_loc(const LocateArgs&, int, int, void*);
int fam_g2_fp32_loc(const LocateArgs&, int, int, void*);
int fam_g3_fp64_loc(const LocateArgs&, int, int, void*);
int fam_g3_fp32_loc(const LocateArgs&, int, int, void*);
int fam_g4_fp64_loc(const LocateArgs&, int, int, void*);
int fam_g4_fp32_loc(const LocateArgs&, int, int, void*);
int fam_g5_fp64_loc(const LocateArgs&, int, int, void*);
int fam_g5_fp32_loc(const LocateArgs&, int, int, void*);
int fam_g2_fp64_terms(int, const TermsArgs&, int, int, void*);
int fam_g2_fp32_terms(int, const TermsArgs&, int, int, void*);
int fam_g3_fp64_terms(int, const TermsArgs&, int, int, void*);
int fam_g3_fp32_terms(int, const TermsArgs&, int, int, void*);
int fam_g4_fp64_terms(int, const TermsArgs&, int, int, void*);
int fam_g4_fp32_terms(int, const TermsArgs&, int, int, void*);
int fam_g5_fp64_terms(int, const TermsArgs&, int, int, void*);
int fam_g5_fp32_terms(int, const TermsArgs&, int, int, void*);
int fam_g2_fp64_staged(int, int, const StageArgs&, const DevParticles&, const int*, int, int, void*);
int fam_g2_fp64_occs(int, int);
int fam_g2_fp32_staged(int, int, const StageArgs&, const DevParticles&, const int*, int, int, void*);
int fam_g2_fp32_occs(int, int);
int fam_g3_fp64_staged(int, int, const StageArgs&, const DevParticles&, const int*, int, int, void*);
int fam_g3_fp64_occs(int, int);
int fam_g3_fp32_staged(int, int, const StageArgs&, const DevParticles&, const int*, int, int, void*);
int fam_g3_fp32_occs(int, int);
int fam_g4_fp64_staged(int, int, const StageArgs&, const DevParticles&, const int*, int, int, void*);
int fam_g4_fp64_occs(int, int);
int fam_g4_fp32_staged(int, int, const StageArgs&, const DevParticles&, const int*, int, int, void*);
int fam_g4_fp32_occs(int, int);
int fam_g5_fp64_staged(int, int, const StageArgs&, const DevParticles&, const int*, int, int, void*);
int fam_g5_fp64_occs(int, int);
int fam_g5_fp32_staged(int, int, const StageArgs&, const DevParticles&, const int*, int, int, void*);
int fam_g5_fp32_occs(int, int);
int fam_g2_fp64_find(const FindArgs&, int, int, void*);
int fam_g2_fp32_find(const FindArgs&, int, int, void*);
int fam_g3_fp64_find(const FindArgs&, int, int, void*);
int fam_g3_fp32_find(const FindArgs&, int, int, void*);
int fam_g4_fp64_find(const FindArgs&, int, int, void*);
int fam_g4_fp32_find(const FindArgs&, int, int, void*);
int fam_g5_fp64_find(const FindArgs&, int, int, void*);
int fam_g5_fp32_find(const FindArgs&, int, int, void*);

#define PT_DISPATCH(g, f64, SUFFIX, ...)                                          \
  ((g) == 2 ? ((f64) ? fam_g2_fp64_##SUFFIX(__VA_ARGS__) : fam_g2_fp32_##SUFFIX(__VA_ARGS__)) \
   : (g) == 3 ? ((f64) ? fam_g3_fp64_##SUFFIX(__VA_ARGS__) : fam_g3_fp32_##SUFFIX(__VA_ARGS__)) \
   : (g) == 4 ? ((f64) ? fam_g4_fp64_##SUFFIX(__VA_ARGS__) : fam_g4_fp32_##SUFFIX(__VA_ARGS__)) \
   : ((f64) ? fam_g5_fp64_##SUFFIX(__VA_ARGS__) : fam_g5_fp32_##SUFFIX(__VA_ARGS__)))

int launch_push(int g, bool f64, int np, const PushArgs& a, int grid, int block, void* s) {
  return PT_DISPATCH(g, f64, push, np, a, grid, block, s);
}
int launch_deposit(int g, bool f64, int np, int mode, const DepositArgs& a, int grid, int block,
                   void* s) {
  return PT_DISPATCH(g, f64, dep, np, mode, a, grid, block, s);
}
int max_active_push(int g, bool f64, int np, int block) {
  return PT_DISPATCH(g, f64, occ, np, block);
}
int launch_find(int g, bool f64, const FindArgs& a, int grid, int block, void* s) {
  return PT_DISPATCH(g, f64, find, a, grid, block, s);
}
int launch_staged(int g, bool f64, int np, int op, const StageArgs& a, const DevParticles& p,
                  const int* perm, int grid, int block, void* s) {
  return PT_DISPATCH(g, f64, staged, np, op, a, p, perm, grid, block, s);
}
int max_active_stage(int g, bool f64, int np, int block) {
  return PT_DISPATCH(g, f64, occs, np, block);
}
int launch_terms(int g, bool f64, int np, const TermsArgs& a, int grid, int block, void* s) {
  return PT_DISPATCH(g, f64, terms, np, a, grid, block, s);
}
int launch_locate(int g, bool f64, int np, const LocateArgs& a, int grid, int block, void* s) {
  (void)np;
  return PT_DISPATCH(g, f64, loc, a, grid, block, s);
}
}  // namespace pt

using namespace pt;

static thread_local std::string g_init_err = "no error";

static pt_status fail(pt_ctx* c, pt_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    g_init_err = buf;
  return st;
}

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(c, PT_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                  __FILE__, __LINE__);                                               \
  } while (0)

// ---------------------------------------------------------------------------
// node sets (host): Legendre-Gauss, Gauss-Lobatto, equidistant; barycentric weights
// ---------------------------------------------------------------------------

// P_n and P_n' at x by the three-term recurrence
static void legendre_pd(int n, double x, double* p, double* dp) {
  double a = 1.0, b = x, da = 0.0, db = 1.0;
  if (n == 0) {
    *p = 1.0;
    *dp = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
    double dc = da + (2 * k - 1) * b;  // P_k' = P_{k-2}' + (2k-1) P_{k-1}
    a = b;
    b = c;
    da = db;
    db = dc;
  }
  *p = b;
  *dp = db;
}

static void solution_nodes(int kind, int n, double* x) {
  if (n == 1) {
    x[0] = 0.0;
    return;
  }
  const double pi = 3.14159265358979323846;
  if (kind == 0) {
    for (int i = 0; i < n; ++i) {
      double z = -std::cos(pi * (4 * i + 3) / (4 * n + 2));
      for (int it = 0; it < 60; ++it) {
        double p, dp;
        legendre_pd(n, z, &p, &dp);
        double dz = p / dp;
        z -= dz;
        if (std::fabs(dz) <= 1e-17) break;
      }
      x[i] = z;
    }
  } else {
    // Gauss-Lobatto: endpoints and the zeros of P_{n-1}' (Newton with the
    // second derivative from Legendre's differential equation)
    int N = n - 1;
    x[0] = -1.0;
    x[N] = 1.0;
    for (int i = 1; i < N; ++i) {
      double z = -std::cos(pi * i / N);
      for (int it = 0; it < 60; ++it) {
        double p, dp;
        legendre_pd(N, z, &p, &dp);
        double d2 = (2 * z * dp - N * (N + 1) * p) / (1 - z * z);
        double dz = dp / d2;
        z -= dz;
        if (std::fabs(dz) <= 1e-17) break;
      }
      x[i] = z;
    }
  }
  std::sort(x, x + n);
}

static void bary(int n, const double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double p = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != i) p *= (x[i] - x[m]);
    w[i] = 1.0 / p;
  }
}

// Quadrature weights of a node set: the w with sum_i w_i P_k(x_i) = int P_k =
// 2 delta_k0 for k < n (exact for every polynomial of degree < n, hence
// w_i = int l_i), solved by Gaussian elimination with partial pivoting.
static void quad_weights(int n, const double* x, double* w) {
  double M[PT_MAXN][PT_MAXN + 1];
  for (int k = 0; k < n; ++k) {
    for (int i = 0; i < n; ++i) {
      double p, dp;
      legendre_pd(k, x[i], &p, &dp);
      M[k][i] = p;
    }
    M[k][n] = k == 0 ? 2.0 : 0.0;
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(M[r][col]) > std::fabs(M[piv][col])) piv = r;
    for (int q = 0; q <= n; ++q) std::swap(M[col][q], M[piv][q]);
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = M[r][col] / M[col][col];
      for (int q = col; q <= n; ++q) M[r][q] -= f * M[col][q];
    }
  }
  for (int i = 0; i < n; ++i) w[i] = M[i][n] / M[i][i];
}

// 5-stage 4th-order 2N-storage Runge-Kutta (Carpenter & Kennedy, NASA TM-109112)
static const double kRK_A[5] = {0.0, -567301805773.0 / 1357537059087.0,
                                -2404267990393.0 / 2016746695238.0,
                                -3550918686646.0 / 2091501179385.0,
                                -1275806237668.0 / 842570457699.0};
static const double kRK_B[5] = {1432997174477.0 / 9575080441755.0,
                                5161836677717.0 / 13612068292357.0,
                                1720146321549.0 / 2090206949498.0,
                                3134564353537.0 / 4481467310338.0,
                                2277821191437.0 / 14882151754819.0};

// ---------------------------------------------------------------------------
// mesh preprocessing
// ---------------------------------------------------------------------------

static int face_node_h(int g, int f, int mm, int kk) {
  int fixed = (f & 1) ? g - 1 : 0;
  switch (f >> 1) {
    case 0: return fixed + g * (mm + g * kk);
    case 1: return mm + g * (fixed + g * kk);
    default: return mm + g * (kk + g * fixed);
  }
}

// inverse of the Bernstein-Vandermonde matrix on equidistant nodes:
// Bezier control values = M * nodal values
static void bezier_matrix(int g, std::vector<double>& M) {
  int p = g - 1;
  std::vector<double> V(g * g), I(g * g, 0.0);
  for (int j = 0; j < g; ++j) {
    double u = p ? (double)j / p : 0.0;
    for (int k = 0; k < g; ++k) {
      double bin = 1.0;
      for (int q = 1; q <= k; ++q) bin = bin * (p - k + q) / q;
      V[j * g + k] = bin * std::pow(u, k) * std::pow(1.0 - u, p - k);
    }
    I[j * g + j] = 1.0;
  }
  // Gauss-Jordan
  for (int c = 0; c < g; ++c) {
    int piv = c;
    for (int r = c + 1; r < g; ++r)
      if (std::fabs(V[r * g + c]) > std::fabs(V[piv * g + c])) piv = r;
    for (int q = 0; q < g; ++q) {
      std::swap(V[c * g + q], V[piv * g + q]);
      std::swap(I[c * g + q], I[piv * g + q]);
    }
    double d = V[c * g + c];
    for (int q = 0; q < g; ++q) {
      V[c * g + q] /= d;
      I[c * g + q] /= d;
    }
    for (int r = 0; r < g; ++r)
      if (r != c) {
        double f = V[r * g + c];
        for (int q = 0; q < g; ++q) {
          V[r * g + q] -= f * V[c * g + q];
          I[r * g + q] -= f * I[c * g + q];
        }
      }
  }
  M = I;
}

static bool inv3h(const double* J, double* Ji) {
  double c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8],
         c02 = J[3] * J[7] - J[4] * J[6];
  double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
  if (!(std::fabs(det) > 0)) return false;
  double id = 1.0 / det;
  Ji[0] = c00 * id;
  Ji[1] = (J[2] * J[7] - J[1] * J[8]) * id;
  Ji[2] = (J[1] * J[5] - J[2] * J[4]) * id;
  Ji[3] = c01 * id;
  Ji[4] = (J[0] * J[8] - J[2] * J[6]) * id;
  Ji[5] = (J[2] * J[3] - J[0] * J[5]) * id;
  Ji[6] = c02 * id;
  Ji[7] = (J[1] * J[6] - J[0] * J[7]) * id;
  Ji[8] = (J[0] * J[4] - J[1] * J[3]) * id;
  return true;
}

template <typename T>
static T* dmalloc(pt_ctx* c, size_t n, cudaError_t* err) {
  void* p = nullptr;
  *err = cudaMalloc(&p, n * sizeof(T) + 16);
  if (*err == cudaSuccess) c->allocs.push_back(p);
  return (T*)p;
}

static pt_status upload_mesh(pt_ctx* c, const pt_mesh_desc* md) {
  const int E = md->nelem, g = md->ngeo + 1, g3 = g * g * g;
  c->nelem = E;
  c->ngeo = md->ngeo;
  c->g = g;
  std::vector<double> xg64((size_t)E * g3 * 3), ce((size_t)E * 3), bil((size_t)E * 72),
      shift((size_t)E * 18);
  std::vector<float> xg32((size_t)E * g3 * 3), xg32lo((size_t)E * g3 * 3), tri((size_t)E * 12), slab((size_t)E * 48, 0.f);
  std::vector<int> fnbr((size_t)E * 6), finfo((size_t)E * 6), tmask((size_t)E, 0);
  std::vector<double> M;
  bezier_matrix(g, M);
  const double bx = c->cfg.band_x;
  const int nmort = md->nmortar;
  if (nmort < 0 || (nmort > 0 && md->mortar == nullptr))
    return fail(nullptr, PT_ERR_ARG, "bad mortar table (%d rows)", nmort);
  std::vector<int> big_of((size_t)nmort, -1);
  int ncurved = 0;
  for (int e = 0; e < E; ++e) {
    const double* X = md->xgeo + (size_t)e * g3 * 3;
    double cr[8][3], cc[3] = {0, 0, 0};
    for (int q = 0; q < 8; ++q) {
      int a = (q & 1) ? g - 1 : 0, b = (q & 2) ? g - 1 : 0, cz = (q & 4) ? g - 1 : 0;
      for (int r = 0; r < 3; ++r) {
        cr[q][r] = X[3 * (a + g * (b + g * cz)) + r];
        cc[r] += cr[q][r] / 8.0;
      }
    }
    double Rmax = 0.0;
    for (int q = 0; q < g3; ++q)
      for (int r = 0; r < 3; ++r) {
        double v = X[3 * q + r] - cc[r];
        xg64[((size_t)e * g3 + q) * 3 + r] = v;
        const float vh = (float)v;
        xg32[(size_t)e * 3 * g3 + r * g3 + q] = vh;
        xg32lo[(size_t)e * 3 * g3 + r * g3 + q] = (float)(v - (double)vh);
        Rmax = std::max(Rmax, std::fabs(v));
      }
    for (int r = 0; r < 3; ++r) ce[3 * e + r] = cc[r];
    // trilinear start table
    double Jc[9] = {0}, Ji[9];
    for (int q = 0; q < 8; ++q)
      for (int r = 0; r < 3; ++r)
        for (int d = 0; d < 3; ++d) Jc[3 * r + d] += ((q >> d) & 1 ? 1.0 : -1.0) * cr[q][r] / 8.0;
    if (!inv3h(Jc, Ji))
      return fail(nullptr, PT_ERR_ARG, "element %d: degenerate corner Jacobian", e);
    // coordinates that equal the trilinear interpolant of the corners at every
    // node (to 1e-14 of the element radius) use the 8-corner form on the GPU
    for (int r = 0; r < 3; ++r) {
      double dev = 0.0;
      for (int cz = 0; cz < g; ++cz)
        for (int b = 0; b < g; ++b)
          for (int a = 0; a < g; ++a) {
            double xi[3] = {-1.0 + 2.0 * a / (g - 1), -1.0 + 2.0 * b / (g - 1),
                            -1.0 + 2.0 * cz / (g - 1)};
            double t = 0.0;
            for (int q = 0; q < 8; ++q) {
              double w = 1.0;
              for (int d = 0; d < 3; ++d) w *= 0.5 * (1.0 + (((q >> d) & 1) ? xi[d] : -xi[d]));
              t += w * (cr[q][r] - cc[r]);
            }
            dev = std::max(dev, std::fabs(xg64[((size_t)e * g3 + a + g * (b + g * cz)) * 3 + r] - t));
          }
      if (dev <= 1e-14 * Rmax) tmask[e] |= 1 << r;
    }
    for (int r = 0; r < 3; ++r) tri[12 * e + r] = 0.f;
    for (int q = 0; q < 9; ++q) tri[12 * e + 3 + q] = (float)Ji[q];
    // faces
    for (int f = 0; f < 6; ++f) {
      const int k6 = 6 * e + f;
      int bc = md->bc[k6];
      int nb = md->neighbor[k6], nf = md->nbr_face[k6];
      if (bc < 0 || bc > 4) return fail(nullptr, PT_ERR_ARG, "element %d face %d: bad bc %d", e, f, bc);
      if (bc == PT_BC_INTERNAL || bc == PT_BC_PERIODIC) {
        if (nb < 0 || nb >= E || nf < 0 || nf > 5)
          return fail(nullptr, PT_ERR_ARG, "element %d face %d: bad neighbour %d/%d", e, f, nb, nf);
        if (md->bc[6 * nb + nf] == PT_BC_MORTAR) {
          // small side of a mortar: the big face's row must list this face
          const int row = md->neighbor[6 * nb + nf];
          bool listed = false;
          if (bc == PT_BC_INTERNAL && row >= 0 && row < nmort)
            for (int q = 0; q < 4; ++q)
              listed |= md->mortar[9 * (size_t)row + 1 + q] == e &&
                        md->mortar[9 * (size_t)row + 5 + q] == f;
          if (!listed)
            return fail(nullptr, PT_ERR_ARG,
                        "element %d face %d: not a small face of the mortar of element %d", e, f,
                        nb);
        } else if (md->neighbor[6 * nb + nf] != e || md->nbr_face[6 * nb + nf] != f) {
          return fail(nullptr, PT_ERR_ARG, "element %d face %d: neighbour %d does not point back", e,
                      f, nb);
        }
      } else if (bc == PT_BC_MORTAR) {
        if (nb < 0 || nb >= nmort)
          return fail(nullptr, PT_ERR_ARG, "element %d face %d: bad mortar row %d", e, f, nb);
        if (big_of[nb] >= 0)
          return fail(nullptr, PT_ERR_ARG, "mortar row %d referenced twice", nb);
        big_of[nb] = k6;
        nf = 0;
      } else {
        nb = -1;
        nf = 0;
      }
      for (int r = 0; r < 3; ++r) {
        double sv = md->shift[18 * e + 3 * f + r];
        if (bc != PT_BC_PERIODIC && sv != 0.0)
          return fail(nullptr, PT_ERR_ARG, "element %d face %d: shift on a non-periodic face", e, f);
        shift[18 * e + 3 * f + r] = bc == PT_BC_PERIODIC ? sv : 0.0;
      }
      // face nodes (local coords)
      std::vector<double> P(g * g * 3);
      for (int kk = 0; kk < g; ++kk)
        for (int mm = 0; mm < g; ++mm)
          for (int r = 0; r < 3; ++r)
            P[3 * (mm + g * kk) + r] =
                xg64[((size_t)e * g3 + face_node_h(g, f, mm, kk)) * 3 + r];
      const double* P00 = &P[0];
      const double* P10 = &P[3 * (g - 1)];
      const double* P01 = &P[3 * g * (g - 1)];
      const double* P11 = &P[3 * (g - 1 + g * (g - 1))];
      double* Bf = &bil[72 * (size_t)e + 12 * f];
      for (int r = 0; r < 3; ++r) {
        Bf[r] = 0.25 * (P00[r] - P10[r] - P01[r] + P11[r]);
        Bf[3 + r] = 0.25 * (-P00[r] + P10[r] - P01[r] + P11[r]);
        Bf[6 + r] = 0.25 * (-P00[r] - P10[r] + P01[r] + P11[r]);
        Bf[9 + r] = 0.25 * (P00[r] + P10[r] + P01[r] + P11[r]);
      }
      // kind: bilinear if every face node lies on the bilinear patch
      double dev = 0.0, amax = 0.0;
      for (int kk = 0; kk < g; ++kk)
        for (int mm = 0; mm < g; ++mm) {
          double s = g > 1 ? -1.0 + 2.0 * mm / (g - 1) : 0.0;
          double t = g > 1 ? -1.0 + 2.0 * kk / (g - 1) : 0.0;
          for (int r = 0; r < 3; ++r) {
            double b = Bf[r] * s * t + Bf[3 + r] * s + Bf[6 + r] * t + Bf[9 + r];
            dev = std::max(dev, std::fabs(P[3 * (mm + g * kk) + r] - b));
          }
        }
      for (int r = 0; r < 3; ++r) amax = std::max(amax, std::fabs(Bf[r]));
      int kind = dev <= 1e-13 * Rmax ? (amax <= 1e-13 * Rmax ? PT_FACE_PLANAR : PT_FACE_BILINEAR)
                                     : PT_FACE_CURVED;
      ncurved += kind == PT_FACE_CURVED;
      fnbr[k6] = nb;
      finfo[k6] = bc | (kind << 3) | (nf << 5);
      // slab: centre normal b x c rounded to FP32, range over the Bezier
      // control points (their convex hull contains the face), widened
      double nrm[3] = {Bf[4] * Bf[8] - Bf[5] * Bf[7], Bf[5] * Bf[6] - Bf[3] * Bf[8],
                       Bf[3] * Bf[7] - Bf[4] * Bf[6]};
      double nn = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
      if (!(nn > 0)) return fail(nullptr, PT_ERR_ARG, "element %d face %d: degenerate face", e, f);
      float nf32[3];
      for (int r = 0; r < 3; ++r) {
        nf32[r] = (float)(nrm[r] / nn);
        nrm[r] = nf32[r];
      }
      double lo = 1e300, hi = -1e300;
      for (int km = 0; km < g; ++km)
        for (int kt = 0; kt < g; ++kt) {
          double cp[3] = {0, 0, 0};
          for (int mm = 0; mm < g; ++mm)
            for (int kk = 0; kk < g; ++kk)
              for (int r = 0; r < 3; ++r)
                cp[r] += M[km * g + mm] * M[kt * g + kk] * P[3 * (mm + g * kk) + r];
          double pr = nrm[0] * cp[0] + nrm[1] * cp[1] + nrm[2] * cp[2];
          lo = std::min(lo, pr);
          hi = std::max(hi, pr);
        }
      double margin = bx + 4e-6 * Rmax + 1e-12;
      // bound on the distance between the face and its bilinear patch: the
      // Bezier control points of their difference enclose it
      double devmax = 0.0;
      if (kind == PT_FACE_CURVED) {
        for (int km = 0; km < g; ++km)
          for (int kt = 0; kt < g; ++kt) {
            double cp[3] = {0, 0, 0};
            for (int mm = 0; mm < g; ++mm)
              for (int kk = 0; kk < g; ++kk) {
                double s = -1.0 + 2.0 * mm / (g - 1), t = -1.0 + 2.0 * kk / (g - 1);
                for (int r = 0; r < 3; ++r) {
                  double bl = Bf[r] * s * t + Bf[3 + r] * s + Bf[6 + r] * t + Bf[9 + r];
                  cp[r] += M[km * g + mm] * M[kt * g + kk] * (P[3 * (mm + g * kk) + r] - bl);
                }
              }
            devmax = std::max(devmax, std::sqrt(cp[0] * cp[0] + cp[1] * cp[1] + cp[2] * cp[2]));
          }
      }
      float* S = &slab[48 * (size_t)e + 8 * f];
      S[0] = nf32[0];
      S[1] = nf32[1];
      S[2] = nf32[2];
      S[3] = (float)(lo - margin);
      S[4] = (float)(hi + margin);
      S[5] = (float)Rmax;
      S[6] = (float)(devmax * (1.0 + 1e-6) + 1e-12 * Rmax);
      // faces that reference-space localisation must still track physically
      S[7] = (bc == PT_BC_WALL || bc == PT_BC_OPEN) ? 1.f : 0.f;
    }
  }
  c->ncurved = ncurved;
  // mortar rows: every listed small face points back at the big face
  for (int r = 0; r < nmort; ++r) {
    const int32_t* mt = md->mortar + 9 * (size_t)r;
    if (big_of[r] < 0) return fail(nullptr, PT_ERR_ARG, "mortar row %d: no big face", r);
    if (mt[0] < PT_MORTAR_FOUR || mt[0] > PT_MORTAR_T)
      return fail(nullptr, PT_ERR_ARG, "mortar row %d: bad type %d", r, mt[0]);
    const int ns = mt[0] == PT_MORTAR_FOUR ? 4 : 2;
    for (int q = 0; q < 4; ++q) {
      const int es = mt[1 + q], fs = mt[5 + q];
      if (q >= ns) {
        if (es != -1 || fs != -1)
          return fail(nullptr, PT_ERR_ARG, "mortar row %d: entry %d must be unused", r, q);
        continue;
      }
      if (es < 0 || es >= E || fs < 0 || fs > 5)
        return fail(nullptr, PT_ERR_ARG, "mortar row %d: bad small face %d/%d", r, es, fs);
      const int ks = 6 * es + fs;
      if (md->bc[ks] != PT_BC_INTERNAL || 6 * md->neighbor[ks] + md->nbr_face[ks] != big_of[r])
        return fail(nullptr, PT_ERR_ARG, "mortar row %d: small face %d/%d does not point back", r,
                    es, fs);
    }
  }
  std::vector<int> mort((size_t)std::max(nmort, 1) * 9, -1);
  if (nmort > 0) std::memcpy(mort.data(), md->mortar, sizeof(int) * 9 * (size_t)nmort);
  cudaError_t err;
  pt_ctx* cc = c;
  c->d_xg64 = dmalloc<double>(cc, xg64.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->d_xg32 = dmalloc<float>(cc, xg32.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->d_xg32lo = dmalloc<float>(cc, xg32lo.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->d_ce = dmalloc<double>(cc, ce.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->d_tri = dmalloc<float>(cc, tri.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->d_tmask = dmalloc<int>(cc, tmask.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->d_fnbr = dmalloc<int>(cc, fnbr.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->d_finfo = dmalloc<int>(cc, finfo.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->d_slab = dmalloc<float>(cc, slab.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->d_bil = dmalloc<double>(cc, bil.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  std::vector<float> bil32(bil.size());
  for (size_t i = 0; i < bil.size(); ++i) bil32[i] = (float)bil[i];
  c->d_bil32 = dmalloc<float>(cc, bil32.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->d_shift = dmalloc<double>(cc, shift.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->d_mort = dmalloc<int>(cc, mort.size(), &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  c->nmortar = nmort;
  c->d_stats = dmalloc<unsigned long long>(cc, PT_C_COUNT, &err);
  if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
  struct {
    void* d;
    const void* h;
    size_t b;
  } cp[] = {{c->d_xg64, xg64.data(), xg64.size() * 8}, {c->d_xg32, xg32.data(), xg32.size() * 4},
            {c->d_xg32lo, xg32lo.data(), xg32lo.size() * 4},
            {c->d_ce, ce.data(), ce.size() * 8},       {c->d_tri, tri.data(), tri.size() * 4},
            {c->d_tmask, tmask.data(), tmask.size() * 4},
            {c->d_fnbr, fnbr.data(), fnbr.size() * 4}, {c->d_finfo, finfo.data(), finfo.size() * 4},
            {c->d_slab, slab.data(), slab.size() * 4}, {c->d_bil, bil.data(), bil.size() * 8},
            {c->d_bil32, bil32.data(), bil32.size() * 4},
            {c->d_shift, shift.data(), shift.size() * 8},
            {c->d_mort, mort.data(), mort.size() * 4}};
  for (auto& q : cp) {
    err = cudaMemcpy(q.d, q.h, q.b, cudaMemcpyHostToDevice);
    if (err) return fail(nullptr, PT_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(err));
  }
  return PT_OK;
}

static void fill_consts(const pt_ctx* c, DevConsts& k) {
  std::memset(&k, 0, sizeof k);
  double gn[PT_MAXG], gw[PT_MAXG];
  for (int a = 0; a < c->g; ++a) gn[a] = c->g > 1 ? -1.0 + 2.0 * a / (c->g - 1) : 0.0;
  bary(c->g, gn, gw);
  {
    std::vector<double> M;
    bezier_matrix(c->g, M);
    for (int q = 0; q < c->g * c->g; ++q) k.gbz[q] = M[q];
  }
  for (int a = 0; a < c->g; ++a) {
    k.gn[a] = gn[a];
    k.gw[a] = gw[a];
    k.gn32[a] = (float)gn[a];
    k.gw32[a] = (float)gw[a];
    k.gn_hi[a] = (float)gn[a];
    k.gn_lo[a] = (float)(gn[a] - (double)k.gn_hi[a]);
    k.gw_hi[a] = (float)gw[a];
    k.gw_lo[a] = (float)(gw[a] - (double)k.gw_hi[a]);
  }
  for (int i = 0; i < c->N + 1 && c->N >= 0; ++i) {
    k.sn[i] = c->sn[i];
    k.sw[i] = c->sw[i];
    k.sn32[i] = (float)c->sn[i];
    k.sw32[i] = (float)c->sw[i];
    k.sq[i] = c->sq[i];
  }
  for (int i = 0; i < 5; ++i) {
    k.A[i] = kRK_A[i];
    k.B[i] = kRK_B[i];
    k.A32[i] = (float)kRK_A[i];
    k.B32[i] = (float)kRK_B[i];
  }
  k.mu = c->cfg.mu;
  k.rho_p = c->cfg.rho_p;
  for (int r = 0; r < 3; ++r) {
    k.g[r] = c->cfg.g[r];
    k.mask[r] = c->cfg.drag_mask[r];
  }
  k.newton_tol = c->cfg.newton_tol;
  k.band_ref = c->cfg.band_ref;
  k.band_x = c->cfg.band_x;
  k.lost_tol = c->cfg.lost_tol;
  k.drag_law = c->cfg.drag_law;
  k.lift = c->cfg.lift;
  k.track = c->cfg.track;
  k.buoyancy = c->cfg.buoyancy;
  k.curved_clip = c->cfg.curved_faces;
  {
    // Haider & Levenspiel (1989) fits in the sphericity
    const double f = c->cfg.sphericity;
    k.hl[0] = std::exp(2.3288 - 6.4581 * f + 2.4486 * f * f);
    k.hl[1] = 0.0964 + 0.5565 * f;
    k.hl[2] = std::exp(4.905 - 13.8944 * f + 18.4222 * f * f - 10.2599 * f * f * f);
    k.hl[3] = std::exp(1.4681 + 12.2584 * f - 20.7322 * f * f + 15.8855 * f * f * f);
  }
  k.max_newton = c->cfg.max_newton;
  k.max_cross = c->cfg.max_cross;
  k.guess = c->cfg.guess;
}

static DevMesh dev_mesh(const pt_ctx* c) {
  DevMesh m;
  m.nelem = c->nelem;
  m.g = c->g;
  m.xg64 = c->d_xg64;
  m.xg32 = c->d_xg32;
  m.xg32lo = c->d_xg32lo;
  m.ce = c->d_ce;
  m.tri = c->d_tri;
  m.tmask = c->d_tmask;
  m.fnbr = c->d_fnbr;
  m.finfo = c->d_finfo;
  m.slab = c->d_slab;
  m.bil = c->d_bil;
  m.bil32 = c->d_bil32;
  m.shift = c->d_shift;
  m.mort = c->d_mort;
  m.mlp_pre = c->d_mlp_pre;
  return m;
}

DevMLP pt_dev_mlp(const pt_ctx* c);
void pt_fill_consts(const pt_ctx* c, DevConsts& k) { fill_consts(c, k); }
DevMesh pt_dev_mesh(const pt_ctx* c) { return dev_mesh(c); }

static pt_status check_config(const pt_config* cfg) {
  if (!cfg) return fail(nullptr, PT_ERR_ARG, "config is NULL");
  if (cfg->precision != PT_FP64 && cfg->precision != PT_FP32)
    return fail(nullptr, PT_ERR_ARG, "precision must be PT_FP64 or PT_FP32");
  if (cfg->drag_law < 0 || cfg->drag_law > 2) return fail(nullptr, PT_ERR_ARG, "bad drag_law");
  if (cfg->drag_law == PT_DRAG_HAIDER_LEVENSPIEL &&
      !(cfg->sphericity > 0.0 && cfg->sphericity <= 1.0))
    return fail(nullptr, PT_ERR_ARG, "sphericity must be in (0, 1]");
  if (cfg->lift != 0 && cfg->lift != 1) return fail(nullptr, PT_ERR_ARG, "lift must be 0 or 1");
  if (cfg->curved_faces != 0 && cfg->curved_faces != 1)
    return fail(nullptr, PT_ERR_ARG, "curved_faces must be 0 or 1");
  if (cfg->schedule < PT_SCHEDULE_AUTO || cfg->schedule > PT_SCHEDULE_STAGED)
    return fail(nullptr, PT_ERR_ARG, "schedule must be a pt_schedule value");
  if (cfg->buoyancy != 0 && cfg->buoyancy != 1)
    return fail(nullptr, PT_ERR_ARG, "buoyancy must be 0 or 1");
  if (cfg->track != PT_TRACK_PHYSICAL && cfg->track != PT_TRACK_REFERENCE)
    return fail(nullptr, PT_ERR_ARG, "track must be PT_TRACK_PHYSICAL or PT_TRACK_REFERENCE");
  if (cfg->guess != 0 && cfg->guess != 1) return fail(nullptr, PT_ERR_ARG, "bad guess");
  if (!(cfg->mu > 0) || !(cfg->rho_p > 0)) return fail(nullptr, PT_ERR_ARG, "mu, rho_p must be > 0");
  if (cfg->max_newton < 1 || cfg->max_cross < 1) return fail(nullptr, PT_ERR_ARG, "caps must be >= 1");
  if (!(cfg->newton_tol > 0) || !(cfg->band_ref >= 0) || !(cfg->band_x >= 0) ||
      !(cfg->lost_tol >= 0))
    return fail(nullptr, PT_ERR_ARG, "bad tolerance");
  if (cfg->block < 0 || cfg->block > 128 || (cfg->block % 32))
    return fail(nullptr, PT_ERR_ARG, "block must be a multiple of 32 in [0, 128]");
  if (cfg->rebin_every < 0) return fail(nullptr, PT_ERR_ARG, "rebin_every must be >= 0");
  return PT_OK;
}

extern "C" {

void pt_config_default(pt_config* cfg) {
  std::memset(cfg, 0, sizeof *cfg);
  cfg->mu = 1e-5;
  cfg->rho_p = 1000.0;
  cfg->drag_mask[0] = cfg->drag_mask[1] = cfg->drag_mask[2] = 1.0;
  cfg->newton_tol = 1e-12;
  cfg->band_ref = 1e-10;
  cfg->band_x = 1e-10;
  cfg->lost_tol = 1e-6;
  cfg->precision = PT_FP64;
  cfg->drag_law = PT_DRAG_STOKES;
  cfg->guess = PT_GUESS_TRILINEAR;
  cfg->max_newton = 50;
  cfg->max_cross = 64;
  cfg->rebin_every = 0;
  cfg->block = 0;
  cfg->lift = 0;
  cfg->sphericity = 1.0;
}

pt_status pt_init_mesh(pt_ctx** out, const pt_mesh_desc* md, const pt_config* cfg, void* stream) {
  if (!out) return fail(nullptr, PT_ERR_ARG, "ctx out-pointer is NULL");
  *out = nullptr;
  if (!md || !md->xgeo || !md->neighbor || !md->nbr_face || !md->bc || !md->shift)
    return fail(nullptr, PT_ERR_ARG, "mesh descriptor or one of its arrays is NULL");
  if (md->nelem <= 0) return fail(nullptr, PT_ERR_ARG, "nelem must be > 0");
  if (md->ngeo < 1 || md->ngeo > 4) return fail(nullptr, PT_ERR_ARG, "ngeo must be 1..4");
  if (md->nelem > (1 << 28)) return fail(nullptr, PT_ERR_ARG, "nelem too large");
  pt_status s = check_config(cfg);
  if (s) return s;
  pt_ctx* c = new pt_ctx();
  c->cfg = *cfg;
  c->stream = (cudaStream_t)stream;
  cudaGetDevice(&c->dev);
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev);
  s = upload_mesh(c, md);
  if (s) {
    pt_destroy(c);
    return s;
  }
  *out = c;
  return PT_OK;
}

pt_status pt_set_config(pt_ctx* c, const pt_config* cfg) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  pt_status s = check_config(cfg);
  if (s) {
    c->err = g_init_err;
    return s;
  }
  if (cfg->band_x != c->cfg.band_x)
    return fail(c, PT_ERR_ARG, "band_x is fixed at init (it sizes the face slabs)");
  c->cfg = *cfg;
  return PT_OK;
}

pt_status pt_set_fluid(pt_ctx* c, int32_t N, int32_t node_type, const void* U) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  if (N < 1 || N > 7) return fail(c, PT_ERR_ARG, "N must be 1..7");
  if (node_type != 0 && node_type != 1) return fail(c, PT_ERR_ARG, "node_type must be 0 or 1");
  if (!U) return fail(c, PT_ERR_ARG, "U is NULL");
  if (reinterpret_cast<uintptr_t>(U) % 16 != 0)
    return fail(c, PT_ERR_ARG, "U must be 16-byte aligned (vector loads)");
  c->N = N;
  c->node_type = node_type;
  c->U = U;
  solution_nodes(node_type, N + 1, c->sn);
  bary(N + 1, c->sn, c->sw);
  quad_weights(N + 1, c->sn, c->sq);
  return PT_OK;
}

}  // extern "C"

// scratch for binning + permutation, grown on demand
static pt_status ensure_scratch(pt_ctx* c, int64_t n) {
  size_t need = bin_scratch_ints(c->nelem);
  if (c->scratch_ints < need) {
    if (c->d_scratch) cudaFree(c->d_scratch);
    c->d_scratch = nullptr;
    CK(cudaMalloc(&c->d_scratch, need * sizeof(int)));
    c->scratch_ints = need;
  }
  if (c->perm_cap < n) {
    if (c->d_perm) cudaFree(c->d_perm);
    c->d_perm = nullptr;
    CK(cudaMalloc(&c->d_perm, std::max<int64_t>(n, 1) * sizeof(int)));
    c->perm_cap = n;
  }
  return PT_OK;
}

static int push_block(pt_ctx* c) { return c->cfg.block > 0 ? c->cfg.block : 128; }
// the push kernel is compiled for blocks of at most 128 threads

static int grid_for(pt_ctx* c, int64_t n, int block, int occ) {
  int64_t want = (n + block - 1) / block;
  int64_t cap = (int64_t)c->nsm * std::max(occ, 1);
  return (int)std::max<int64_t>(1, std::min(want, cap));
}

__global__ void k_status_counts(const unsigned* st, int64_t n, unsigned long long* stats) {
  unsigned long long a[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned s = st[i];
    a[0] += (s & PT_ST_NEAR_FACE) != 0;
    a[1] += (s & PT_ST_NEWTON_FAIL) != 0;
    a[2] += (s & PT_ST_LOST) != 0;
    a[3] += (s & PT_ST_CROSS_CAP) != 0;
    a[4] += (s & PT_ST_OPEN) != 0;
    a[5] += (s & PT_ST_REP800) != 0;
    a[6] += (s & PT_ST_NEAR_WALL) != 0;
  }
  for (int q = 0; q < 7; ++q) {
    unsigned long long v = a[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v)
      atomicAdd(stats + (q < 6 ? PT_C_NEAR + q : PT_C_NEARWALL), v);
  }
}

template <typename R>
__global__ void k_dt_check(const R* d, int64_t n, double lim, double rho_p, double mu,
                           unsigned long long* stats) {
  unsigned long long a = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double dd = (double)d[i];
    double tau = rho_p * dd * dd / (18.0 * mu);
    a += lim > 2.75 * tau;
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0 && a) atomicAdd(stats + PT_C_DTWARN, a);
}

static pt_status validate_particles(pt_ctx* c, const pt_particles* p) {
  if (!p) return fail(c, PT_ERR_ARG, "particles is NULL");
  if (p->n < 0 || p->n > (int64_t)INT32_MAX) return fail(c, PT_ERR_ARG, "bad particle count");
  if (p->n > 0 && (!p->x || !p->v || !p->d || !p->elem || !p->hits || !p->status))
    return fail(c, PT_ERR_ARG, "a particle array is NULL");
  return PT_OK;
}

pt_status pt_validate_particles(pt_ctx* c, const pt_particles* p) {
  return validate_particles(c, p);
}

static pt_status read_stats(pt_ctx* c, const pt_particles* p, double dt, pt_stats* out) {
  const int64_t n = p->n;
  if (n > 0) {
    int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->nsm * 8);
    k_status_counts<<<g, 256, 0, c->stream>>>(p->status, n, c->d_stats);
    if (c->cfg.precision == PT_FP64)
      k_dt_check<double><<<g, 256, 0, c->stream>>>((const double*)p->d, n, dt, c->cfg.rho_p,
                                                   c->cfg.mu, c->d_stats);
    else
      k_dt_check<float><<<g, 256, 0, c->stream>>>((const float*)p->d, n, dt, c->cfg.rho_p,
                                                  c->cfg.mu, c->d_stats);
  }
  unsigned long long h[PT_C_COUNT];
  CK(cudaMemcpyAsync(h, c->d_stats, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::memset(out, 0, sizeof *out);
  out->particle_steps = (int64_t)h[PT_C_STEPS];
  out->crossings = (int64_t)h[PT_C_CROSS];
  out->wall_hits = (int64_t)h[PT_C_HITS];
  out->newton_it_fp32 = (int64_t)h[PT_C_IT32];
  out->newton_it_fp64 = (int64_t)h[PT_C_IT64];
  out->slow_track = (int64_t)h[PT_C_SLOW];
  out->near_face = (int64_t)h[PT_C_NEAR];
  out->newton_fail = (int64_t)h[PT_C_NFAIL];
  out->lost = (int64_t)h[PT_C_LOST];
  out->cross_cap = (int64_t)h[PT_C_CCAP];
  out->open = (int64_t)h[PT_C_OPEN];
  out->rep800 = (int64_t)h[PT_C_REP];
  out->dt_warn = (int64_t)h[PT_C_DTWARN];
  out->near_wall = (int64_t)h[PT_C_NEARWALL];
  if (h[PT_C_TIMEOUT])
    return fail(c, PT_ERR_TIMEOUT, "%llu tensor-core waits gave up", (unsigned long long)h[PT_C_TIMEOUT]);
  if (out->newton_fail) return fail(c, PT_ERR_NEWTON, "%lld particles failed the inverse map",
                                    (long long)out->newton_fail);
  if (out->lost) return fail(c, PT_ERR_LOST, "%lld particles lost", (long long)out->lost);
  if (out->cross_cap)
    return fail(c, PT_ERR_CROSS, "%lld particles hit the crossing cap", (long long)out->cross_cap);
  if (out->dt_warn) return PT_WARN_DT;
  return PT_OK;
}

static cudaEvent_t take_event(pt_ctx* c, int kind = 0) {
  cudaEvent_t e = nullptr;
  if (!c->ev_free.empty()) {
    e = c->ev_free.back();
    c->ev_free.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    return nullptr;
  }
  c->ev_used[kind].push_back(e);
  return e;
}

// particles from which PT_SCHEDULE_AUTO takes the staged schedule
static const int64_t kStagedMin = (int64_t)1 << 18;

static bool use_staged(const pt_ctx* c, int64_t n) {
  if (c->cfg.schedule == PT_SCHEDULE_STAGED) return true;
  if (c->cfg.schedule == PT_SCHEDULE_RESIDENT) return false;
  return n >= kStagedMin;
}

// Carves the staged schedule's state buffers for n particles out of one
// allocation (grown on demand).
static pt_status stage_args(pt_ctx* c, int64_t n, StageArgs& a) {
  const bool f64 = c->cfg.precision == PT_FP64;
  const size_t rs = f64 ? 8 : 4;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  size_t bytes = 0;
  if (f64) bytes += al(24 * nn);                      // x
  else bytes += 2 * al(12 * nn);                      // xh, xl
  bytes += 3 * al(3 * rs * nn) + al(rs * nn);         // v, kx, kv, d
  bytes += al((f64 ? 24 : 24) * nn);                  // xe
  bytes += f64 ? 0 : al(12 * nn) + 2 * al(12 * nn);   // guess, converged xi (hi, lo)
  bytes += 4 * al(4 * nn) + 256;                      // e, hits, st, list, counters
  if (c->state_cap < n || !c->d_state) {
    if (c->d_state) cudaFree(c->d_state);
    c->d_state = nullptr;
    c->state_cap = 0;
    CK(cudaMalloc(&c->d_state, bytes));
    c->state_cap = n;
  }
  char* b = (char*)c->d_state;
  auto take = [&](size_t sz) {
    char* q = b;
    b += al(sz);
    return (void*)q;
  };
  a.x = nullptr;
  a.xh = a.xl = nullptr;
  a.guess = nullptr;
  a.xih = a.xil = nullptr;
  if (f64) {
    a.x = (double*)take(24 * nn);
  } else {
    a.xh = (float*)take(12 * nn);
    a.xl = (float*)take(12 * nn);
  }
  a.v = take(3 * rs * nn);
  a.kx = take(3 * rs * nn);
  a.kv = take(3 * rs * nn);
  a.d = take(rs * nn);
  a.xe = take(24 * nn);
  if (!f64) {
    a.guess = (float*)take(12 * nn);
    a.xih = (float*)take(12 * nn);
    a.xil = (float*)take(12 * nn);
  }
  a.e = (int*)take(4 * nn);
  a.hits = (int*)take(4 * nn);
  a.st = (unsigned*)take(4 * nn);
  a.list = (unsigned*)take(4 * nn);
  a.count = (unsigned*)b;
  a.count_next = a.count + 1;
  return PT_OK;
}

// The staged schedule: per chunk of rebin_every steps, binning, the sorted
// copy of the particle state, per RK stage (the learned start,) the stage
// kernel and the exact-tracking kernel over its list, and the copy back.
// Launch shapes of the staged schedule for n particles.
struct StagedLaunch {
  bool f64 = false, mlp = false;
  int np = 0, grid = 1, block = 128, gmove = 1, gtrack = 1, gguess = 1;
  DevParticles dp{};
  unsigned* ctr = nullptr;  // two list counters, used by alternate stages
};

static pt_status staged_prepare(pt_ctx* c, const pt_particles* p, double dt, StageArgs& a,
                                StagedLaunch& L) {
  const int64_t n = p->n;
  L.f64 = c->cfg.precision == PT_FP64;
  L.mlp = !L.f64 && c->cfg.guess == PT_GUESS_MLP;
  L.np = c->N + 1;
  pt_status s = stage_args(c, n, a);
  if (s) return s;
  a.m = dev_mesh(c);
  fill_consts(c, a.k);
  a.mlp = pt_dev_mlp(c);
  a.U = c->U;
  a.n = n;
  a.dt = dt;
  a.stats = c->d_stats;
  L.dp = {n, p->x, p->v, p->d, p->elem, p->hits, p->status};
  const int occ = max_active_stage(c->g, L.f64, L.np, L.block);
  L.grid = grid_for(c, n, L.block, occ);
  L.gmove = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->nsm * 8));
  L.gtrack = c->nsm * 4;
  L.gguess = (int)std::max<int64_t>(1, std::min<int64_t>((n + 127) / 128, (int64_t)c->nsm * 4));
  L.ctr = a.count;
  return PT_OK;
}

// binning and the sorted copy of the caller's particles
static int staged_begin(pt_ctx* c, const pt_particles* p, StageArgs& a, const StagedLaunch& L) {
  int rc = bin_by_element(p->elem, p->n, c->nelem, c->d_scratch, c->d_perm, nullptr, c->nsm,
                          c->stream);
  c->launches += 5;
  if (!rc) rc = launch_staged(c->g, L.f64, L.np, PT_SOP_GATHER, a, L.dp, c->d_perm, L.gmove, 256,
                              c->stream);
  c->launches += 1;
  return rc;
}

// RK stage st (k: running stage count, which selects the list counter)
static int staged_stage(pt_ctx* c, StageArgs& a, const StagedLaunch& L, int st, int k) {
  a.stage = st;
  a.count = L.ctr + (k & 1);
  a.count_next = L.ctr + ((k + 1) & 1);
  // each kernel between an event pair of its kind when profiling
  auto timed = [&](int kind, int op, int g, int b) {
    cudaEvent_t q0 = c->profile ? take_event(c, kind) : nullptr;
    cudaEvent_t q1 = c->profile ? take_event(c, kind) : nullptr;
    if (q0) cudaEventRecord(q0, c->stream);
    const int r = launch_staged(c->g, L.f64, L.np, op, a, L.dp, c->d_perm, g, b, c->stream);
    if (q1) cudaEventRecord(q1, c->stream);
    c->launches += 1;
    return r;
  };
  int rc = 0;
  if (L.mlp) rc = timed(2, PT_SOP_GUESS, L.gguess, 128);
  if (!rc) rc = timed(1, PT_SOP_STAGE, L.grid, L.block);
  if (!rc) rc = timed(3, PT_SOP_TRACK, L.gtrack, 128);
  return rc;
}

static int staged_end(pt_ctx* c, StageArgs& a, const StagedLaunch& L) {
  c->launches += 1;
  return launch_staged(c->g, L.f64, L.np, PT_SOP_SCATTER, a, L.dp, c->d_perm, L.gmove, 256,
                       c->stream);
}

// The staged schedule: per chunk of rebin_every steps, binning, the sorted
// copy of the particle state, per RK stage (the learned start,) the stage
// kernel and the exact-tracking kernel over its list, and the copy back.
static pt_status push_staged(pt_ctx* c, const pt_particles* p, int32_t nsteps, double dt) {
  StageArgs a;
  StagedLaunch L;
  pt_status s = staged_prepare(c, p, dt, a, L);
  if (s) return s;
  CK(cudaMemsetAsync(L.ctr, 0, 2 * sizeof(unsigned), c->stream));
  const int chunk = c->cfg.rebin_every > 0 ? c->cfg.rebin_every : 10;
  int k = 0;
  for (int s0 = 0; s0 < nsteps; s0 += chunk) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profile) {
      e0 = take_event(c);
      e1 = take_event(c);
    }
    if (e0) cudaEventRecord(e0, c->stream);
    int rc = staged_begin(c, p, a, L);
    const int ns = std::min(chunk, nsteps - s0);
    for (int step = 0; step < ns && !rc; ++step)
      for (int st = 0; st < 5 && !rc; ++st, ++k) rc = staged_stage(c, a, L, st, k);
    if (!rc) rc = staged_end(c, a, L);
    if (e1) cudaEventRecord(e1, c->stream);
    if (rc) return fail(c, PT_ERR_CUDA, "staged push launch: %s",
                        cudaGetErrorString((cudaError_t)rc));
  }
  return PT_OK;
}

pt_status pt_push_impl(pt_ctx* c, const pt_particles* p, int32_t nsteps, double dt,
                       pt_stats* out) {
  const int64_t n = p->n;
  CK(cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * PT_C_COUNT, c->stream));
  if (n > 0 && nsteps > 0 && use_staged(c, n)) {
    pt_status s = ensure_scratch(c, n);
    if (s) return s;
    s = push_staged(c, p, nsteps, dt);
    if (s) return s;
  } else if (n > 0 && nsteps > 0) {
    pt_status s = ensure_scratch(c, n);
    if (s) return s;
    const bool f64 = c->cfg.precision == PT_FP64;
    const int np = c->N + 1;
    const int block = push_block(c);
    int occ = max_active_push(c->g, f64, np, block);
    int grid = grid_for(c, n, block, occ);
    PushArgs a;
    a.m = dev_mesh(c);
    fill_consts(c, a.k);
    a.p = {n, p->x, p->v, p->d, p->elem, p->hits, p->status};
    a.mlp = pt_dev_mlp(c);
    a.U = c->U;
    a.dt = dt;
    a.stats = c->d_stats;
    const int chunk = c->cfg.rebin_every > 0 ? c->cfg.rebin_every : 10;
    for (int s0 = 0; s0 < nsteps; s0 += chunk) {
      int rc = bin_by_element(p->elem, n, c->nelem, c->d_scratch, c->d_perm, nullptr, c->nsm,
                              c->stream);
      if (rc) return fail(c, PT_ERR_CUDA, "binning: %s", cudaGetErrorString((cudaError_t)rc));
      c->launches += 5;  // histogram, three scan kernels, scatter
      a.perm = c->d_perm;
      a.nsteps = std::min(chunk, nsteps - s0);
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (c->profile) {
        e0 = take_event(c);
        e1 = take_event(c);
        if (e0) cudaEventRecord(e0, c->stream);
      }
      rc = launch_push(c->g, f64, np, a, grid, block, c->stream);
      c->launches += 1;
      if (e1) cudaEventRecord(e1, c->stream);
      if (rc) return fail(c, PT_ERR_CUDA, "push launch: %s", cudaGetErrorString((cudaError_t)rc));
    }
  }
  if (out) return read_stats(c, p, dt, out);
  return PT_OK;
}

extern "C" {

pt_status pt_push(pt_ctx* c, const pt_particles* p, int32_t nsteps, double dt, pt_stats* out) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  if (c->N < 0 || !c->U) return fail(c, PT_ERR_STATE, "pt_set_fluid was not called");
  pt_status s = validate_particles(c, p);
  if (s) return s;
  if (nsteps < 0) return fail(c, PT_ERR_ARG, "nsteps must be >= 0");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(c, PT_ERR_ARG, "dt must be finite and > 0");
  if (c->cfg.guess == PT_GUESS_MLP && (c->g != 4 || !c->mlp_ready))
    return fail(c, PT_ERR_STATE, "learned guess needs ngeo = 3 and a trained network");
  if (c->cfg.guess == PT_GUESS_MLP && push_block(c) > 128)
    return fail(c, PT_ERR_ARG, "the learned guess needs a push block of at most 128 threads");
  if (c->stage_next != 0)
    return fail(c, PT_ERR_STATE, "a pt_push_stage sequence is open (stage %d expected)",
                c->stage_next);
  return pt_push_impl(c, p, nsteps, dt, out);
}

pt_status pt_push_stage(pt_ctx* c, const pt_particles* p, int32_t stage, double dt,
                        pt_stats* out) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  if (c->N < 0 || !c->U) return fail(c, PT_ERR_STATE, "pt_set_fluid was not called");
  pt_status s = validate_particles(c, p);
  if (s) return s;
  if (!(dt > 0) || !std::isfinite(dt)) return fail(c, PT_ERR_ARG, "dt must be finite and > 0");
  if (stage < 0 || stage > 4) return fail(c, PT_ERR_ARG, "stage must be 0..4");
  if (stage != c->stage_next)
    return fail(c, PT_ERR_STATE, "pt_push_stage: stage %d expected, %d given", c->stage_next, stage);
  if (stage > 0 && (std::memcmp(&c->stage_p, p, sizeof *p) != 0 || dt != c->stage_dt))
    return fail(c, PT_ERR_ARG, "pt_push_stage: the particles and dt of stage 0 are required");
  if (c->cfg.guess == PT_GUESS_MLP && (c->g != 4 || !c->mlp_ready))
    return fail(c, PT_ERR_STATE, "learned guess needs ngeo = 3 and a trained network");
  const int64_t n = p->n;
  StageArgs a;
  StagedLaunch L;
  if (stage == 0) {
    CK(cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * PT_C_COUNT, c->stream));
    s = ensure_scratch(c, std::max<int64_t>(n, 1));
    if (s) return s;
  }
  s = staged_prepare(c, p, dt, a, L);
  if (s) return s;
  int rc = 0;
  if (n > 0) {
    if (stage == 0) {
      CK(cudaMemsetAsync(L.ctr, 0, 2 * sizeof(unsigned), c->stream));
      rc = staged_begin(c, p, a, L);
    }
    if (!rc) rc = staged_stage(c, a, L, stage, stage);
    if (!rc && stage == 4) rc = staged_end(c, a, L);
    if (rc) {
      c->stage_next = 0;
      return fail(c, PT_ERR_CUDA, "pt_push_stage launch: %s", cudaGetErrorString((cudaError_t)rc));
    }
  }
  c->stage_p = *p;
  c->stage_dt = dt;
  c->stage_next = (stage + 1) % 5;
  if (stage == 4 && out) return read_stats(c, p, dt, out);
  return PT_OK;
}

pt_status pt_push_host(pt_ctx* c, const pt_particles* h, int32_t nsteps, double dt,
                       pt_stats* out) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  pt_status s = validate_particles(c, h);
  if (s) return s;
  const int64_t n = h->n;
  const size_t rs = c->cfg.precision == PT_FP64 ? 8 : 4;
  const size_t bytes = n * (24 + 3 * rs + rs + 12);
  if (c->stage_bytes < bytes) {
    if (c->d_stage) cudaFree(c->d_stage);
    c->d_stage = nullptr;
    CK(cudaMalloc(&c->d_stage, std::max<size_t>(bytes, 64) + 256));
    c->stage_bytes = bytes;
  }
  char* b = (char*)c->d_stage;
  pt_particles d;
  d.n = n;
  d.x = (double*)b;
  b += 24 * n;
  d.v = b;
  b += 3 * rs * n;
  d.d = b;
  b += rs * n;
  d.elem = (int32_t*)b;
  b += 4 * n;
  d.hits = (int32_t*)b;
  b += 4 * n;
  d.status = (uint32_t*)b;
  cudaStream_t st = c->stream;
  CK(cudaMemcpyAsync(d.x, h->x, 24 * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.v, h->v, 3 * rs * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync((void*)d.d, h->d, rs * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.elem, h->elem, 4 * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.hits, h->hits, 4 * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.status, h->status, 4 * n, cudaMemcpyHostToDevice, st));
  pt_stats tmp;
  s = pt_push(c, &d, nsteps, dt, out ? &tmp : nullptr);
  if (s && s != PT_WARN_DT && s != PT_ERR_NEWTON && s != PT_ERR_LOST && s != PT_ERR_CROSS)
    return s;
  CK(cudaMemcpyAsync(h->x, d.x, 24 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->v, d.v, 3 * rs * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->elem, d.elem, 4 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->hits, d.hits, 4 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->status, d.status, 4 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (out) *out = tmp;
  return s;
}

pt_status pt_locate(pt_ctx* c, int64_t n, const double* x, const int32_t* elem, double* xi,
                    int32_t* iters, uint32_t* status) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  if (n < 0) return fail(c, PT_ERR_ARG, "n must be >= 0");
  if (n > 0 && (!x || !elem || !xi)) return fail(c, PT_ERR_ARG, "NULL array");
  if (c->cfg.guess == PT_GUESS_MLP && (c->g != 4 || !c->mlp_ready))
    return fail(c, PT_ERR_STATE, "learned guess needs ngeo = 3 and a trained network");
  if (n == 0) return PT_OK;
  LocateArgs a;
  a.m = dev_mesh(c);
  fill_consts(c, a.k);
  a.mlp = pt_dev_mlp(c);
  a.n = n;
  a.x = x;
  a.elem = elem;
  a.xi = xi;
  a.iters = iters;
  a.status = status;
  int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)c->nsm * 16);
  int rc = launch_locate(c->g, c->cfg.precision == PT_FP64, 0, a, grid, 128, c->stream);
  if (rc) return fail(c, PT_ERR_CUDA, "locate launch: %s", cudaGetErrorString((cudaError_t)rc));
  return PT_OK;
}

pt_status pt_mlp_start(pt_ctx* c, int64_t n, const double* x, const int32_t* elem, float* guess,
                       int32_t engine) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  if (n < 0 || (n > 0 && (!x || !elem || !guess))) return fail(c, PT_ERR_ARG, "bad arrays");
  if (engine != 0 && engine != 1) return fail(c, PT_ERR_ARG, "engine must be 0 or 1");
  if (c->g != 4 || !c->mlp_ready || c->cfg.precision != PT_FP32)
    return fail(c, PT_ERR_STATE, "learned start needs ngeo = 3, PT_FP32 and a trained network");
  if (n == 0) return PT_OK;
  StageArgs a;
  std::memset(&a, 0, sizeof a);
  a.m = dev_mesh(c);
  fill_consts(c, a.k);
  a.mlp = pt_dev_mlp(c);
  a.n = n;
  a.x = const_cast<double*>(x);
  a.e = const_cast<int*>(elem);
  a.st = nullptr;
  a.guess = guess;
  a.stats = c->d_stats;
  CK(cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * PT_C_COUNT, c->stream));
  const DevParticles dp = {0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 127) / 128, (int64_t)c->nsm * 4));
  const int rc = launch_staged(c->g, false, c->N + 1, engine ? PT_SOP_GUESS_X_TC : PT_SOP_GUESS_X_WARP,
                               a, dp, nullptr, grid, 128, c->stream);
  if (rc) return fail(c, PT_ERR_CUDA, "learned start launch: %s", cudaGetErrorString((cudaError_t)rc));
  unsigned long long h[PT_C_COUNT];
  CK(cudaMemcpyAsync(h, c->d_stats, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (h[PT_C_TIMEOUT]) return fail(c, PT_ERR_TIMEOUT, "tensor-core wait gave up");
  return PT_OK;
}

pt_status pt_stage_terms(pt_ctx* c, const pt_particles* p, double dt, double* xi, void* U,
                         void* acc, void* dx, void* dv) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  if (c->N < 0 || !c->U) return fail(c, PT_ERR_STATE, "pt_set_fluid was not called");
  pt_status s = validate_particles(c, p);
  if (s) return s;
  const int64_t n = p->n;
  if (n > 0 && (!xi || !U || !acc || !dx || !dv)) return fail(c, PT_ERR_ARG, "NULL output");
  if (n == 0) return PT_OK;
  TermsArgs a;
  a.m = dev_mesh(c);
  fill_consts(c, a.k);
  a.p = {n, p->x, p->v, p->d, p->elem, p->hits, p->status};
  a.U = c->U;
  a.dt = dt;
  a.xi = xi;
  a.Uo = U;
  a.acc = acc;
  a.dx = dx;
  a.dv = dv;
  const int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)c->nsm * 16);
  const int rc = launch_terms(c->g, c->cfg.precision == PT_FP64, c->N + 1, a, grid, 128,
                              c->stream);
  if (rc) return fail(c, PT_ERR_CUDA, "terms launch: %s", cudaGetErrorString((cudaError_t)rc));
  return PT_OK;
}

pt_status pt_deposit(pt_ctx* c, const pt_particles* p, int32_t mode, float* S) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  if (c->N < 0 || !c->U) return fail(c, PT_ERR_STATE, "pt_set_fluid was not called");
  pt_status s = validate_particles(c, p);
  if (s) return s;
  if (mode & ~(PT_DEPOSIT_SEGMENTED | PT_DEPOSIT_NEAREST))
    return fail(c, PT_ERR_ARG,
                "mode must be PT_DEPOSIT_ATOMIC or PT_DEPOSIT_SEGMENTED, optionally | "
                "PT_DEPOSIT_NEAREST");
  if (!S) return fail(c, PT_ERR_ARG, "S is NULL");
  if (c->stage_next != 0)
    return fail(c, PT_ERR_STATE, "a pt_push_stage sequence is open (stage %d expected)",
                c->stage_next);
  const int np = c->N + 1;
  const size_t n3 = (size_t)np * np * np;
  const int64_t n = p->n;
  s = ensure_scratch(c, n);
  if (s) return s;
  int* offs = nullptr;
  int rc = bin_by_element(p->elem, n, c->nelem, c->d_scratch, c->d_perm, &offs, c->nsm, c->stream);
  if (rc) return fail(c, PT_ERR_CUDA, "binning: %s", cudaGetErrorString((cudaError_t)rc));
  DepositArgs a;
  a.m = dev_mesh(c);
  fill_consts(c, a.k);
  a.p = {n, p->x, p->v, p->d, p->elem, p->hits, p->status};
  a.U = c->U;
  a.perm = c->d_perm;
  a.offs = offs;
  a.S = S;
  a.src = nullptr;
  const bool f64 = c->cfg.precision == PT_FP64;
  if (mode & PT_DEPOSIT_SEGMENTED) {
    // two passes: the sources of all particles, then the per-element sums,
    // each element's particles in index order
    if (c->src_cap < n) {
      if (c->d_src) cudaFree(c->d_src);
      if (c->d_perm2) cudaFree(c->d_perm2);
      c->d_src = nullptr;
      c->d_perm2 = nullptr;
      c->src_cap = 0;
      CK(cudaMalloc(&c->d_src, sizeof(float4) * 2 * std::max<int64_t>(n, 1)));
      CK(cudaMalloc(&c->d_perm2, sizeof(int) * std::max<int64_t>(n, 1)));
      c->src_cap = n;
    }
    a.src = c->d_src;
    rc = sort_segments(c->d_perm, offs, c->nelem, c->d_perm2, c->nsm, c->stream);
    if (rc) return fail(c, PT_ERR_CUDA, "segment sort: %s", cudaGetErrorString((cudaError_t)rc));
    a.perm = c->d_perm2;
  }
  if (!(mode & PT_DEPOSIT_SEGMENTED)) {
    CK(cudaMemsetAsync(S, 0, sizeof(float) * 4 * n3 * c->nelem, c->stream));
    if (n == 0) return PT_OK;
    int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)c->nsm * 16);
    rc = launch_deposit(c->g, f64, np, mode, a, grid, 128, c->stream);
  } else {
    int grid = std::min(c->nelem, c->nsm * 32);
    rc = launch_deposit(c->g, f64, np, mode | 4, a, grid, 256, c->stream);
  }
  if (rc) return fail(c, PT_ERR_CUDA, "deposit launch: %s", cudaGetErrorString((cudaError_t)rc));
  return PT_OK;
}

// Background grid of pt_find_element: every element is listed in the cells its
// control box meets.  The box of an element is the box of the Bezier control
// points of its map (the element lies in their convex hull).  The cell size
// starts at the mean element size and shrinks until no cell lists more than
// PT_FIND_MAXC elements.
static pt_status build_find_grid(pt_ctx* c) {
  const int E = c->nelem, g = c->g, g3 = g * g * g;
  std::vector<double> xg((size_t)E * g3 * 3), ce((size_t)E * 3);
  CK(cudaMemcpy(xg.data(), c->d_xg64, xg.size() * 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(ce.data(), c->d_ce, ce.size() * 8, cudaMemcpyDeviceToHost));
  std::vector<double> M;
  bezier_matrix(g, M);
  std::vector<double> box((size_t)E * 6);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  std::vector<double> t1(g3), t2(g3);
  for (int e = 0; e < E; ++e) {
    double* b = &box[6 * (size_t)e];
    for (int r = 0; r < 3; ++r) {
      b[r] = 1e300;
      b[3 + r] = -1e300;
      // control values of coordinate r: M applied along each direction
      for (int q = 0; q < g3; ++q) t1[q] = xg[((size_t)e * g3 + q) * 3 + r];
      for (int dir = 0; dir < 3; ++dir) {
        const int st = dir == 0 ? 1 : dir == 1 ? g : g * g;
        for (int q = 0; q < g3; ++q) {
          const int i = (q / st) % g, base = q - i * st;
          double v = 0.0;
          for (int j = 0; j < g; ++j) v += M[i * g + j] * t1[base + j * st];
          t2[q] = v;
        }
        t1.swap(t2);
      }
      for (int q = 0; q < g3; ++q) {
        b[r] = std::min(b[r], t1[q] + ce[3 * e + r]);
        b[3 + r] = std::max(b[3 + r], t1[q] + ce[3 * e + r]);
      }
      lo[r] = std::min(lo[r], b[r]);
      hi[r] = std::max(hi[r], b[3 + r]);
    }
  }
  double vol = 1.0, pad[3];
  for (int r = 0; r < 3; ++r) {
    pad[r] = 1e-9 * (hi[r] - lo[r]) + 1e-300;
    lo[r] -= pad[r];
    hi[r] += pad[r];
    vol *= hi[r] - lo[r];
  }
  double h = std::cbrt(vol / E);
  for (int attempt = 0; attempt < 8; ++attempt, h /= 1.5) {
    int dims[3];
    size_t ncell = 1;
    for (int r = 0; r < 3; ++r) {
      dims[r] = std::max(1, (int)std::ceil((hi[r] - lo[r]) / h));
      ncell *= (size_t)dims[r];
    }
    if (ncell > (size_t)64 * E + 4096) break;
    std::vector<int> start(ncell + 1, 0);
    auto cells_of = [&](int e, int* c0, int* c1) {
      for (int r = 0; r < 3; ++r) {
        c0[r] = std::max(0, std::min(dims[r] - 1, (int)((box[6 * (size_t)e + r] - 1e-12 * h - lo[r]) / h)));
        c1[r] = std::max(0, std::min(dims[r] - 1, (int)((box[6 * (size_t)e + 3 + r] + 1e-12 * h - lo[r]) / h)));
      }
    };
    for (int e = 0; e < E; ++e) {
      int c0[3], c1[3];
      cells_of(e, c0, c1);
      for (int k = c0[2]; k <= c1[2]; ++k)
        for (int j = c0[1]; j <= c1[1]; ++j)
          for (int i = c0[0]; i <= c1[0]; ++i) start[i + (size_t)dims[0] * (j + (size_t)dims[1] * k) + 1]++;
    }
    int maxc = 0;
    for (size_t q = 0; q < ncell; ++q) maxc = std::max(maxc, start[q + 1]);
    if (maxc > PT_FIND_MAXC) continue;
    for (size_t q = 0; q < ncell; ++q) start[q + 1] += start[q];
    std::vector<int> cur(start.begin(), start.end() - 1), list(start[ncell]);
    for (int e = 0; e < E; ++e) {
      int c0[3], c1[3];
      cells_of(e, c0, c1);
      for (int k = c0[2]; k <= c1[2]; ++k)
        for (int j = c0[1]; j <= c1[1]; ++j)
          for (int i = c0[0]; i <= c1[0]; ++i)
            list[cur[i + (size_t)dims[0] * (j + (size_t)dims[1] * k)]++] = e;
    }
    cudaError_t err;
    c->d_cell_start = dmalloc<int>(c, start.size(), &err);
    if (err) return fail(c, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
    c->d_cell_elem = dmalloc<int>(c, std::max<size_t>(list.size(), 1), &err);
    if (err) return fail(c, PT_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(err));
    CK(cudaMemcpy(c->d_cell_start, start.data(), start.size() * 4, cudaMemcpyHostToDevice));
    if (!list.empty())
      CK(cudaMemcpy(c->d_cell_elem, list.data(), list.size() * 4, cudaMemcpyHostToDevice));
    for (int r = 0; r < 3; ++r) {
      c->grid_lo[r] = lo[r];
      c->grid_ih[r] = 1.0 / h;
      c->grid_dims[r] = dims[r];
    }
    c->grid_ready = true;
    return PT_OK;
  }
  return fail(c, PT_ERR_ARG, "pt_find_element: elements too distorted for the background grid");
}

pt_status pt_find_element(pt_ctx* c, int64_t n, const double* x, int32_t* elem, double* xi,
                          uint32_t* status) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  if (n < 0) return fail(c, PT_ERR_ARG, "n must be >= 0");
  if (n > 0 && (!x || !elem || !xi)) return fail(c, PT_ERR_ARG, "NULL array");
  if (!c->grid_ready) {
    pt_status s = build_find_grid(c);
    if (s) return s;
  }
  if (n == 0) return PT_OK;
  FindArgs a;
  a.m = dev_mesh(c);
  fill_consts(c, a.k);
  a.n = n;
  a.x = x;
  a.elem = elem;
  a.xi = xi;
  a.status = status;
  for (int r = 0; r < 3; ++r) {
    a.lo[r] = c->grid_lo[r];
    a.ih[r] = c->grid_ih[r];
    a.dims[r] = c->grid_dims[r];
  }
  a.cell_start = c->d_cell_start;
  a.cell_elem = c->d_cell_elem;
  int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)c->nsm * 16);
  int rc = launch_find(c->g, c->cfg.precision == PT_FP64, a, grid, 128, c->stream);
  if (rc) return fail(c, PT_ERR_CUDA, "find launch: %s", cudaGetErrorString((cudaError_t)rc));
  return PT_OK;
}

pt_status pt_profile(pt_ctx* c, int32_t enable) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  c->profile = enable != 0;
  return PT_OK;
}

pt_status pt_profile_read_kind(pt_ctx* c, int32_t kind, double* ms, int64_t* launches) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  if (kind < 0 || kind > 3) return fail(c, PT_ERR_ARG, "kind must be 0..3");
  CK(cudaStreamSynchronize(c->stream));
  double tot = 0.0;
  int64_t k = 0;
  std::vector<cudaEvent_t>& u = c->ev_used[kind];
  for (size_t i = 0; i + 1 < u.size(); i += 2) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, u[i], u[i + 1]) == cudaSuccess) {
      tot += t;
      ++k;
    }
  }
  for (cudaEvent_t e : u) c->ev_free.push_back(e);
  u.clear();
  if (ms) *ms = tot;
  if (launches) *launches = k;
  return PT_OK;
}

pt_status pt_profile_read(pt_ctx* c, double* ms, int64_t* launches) {
  if (!c) return fail(nullptr, PT_ERR_ARG, "ctx is NULL");
  pt_status s = pt_profile_read_kind(c, 0, ms, launches);
  if (s) return s;
  for (int k = 1; k < 4; ++k) pt_profile_read_kind(c, k, nullptr, nullptr);  // clear the rest
  return PT_OK;
}

pt_status pt_read_histograms(pt_ctx* c, pt_histograms* out) {
  if (!c || !out) return fail(c, PT_ERR_ARG, "NULL argument");
  unsigned long long h[PT_C_COUNT];
  CK(cudaMemcpyAsync(h, c->d_stats, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 8; ++k) {
    out->newton_fp32[k] = (int64_t)h[PT_C_H32 + k];
    out->newton_final[k] = (int64_t)h[PT_C_H64 + k];
  }
  for (int k = 0; k < 4; ++k) out->crossings[k] = (int64_t)h[PT_C_HCR + k];
  return PT_OK;
}

pt_status pt_launch_count(pt_ctx* c, int64_t* n) {
  if (!c || !n) return fail(c, PT_ERR_ARG, "NULL argument");
  *n = c->launches;
  c->launches = 0;
  return PT_OK;
}

pt_status pt_destroy(pt_ctx* c) {
  if (!c) return PT_OK;
  for (auto& u : c->ev_used)
    for (cudaEvent_t e : u) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  for (void* q : c->allocs) cudaFree(q);
  if (c->d_scratch) cudaFree(c->d_scratch);
  if (c->d_perm) cudaFree(c->d_perm);
  if (c->d_stage) cudaFree(c->d_stage);
  if (c->d_src) cudaFree(c->d_src);
  if (c->d_perm2) cudaFree(c->d_perm2);
  if (c->d_state) cudaFree(c->d_state);
  pt_mlp_release(c);
  pt_batch_release(c);
  delete c;
  return PT_OK;
}

const char* pt_last_error(const pt_ctx* c) {
  if (!c) return g_init_err.c_str();
  return c->err.c_str();
}

}  // extern "C"
