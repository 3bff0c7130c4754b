/*
 * oracle.h -- plain FP64 CPU oracle for the per-particle push of a high-order
 * DG point-particle solver (Kopper, Schwarz et al., "A framework for
 * high-fidelity particle tracking on massively parallel systems",
 * arXiv 2211.05458).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code; only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * Every routine is a direct, unoptimised restatement of the paper's definitions:
 *   - element map and Newton inverse      Sec. 3.1 (Eq. dgsem_curvedfaces), Sec. 3.2.1
 *   - tensor-product interpolation         Sec. 3.2.1, Eq. part_interpolation
 *   - drag force and relaxation time       Sec. 2.2, Eqs. stokesnumber, dragforce, dragfactor
 *   - low-storage RK time integration      Sec. 3.1 (Carpenter & Kennedy 1994), Sec. 3.2.2
 *   - physical-space tracking              Sec. 3.2.3, Eq. parttrajectory
 *   - face intersection (Bezier surfaces)  Sec. 3.2.4, Eq. intersection
 *   - specular wall reflection             Sec. 2.4
 *   - two-way coupling source              Sec. 2.3, Eq. theory:source
 * plus an FP64 multilayer perceptron (forward, backward, Adam) used to check the
 * learned initial-guess network, which has no counterpart in the paper.
 */
#ifndef PT_ORACLE_H
#define PT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status bits, one word per particle */
enum {
  OR_ST_NEWTON_FAIL = 1u << 0,
  OR_ST_LOST        = 1u << 1,
  OR_ST_CROSS_CAP   = 1u << 2,
  OR_ST_NEAR_FACE   = 1u << 3,
  OR_ST_REP800      = 1u << 4,
  OR_ST_OPEN        = 1u << 5,
  OR_ST_NEAR_WALL   = 1u << 6  /* a near-face event on a wall or open face */
};
#define OR_ST_FROZEN (OR_ST_NEWTON_FAIL | OR_ST_LOST | OR_ST_CROSS_CAP | OR_ST_OPEN)

typedef struct {
  double mu;          /* dynamic viscosity                                  */
  double rho_p;       /* particle material density                          */
  int    drag_law;    /* 0 Stokes (f_D = 1), 1 Schiller-Naumann, 2 Haider-Levenspiel */
  int    max_newton;  /* Newton iteration cap                               */
  double g[3];        /* gravitational acceleration                         */
  double mask[3];     /* per-axis multiplier on the drag term (1,1,1)       */
  int    max_cross;   /* face-crossing cap per RK stage                     */
  int    pad;
  double newton_tol;  /* |dxi|_inf convergence threshold                    */
  double band_ref;    /* near-face band in reference units                  */
  double band_x;      /* near-face band in physical length                  */
  double lost_tol;    /* xi outside [-1-lost_tol, 1+lost_tol] => lost       */
  int    lift;        /* 1: Saffman lift with Mei's correction (Sec. 2.2)   */
  int    buoyancy;    /* 1: gravity acts on m_p - m_f (Eq. theory:maxey)      */
  double sphericity;  /* drag_law 2 (Haider-Levenspiel): particle sphericity */
} or_params;

typedef struct or_ctx or_ctx;

/* mesh: xgeo[nelem][(ngeo+1)^3][3], node (a,b,c) at index a+g*(b+g*c) on
 * equidistant reference nodes; neighbor/nbr_face/bc[nelem][6]; shift[nelem][6][3].
 * Local faces: 0: xi1=-1, 1: xi1=+1, 2: xi2=-1, 3: xi2=+1, 4: xi3=-1, 5: xi3=+1.
 * bc: 0 internal, 1 wall, 2 periodic, 3 open, 4 mortar (or_set_mortars).  Arrays are copied. */
or_ctx* or_create(int nelem, int ngeo, const double* xgeo, const int32_t* neighbor,
                  const int32_t* nbr_face, const int32_t* bc, const double* shift);
void    or_destroy(or_ctx* c);
/* non-conforming faces (Sec. 3.2.3): a face with bc 4 is the big side of a
 * mortar; its neighbor entry is a row m of mortar[nmortar][9]:
 *   [0] type 1: four small faces, small face k = i_s + 2 i_t covers the part of
 *       the big face with s < 0 (i_s = 0) or s > 0 (i_s = 1), likewise t;
 *       type 2: two small faces, k = i_s; type 3: two small faces, k = i_t
 *       ((s,t) the big face's parameters)
 *   [1..4] small elements, [5..8] their local faces (unused entries -1).
 * Each small face is an internal face whose neighbour is the big element.
 * The table is copied.  Returns 0 on a malformed table. */
int     or_set_mortars(or_ctx* c, int nmortar, const int32_t* mortar);
/* fluid: U[nelem][5][(N+1)^3] with node (i,j,k) at i+n*(j+n*k); node_type 0 Gauss, 1 GLL.
 * The array is copied. */
int     or_set_fluid(or_ctx* c, int N, int node_type, const double* U);

void    or_nodes(int kind, int n, double* out);             /* 0 Gauss, 1 GLL, 2 equidistant */
double  or_lagrange(int n, const double* xn, int i, double x);
double  or_lagrange_deriv(int n, const double* xn, int i, double x);
void    or_elem_map(const or_ctx* c, int e, const double xi[3], double x[3], double J[9]);
int     or_newton(const or_ctx* c, const or_params* p, int e, const double x[3],
                  double xi[3], int* iters);
void    or_interp(const or_ctx* c, int e, const double xi[3], double U[5]);
void    or_interp_grad(const or_ctx* c, int e, const double xi[3], double U[5], double dU[15]);
void    or_velocity_gradient(const or_ctx* c, int e, const double xi[3], double G[9]);
double  or_drag_factor(const or_params* p, double re);
void    or_saffman_force(const or_params* p, double rho, const double rel[3],
                         const double omega[3], double d, double F[3]);
int     or_face_hits(const or_ctx* c, int e, int f, const double x0[3], const double x1[3],
                     double band, double* out, int maxout);
void    or_face_ctrl(const or_ctx* c, int e, int f, double* out);
int     or_locate_bruteforce(const or_ctx* c, const or_params* p, const double x[3],
                             double tol, int32_t* elems, int maxout);

void    or_push(const or_ctx* c, const or_params* p, int64_t np, double* x, double* v,
                const double* d, int32_t* elem, int32_t* hits, uint32_t* status,
                int nsteps, double dt);
int     or_stage1(const or_ctx* c, const or_params* p, int e, const double x[3],
                  const double v[3], double d, double dt, double out[17]);
void    or_deposit(const or_ctx* c, const or_params* p, int64_t np, const double* x,
                   const double* v, const double* d, const int32_t* elem,
                   const uint32_t* status, double* S);

void    or_quad_weights(int kind, int n, const double* x, double* w);
void    or_deposit_nearest(const or_ctx* c, const or_params* p, int64_t np, const double* x,
                           const double* v, const double* d, const int32_t* elem,
                           const uint32_t* status, double* S);
int64_t or_dt_violations(const or_params* p, int64_t np, const double* d, double dt);
void    or_lserk_coeffs(double* A, double* B, double* C);
void    or_mlp_features(const or_ctx* c, int e, const double x[3], double feat[51]);
void    or_mlp_forward(const double* theta, int B, const double* in, double* out);
double  or_mlp_loss_grad(const double* theta, int B, const double* in, const double* target,
                         double* grad);
void    or_adam(int n, double* theta, const double* g, double* m, double* v, int t,
                double lr, double b1, double b2, double eps);
int     or_mlp_nparams(void);

#ifdef __cplusplus
}
#endif
#endif
