/*
 * pt.h -- C ABI of libpt, a single-GPU (GB300, sm_103a) implementation of the
 * per-particle push of a high-order DG point-particle solver, after Kopper,
 * Schwarz et al., "A framework for high-fidelity particle tracking on
 * massively parallel systems" (arXiv 2211.05458).
 *
 * Conventions used by every entry point
 *   - All pointers are plain host or device pointers as stated per argument;
 *     no CUDA or framework types cross the boundary (streams are void*).
 *   - Device arrays are caller-owned unless stated otherwise and must stay
 *     valid until the work queued on the context's stream has finished.
 *   - Every call returns a pt_status; no exception or abort crosses the ABI.
 *     On error pt_last_error() returns a message for the context (or for the
 *     failed pt_init_mesh when called with NULL).
 *   - Work is queued on the context's stream; a call synchronises only where
 *     it says so (reading statistics back, the *_host variants).
 *   - Particle arrays are structure-of-arrays: a vector quantity of n
 *     particles is 3 contiguous component arrays, x[0..n), x[n..2n), x[2n..3n).
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pt_ctx pt_ctx;

typedef enum {
  PT_OK = 0,
  PT_ERR_ARG = 1,      /* invalid argument, nothing was queued              */
  PT_ERR_CUDA = 2,     /* a CUDA call failed (message in pt_last_error)     */
  PT_ERR_NEWTON = 3,   /* some particles' inverse map did not converge      */
  PT_ERR_LOST = 4,     /* some particles ended outside their element        */
  PT_ERR_CROSS = 5,    /* some particles hit the face-crossing cap          */
  PT_ERR_TIMEOUT = 6,  /* reserved: a bounded device wait gave up           */
  PT_ERR_STATE = 7,    /* call order violated (e.g. push before set_fluid)  */
  PT_WARN_DT = 16      /* dt > 2.75 tau_p for some particle (two-way limit) */
} pt_status;

/* per-particle status bits (pt_particles.status) */
enum {
  PT_ST_NEWTON_FAIL = 1u << 0, /* inverse map failed: particle frozen      */
  PT_ST_LOST = 1u << 1,        /* xi outside the element: particle frozen  */
  PT_ST_CROSS_CAP = 1u << 2,   /* crossing cap reached: particle frozen    */
  PT_ST_NEAR_FACE = 1u << 3,   /* came within the near-face band           */
  PT_ST_REP800 = 1u << 4,      /* Re_p >= 800 seen (drag law out of range)  */
  PT_ST_OPEN = 1u << 5,        /* left through an open boundary: frozen    */
  PT_ST_NEAR_WALL = 1u << 6    /* came within the near-face band of a wall
                                  or open face (a subset of PT_ST_NEAR_FACE):
                                  the wall-hit count and the reflected path
                                  may then depend on rounding               */
};

/* boundary kinds (pt_mesh_desc.bc); PT_BC_MORTAR marks the big side of a
 * non-conforming face (Sec. 3.2.3), see pt_mesh_desc.mortar */
enum { PT_BC_INTERNAL = 0, PT_BC_WALL = 1, PT_BC_PERIODIC = 2, PT_BC_OPEN = 3, PT_BC_MORTAR = 4 };
/* mortar types (pt_mesh_desc.mortar[m][0]) */
enum { PT_MORTAR_FOUR = 1, PT_MORTAR_S = 2, PT_MORTAR_T = 3 };

typedef enum { PT_FP64 = 0, PT_FP32 = 1 } pt_precision;
typedef enum {
  PT_DRAG_STOKES = 0,            /* f_D = 1                                  */
  PT_DRAG_SCHILLER_NAUMANN = 1,  /* f_D = 1 + 0.15 Re^0.687 (Sec. 2.2)       */
  PT_DRAG_HAIDER_LEVENSPIEL = 2  /* four-parameter law in the sphericity     */
} pt_drag_law;
typedef enum { PT_GUESS_TRILINEAR = 0, PT_GUESS_MLP = 1 } pt_guess;
/* How a stage segment finds its new element (Sec. 3.2.3).  PHYSICAL: every
 * face the segment may cross is intersected (Eq. parttrajectory).  REFERENCE:
 * only wall and open faces are intersected; otherwise the end point is
 * located by the inverse map in the current element and, when it lies
 * outside, by walking across the face of the largest |xi_d| (translated on a
 * periodic face) and mapping again (the paper's "localisation in reference
 * space" with face neighbours instead of a background mesh). */
typedef enum { PT_TRACK_PHYSICAL = 0, PT_TRACK_REFERENCE = 1 } pt_track;
/* Kernel schedule of pt_push.  RESIDENT: one kernel per pt_push chunk keeps
 * every particle in registers for all its stages.  STAGED: one kernel per RK
 * stage over the particle state in element-sorted order (held in library-
 * owned device buffers of about 116 bytes per particle in PT_FP32 mode, 144 in
 * PT_FP64 mode), the stage segments that may cross a face collected in a
 * compacted list and intersected by a second kernel on full warps.  AUTO:
 * STAGED from 2^18 particles on, RESIDENT below (launch latency dominates
 * small pushes).  Both run the same arithmetic in the same order per
 * particle. */
typedef enum { PT_SCHEDULE_AUTO = 0, PT_SCHEDULE_RESIDENT = 1, PT_SCHEDULE_STAGED = 2 } pt_schedule;
typedef enum {
  PT_DEPOSIT_ATOMIC = 0,     /* FP32 atomics                                   */
  PT_DEPOSIT_SEGMENTED = 1,  /* element-sorted, fixed summation order          */
  PT_DEPOSIT_NEAREST = 2     /* flag: nearest-node projection (Sec. 2.3)       */
} pt_deposit_mode;

/* Mesh of curved hexahedra (Sec. 3.1, Eq. dgsem_curvedfaces).  All arrays are
 * host memory, read during pt_init_mesh and copied; the caller keeps ownership.
 *   xgeo     [nelem][(ngeo+1)^3][3]  geometry nodes, node (a,b,c) at index
 *                                    a + g*(b + g*c), g = ngeo+1, on
 *                                    equidistant reference points in [-1,1]
 *   neighbor [nelem][6]   element across local face f (-1 on walls / open)
 *   nbr_face [nelem][6]   that element's local index of the shared face
 *   bc       [nelem][6]   PT_BC_* of face f
 *   shift    [nelem][6][3] translation added to a particle crossing a
 *                          periodic face (ignored for other kinds)
 *   nmortar  number of rows of mortar (0 for a conforming mesh)
 *   mortar   [nmortar][9]  non-conforming faces (Sec. 3.2.3): the big side
 *            (e, f) of a mortar has bc PT_BC_MORTAR, neighbor[e][f] = its row
 *            m and nbr_face[e][f] = -1; row m holds
 *              [0]    PT_MORTAR_FOUR: four small faces, small face k = i_s + 2 i_t
 *                     covers the part of the big face with s < 0 (i_s = 0) or
 *                     s > 0 (i_s = 1), likewise t; PT_MORTAR_S: two, k = i_s;
 *                     PT_MORTAR_T: two, k = i_t ((s,t): the big face's parameters)
 *              [1..4] the small elements, [5..8] their local faces (-1 unused)
 *            Every small face is PT_BC_INTERNAL with the big element and face as
 *            neighbour.  Small faces must tile the big face (to rounding).
 *            Mortar faces are not periodic (zero shift).  May be NULL if
 *            nmortar = 0.
 * Local faces: 0: xi1=-1, 1: xi1=+1, 2: xi2=-1, 3: xi2=+1, 4: xi3=-1, 5: xi3=+1;
 * face parameters (s,t) run along the two free reference directions in order. */
typedef struct {
  int32_t nelem;
  int32_t ngeo;
  const double* xgeo;
  const int32_t* neighbor;
  const int32_t* nbr_face;
  const int32_t* bc;
  const double* shift;
  int32_t nmortar;
  const int32_t* mortar;
} pt_mesh_desc;

/* Run-time configuration.  pt_config_default() fills the documented defaults. */
typedef struct {
  double mu;            /* dynamic viscosity (default 1e-5)                        */
  double rho_p;         /* particle material density (default 1000)               */
  double g[3];          /* gravity (default 0)                                     */
  double drag_mask[3];  /* per-axis factor on the drag term (default 1,1,1)       */
  double newton_tol;    /* |dxi|_inf convergence of the inverse map (1e-12)       */
  double band_ref;      /* near-face band, reference units (1e-10)                */
  double band_x;        /* near-face band, physical length (1e-10)                */
  double lost_tol;      /* xi outside [-1-lost_tol, 1+lost_tol] => lost (1e-6)    */
  int32_t precision;    /* pt_precision (default PT_FP64)                          */
  int32_t drag_law;     /* pt_drag_law (default PT_DRAG_STOKES)                    */
  int32_t guess;        /* pt_guess (default PT_GUESS_TRILINEAR)                   */
  int32_t max_newton;   /* Newton iteration cap (default 50)                       */
  int32_t max_cross;    /* face-crossing cap per RK stage (default 64)             */
  int32_t rebin_every;  /* steps between particle re-binning; 0 = library choice   */
  int32_t block;        /* threads per block of the push kernel (32..128); 0 = 128 */
  int32_t lift;         /* 1: add the Saffman lift with Mei's correction (Sec. 2.2),
                           F_S = 6.46/4 C_S d^2 sqrt(rho mu/|w|) (u - v) x w, w = curl u;
                           also deposited by pt_deposit (default 0)                */
  double sphericity;    /* PT_DRAG_HAIDER_LEVENSPIEL: particle sphericity in (0, 1]
                           (default 1): f_D = 1 + A Re^B + (Re/24) C / (1 + D/Re)
                           with A..D the Haider & Levenspiel (1989) fits          */
  int32_t track;        /* pt_track (default PT_TRACK_PHYSICAL)                    */
  int32_t buoyancy;     /* 1: gravity acts on m_p - m_f, i.e. g (1 - rho/rho_p)
                           with the interpolated fluid density (Eq. theory:maxey);
                           0: g acts on m_p alone (default 0)                     */
  int32_t curved_faces; /* intersection with curved faces (Sec. 3.2.4): 0 Newton from
                           the roots of the face's bilinear patch (default; a
                           crossing it misses is found by the walk after the
                           stage); 1 Bezier clipping of the face's control net   */
  int32_t schedule;     /* pt_schedule: how pt_push maps the stages to kernels
                           (default PT_SCHEDULE_AUTO); results do not depend on it */
  int32_t reserved[2];
} pt_config;

/* Particles, structure of arrays, all device memory, caller-owned, updated in
 * place by pt_push.  Floating-point arrays marked "real" are double in
 * PT_FP64 mode and float in PT_FP32 mode; positions are always double.
 *   n       number of particles (>= 0)
 *   x       double [3][n] positions (in/out)
 *   v       real   [3][n] velocities (in/out)
 *   d       real   [n]    diameters (in)
 *   elem    int32  [n]    owning element (in/out; must own x on entry)
 *   hits    int32  [n]    wall-impact counters (in/out)
 *   status  uint32 [n]    PT_ST_* bits (in/out; frozen particles are skipped) */
typedef struct {
  int64_t n;
  double* x;
  void* v;
  const void* d;
  int32_t* elem;
  int32_t* hits;
  uint32_t* status;
} pt_particles;

/* Totals over one pt_push call (host struct). */
typedef struct {
  int64_t particle_steps;   /* live particles x steps                        */
  int64_t crossings;        /* internal + periodic face crossings            */
  int64_t wall_hits;        /* specular reflections                          */
  int64_t newton_it_fp32;   /* FP32 Newton iterations (FP32 mode)            */
  int64_t newton_it_fp64;   /* FP64 Newton iterations / refinements          */
  int64_t slow_track;       /* stage segments that needed face intersection  */
  int64_t near_face;        /* particles with PT_ST_NEAR_FACE set at the end */
  int64_t newton_fail;      /* particles frozen by each cause, at the end    */
  int64_t lost;
  int64_t cross_cap;
  int64_t open;
  int64_t rep800;
  int64_t dt_warn;          /* particles with dt > 2.75 tau_p                */
  int64_t near_wall;        /* particles with PT_ST_NEAR_WALL set at the end */
  int64_t reserved[2];
} pt_stats;

/* Histograms of the last pt_push (host struct), kept by the staged schedule
 * (all zero after a push with the resident one):
 *   newton_fp32[k]  particle-stages whose inverse map took k FP32 Newton
 *                   iterations (k = 0..6; [7]: 7 or more)
 *   newton_final[k] the same for the final iterations (double-float residuals
 *                   in PT_FP32 mode; every FP64 iteration in PT_FP64 mode)
 *   crossings[k]    exactly tracked stage segments with k face crossings
 *                   (k = 0..2; [3]: 3 or more)                             */
typedef struct {
  int64_t newton_fp32[8];
  int64_t newton_final[8];
  int64_t crossings[4];
} pt_histograms;

/* Fills *cfg with the defaults listed in pt_config. */
void pt_config_default(pt_config* cfg);

/* Creates a context on the current CUDA device: copies the mesh to the GPU and
 * builds the per-face tables (face kind by bounding box, Sec. 3.2.4; bilinear
 * coefficients; bounding slabs), the element centres and trilinear start
 * tables.  stream: cudaStream_t used for all later work (NULL = default).
 * Returns PT_ERR_ARG for inconsistent connectivity (a neighbour that does not
 * point back, an out-of-range element or face index, a non-periodic face with
 * a shift, a malformed mortar row or one not referenced by exactly one big
 * face, unsupported ngeo (1..4)).  *ctx is NULL on error. */
pt_status pt_init_mesh(pt_ctx** ctx, const pt_mesh_desc* mesh, const pt_config* cfg,
                       void* stream);

/* Replaces the configuration (same rules as at init). */
pt_status pt_set_config(pt_ctx* ctx, const pt_config* cfg);

/* Registers the fluid state (Sec. 3.1, Eq. dgsem_interpolation): N in 1..7,
 * node_type 0 = Legendre-Gauss, 1 = Legendre-Gauss-Lobatto,
 * U_dev [nelem][5][(N+1)^3] device array of (rho, rho u1, rho u2, rho u3,
 * rho e) with node (i,j,k) at i + n*(j + n*k); double in PT_FP64 mode, float
 * in PT_FP32 mode, 16-byte aligned (PT_ERR_ARG otherwise).  Caller-owned;
 * read by every later push / deposit. */
pt_status pt_set_fluid(pt_ctx* ctx, int32_t N, int32_t node_type, const void* U_dev);

/* Advances every live particle by nsteps steps of the 5-stage, 4th-order
 * low-storage RK scheme of Carpenter & Kennedy (Sec. 3.1) with time step dt.
 * The fluid state registered by pt_set_fluid is frozen during a call: all
 * nsteps x 5 stages interpolate the same U.  A solver that updates U every
 * time step calls pt_push with nsteps = 1 between its own updates (binning
 * and, in the staged schedule, the sorted copy of the particle state are then
 * paid per step); the paper's fully coupled loop, in which the fluid and the
 * particles advance stage by stage together, is not offered.
 * Per stage and particle (Sec. 3.2): inverse map x -> xi by Newton, tensor-
 * product interpolation of rho and rho u at xi (Eq. part_interpolation),
 * drag (Eqs. dragforce, dragfactor) plus gravity, the RK update of x and v,
 * and tracking of the straight stage segment (Eq. parttrajectory) through
 * element faces with specular reflection at walls (Sec. 2.4), periodic
 * translation, removal at open faces and, across the big side of a mortar,
 * entry by the small face the segment crosses (Sec. 3.2.3).
 * out: host pointer or NULL; when non-NULL the call synchronises the stream
 * and fills the totals.  Returns PT_OK, or (only when out != NULL) the first
 * of PT_ERR_NEWTON / PT_ERR_LOST / PT_ERR_CROSS whose count is non-zero, or
 * PT_WARN_DT.  Particle order is preserved; the library bins particles by
 * element internally. */
pt_status pt_push(pt_ctx* ctx, const pt_particles* p, int32_t nsteps, double dt,
                  pt_stats* out);

/* One RK stage for a solver that advances the fluid and the particles stage
 * by stage together (Sec. 3.2.2: the particles use the fluid's RK scheme,
 * each stage interpolating the fluid state of that stage).  Call with
 * stage = 0, 1, 2, 3, 4 in turn, the same particle arrays and dt, updating
 * the fluid state registered by pt_set_fluid (in place or by another
 * pt_set_fluid with the same N) between the calls.  Stage 0 bins the
 * particles and copies them into library-owned device buffers (the staged
 * schedule's state); stages 0..4 each run the inverse map, interpolation,
 * drag, RK stage and tracking on that state; stage 4 copies the state back
 * into the caller's arrays, which hold the step's start state until then.
 * With a fluid state that does not change, the five calls give bitwise the
 * result of pt_push with nsteps = 1 in the staged schedule.  out: as pt_push,
 * read at stage 4 (NULL otherwise).  PT_ERR_STATE for a stage out of order;
 * PT_ERR_ARG for other particle arrays or another dt than at stage 0;
 * pt_push and pt_deposit return PT_ERR_STATE while a sequence is open. */
pt_status pt_push_stage(pt_ctx* ctx, const pt_particles* p, int32_t stage, double dt,
                        pt_stats* out);

/* As pt_push, but the particle arrays are HOST memory (same layout); the
 * library stages them through its own device buffers, copies the results
 * back and synchronises.  Intended for callers without device buffers. */
pt_status pt_push_host(pt_ctx* ctx, const pt_particles* p_host, int32_t nsteps, double dt,
                       pt_stats* out);

/* Two-way coupling source (Sec. 2.3, Eq. theory:source): each live particle's
 * drag F = m_p f_D (u - v) / tau_p contributes momentum -F and energy -F.v_p.
 * S_dev [nelem][4][(N+1)^3] float, device, caller-owned, overwritten.
 * Projection: by default the amounts are spread over the nodes of the
 * particle's element with weights l_i(xi1) l_j(xi2) l_k(xi3) (nodal amounts);
 * with the PT_DEPOSIT_NEAREST flag the whole source goes to the node nearest
 * to xi (per reference direction, the lower node on a tie) as the density
 * a / V_ijk, V_ijk = w_i w_j w_k |det J(xi_ijk)| the node's quadrature share
 * of the element volume (the paper's projection operator).  Summation:
 * PT_DEPOSIT_ATOMIC adds with FP32 atomics (order-dependent rounding);
 * PT_DEPOSIT_SEGMENTED sums each element's particles in index order (bitwise
 * reproducible): it sorts each element's particles by index (O(m log^2 m)
 * for m particles in an element), computes every particle's source into a
 * library-owned device buffer of 36 bytes per particle (grown on demand,
 * released by pt_destroy), then reduces per element.  Other mode bits: PT_ERR_ARG. */
pt_status pt_deposit(pt_ctx* ctx, const pt_particles* p, int32_t mode, float* S_dev);

/* pt_deposit without any device allocation (the paper has no counterpart).
 * Some callers cannot call cudaMalloc: a flow solver that has handed the
 * device memory to its own pool allocator, or a time loop that must not
 * allocate once it runs (a device allocation can synchronise the device and
 * fragment such a pool).  This entry point takes the same modes, S_dev layout
 * and ownership as pt_deposit, but keeps its scratch -- the element binning
 * counters and two particle orders -- in one fixed array of about 9.9 MB of
 * device memory that the library reserves on every GPU that loads it, until
 * the process exits.  The segmented mode computes each particle's source
 * inside the per-element reduction (one pass, no 32-byte-per-particle buffer)
 * with the same factors and order as pt_deposit: in PT_FP32 mode the result is
 * bitwise that of pt_deposit; in PT_FP64 mode it agrees to FP32 rounding of
 * the weights; either way it is bitwise reproducible from call to call.  The
 * atomic mode is pt_deposit's atomic mode.  Limits: at most 131072 elements
 * and 1048576 particles; larger problems return PT_ERR_ARG (use pt_deposit).
 * The array's device address differs per CUDA context; every call outside a
 * stream capture looks it up again in the current context, and a call being
 * captured into a graph uses the address of the last call outside capture on
 * that device (PT_ERR_CUDA if there was none): make one call outside capture
 * first.  Every call reuses the same array and clears what must start at
 * zero; calls whose work overlaps on the GPU (other streams, other contexts)
 * race on it. */
pt_status pt_deposit_noalloc(pt_ctx* ctx, const pt_particles* p, int32_t mode, float* S_dev);

/* The terms of the first RK stage of each particle, evaluated by the push's
 * own code but without tracking, so that each result of the precision split
 * (Sec. 3.2.1 inverse map, Eq. part_interpolation, Sec. 2.2 drag, Sec. 3.1
 * RK update) can be compared with FP64 values: xi_dev double [3][n] the
 * inverse map of x in elem (trilinear start, the context's precision);
 * U_dev real [4][n] rho, rho u1, rho u2, rho u3 at xi; acc_dev real [3][n]
 * the particle's acceleration (drag, gravity, lift as configured); dx_dev and
 * dv_dev real [3][n] the stage increments B_1 dt v and B_1 dt a ("real" is
 * the context's precision).  p->status receives PT_ST_NEWTON_FAIL or
 * PT_ST_LOST where no terms could be formed (outputs then unchanged), else
 * 0 or PT_ST_REP800; x, v, elem are not changed.  All device, caller-owned. */
pt_status pt_stage_terms(pt_ctx* ctx, const pt_particles* p, double dt, double* xi_dev,
                         void* U_dev, void* acc_dev, void* dx_dev, void* dv_dev);

/* Point location without a known element (Sec. 3.2.3, localisation in
 * reference space): for each x the candidates are the elements listed in x's
 * cell of a uniform background grid (an element is listed in every cell its
 * Bezier control box meets), tried closest element centre first with the
 * inverse map; the first with max |xi| <= 1 + lost_tol owns x.  x_dev double
 * [3][n] device; elem_dev int32 [n] out (-1: no element contains x);
 * xi_dev double [3][n] out (0 where not found); status_dev uint32 [n] out or
 * NULL (0, or PT_ST_LOST where not found).  The first call builds the grid
 * (host work over all elements, device memory released by pt_destroy);
 * PT_ERR_ARG if the elements are too distorted for a grid of at most 64
 * candidates per cell.  A point on a face shared by several elements gets one
 * of them. */
pt_status pt_find_element(pt_ctx* ctx, int64_t n, const double* x_dev, int32_t* elem_dev,
                          double* xi_dev, uint32_t* status_dev);

/* Inverse map only (Sec. 3.2.1): for each i, xi of x[:,i] in element elem[i].
 * x_dev double [3][n], elem_dev int32 [n], xi_dev double [3][n] out,
 * iters_dev int32 [n] out (Newton iterations, FP32 + FP64), status_dev uint32
 * [n] out (PT_ST_NEWTON_FAIL on failure).  Uses the context's precision and
 * guess mode.  All device, caller-owned. */
pt_status pt_locate(pt_ctx* ctx, int64_t n, const double* x_dev, const int32_t* elem_dev,
                    double* xi_dev, int32_t* iters_dev, uint32_t* status_dev);

/* Learned initial guess (no counterpart in the paper).  A 51-64-64-64-3 GELU
 * network maps [xi_tri (3), 48 geometry deviations] to a correction of the
 * trilinear Newton start; see pt_mlp_features for the inputs (ngeo = 3 only).
 *
 * pt_mlp_make_pairs: n training pairs on the device.  Elements and reference
 * points are drawn by a counter-based generator from seed; x = chi(xi) and the
 * label xi comes from the FP64 Newton inverse.  in_dev float [n][51] (raw
 * features), target_dev float [n][3] (xi_newton - xi_tri).
 * pt_mlp_train: Adam (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the MSE, batch
 * rows per step, epochs passes in an order drawn from seed; inputs are
 * standardised by statistics taken from in_dev and targets scaled by their
 * rms.  loss_host: host float[epochs] mean loss per epoch, or NULL.
 * Synchronises.  After training the BF16 copy used by the push is refreshed. */
pt_status pt_mlp_make_pairs(pt_ctx* ctx, int64_t n, uint64_t seed, float* in_dev,
                            float* target_dev);
pt_status pt_mlp_train(pt_ctx* ctx, int64_t n, const float* in_dev, const float* target_dev,
                       int32_t epochs, int32_t batch, float lr, uint64_t seed, float* loss_host);
/* Raw features of x in elem (same definition as the learned guess uses):
 * x_dev double [3][n], elem_dev int32 [n], feat_dev float [n][51]. */
pt_status pt_mlp_features(pt_ctx* ctx, int64_t n, const double* x_dev, const int32_t* elem_dev,
                          float* feat_dev);
/* Network parameters as one flat float array (11843 values: W1[64][51], b1,
 * W2[64][64], b2, W3[64][64], b3, W4[3][64], b4) plus the normalisation
 * (in_mean[51], in_std[51], out_scale[3]).  Host pointers.  set refreshes the
 * BF16 copy. */
int32_t pt_mlp_nparams(void);
pt_status pt_mlp_set(pt_ctx* ctx, const float* theta_host, const float* norm_host);
pt_status pt_mlp_get(pt_ctx* ctx, float* theta_host, float* norm_host);
/* The learned Newton start of x_dev double [3][n] in elem_dev int32 [n]:
 * guess_dev float [3][n] receives xi_tri + the network's correction, as the
 * push uses it (an owner out of range leaves its column unchanged).  engine 1:
 * the tensor-core form of the staged schedule (tcgen05, 128 particles per
 * CTA, accumulators in tensor memory); 0: the warp-level mma.sync form of the
 * resident schedule.  Needs ngeo = 3, PT_FP32 and a trained or set network
 * (PT_ERR_STATE otherwise); PT_ERR_TIMEOUT if a tensor-core wait gave up.
 * Synchronises. */
pt_status pt_mlp_start(pt_ctx* ctx, int64_t n, const double* x_dev, const int32_t* elem_dev,
                       float* guess_dev, int32_t engine);

/* FP32 forward pass and loss gradient of the network on already-normalised
 * inputs (the kernels training uses): in_dev float [B][51], out_dev [B][3];
 * grad_dev float [11843] overwritten with d(mean squared error)/d theta for
 * targets target_dev [B][3]; loss_host receives the loss (synchronises). */
pt_status pt_mlp_forward(pt_ctx* ctx, int32_t B, const float* in_dev, float* out_dev);
pt_status pt_mlp_grad(pt_ctx* ctx, int32_t B, const float* in_dev, const float* target_dev,
                      float* grad_dev, float* loss_host);

/* Batched push: nbox independent contexts (PT_FP32, ngeo = 1, N in 3..7),
 * each with its own particles.  The boxes are grouped by N; per step chunk
 * one binning of all particles, then one persistent launch per group with the
 * kernel instantiated for that N, the groups' launches running concurrently.
 * The first call tunes each group's block size (64, 96 or 128 threads, timed
 * on successive chunks); later calls replay the sequence captured once per
 * (nsteps, dt) in a CUDA graph on ctxs[0]'s stream.  out: host array of nbox
 * pt_stats or NULL (synchronises). */
pt_status pt_push_batch(pt_ctx* const* ctxs, const pt_particles* parts, int32_t nbox,
                        int32_t nsteps, double dt, pt_stats* out);
/* The batched push's tuning, per degree group (in increasing N): N_out[i], the
 * chosen block size block_out[i] (0 while tuning) and the measured ms per step
 * of the three candidates ms_out[3 i + k]; *ngroups receives the number of
 * groups (0 before the first pt_push_batch with ctx0 first).  Arrays may be
 * NULL; at most max_groups entries are written. */
pt_status pt_batch_tuning(pt_ctx* ctx0, int32_t* N_out, int32_t* block_out, float* ms_out,
                          int32_t max_groups, int32_t* ngroups);

/* Kernel timing (diagnostics).  pt_profile(ctx, 1) makes every later push
 * record a CUDA event pair around each launch of the push kernel on the
 * context's stream; pt_profile_read synchronises, returns the summed device
 * time of those launches in milliseconds and their number, and clears the
 * record.  pt_profile(ctx, 0) stops recording. */
pt_status pt_profile(pt_ctx* ctx, int32_t enable);
pt_status pt_profile_read(pt_ctx* ctx, double* kernel_ms, int64_t* launches);
/* As pt_profile_read for one kind of kernel, clearing only that record:
 * kind 0 the push (the resident kernel, or a whole chunk of the staged
 * schedule from its binning to the copy back), 1 the staged schedule's
 * stage kernels, 2 its learned-start kernels, 3 its exact-tracking kernels.
 * (pt_profile_read reads kind 0 and clears all four.) */
pt_status pt_profile_read_kind(pt_ctx* ctx, int32_t kind, double* kernel_ms, int64_t* launches);

/* Reads the histograms of the last pt_push into *out (synchronises). */
pt_status pt_read_histograms(pt_ctx* ctx, pt_histograms* out);

/* Kernel launches this context queued (every kernel of every call) since the
 * last pt_launch_count; *n receives the count, which is then cleared. */
pt_status pt_launch_count(pt_ctx* ctx, int64_t* n);

/* Measured arithmetic throughput of the current device (diagnostics, no
 * counterpart in the paper): kind 0 FP32, 1 FP64 fused multiply-adds on every
 * SM (eight independent chains per thread), best of three timed launches after
 * a warm-up; *tflops receives TFLOP/s (2 flops per multiply-add).  Queued on
 * stream (a cudaStream_t, NULL = default) and synchronised.  The ALU roofline
 * of the push is reported against it. */
pt_status pt_measure_peak(int32_t kind, void* stream, double* tflops);

/* Releases the context and its device memory (not the caller's arrays). */
pt_status pt_destroy(pt_ctx* ctx);

/* Last error message of ctx (or of the last failed pt_init_mesh if ctx is
 * NULL); never NULL. */
const char* pt_last_error(const pt_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PT_H */
