// pt_internal.h -- device-side views and launch arguments shared by the
// translation units of libpt.  Not part of the public ABI (see include/pt.h).
#pragma once
#include <cstdint>

#include "pt.h"

#define PT_MAXG 5  // geometry nodes per direction (NGeo <= 4)
#define PT_MAXN 8  // solution nodes per direction (N <= 7)
#define PT_MLP_IN 51
#define PT_MLP_H 64
#define PT_MLP_OUT 3
#define PT_MLP_NP (PT_MLP_H * PT_MLP_IN + PT_MLP_H + 2 * (PT_MLP_H * PT_MLP_H + PT_MLP_H) + \
                   PT_MLP_OUT * PT_MLP_H + PT_MLP_OUT)

// face kinds (by bounding-box flatness / bilinearity of the face nodes)
enum { PT_FACE_PLANAR = 0, PT_FACE_BILINEAR = 1, PT_FACE_CURVED = 2 };
// packed face record (DevMesh::finfo)
__host__ __device__ __forceinline__ int finfo_bc(int info) { return info & 7; }
__host__ __device__ __forceinline__ int finfo_kind(int info) { return (info >> 3) & 3; }
__host__ __device__ __forceinline__ int finfo_nf(int info) { return (info >> 5) & 7; }

// stats counter slots (device uint64 array)
enum {
  PT_C_STEPS = 0, PT_C_CROSS, PT_C_HITS, PT_C_IT32, PT_C_IT64, PT_C_SLOW,
  PT_C_NEAR, PT_C_NFAIL, PT_C_LOST, PT_C_CCAP, PT_C_OPEN, PT_C_REP, PT_C_DTWARN, PT_C_NEARWALL,
  PT_C_TIMEOUT,
  // histograms of the staged schedule: particle-stages by FP32 Newton
  // iterations (0..6, 7+), by final iterations (0..6, 7+), exactly tracked
  // segments by crossings (0, 1, 2, 3+)
  PT_C_H32 = 16, PT_C_H64 = 24, PT_C_HCR = 32,
  PT_C_COUNT = 40
};

#define PT_ST_FROZEN (PT_ST_NEWTON_FAIL | PT_ST_LOST | PT_ST_CROSS_CAP | PT_ST_OPEN)

// Mesh tables on the device.  Geometry is stored relative to each element's
// centre ce (the mean of its 8 corner nodes), which keeps FP64 residuals and
// face intersections at the element's own scale.
struct DevMesh {
  int nelem;
  int g;                  // NGeo + 1
  const double* xg64;     // [E][g^3][3]   nodes - ce
  const float* xg32;      // [E][3][g^3]   nodes - ce, FP32, coordinate-major
  const float* xg32lo;    // [E][3][g^3]   (nodes - ce) - xg32: low parts of a double-float copy
  const double* ce;       // [E][3]
  const float* tri;       // [E][12]       trilinear centre (3) and inverse Jacobian (9)
  const int* tmask;       // [E]           bit q: coordinate q is trilinear in xi (8-corner form)
  const int* fnbr;        // [E][6]        neighbour element (mortar row on a PT_BC_MORTAR face)
  const int* finfo;       // [E][6]        bc | kind << 3 | nbr_face << 5
  const int* mort;        // [M][9]        mortar rows as in pt_mesh_desc (null if none)
  const float* slab;      // [E][6][8]     unit normal (3), lo, hi, -, -, - (local coords)
  const double* bil;      // [E][6][12]    p(s,t) = a st + b s + c t + d (local coords)
  const float* bil32;     // [E][6][12]    FP32 copy of bil (screening)
  const double* shift;    // [E][6][3]
  const float* mlp_pre;   // [E][64]       element part of the first MLP layer, or null
};

// Constants of one run: node sets, RK table, physics and tolerances.
struct DevConsts {
  double gn[PT_MAXG], gw[PT_MAXG];   // geometry nodes / barycentric weights
  float gn32[PT_MAXG], gw32[PT_MAXG];
  float gn_hi[PT_MAXG], gn_lo[PT_MAXG], gw_hi[PT_MAXG], gw_lo[PT_MAXG];  // double-float copies
  double sn[PT_MAXN], sw[PT_MAXN];   // solution nodes / barycentric weights
  float sn32[PT_MAXN], sw32[PT_MAXN];
  double sq[PT_MAXN];                // quadrature weights of the solution nodes
  double A[5], B[5];
  float A32[5], B32[5];
  double mu, rho_p, g[3], mask[3];
  double newton_tol, band_ref, band_x, lost_tol;
  double hl[4];                      // Haider-Levenspiel A, B, C, D
  int drag_law, max_newton, max_cross, guess, lift, track, buoyancy, curved_clip;
  double gbz[PT_MAXG * PT_MAXG];     // Bezier control values = gbz x nodal values
};

struct DevParticles {
  int64_t n;
  double* x;
  void* v;
  const void* d;
  int* elem;
  int* hits;
  unsigned* status;
};

// BF16 network for the learned guess: layers 2 and 3 as bf16 [out][in] in
// global memory (staged to shared memory per block); the small FP32 parts
// travel by value in the kernel parameters (constant bank).
struct DevMLP {
  const uint16_t* w2;     // [64][64] bf16
  const uint16_t* w3;     // [64][64] bf16
  float w1x[64 * 3];      // first-layer columns of the xi_tri inputs / in_std
  float b2[64];
  float b3[64];
  float w4[3 * 64];       // output layer scaled by the output scale
  float b4[4];
};

struct PushArgs {
  DevMesh m;
  DevConsts k;
  DevParticles p;
  DevMLP mlp;
  const void* U;          // fluid state, [E][5][n^3], double or float per mode
  const int* perm;        // particle visiting order (sorted by element) or null
  int nsteps;
  double dt;
  unsigned long long* stats;
};

struct LocateArgs {
  DevMesh m;
  DevConsts k;
  DevMLP mlp;
  int64_t n;
  const double* x;
  const int* elem;
  double* xi;
  int* iters;
  unsigned* status;
};

// point location without a known element: background grid of element lists
#define PT_FIND_MAXC 64  // candidates per grid cell at most
struct FindArgs {
  DevMesh m;
  DevConsts k;
  int64_t n;
  const double* x;        // [3][n]
  int* elem;              // [n] out, -1 if not found
  double* xi;             // [3][n] out
  unsigned* status;       // [n] out, 0 or PT_ST_LOST
  double lo[3], ih[3];    // grid origin and inverse cell size
  int dims[3];
  const int* cell_start;  // [ncell + 1]
  const int* cell_elem;   // elements whose control box meets the cell
};

struct DepositArgs {
  DevMesh m;
  DevConsts k;
  DevParticles p;
  const void* U;
  const int* perm;        // sorted order (segmented mode)
  const int* offs;        // [E+1] element segment offsets (segmented mode)
  float* S;               // [E][4][n^3]
  float4* src;            // [2 n] per-particle sources of the two-pass segmented mode
};

// One RK stage of the staged schedule: the particle state in element-sorted
// order (library-owned structure-of-arrays, index t), the list of stage
// segments that need exact tracking or the walk, and the counters.
struct StageArgs {
  DevMesh m;
  DevConsts k;
  DevMLP mlp;
  const void* U;          // fluid state
  int64_t n;
  double* x;              // FP64 mode: [3][n] positions
  float* xh;              // FP32 mode: [3][n] double-float offset from the owner's
  float* xl;              //            centre, high and low parts
  void* v;                // [3][n] velocity, mode precision
  void* kx;               // [3][n] RK registers of x and v
  void* kv;
  const void* d;          // [n] diameters
  void* xe;               // stage end of listed particles: FP64 [3][n]; FP32 [6][n] hi, lo
  int* e;                 // [n] owner
  int* hits;              // [n]
  unsigned* st;           // [n] status bits
  float* guess;           // [3][n] learned start (MLP) or null
  float* xih;             // FP32 mode, split stage: [3][n] converged xi, double-float
  float* xil;
  unsigned* list;         // [n] listed positions (| 1 << 31: walk only)
  unsigned* count;        // entries in list
  unsigned* count_next;   // the next stage's counter (cleared by this stage)
  int stage;              // 0..4
  double dt;
  unsigned long long* stats;
};

// first-stage terms of each particle (pt_stage_terms): p.status receives the
// status bits, the other outputs are [q][n] arrays in the mode's precision
struct TermsArgs {
  DevMesh m;
  DevConsts k;
  DevParticles p;
  const void* U;
  double dt;
  double* xi;             // [3][n]
  void* Uo;               // [4][n] rho, rho u1, rho u2, rho u3 at xi
  void* acc;              // [3][n]
  void* dx;               // [3][n] B_1 dt v
  void* dv;               // [3][n] B_1 dt a
};

// kernel entry points, one family per (g, mode) translation unit
namespace pt {
int launch_push(int g, bool fp64, int np, const PushArgs& a, int grid, int block, void* stream);
int launch_find(int g, bool fp64, const FindArgs& a, int grid, int block, void* stream);
int launch_locate(int g, bool fp64, int np, const LocateArgs& a, int grid, int block,
                  void* stream);
int launch_deposit(int g, bool fp64, int np, int mode, const DepositArgs& a, int grid, int block,
                   void* stream);
int max_active_push(int g, bool fp64, int np, int block);
int launch_terms(int g, bool fp64, int np, const TermsArgs& a, int grid, int block, void* stream);
// staged schedule: op 0 gather, 1 stage, 2 track, 3 learned start, 4 scatter back
// (5, 6: the learned start of global positions a.x, tensor-core and warp-MMA
// forms, for pt_mlp_start)
enum { PT_SOP_GATHER = 0, PT_SOP_STAGE = 1, PT_SOP_TRACK = 2, PT_SOP_GUESS = 3, PT_SOP_SCATTER = 4,
       PT_SOP_GUESS_X_TC = 5, PT_SOP_GUESS_X_WARP = 6 };
int launch_staged(int g, bool fp64, int np, int op, const StageArgs& a, const DevParticles& p,
                  const int* perm, int grid, int block, void* stream);
int max_active_stage(int g, bool fp64, int np, int block);
}  // namespace pt
