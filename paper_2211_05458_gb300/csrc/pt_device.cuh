// pt_device.cuh -- device building blocks of the particle push (arXiv 2211.05458):
// Lagrange bases, the inverse map x -> xi (Sec. 3.2.1), interpolation of the
// nodal state (Eq. part_interpolation), drag (Sec. 2.2) and the physical-
// space tracking with face intersection (Secs. 3.2.3, 3.2.4) and the specular
// wall model (Sec. 2.4).  Everything is templated on the number of geometry
// nodes G = NGeo+1 and solution nodes NP = N+1 so loops unroll into registers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "pt_df.cuh"
#include "pt_internal.h"

// 1: evaluate the per-dimension Lagrange bases of the Newton residuals in a
// rolled loop (one copy of the code, values through local memory), which
// shrinks the hot loop's instruction footprint
#ifndef PT_ROLL_BASIS
#define PT_ROLL_BASIS 1
#endif
// 1: run-time indices into small register arrays of the interpolation
// (PT_PICK_INTERP) and of the element map (PT_PICK_MAP) go through chains of
// selects instead of dynamic indexing, which keeps the arrays out of local
// memory at the cost of more live registers
#ifndef PT_PICK_INTERP
#define PT_PICK_INTERP 0
#endif
#ifndef PT_PICK_MAP
#define PT_PICK_MAP 0
#endif
// FP32 Newton iterations of the FP32 mode stop once the step is below this;
// the final iterations (double-float residuals, last FP32 inverse Jacobian)
// take over and converge linearly with a factor of about the step at which
// that Jacobian was evaluated
#ifndef PT_NEWTON_SWITCH
#define PT_NEWTON_SWITCH 1e-5f
#endif
// 1: screen each touched face in FP32 before its exact FP64 solve
#ifndef PT_FACE_SCREEN
#define PT_FACE_SCREEN 1
#endif
// 1 (FP32 mode): an internal or periodic crossing that the FP32 screen finds
// unambiguous is taken without the FP64 solve (see track_slow)
#ifndef PT_FP32_DECIDE
#define PT_FP32_DECIDE 1
#endif

namespace pt {

template <typename T>
__device__ __forceinline__ T tabs(T a) {
  return a < T(0) ? -a : a;
}

template <typename T>
__device__ __forceinline__ T tmax3(T a, T b, T c) {
  return fmax(fmax(tabs(a), tabs(b)), tabs(c));
}

// a[i] for a run-time i without indexing the array dynamically (which would
// put it in local memory): a chain of selects over the unrolled indices
template <int N, typename T>
__device__ __forceinline__ T pick(const T* a, int i) {
  T v = a[0];
#pragma unroll
  for (int j = 1; j < N; ++j)
    if (j == i) v = a[j];
  return v;
}

// a[i] = v for a run-time i, likewise
template <int N, typename T>
__device__ __forceinline__ void put(T* a, int i, T v) {
#pragma unroll
  for (int j = 0; j < N; ++j)
    if (j == i) a[j] = v;
}

template <typename T>
__device__ __forceinline__ T tfma(T a, T b, T c);
template <>
__device__ __forceinline__ float tfma<float>(float a, float b, float c) {
  return fmaf(a, b, c);
}
template <>
__device__ __forceinline__ double tfma<double>(double a, double b, double c) {
  return fma(a, b, c);
}

// node set of the right precision from the constants
template <typename T>
struct Nodes;
template <>
struct Nodes<float> {
  __device__ static const float* geo(const DevConsts& k) { return k.gn32; }
  __device__ static const float* geow(const DevConsts& k) { return k.gw32; }
  __device__ static const float* sol(const DevConsts& k) { return k.sn32; }
  __device__ static const float* solw(const DevConsts& k) { return k.sw32; }
};
template <>
struct Nodes<double> {
  __device__ static const double* geo(const DevConsts& k) { return k.gn; }
  __device__ static const double* geow(const DevConsts& k) { return k.gw; }
  __device__ static const double* sol(const DevConsts& k) { return k.sn; }
  __device__ static const double* solw(const DevConsts& k) { return k.sw; }
};

// Lagrange basis in barycentric product form: l_i(x) = w_i prod_{m != i} (x - x_m),
// w_i = 1 / prod_{m != i} (x_i - x_m).  Prefix and suffix products avoid the
// division of the second barycentric form, so the values at the nodes are exact.
template <int NP, typename T>
__device__ __forceinline__ void lagr(T x, const T* nodes, const T* w, T* l) {
  T d[NP];
#pragma unroll
  for (int m = 0; m < NP; ++m) d[m] = x - nodes[m];
  T pre = T(1);
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    l[i] = pre;
    pre *= d[i];
  }
  T suf = T(1);
#pragma unroll
  for (int i = NP - 1; i >= 0; --i) {
    l[i] *= suf * w[i];
    suf *= d[i];
  }
}

// values and first derivatives (dual-number prefix / suffix products)
template <int NP, typename T>
__device__ __forceinline__ void lagr_d(T x, const T* nodes, const T* w, T* l, T* dl) {
  T d[NP], P[NP], dP[NP];
#pragma unroll
  for (int m = 0; m < NP; ++m) d[m] = x - nodes[m];
  T p = T(1), dp = T(0);
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    P[i] = p;
    dP[i] = dp;
    dp = tfma(dp, d[i], p);
    p *= d[i];
  }
  T s = T(1), ds = T(0);
#pragma unroll
  for (int i = NP - 1; i >= 0; --i) {
    l[i] = w[i] * P[i] * s;
    dl[i] = w[i] * tfma(dP[i], s, P[i] * ds);
    ds = tfma(ds, d[i], s);
    s *= d[i];
  }
}

// Read-only load: through the non-coherent path from global memory, or (SH)
// a generic load, for data that may sit in shared memory.
template <bool SH, typename V>
__device__ __forceinline__ V ldx(const V* p) {
  if constexpr (SH)
    return *p;
  else
    return __ldg(p);
}

// G consecutive floats starting at p (p is 16-byte aligned when G == 4 and
// 8-byte aligned when G is even: row starts are multiples of G in arrays whose
// per-element blocks are multiples of 16 bytes)
template <int G, bool SH = false>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float* v) {
  if constexpr (G == 4) {
    const float4 q = ldx<SH>(reinterpret_cast<const float4*>(p));
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else if constexpr (G % 2 == 0) {
#pragma unroll
    for (int i = 0; i < G; i += 2) {
      const float2 q = ldx<SH>(reinterpret_cast<const float2*>(p + i));
      v[i] = q.x;
      v[i + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < G; ++i) v[i] = ldx<SH>(p + i);
  }
}

template <typename T>
__device__ __forceinline__ bool inv3(const T* J, T* Ji) {
  T c00 = J[4] * J[8] - J[5] * J[7];
  T c01 = J[5] * J[6] - J[3] * J[8];
  T c02 = J[3] * J[7] - J[4] * J[6];
  T det = J[0] * c00 + J[1] * c01 + J[2] * c02;
  if (!(tabs(det) > T(0))) return false;
  T id = T(1) / det;
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
__device__ __forceinline__ void matvec3(const T* M, const T* v, T* o) {
#pragma unroll
  for (int r = 0; r < 3; ++r) o[r] = M[3 * r] * v[0] + M[3 * r + 1] * v[1] + M[3 * r + 2] * v[2];
}

// ---------------------------------------------------------------------------
// element map chi(xi) = sum_abc X_abc l_a(xi1) l_b(xi2) l_c(xi3), sum-factorised
// ---------------------------------------------------------------------------

// FP32, nodes coordinate-major [3][G^3]; chi and Jacobian J[r][q] = d chi_r / d xi_q
template <int G>
__device__ __forceinline__ int corner_node(int q) {
  return ((q & 1) ? G - 1 : 0) + G * (((q & 2) ? G - 1 : 0) + G * ((q & 4) ? G - 1 : 0));
}

// FP32, nodes coordinate-major [3][G^3]; chi and Jacobian J[r][q] = d chi_r / d xi_q.
// Coordinates flagged in tm are trilinear in xi: their 8-corner form is used.
// Per-thread scratch for the per-dimension bases: SS = 0 keeps them in a
// local array (computed in a rolled loop, read through local memory); SS > 0
// puts them in shared memory at sb[row * SS] (sb: this thread's column of a
// [rows][SS] block array), which keeps local memory out of the L1 cache.
// With a shared-memory scratch (SS > 0), the small per-thread results that
// the rolled loops index at run time (chi, J, a residual, the interpolation's
// third-direction basis and its outputs) also go through rows of the scratch
// from kScratchOut on instead of through local memory (PT_SMEM_OUT = 1).
#ifndef PT_SMEM_OUT
#define PT_SMEM_OUT 1
#endif
constexpr int kScratchOut = 6 * PT_MAXG;
constexpr int kScratchRows = kScratchOut + 12;

template <int SS>
struct BasisStore {
  float* sb;
  float loc[SS > 0 ? 1 : 6 * PT_MAXG];
  __device__ __forceinline__ float* row(int r) { return SS > 0 ? sb + r * SS : loc + r; }
  __device__ __forceinline__ float get(int r) const { return SS > 0 ? sb[r * SS] : loc[r]; }
};

template <int G, int SS = 0, bool SH = false>
__device__ __forceinline__ void map_j32(const float* __restrict__ X, const float* xi, int tm,
                                        const DevConsts& k, float* chi, float* J,
                                        float* sb = nullptr) {
  constexpr int G3 = G * G * G;
  // rows d G + i: l_i(xi_d); rows (3 + d) G + i: l_i'(xi_d)
  BasisStore<SS> bs;
  bs.sb = sb;
  if (tm != 7) {
#if PT_ROLL_BASIS
#pragma unroll 1
#else
#pragma unroll
#endif
    for (int d = 0; d < 3; ++d) {
      float l[G], dl[G];
      lagr_d<G, float>(xi[d], k.gn32, k.gw32, l, dl);
#pragma unroll
      for (int i = 0; i < G; ++i) {
        *bs.row(d * G + i) = l[i];
        *bs.row((3 + d) * G + i) = dl[i];
      }
    }
  }
#define PT_L(d, i) bs.get((d) * G + (i))
#define PT_D(d, i) bs.get((3 + (d)) * G + (i))
  const float hp[3] = {0.5f * (1.f + xi[0]), 0.5f * (1.f + xi[1]), 0.5f * (1.f + xi[2])};
  const float hm[3] = {0.5f * (1.f - xi[0]), 0.5f * (1.f - xi[1]), 0.5f * (1.f - xi[2])};
  // one coordinate at a time; the loops over c and r stay rolled so that the
  // hot loop's code stays small
#pragma unroll 1
  for (int r = 0; r < 3; ++r) {
    const float* Xr = X + r * G3;
    float cr = 0.f, j0 = 0.f, j1 = 0.f, j2 = 0.f;
    if ((tm >> r) & 1) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float xv = ldx<SH>(Xr + corner_node<G>(q));
        const float a0 = (q & 1) ? hp[0] : hm[0], a1 = (q & 2) ? hp[1] : hm[1],
                    a2 = (q & 4) ? hp[2] : hm[2];
        const float s0 = (q & 1) ? 0.5f : -0.5f, s1 = (q & 2) ? 0.5f : -0.5f,
                    s2 = (q & 4) ? 0.5f : -0.5f;
        cr = fmaf(xv, a0 * a1 * a2, cr);
        j0 = fmaf(xv, s0 * a1 * a2, j0);
        j1 = fmaf(xv, a0 * s1 * a2, j1);
        j2 = fmaf(xv, a0 * a1 * s2, j2);
      }
    } else {
#pragma unroll 1
      for (int c = 0; c < G; ++c) {
        float T0 = 0.f, T1 = 0.f, T2 = 0.f;
#pragma unroll
        for (int b = 0; b < G; ++b) {
          float sv = 0.f, s1 = 0.f, row[G];
          load_row<G, SH>(Xr + G * (b + G * c), row);
#pragma unroll
          for (int a = 0; a < G; ++a) {
            sv = fmaf(row[a], PT_L(0, a), sv);
            s1 = fmaf(row[a], PT_D(0, a), s1);
          }
          T0 = fmaf(sv, PT_L(1, b), T0);
          T1 = fmaf(s1, PT_L(1, b), T1);
          T2 = fmaf(sv, PT_D(1, b), T2);
        }
        const float lc = PT_L(2, c), dc = PT_D(2, c);
        cr = fmaf(T0, lc, cr);
        j0 = fmaf(T1, lc, j0);
        j1 = fmaf(T2, lc, j1);
        j2 = fmaf(T0, dc, j2);
      }
    }
#if PT_PICK_MAP
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (q == r) {
        chi[q] = cr;
        J[3 * q] = j0;
        J[3 * q + 1] = j1;
        J[3 * q + 2] = j2;
      }
#else
    if constexpr (SS > 0 && PT_SMEM_OUT) {
      sb[(kScratchOut + r) * SS] = cr;
      sb[(kScratchOut + 3 + 3 * r) * SS] = j0;
      sb[(kScratchOut + 4 + 3 * r) * SS] = j1;
      sb[(kScratchOut + 5 + 3 * r) * SS] = j2;
    } else {
      chi[r] = cr;
      J[3 * r] = j0;
      J[3 * r + 1] = j1;
      J[3 * r + 2] = j2;
    }
#endif
  }
  if constexpr (SS > 0 && PT_SMEM_OUT && !PT_PICK_MAP) {
#pragma unroll
    for (int q = 0; q < 3; ++q) chi[q] = sb[(kScratchOut + q) * SS];
#pragma unroll
    for (int q = 0; q < 9; ++q) J[q] = sb[(kScratchOut + 3 + q) * SS];
  }
}
#undef PT_L
#undef PT_D

// FP64, nodes point-major [G^3][3]; with WJ also the Jacobian
template <int G, bool WJ>
__device__ __forceinline__ void map64(const double* __restrict__ X, const double* xi,
                                      const DevConsts& k, double* chi, double* J) {
  double l0[G], d0[G], l1[G], d1[G], l2[G], d2[G];
  if (WJ) {
    lagr_d<G, double>(xi[0], k.gn, k.gw, l0, d0);
    lagr_d<G, double>(xi[1], k.gn, k.gw, l1, d1);
    lagr_d<G, double>(xi[2], k.gn, k.gw, l2, d2);
  } else {
    lagr<G, double>(xi[0], k.gn, k.gw, l0);
    lagr<G, double>(xi[1], k.gn, k.gw, l1);
    lagr<G, double>(xi[2], k.gn, k.gw, l2);
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    chi[r] = 0.0;
    if (WJ) J[3 * r] = J[3 * r + 1] = J[3 * r + 2] = 0.0;
  }
#pragma unroll 1
  for (int c = 0; c < G; ++c) {
    double T0[3] = {0, 0, 0}, T1[3] = {0, 0, 0}, T2[3] = {0, 0, 0};
#pragma unroll 1
    for (int b = 0; b < G; ++b) {
      double s[3] = {0, 0, 0}, s1[3] = {0, 0, 0};
#pragma unroll
      for (int a = 0; a < G; ++a) {
        const double* P = X + 3 * (a + G * (b + G * c));
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          double xv = __ldg(P + r);
          s[r] = fma(xv, l0[a], s[r]);
          if (WJ) s1[r] = fma(xv, d0[a], s1[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        T0[r] = fma(s[r], l1[b], T0[r]);
        if (WJ) {
          T1[r] = fma(s1[r], l1[b], T1[r]);
          T2[r] = fma(s[r], d1[b], T2[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      chi[r] = fma(T0[r], l2[c], chi[r]);
      if (WJ) {
        J[3 * r] = fma(T1[r], l2[c], J[3 * r]);
        J[3 * r + 1] = fma(T2[r], l2[c], J[3 * r + 1]);
        J[3 * r + 2] = fma(T0[r], d2[c], J[3 * r + 2]);
      }
    }
  }
}

// trilinear start xi0 = Jc^{-1} (x_loc - xc), from the per-element table
__device__ __forceinline__ void trilinear_guess(const DevMesh& m, int e, const float* xf,
                                                float* xi) {
  const float* t = m.tri + 12 * (size_t)e;
  float r[3] = {xf[0] - __ldg(t), xf[1] - __ldg(t + 1), xf[2] - __ldg(t + 2)};
#pragma unroll
  for (int q = 0; q < 3; ++q)
    xi[q] = __ldg(t + 3 + 3 * q) * r[0] + __ldg(t + 4 + 3 * q) * r[1] + __ldg(t + 5 + 3 * q) * r[2];
}

// Full FP64 Newton: chi(xi) - x = 0, |dxi|_inf < tol (Sec. 3.2.1).
template <int G>
__device__ __forceinline__ bool newton64(const double* X64, const double* xl, double* xi,
                                         const DevConsts& k, int maxit, int& it64) {
  #pragma unroll 1
  for (int it = 0; it < maxit; ++it) {
    double chi[3], J[9], Ji[9], r[3], d[3];
    map64<G, true>(X64, xi, k, chi, J);
    if (!inv3(J, Ji)) return false;
#pragma unroll
    for (int q = 0; q < 3; ++q) r[q] = chi[q] - xl[q];
    matvec3(Ji, r, d);
#pragma unroll
    for (int q = 0; q < 3; ++q) xi[q] -= d[q];
    ++it64;
    double md = tmax3(d[0], d[1], d[2]);
    if (md < k.newton_tol) return true;
    if (!(tmax3(xi[0], xi[1], xi[2]) <= 4.0)) return false;
  }
  return false;
}

// Lagrange basis on the geometry nodes in double-float (nodes and barycentric
// weights carried as hi + lo pairs)
template <int NP>
__device__ __forceinline__ void lagr_df(df x, const DevConsts& k, df* l) {
  df d[NP];
#pragma unroll
  for (int m = 0; m < NP; ++m) d[m] = df_sub(x, df{k.gn_hi[m], k.gn_lo[m]});
  df pre = df_from(1.f);
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    l[i] = pre;
    if (i + 1 < NP) pre = df_mul(pre, d[i]);
  }
  df suf = df_from(1.f);
#pragma unroll
  for (int i = NP - 1; i >= 0; --i) {
    l[i] = df_mul(df_mul(l[i], suf), df{k.gw_hi[i], k.gw_lo[i]});
    if (i > 0) suf = df_mul(suf, d[i]);
  }
}

// Residual chi(xi) - x of the element map in double-float, sum-factorised;
// nodes as hi [3][G^3] + lo [3][G^3] (relative to the element centre);
// coordinates flagged in tm use the 8-corner trilinear form.
template <int G, int SS = 0, bool SH = false>
__device__ __forceinline__ void resid_df(const float* __restrict__ Xh,
                                         const float* __restrict__ Xl, const df* xi, int tm,
                                         const df* xloc, const DevConsts& k, float* r,
                                         float* sb = nullptr) {
  constexpr int G3 = G * G * G;
  // rows d G + i: high part of l_i(xi_d); rows (3 + d) G + i: low part
  BasisStore<SS> bs;
  bs.sb = sb;
  if (tm != 7) {
#if PT_ROLL_BASIS
#pragma unroll 1
#else
#pragma unroll
#endif
    for (int d = 0; d < 3; ++d) {
      df l[G];
      lagr_df<G>(xi[d], k, l);
#pragma unroll
      for (int i = 0; i < G; ++i) {
        *bs.row(d * G + i) = l[i].hi;
        *bs.row((3 + d) * G + i) = l[i].lo;
      }
    }
  }
#define PT_LDF(d, i) df{bs.get((d) * G + (i)), bs.get((3 + (d)) * G + (i))}
  df w8[8];
  if (tm != 0) {
    df hp[3], hm[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const df up = df_add(df_from(1.f), xi[d]);
      const df dn = df_sub(df_from(1.f), xi[d]);
      hp[d] = df{0.5f * up.hi, 0.5f * up.lo};
      hm[d] = df{0.5f * dn.hi, 0.5f * dn.lo};
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const df w01 = df_mul((q & 1) ? hp[0] : hm[0], (q & 2) ? hp[1] : hm[1]);
      w8[q] = df_mul(w01, hm[2]);
      w8[q + 4] = df_mul(w01, hp[2]);
    }
  }
#pragma unroll 1
  for (int q = 0; q < 3; ++q) {
    const float* Ph = Xh + q * G3;
    const float* Pl = Xl + q * G3;
    df_acc a3;
    dacc_init(a3);
    if ((tm >> q) & 1) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int i = corner_node<G>(c);
        dacc_fma(a3, df{ldx<SH>(Ph + i), ldx<SH>(Pl + i)}, w8[c]);
      }
    } else {
#pragma unroll 1
      for (int c = 0; c < G; ++c) {
        df_acc a2;
        dacc_init(a2);
#pragma unroll
        for (int b = 0; b < G; ++b) {
          df_acc a1;
          dacc_init(a1);
          float rh[G], rl[G];
          load_row<G, SH>(Ph + G * (b + G * c), rh);
          load_row<G, SH>(Pl + G * (b + G * c), rl);
#pragma unroll
          for (int a = 0; a < G; ++a) dacc_fma(a1, df{rh[a], rl[a]}, PT_LDF(0, a));
          dacc_fma(a2, dacc_result(a1), PT_LDF(1, b));
        }
        dacc_fma(a3, dacc_result(a2), PT_LDF(2, c));
      }
    }
#if PT_PICK_MAP
    const df rr = df_sub(dacc_result(a3), pick<3>(xloc, q));
    put<3>(r, q, __fadd_rn(rr.hi, rr.lo));
#else
    const df rr = df_sub(dacc_result(a3), xloc[q]);
    if constexpr (SS > 0 && PT_SMEM_OUT)
      sb[(kScratchOut + q) * SS] = __fadd_rn(rr.hi, rr.lo);
    else
      r[q] = __fadd_rn(rr.hi, rr.lo);
#endif
  }
  if constexpr (SS > 0 && PT_SMEM_OUT && !PT_PICK_MAP) {
#pragma unroll
    for (int q = 0; q < 3; ++q) r[q] = sb[(kScratchOut + q) * SS];
  }
#undef PT_LDF
}

// Lagrange basis at z (l) and its increment dl = l(z + dz) - l(z), the latter
// without cancellation: with f_m = z - x_m and F_m = f_m + dz, the product
// difference telescopes, prod F - prod f = dz sum_j (prod_{i<j} f_i)(prod_{i>j} F_i),
// so dl carries the relative accuracy of FP32 however small dz is.
template <int G>
__device__ __forceinline__ void lagr_inc(float z, float dz, const float* xn, const float* w,
                                         float* l, float* dl) {
  float f[G], F[G];
#pragma unroll
  for (int m = 0; m < G; ++m) {
    f[m] = z - xn[m];
    F[m] = f[m] + dz;
  }
#pragma unroll
  for (int a = 0; a < G; ++a) {
    float suf[G], sp = 1.f;
#pragma unroll
    for (int m = G - 1; m >= 0; --m) {
      suf[m] = sp;
      if (m != a) sp *= F[m];
    }
    float pre = 1.f, acc = 0.f;
#pragma unroll
    for (int m = 0; m < G; ++m) {
      if (m == a) continue;
      acc = fmaf(pre, suf[m], acc);
      pre *= f[m];
    }
    l[a] = w[a] * pre;
    dl[a] = w[a] * dz * acc;
  }
}

// Increment of the element map between two nearby points, dchi = chi(z + dz) -
// chi(z), in FP32 without cancellation: with L = l + dl the bases at z + dz,
//   prod L - prod l = dl0 L1 L2 + l0 dl1 L2 + l0 l1 dl2
// (and likewise for the 8-corner form of trilinear coordinates), so every term
// carries a factor dl and the result has FP32 relative accuracy.  Used for the
// second residual of the final Newton iterations: r(z + dz) = r(z) + dchi, with
// r(z) from the double-float residual.  Nodes: FP32 high parts, relative to the
// element centre (the low parts change dchi by ~1e-8 of itself).
template <int G, bool SH = false, int SS = 0>
__device__ __forceinline__ void map_inc32(const float* __restrict__ X, const float* z,
                                          const float* dz, int tm, const DevConsts& k,
                                          float* dchi, float* sb = nullptr) {
  constexpr int G3 = G * G * G;
  float l0[G], dl0[G], l1[G], dl1[G], l2[G], dl2[G];
  lagr_inc<G>(z[0], dz[0], k.gn32, k.gw32, l0, dl0);
  lagr_inc<G>(z[1], dz[1], k.gn32, k.gw32, l1, dl1);
  lagr_inc<G>(z[2], dz[2], k.gn32, k.gw32, l2, dl2);
  float hp[3], hm[3], dh[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    hp[d] = 0.5f * (1.f + z[d]);
    hm[d] = 0.5f * (1.f - z[d]);
    dh[d] = 0.5f * dz[d];
  }
#pragma unroll 1
  for (int q = 0; q < 3; ++q) {
    const float* Xq = X + q * G3;
    float acc = 0.f;
    if ((tm >> q) & 1) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float a0 = (c & 1) ? hp[0] : hm[0], a1 = (c & 2) ? hp[1] : hm[1],
                    a2 = (c & 4) ? hp[2] : hm[2];
        const float d0 = (c & 1) ? dh[0] : -dh[0], d1 = (c & 2) ? dh[1] : -dh[1],
                    d2 = (c & 4) ? dh[2] : -dh[2];
        const float A1 = a1 + d1, A2 = a2 + d2;
        const float dw = d0 * A1 * A2 + a0 * d1 * A2 + a0 * a1 * d2;
        acc = fmaf(ldx<SH>(Xq + corner_node<G>(c)), dw, acc);
      }
    } else {
      float t1 = 0.f, t2 = 0.f, t3 = 0.f;
#pragma unroll 1
      for (int c = 0; c < G; ++c) {
        float s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
        for (int b = 0; b < G; ++b) {
          float row[G];
          load_row<G, SH>(Xq + G * (b + G * c), row);
          float A = 0.f, B = 0.f;
#pragma unroll
          for (int a = 0; a < G; ++a) {
            A = fmaf(row[a], dl0[a], A);
            B = fmaf(row[a], l0[a], B);
          }
          s1 = fmaf(A, l1[b] + dl1[b], s1);
          s2 = fmaf(B, dl1[b], s2);
          s3 = fmaf(B, l1[b], s3);
        }
        float lc = l2[0], dc = dl2[0];
#pragma unroll
        for (int j = 1; j < G; ++j)
          if (j == c) {
            lc = l2[j];
            dc = dl2[j];
          }
        t1 = fmaf(s1, lc + dc, t1);
        t2 = fmaf(s2, lc + dc, t2);
        t3 = fmaf(s3, dc, t3);
      }
      acc = t1 + t2 + t3;
    }
#if PT_PICK_MAP
    put<3>(dchi, q, acc);
#else
    if constexpr (SS > 0 && PT_SMEM_OUT)
      sb[(kScratchOut + q) * SS] = acc;
    else
      dchi[q] = acc;
#endif
  }
  if constexpr (SS > 0 && PT_SMEM_OUT && !PT_PICK_MAP) {
#pragma unroll
    for (int q = 0; q < 3; ++q) dchi[q] = sb[(kScratchOut + q) * SS];
  }
}

template <int G>
__device__ __noinline__ bool newton64_cold(const double* X64, const double* xl, double* xi,
                                           const DevConsts& k, int& it64) {
  return newton64<G>(X64, xl, xi, k, k.max_newton, it64);
}

// Mixed-precision Newton on a double-float local position xd (relative to the
// element centre): FP32 iterations (chi and J in FP32) until the step is below
// 1e-5, then double-float residuals with the last FP32 inverse Jacobian until
// the step is below newton_tol.  Returns the double-float xi in zd; a full
// FP64 Newton is the (out-of-line) fallback.
// Xs: optional copy of the element's FP32 nodes, high parts [3][G^3], then the
// low parts from the next 16-byte boundary (read with generic loads when SH).
template <int G, int SS = 0, bool SH = false>
__device__ __forceinline__ bool newton_df(const DevMesh& m, const DevConsts& k, int e,
                                          const df* xd, const float* guess, df* zd, int& it32,
                                          int& it64, float* sb = nullptr,
                                          const float* Xs = nullptr) {
  constexpr int G3 = G * G * G;
  const float* X32 = Xs ? Xs : m.xg32 + (size_t)e * 3 * G3;
  const float* X32l = Xs ? Xs + ((3 * G3 + 3) & ~3) : m.xg32lo + (size_t)e * 3 * G3;
  const int tm = __ldg(m.tmask + e);
  float z[3] = {guess[0], guess[1], guess[2]};
  float Ji[9];
  bool have = false;
  #pragma unroll 1
  for (int it = 0; it < 8; ++it) {
    float chi[3], J[9], r[3], d[3];
    map_j32<G, SS, SH>(X32, z, tm, k, chi, J, sb);
    if (!inv3(J, Ji)) break;
    have = true;
#pragma unroll
    for (int q = 0; q < 3; ++q) r[q] = chi[q] - xd[q].hi;
    matvec3(Ji, r, d);
#pragma unroll
    for (int q = 0; q < 3; ++q) z[q] -= d[q];
    ++it32;
    if (!(tmax3(z[0], z[1], z[2]) <= 4.f)) {
      have = false;
      break;
    }
    if (tmax3(d[0], d[1], d[2]) < PT_NEWTON_SWITCH) break;
  }
  if (have) {
#pragma unroll
    for (int q = 0; q < 3; ++q) zd[q] = df_from(z[q]);
    const float tol = (float)k.newton_tol;
    // Each step needs the residual at the current iterate.  The first is the
    // double-float residual at the FP32 iterate z.  After a first step d with
    // |d| <= 4e-7 the next residual is r(z) + [chi(z - d) - chi(z)], the
    // bracket an exact FP32 increment (it carries ~1e-7 of a term of size
    // |J d|, far below the tolerance); later residuals are double-float again.
    float rp[3] = {0.f, 0.f, 0.f}, dz[3] = {0.f, 0.f, 0.f};
    bool inc = false;
#pragma unroll 1
    for (int it = 0; it < 6; ++it) {
      float r[3], d[3];
      if (inc) {
        float dchi[3];
        map_inc32<G, SH, SS>(X32, z, dz, tm, k, dchi, sb);
#pragma unroll
        for (int q = 0; q < 3; ++q) r[q] = rp[q] + dchi[q];
      } else {
        resid_df<G, SS, SH>(X32, X32l, zd, tm, xd, k, r, sb);
      }
      matvec3(Ji, r, d);
#pragma unroll
      for (int q = 0; q < 3; ++q) zd[q] = df_sub(zd[q], df_from(d[q]));
      ++it64;
      const float md = tmax3(d[0], d[1], d[2]);
      if (md < tol) return true;
      inc = it == 0 && md <= 4e-7f;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        rp[q] = r[q];
        dz[q] = -d[q];
      }
    }
  }
  // fallback: full FP64 Newton
  double xl[3], xi[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    xl[q] = df_to_double(xd[q]);
    xi[q] = have ? df_to_double(zd[q]) : (double)guess[q];
  }
  if (!(tmax3(xi[0], xi[1], xi[2]) <= 4.0)) xi[0] = xi[1] = xi[2] = 0.0;
  const bool ok = newton64_cold<G>(m.xg64 + (size_t)e * 3 * G3, xl, xi, k, it64);
#pragma unroll
  for (int q = 0; q < 3; ++q) zd[q] = df_from_double(xi[q]);
  return ok;
}

// As newton_df for a local position in FP64 (xl) and a FP64 result.
template <int G>
__device__ __forceinline__ bool newton_mixed(const DevMesh& m, const DevConsts& k, int e,
                                             const double* xl, const float* guess, double* xi,
                                             int& it32, int& it64) {
  df xd[3], zd[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) xd[q] = df_from_double(xl[q]);
  const bool ok = newton_df<G>(m, k, e, xd, guess, zd, it32, it64);
#pragma unroll
  for (int q = 0; q < 3; ++q) xi[q] = df_to_double(zd[q]);
  return ok;
}

// ---------------------------------------------------------------------------
// interpolation of rho and rho u (Eq. part_interpolation), sum-factorised
// ---------------------------------------------------------------------------

// 1: the FP32 interpolation at N = 5 takes two variables per pass (their row
// loads independent: twice the loads in flight; +5 % at the 64^3 workload)
#ifndef PT_INTERP_V2
#define PT_INTERP_V2 1
#endif
template <int NP, typename T, bool SH = false, int SS = 0>
__device__ __forceinline__ void interp4(const T* __restrict__ Ue, const T* l1, const T* l2,
                                        const T* l3, T* out, float* sb = nullptr) {
  constexpr int N3 = NP * NP * NP;
#if PT_INTERP_V2
  // two variables per pass: their row loads are independent, which doubles
  // the loads in flight per iteration
  if constexpr (std::is_same<T, float>::value && NP == 6) {
    // rows kScratchOut + kk: l3; kScratchOut + NP + v: the results
    constexpr bool kS = SS > 0 && PT_SMEM_OUT;
    if constexpr (kS) {
#pragma unroll
      for (int kk = 0; kk < NP; ++kk) sb[(kScratchOut + kk) * SS] = l3[kk];
    }
#pragma unroll 1
    for (int v = 0; v < 4; v += 2) {
      const float* Ua = Ue + v * N3;
      const float* Ub = Ua + N3;
      float acca = 0.f, accb = 0.f;
#pragma unroll 1
      for (int kk = 0; kk < NP; ++kk) {
        float ta = 0.f, tb = 0.f;
#pragma unroll
        for (int j = 0; j < NP; j += 2) {
          const float4* qa = reinterpret_cast<const float4*>(Ua + NP * (j + NP * kk));
          const float4* qb = reinterpret_cast<const float4*>(Ub + NP * (j + NP * kk));
          const float4 a0 = ldx<SH>(qa), a1 = ldx<SH>(qa + 1), a2 = ldx<SH>(qa + 2);
          const float4 b0 = ldx<SH>(qb), b1 = ldx<SH>(qb + 1), b2 = ldx<SH>(qb + 2);
          const float ra0[6] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y};
          const float ra1[6] = {a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
          const float rb0[6] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y};
          const float rb1[6] = {b1.z, b1.w, b2.x, b2.y, b2.z, b2.w};
          float sa0 = 0.f, sa1 = 0.f, sb0 = 0.f, sb1 = 0.f;
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            sa0 = fmaf(ra0[i], l1[i], sa0);
            sa1 = fmaf(ra1[i], l1[i], sa1);
            sb0 = fmaf(rb0[i], l1[i], sb0);
            sb1 = fmaf(rb1[i], l1[i], sb1);
          }
          ta = fmaf(sa0, l2[j], ta);
          ta = fmaf(sa1, l2[j + 1], ta);
          tb = fmaf(sb0, l2[j], tb);
          tb = fmaf(sb1, l2[j + 1], tb);
        }
        const float lk = kS ? sb[(kScratchOut + kk) * SS] : l3[kk];
        acca = fmaf(ta, lk, acca);
        accb = fmaf(tb, lk, accb);
      }
      if constexpr (kS) {
        sb[(kScratchOut + NP + v) * SS] = acca;
        sb[(kScratchOut + NP + 1 + v) * SS] = accb;
      } else {
        out[v] = acca;
        out[v + 1] = accb;
      }
    }
    if constexpr (kS) {
#pragma unroll
      for (int v = 0; v < 4; ++v) out[v] = sb[(kScratchOut + NP + v) * SS];
    }
    return;
  }
#endif
  // FP32 rows of 6 nodes: two rows (48 bytes, 16-byte aligned at even rows
  // since every variable block is a multiple of 16 bytes) in three 16-byte
  // loads; rows of 4 or 8 nodes in 16-byte loads
  constexpr bool kPair = std::is_same<T, float>::value && NP == 6;
#pragma unroll 1
  for (int v = 0; v < 4; ++v) {
    const T* Uv = Ue + v * N3;
    T acc = T(0);
#pragma unroll 1
    for (int kk = 0; kk < NP; ++kk) {
      T t2 = T(0);
      if constexpr (kPair) {
#pragma unroll
        for (int j = 0; j < NP; j += 2) {
          const float4* q = reinterpret_cast<const float4*>(Uv + NP * (j + NP * kk));
          const float4 q0 = ldx<SH>(q), q1 = ldx<SH>(q + 1), q2 = ldx<SH>(q + 2);
          const float r0[6] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y};
          const float r1[6] = {q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
          T t1 = T(0), u1 = T(0);
#pragma unroll
          for (int i = 0; i < NP; ++i) t1 = tfma((T)r0[i], l1[i], t1);
#pragma unroll
          for (int i = 0; i < NP; ++i) u1 = tfma((T)r1[i], l1[i], u1);
          t2 = tfma(t1, l2[j], t2);
          t2 = tfma(u1, l2[j + 1], t2);
        }
      } else {
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          const T* row = Uv + NP * (j + NP * kk);
          T t1 = T(0);
          if constexpr (std::is_same<T, float>::value && NP % 4 == 0) {
#pragma unroll
            for (int i = 0; i < NP; i += 4) {
              const float4 q = ldx<SH>(reinterpret_cast<const float4*>(row + i));
              t1 = tfma((T)q.x, l1[i], t1);
              t1 = tfma((T)q.y, l1[i + 1], t1);
              t1 = tfma((T)q.z, l1[i + 2], t1);
              t1 = tfma((T)q.w, l1[i + 3], t1);
            }
          } else if constexpr (std::is_same<T, float>::value && NP % 2 == 0) {
            float rv[NP];
            load_row<NP, SH>(reinterpret_cast<const float*>(row), rv);
#pragma unroll
            for (int i = 0; i < NP; ++i) t1 = tfma((T)rv[i], l1[i], t1);
          } else {
#pragma unroll
            for (int i = 0; i < NP; ++i) t1 = tfma(ldx<SH>(row + i), l1[i], t1);
          }
          t2 = tfma(t1, l2[j], t2);
        }
      }
#if PT_PICK_INTERP
      acc = tfma(t2, pick<NP>(l3, kk), acc);
    }
    put<4>(out, v, acc);
#else
      acc = tfma(t2, l3[kk], acc);
    }
    out[v] = acc;
#endif
  }
}

// power in the working precision
__device__ __forceinline__ float tpow(float a, float b) { return powf(a, b); }
__device__ __forceinline__ double tpow(double a, double b) { return pow(a, b); }

// drag factor f_D (Sec. 2.2): 1 (Stokes), 1 + 0.15 Re_p^0.687 (Schiller-
// Naumann) or 1 + A Re^B + (Re/24) C / (1 + D/Re) (Haider-Levenspiel, A..D in
// k.hl); called for laws 1 and 2
template <typename T>
__device__ __forceinline__ T drag_factor(const DevConsts& k, T re) {
  if (k.drag_law == 1) return T(1) + T(0.15) * tpow(re, T(0.687));
  if (!(re > T(0))) return T(1);
  return T(1) + (T)k.hl[0] * tpow(re, (T)k.hl[1]) +
         re / T(24) * (T)k.hl[2] / (T(1) + (T)k.hl[3] / re);
}

// ---------------------------------------------------------------------------
// tracking (Secs. 3.2.3-3.2.4, 2.4)
// ---------------------------------------------------------------------------

// Node (mm, kk) of local face f is base + mm sm + kk sk (mm along the face's
// first in-plane direction, kk along its second).
template <int G>
__device__ __forceinline__ void face_strides(int f, int& base, int& sm, int& sk) {
  const int fixed = (f & 1) ? G - 1 : 0;
  const int dir = f >> 1;
  base = fixed * (dir == 0 ? 1 : dir == 1 ? G : G * G);
  sm = dir == 0 ? G : 1;
  sk = dir == 2 ? G : G * G;
}

// curved face p(s,t) and its tangents from the element's Lagrange nodes
template <int G>
__device__ __forceinline__ void face_eval(const double* X64, int f, double s, double t,
                                          const DevConsts& k, double* p, double* ps,
                                          double* pt) {
  double ls[G], ds[G], lt[G], dt[G];
  lagr_d<G, double>(s, k.gn, k.gw, ls, ds);
  lagr_d<G, double>(t, k.gn, k.gw, lt, dt);
#pragma unroll
  for (int r = 0; r < 3; ++r) p[r] = ps[r] = pt[r] = 0.0;
  int base, sm, sk;
  face_strides<G>(f, base, sm, sk);
#pragma unroll
  for (int kk = 0; kk < G; ++kk)
#pragma unroll
    for (int mm = 0; mm < G; ++mm) {
      const double* P = X64 + 3 * (base + mm * sm + kk * sk);
      double w = ls[mm] * lt[kk], wsv = ds[mm] * lt[kk], wtv = ls[mm] * dt[kk];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        double xv = __ldg(P + r);
        p[r] = fma(xv, w, p[r]);
        ps[r] = fma(xv, wsv, ps[r]);
        pt[r] = fma(xv, wtv, pt[r]);
      }
    }
}

__device__ __forceinline__ void cross3d(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot3d(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Roots of the ray (origin xs, unit direction td, frame n1, n2) with the
// bilinear patch p(s,t) = a st + b s + c t + d: the two plane equations
// n_k.(p - xs) = 0 are eliminated to one quadratic (Ramsey et al. 2004).
// Writes up to 2 (s, t, alpha) triples; returns their number.
__device__ __forceinline__ int bilinear_roots(const double* B, const double* xs, const double* td,
                                              const double* n1, const double* n2, double* rs,
                                              double* rt, double* ra) {
  const double* a = B;
  const double* b = B + 3;
  const double* c = B + 6;
  double dd[3] = {B[9] - xs[0], B[10] - xs[1], B[11] - xs[2]};
  double A1 = dot3d(n1, a), B1 = dot3d(n1, b), C1 = dot3d(n1, c), D1 = dot3d(n1, dd);
  double A2 = dot3d(n2, a), B2 = dot3d(n2, b), C2 = dot3d(n2, c), D2 = dot3d(n2, dd);
  double scl = fabs(A1) + fabs(B1) + fabs(C1) + fabs(D1) + fabs(A2) + fabs(B2) + fabs(C2) +
               fabs(D2);
  if (!(scl > 0.0)) return 0;
  int nr = 0;
  #pragma unroll 1
  for (int pass = 0; pass < 2 && nr == 0; ++pass) {
    // pass 0 eliminates t (quadratic in s), pass 1 eliminates s (quadratic in t)
    double P1 = pass ? C1 : B1, Q1 = pass ? B1 : C1, P2 = pass ? C2 : B2, Q2 = pass ? B2 : C2;
    double q2 = P1 * A2 - P2 * A1;
    double q1 = P1 * Q2 + D1 * A2 - P2 * Q1 - D2 * A1;
    double q0 = D1 * Q2 - D2 * Q1;
    double r[2];
    int k = 0;
    if (fabs(q2) <= 1e-14 * scl * scl) {
      if (fabs(q1) > 0.0) r[k++] = -q0 / q1;
    } else {
      double disc = q1 * q1 - 4.0 * q2 * q0;
      if (disc >= 0.0) {
        double sq = sqrt(disc);
        double qq = -0.5 * (q1 + (q1 >= 0.0 ? sq : -sq));
        if (qq != 0.0) {
          r[k++] = qq / q2;
          r[k++] = q0 / qq;
        } else {
          r[k++] = 0.0;
        }
      }
    }
    #pragma unroll 1
    for (int i = 0; i < k; ++i) {
      double u = r[i];
      double den1 = A1 * u + Q1, den2 = A2 * u + Q2, w;
      if (fabs(den1) >= fabs(den2)) {
        if (fabs(den1) <= 1e-14 * scl) continue;
        w = -(P1 * u + D1) / den1;
      } else {
        if (fabs(den2) <= 1e-14 * scl) continue;
        w = -(P2 * u + D2) / den2;
      }
      double s = pass ? w : u, t = pass ? u : w;
      double pp[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) pp[q] = a[q] * s * t + b[q] * s + c[q] * t + B[9 + q] - xs[q];
      rs[nr] = s;
      rt[nr] = t;
      ra[nr] = dot3d(td, pp);
      nr++;
    }
  }
  return nr;
}

// FP32 version of bilinear_roots used to screen faces before the exact FP64
// solve; sets ill when a root is ill-conditioned in FP32 (near-tangent ray,
// vanishing denominator), in which case the caller must not trust it.
__device__ __forceinline__ int bilinear_roots_f32(const float* B, const float* xs, const float* td,
                                                  const float* n1, const float* n2, float* rs,
                                                  float* rt, float* ra, bool& ill) {
  const float* a = B;
  const float* b = B + 3;
  const float* c = B + 6;
  const float dd[3] = {B[9] - xs[0], B[10] - xs[1], B[11] - xs[2]};
  auto dot = [](const float* u, const float* w) { return u[0] * w[0] + u[1] * w[1] + u[2] * w[2]; };
  const float A1 = dot(n1, a), B1 = dot(n1, b), C1 = dot(n1, c), D1 = dot(n1, dd);
  const float A2 = dot(n2, a), B2 = dot(n2, b), C2 = dot(n2, c), D2 = dot(n2, dd);
  const float scl = fabsf(A1) + fabsf(B1) + fabsf(C1) + fabsf(D1) + fabsf(A2) + fabsf(B2) +
                    fabsf(C2) + fabsf(D2);
  if (!(scl > 0.f)) {
    ill = true;
    return 0;
  }
  const float q2 = B1 * A2 - B2 * A1;
  const float q1 = B1 * C2 + D1 * A2 - B2 * C1 - D2 * A1;
  const float q0 = D1 * C2 - D2 * C1;
  float r[2];
  int k = 0;
  if (fabsf(q2) <= 1e-4f * scl * scl) {
    if (fabsf(q1) <= 1e-3f * scl * scl) {
      ill = true;
      return 0;
    }
    r[k++] = -q0 / q1;
  } else {
    const float disc = q1 * q1 - 4.f * q2 * q0;
    if (fabsf(disc) <= 1e-3f * q1 * q1 + 1e-6f * scl * scl * scl * scl) ill = true;
    if (disc >= 0.f) {
      const float sq = sqrtf(disc);
      const float qq = -0.5f * (q1 + (q1 >= 0.f ? sq : -sq));
      if (qq != 0.f) {
        r[k++] = qq / q2;
        r[k++] = q0 / qq;
      } else {
        ill = true;
      }
    }
  }
  int nr = 0;
  for (int i = 0; i < k; ++i) {
    const float u = r[i];
    const float den1 = A1 * u + C1, den2 = A2 * u + C2;
    const bool use1 = fabsf(den1) >= fabsf(den2);
    const float den = use1 ? den1 : den2;
    if (fabsf(den) <= 1e-3f * scl) {
      ill = true;
      continue;
    }
    const float w = -((use1 ? B1 : B2) * u + (use1 ? D1 : D2)) / den;
    float pp[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) pp[q] = a[q] * u * w + b[q] * u + c[q] * w + dd[q];
    rs[nr] = u;
    rt[nr] = w;
    ra[nr] = dot(td, pp);
    nr++;
  }
  return nr;
}

// FP32 Newton on F(s,t,alpha) = p(s,t) - xs - alpha td for a curved face, from
// the element's FP32 nodes (coordinate-major); false if it does not settle.
template <int G>
__device__ __forceinline__ bool curved_newton_f32(const float* __restrict__ X32, int f,
                                                  const float* xs, const float* td,
                                                  const DevConsts& k, float& s, float& t,
                                                  float& al) {
  constexpr int G3 = G * G * G;
  #pragma unroll 1
  for (int it = 0; it < 12; ++it) {
    float ls[G], ds[G], lt[G], dt[G];
    lagr_d<G, float>(s, k.gn32, k.gw32, ls, ds);
    lagr_d<G, float>(t, k.gn32, k.gw32, lt, dt);
    float p[3] = {0, 0, 0}, ps[3] = {0, 0, 0}, pt[3] = {0, 0, 0};
    int base, sm, sk;
    face_strides<G>(f, base, sm, sk);
#pragma unroll
    for (int kk = 0; kk < G; ++kk)
#pragma unroll
      for (int mm = 0; mm < G; ++mm) {
        const int q = base + mm * sm + kk * sk;
        const float w = ls[mm] * lt[kk], wsv = ds[mm] * lt[kk], wtv = ls[mm] * dt[kk];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const float xv = __ldg(X32 + r * G3 + q);
          p[r] = fmaf(xv, w, p[r]);
          ps[r] = fmaf(xv, wsv, ps[r]);
          pt[r] = fmaf(xv, wtv, pt[r]);
        }
      }
    float F[3], J[9], Ji[9], dl[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      F[r] = p[r] - xs[r] - al * td[r];
      J[3 * r] = ps[r];
      J[3 * r + 1] = pt[r];
      J[3 * r + 2] = -td[r];
    }
    if (!inv3(J, Ji)) return false;
    matvec3(Ji, F, dl);
    s -= dl[0];
    t -= dl[1];
    al -= dl[2];
    if (fabsf(dl[0]) < 1e-5f && fabsf(dl[1]) < 1e-5f) return true;
    if (!(fabsf(s) < 3.f && fabsf(t) < 3.f)) return false;
  }
  return false;
}

// curved face point p(s,t) alone (FP64), sum-factorised
template <int G>
__device__ __forceinline__ void face_point(const double* X64, int f, double s, double t,
                                           const DevConsts& k, double* p) {
  double ls[G], lt[G];
  lagr<G, double>(s, k.gn, k.gw, ls);
  lagr<G, double>(t, k.gn, k.gw, lt);
  int base, sm, sk;
  face_strides<G>(f, base, sm, sk);
  p[0] = p[1] = p[2] = 0.0;
#pragma unroll
  for (int kk = 0; kk < G; ++kk) {
    double q[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int mm = 0; mm < G; ++mm) {
      const double* P = X64 + 3 * (base + mm * sm + kk * sk);
#pragma unroll
      for (int r = 0; r < 3; ++r) q[r] = fma(__ldg(P + r), ls[mm], q[r]);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) p[r] = fma(q[r], lt[kk], p[r]);
  }
}

// Newton on F(s,t,alpha) = p(s,t) - xs - alpha td for a curved face, started
// from a bilinear root: FP32 iterations on the FP32 nodes until the step is
// below 1e-5, then FP64 residuals with the last FP32 inverse Jacobian (each
// such step gains about six digits) until the step is below 1e-14; a full
// FP64 Newton if either stage does not settle.  Returns true on convergence.
template <int G>
__device__ __forceinline__ bool curved_refine(const double* X64, const float* __restrict__ X32,
                                              int f, const double* xs, const double* td,
                                              const DevConsts& k, double& s, double& t,
                                              double& al, double L) {
  constexpr int G3 = G * G * G;
  {
    float sf = (float)s, tf = (float)t, af = (float)al;
    const float xsf[3] = {(float)xs[0], (float)xs[1], (float)xs[2]};
    const float tdf[3] = {(float)td[0], (float)td[1], (float)td[2]};
    const float atol = 1e-5f * ((float)L + 1.f);
    int base, sm, sk;
    face_strides<G>(f, base, sm, sk);
    float Ji[9];
    bool ok32 = false;
#pragma unroll 1
    for (int it = 0; it < 12; ++it) {
      float ls[G], ds[G], lt[G], dt[G];
      lagr_d<G, float>(sf, k.gn32, k.gw32, ls, ds);
      lagr_d<G, float>(tf, k.gn32, k.gw32, lt, dt);
      float p[3] = {0, 0, 0}, ps[3] = {0, 0, 0}, pt[3] = {0, 0, 0};
#pragma unroll
      for (int kk = 0; kk < G; ++kk)
#pragma unroll
        for (int mm = 0; mm < G; ++mm) {
          const int q = base + mm * sm + kk * sk;
          const float w = ls[mm] * lt[kk], wsv = ds[mm] * lt[kk], wtv = ls[mm] * dt[kk];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const float xv = __ldg(X32 + r * G3 + q);
            p[r] = fmaf(xv, w, p[r]);
            ps[r] = fmaf(xv, wsv, ps[r]);
            pt[r] = fmaf(xv, wtv, pt[r]);
          }
        }
      float F[3], J[9], dl[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        F[r] = p[r] - xsf[r] - af * tdf[r];
        J[3 * r] = ps[r];
        J[3 * r + 1] = pt[r];
        J[3 * r + 2] = -tdf[r];
      }
      if (!inv3(J, Ji)) break;
      matvec3(Ji, F, dl);
      sf -= dl[0];
      tf -= dl[1];
      af -= dl[2];
      if (fabsf(dl[0]) < 1e-5f && fabsf(dl[1]) < 1e-5f && fabsf(dl[2]) < atol) {
        ok32 = true;
        break;
      }
      if (!(fabsf(sf) < 3.f && fabsf(tf) < 3.f)) break;
    }
    if (ok32) {
      double sd = sf, tq = tf, ad = af;
#pragma unroll 1
      for (int it = 0; it < 4; ++it) {
        double p[3];
        face_point<G>(X64, f, sd, tq, k, p);
        float Fr[3], dl[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) Fr[r] = (float)(p[r] - xs[r] - ad * td[r]);
        matvec3(Ji, Fr, dl);
        sd -= dl[0];
        tq -= dl[1];
        ad -= dl[2];
        if (fabs(dl[0]) < 1e-14 && fabs(dl[1]) < 1e-14 && fabs(dl[2]) < 1e-14 * (L + 1.0)) {
          s = sd;
          t = tq;
          al = ad;
          return true;
        }
      }
    }
  }
#pragma unroll 1
  for (int it = 0; it < 20; ++it) {
    double p[3], ps[3], pt[3], F[3], J[9], Ji[9], dl[3];
    face_eval<G>(X64, f, s, t, k, p, ps, pt);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      F[r] = p[r] - xs[r] - al * td[r];
      J[3 * r] = ps[r];
      J[3 * r + 1] = pt[r];
      J[3 * r + 2] = -td[r];
    }
    if (!inv3(J, Ji)) return false;
    matvec3(Ji, F, dl);
    s -= dl[0];
    t -= dl[1];
    al -= dl[2];
    if (fabs(dl[0]) < 1e-14 && fabs(dl[1]) < 1e-14 && fabs(dl[2]) < 1e-14 * (L + 1.0))
      return true;
    if (!(fabs(s) < 3.0 && fabs(t) < 3.0)) return false;
  }
  return false;
}

// ---------------------------------------------------------------------------
// Bezier clipping (Sec. 3.2.4; Nishita, Sederberg & Kakimoto 1990)
// ---------------------------------------------------------------------------

// x-range where the convex hull of the points (x_i, y_i) meets y = 0: the hull
// meets the axis exactly where some segment between two of its points does.
__device__ __forceinline__ bool hull_axis(const double* x, const double* y, int n, double& lo,
                                          double& hi) {
  lo = 1e300;
  hi = -1e300;
  for (int i = 0; i < n; ++i) {
    if (y[i] == 0.0) {
      lo = fmin(lo, x[i]);
      hi = fmax(hi, x[i]);
    }
    for (int j = i + 1; j < n; ++j)
      if ((y[i] < 0.0 && y[j] > 0.0) || (y[i] > 0.0 && y[j] < 0.0)) {
        const double xc = x[i] + (x[j] - x[i]) * (y[i] / (y[i] - y[j]));
        lo = fmin(lo, xc);
        hi = fmax(hi, xc);
      }
  }
  return lo <= hi;
}

// Control values of a tensor Bernstein polynomial restricted to [a, b] in its
// first (dir 0) or second (dir 1) parameter, by two de Casteljau splits.
template <int G>
__device__ __forceinline__ void bz_restrict(double (&D)[G][G], int dir, double a, double b) {
  for (int l = 0; l < G; ++l) {
    double c[G];
    for (int i = 0; i < G; ++i) c[i] = dir == 0 ? D[i][l] : D[l][i];
    // [0, b]: the left control points of the split at b
    double w[G], left[G];
    for (int i = 0; i < G; ++i) w[i] = c[i];
    for (int r = 0; r < G; ++r) {
      left[r] = w[0];
      for (int i = 0; i + 1 < G - r; ++i) w[i] = (1.0 - b) * w[i] + b * w[i + 1];
    }
    // [a/b, 1] of that: the right control points of the split at a/b
    const double t = b > 0.0 ? a / b : 0.0;
    for (int i = 0; i < G; ++i) w[i] = left[i];
    for (int r = 0; r < G; ++r) {
      c[G - 1 - r] = w[G - 1 - r];
      for (int i = 0; i + 1 < G - r; ++i) w[i] = (1.0 - t) * w[i] + t * w[i + 1];
    }
    for (int i = 0; i < G; ++i) {
      if (dir == 0)
        D[i][l] = c[i];
      else
        D[l][i] = c[i];
    }
  }
}

// Interval of the first (dir 0) or second (dir 1) parameter in [0, 1] outside
// which the Bernstein polynomial with control values D has no zero.
template <int G>
__device__ __forceinline__ bool bz_clip(const double (&D)[G][G], int dir, double& lo,
                                        double& hi) {
  double x[2 * G], y[2 * G];
  for (int i = 0; i < G; ++i) {
    double mn = 1e300, mx = -1e300;
    for (int l = 0; l < G; ++l) {
      const double v = dir == 0 ? D[i][l] : D[l][i];
      mn = fmin(mn, v);
      mx = fmax(mx, v);
    }
    x[2 * i] = x[2 * i + 1] = G > 1 ? (double)i / (G - 1) : 0.0;
    y[2 * i] = mn;
    y[2 * i + 1] = mx;
  }
  if (!hull_axis(x, y, 2 * G, lo, hi)) return false;
  lo = fmax(0.0, lo - 1e-12);
  hi = fmin(1.0, hi + 1e-12);
  return lo <= hi;
}

// All crossings of the line xs + alpha td (frame n1, n2 normal to td) with a
// curved face, by Bezier clipping: the face's control net is projected on the
// two planes through the line, and the parameter domain is cut to where the
// convex hulls of both projections can vanish, in s and in t; a domain whose
// area does not at least halve is split in two, and pending domains wait on a
// stack of parameter boxes (their nets are restricted again from the face's).
// A domain below 1e-9 gives a candidate, refined by curved_refine (kept as it
// is if the refinement does not settle).  Writes up to maxr (s, t, alpha) with
// s, t in [-1, 1]; returns their number.
template <int G>
__device__ __noinline__ int bezier_clip_roots(const double* X64, const float* X32, int f,
                                              const double* xs, const double* td,
                                              const double* n1, const double* n2,
                                              const DevConsts& k, double L, double* rs,
                                              double* rt, double* ra, int maxr) {
  constexpr int kStack = 24;
  double full[2][G][G];
  int base, sm, sk;
  face_strides<G>(f, base, sm, sk);
  for (int i = 0; i < G; ++i)
    for (int j = 0; j < G; ++j) {
      double c[3] = {0.0, 0.0, 0.0};
      for (int mm = 0; mm < G; ++mm)
        for (int kk = 0; kk < G; ++kk) {
          const double w = k.gbz[i * G + mm] * k.gbz[j * G + kk];
          const double* P = X64 + 3 * (base + mm * sm + kk * sk);
          for (int r = 0; r < 3; ++r) c[r] = fma(w, __ldg(P + r), c[r]);
        }
      const double q[3] = {c[0] - xs[0], c[1] - xs[1], c[2] - xs[2]};
      full[0][i][j] = n1[0] * q[0] + n1[1] * q[1] + n1[2] * q[2];
      full[1][i][j] = n2[0] * q[0] + n2[1] * q[1] + n2[2] * q[2];
    }
  double box[kStack][4];
  box[0][0] = 0.0;
  box[0][1] = 1.0;
  box[0][2] = 0.0;
  box[0][3] = 1.0;
  int top = 1, nr = 0;
#pragma unroll 1
  for (int visit = 0; visit < 600 && top > 0; ++visit) {
    --top;
    double u0 = box[top][0], u1 = box[top][1], v0 = box[top][2], v1 = box[top][3];
    double D[2][G][G];
    for (int w = 0; w < 2; ++w) {
      for (int i = 0; i < G; ++i)
        for (int j = 0; j < G; ++j) D[w][i][j] = full[w][i][j];
      bz_restrict<G>(D[w], 0, u0, u1);
      bz_restrict<G>(D[w], 1, v0, v1);
    }
    bool split = true;
#pragma unroll 1
    for (int it = 0; it < 16; ++it) {
      double ulo = 0.0, uhi = 1.0, vlo = 0.0, vhi = 1.0;
      bool hit = true;
      for (int w = 0; w < 2 && hit; ++w) {
        double a, b;
        hit = bz_clip<G>(D[w], 0, a, b);
        ulo = fmax(ulo, a);
        uhi = fmin(uhi, b);
        hit = hit && ulo <= uhi;
      }
      for (int w = 0; w < 2 && hit; ++w) {
        double a, b;
        hit = bz_clip<G>(D[w], 1, a, b);
        vlo = fmax(vlo, a);
        vhi = fmin(vhi, b);
        hit = hit && vlo <= vhi;
      }
      if (!hit) {
        split = false;
        break;
      }
      const double wu = u1 - u0, wv = v1 - v0;
      for (int w = 0; w < 2; ++w) {
        bz_restrict<G>(D[w], 0, ulo, uhi);
        bz_restrict<G>(D[w], 1, vlo, vhi);
      }
      u1 = u0 + wu * uhi;
      u0 = u0 + wu * ulo;
      v1 = v0 + wv * vhi;
      v0 = v0 + wv * vlo;
      if (u1 - u0 < 1e-9 && v1 - v0 < 1e-9) {
        double s = u0 + u1 - 1.0, t = v0 + v1 - 1.0;  // 2 * midpoint - 1
        double p[3];
        face_point<G>(X64, f, s, t, k, p);
        double al = td[0] * (p[0] - xs[0]) + td[1] * (p[1] - xs[1]) + td[2] * (p[2] - xs[2]);
        double s2 = s, t2 = t, al2 = al;
        if (curved_refine<G>(X64, X32, f, xs, td, k, s2, t2, al2, L) &&
            fabs(s2 - s) < 1e-6 && fabs(t2 - t) < 1e-6) {
          s = s2;
          t = t2;
          al = al2;
        }
        bool dup = false;
        for (int q = 0; q < nr; ++q)
          if (fabs(rs[q] - s) < 1e-9 && fabs(rt[q] - t) < 1e-9) dup = true;
        if (!dup && nr < maxr) {
          rs[nr] = s;
          rt[nr] = t;
          ra[nr] = al;
          ++nr;
        }
        split = false;
        break;
      }
      if ((uhi - ulo) * (vhi - vlo) > 0.5) break;  // little progress: split
    }
    if (split && top + 2 <= kStack) {
      // halve the longer side of the current box
      double b0[4] = {u0, u1, v0, v1}, b1[4] = {u0, u1, v0, v1};
      if (u1 - u0 >= v1 - v0) {
        b0[1] = b1[0] = 0.5 * (u0 + u1);
      } else {
        b0[3] = b1[2] = 0.5 * (v0 + v1);
      }
      for (int q = 0; q < 4; ++q) {
        box[top][q] = b1[q];
        box[top + 1][q] = b0[q];
      }
      top += 2;
    }
  }
  return nr;
}

template <typename R>
__device__ __forceinline__ void reflect3(R* a, const double* n) {
  double s = 2.0 * ((double)a[0] * n[0] + (double)a[1] * n[1] + (double)a[2] * n[2]);
#pragma unroll
  for (int r = 0; r < 3; ++r) a[r] = (R)((double)a[r] - s * n[r]);
}

struct TrackCounters {
  int cross, hits, slow;
};

// Conservative FP32 test: can the segment a -> b (element-local coordinates,
// extended by the band) touch any face of element e?  Slab of face f:
// lo <= n.(P - ce) <= hi for every point of the face, margins (band plus
// 4e-6 of the element radius, which covers the FP32 rounding of a and b while
// they stay within 8 radii) included; longer segments take the exact path.
__device__ __forceinline__ bool touches_any_slab(const DevMesh& m, int e, const float* a,
                                                 const float* b) {
  const float4* S = reinterpret_cast<const float4*>(m.slab + 48 * (size_t)e);
  const float rlim = 8.f * __ldg(m.slab + 48 * (size_t)e + 5);
  bool hit = !(fmaxf(fmaxf(fabsf(b[0]), fabsf(b[1])), fabsf(b[2])) <= rlim);
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    float4 s0 = __ldg(S + 2 * f), s1 = __ldg(S + 2 * f + 1);
    float pa = s0.x * a[0] + s0.y * a[1] + s0.z * a[2];
    float pb = s0.x * b[0] + s0.y * b[1] + s0.z * b[2];
    hit |= (fmaxf(pa, pb) >= s0.w) && (fminf(pa, pb) <= s1.x);
  }
  return hit;
}

// As touches_any_slab, with the kind of face: bit 0 some face (or a long
// segment), bit 1 a wall or open face (or a long segment).  Slab word 7 flags
// the wall and open faces.
__device__ __forceinline__ int slab_touch(const DevMesh& m, int e, const float* a,
                                          const float* b) {
  const float4* S = reinterpret_cast<const float4*>(m.slab + 48 * (size_t)e);
  const float rlim = 8.f * __ldg(m.slab + 48 * (size_t)e + 5);
  int t = (fmaxf(fmaxf(fabsf(b[0]), fabsf(b[1])), fabsf(b[2])) <= rlim) ? 0 : 3;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    float4 s0 = __ldg(S + 2 * f), s1 = __ldg(S + 2 * f + 1);
    float pa = s0.x * a[0] + s0.y * a[1] + s0.z * a[2];
    float pb = s0.x * b[0] + s0.y * b[1] + s0.z * b[2];
    if ((fmaxf(pa, pb) >= s0.w) && (fminf(pa, pb) <= s1.x)) t |= s1.w != 0.f ? 3 : 1;
  }
  return t;
}

// Tracks the stage segment x -> xe through the mesh.  The ray
// x(alpha) = xs + alpha td, alpha in (a0, L] (Eq. parttrajectory) is tested
// against every face of the current element except the entry face; the
// smallest accepted alpha wins (lowest face index on ties).  Internal face:
// continue in the neighbour on the same ray.  Periodic: same, translated.
// Wall: restart at the hit point with the remaining length, mirroring the
// direction, v, kx and kv by I - 2 n n^T (Sec. 2.4).  Open: stop there.
template <int G, typename R, bool CLIP = false>
__device__ __noinline__ void track_slow(const DevMesh& m, const DevConsts& k, int& e, double* x,
                                        double* xe, R* v, R* kx, R* kv, int& hits, unsigned& st,
                                        TrackCounters& tc);

// a, b: segment ends relative to the element centre in FP32 (for the test only)
template <int G, typename R>
__device__ __forceinline__ void track(const DevMesh& m, const DevConsts& k, int& e, double* x,
                                      double* xe, const float* a, const float* b, R* v, R* kx,
                                      R* kv, int& hits, unsigned& st, TrackCounters& tc) {
  if (!touches_any_slab(m, e, a, b)) {
#pragma unroll
    for (int r = 0; r < 3; ++r) x[r] = xe[r];
    return;
  }
  track_slow<G, R>(m, k, e, x, xe, v, kx, kv, hits, st, tc);
}

// Big side of a mortar (Sec. 3.2.3): the crossing found on the big face is
// searched again on the small faces matched to it -- their own tables and
// geometry, the same ray (a root finder that reports every crossing needs no
// inverted ray) -- and the small face whose accepted crossing lies closest to
// the big face's one (lowest index on ties) becomes the entry face.  If none
// reports it (a rounding-size gap at the small faces' shared edges), the small
// face whose part of the big face holds the big face's crossing parameters
// (bs, bt) is taken.  Out of line: mortar crossings are rare.
template <int G, bool CLIP>
__device__ __noinline__ void mortar_enter(const DevMesh& m, const DevConsts& k, int row, double bs,
                                          double bt, const double* xs, const double* td,
                                          const double* n1, const double* n2, double L, double a0,
                                          double best, int& e, int& fin, double& anew,
                                          unsigned& st) {
  const int* mt = m.mort + 9 * (size_t)row;
  const int type = __ldg(mt);
  const int ns = type == PT_MORTAR_FOUR ? 4 : 2;
  int kb = -1;
  double db = 1e300, ka = best, km = 1.0;
#pragma unroll 1
  for (int q = 0; q < ns; ++q) {
    const int es = __ldg(mt + 1 + q), fs = __ldg(mt + 5 + q);
    const double* ce = m.ce + 3 * (size_t)es;
    const double xl[3] = {xs[0] - __ldg(ce), xs[1] - __ldg(ce + 1), xs[2] - __ldg(ce + 2)};
    const double* X64 = m.xg64 + (size_t)es * 3 * G * G * G;
    const float* X32 = m.xg32 + (size_t)es * 3 * G * G * G;
    const int kind = finfo_kind(__ldg(m.finfo + 6 * (size_t)es + fs));
    constexpr int MR = CLIP ? 4 : 2;
    double rs[MR], rt[MR], ra[MR];
    int nr;
    if (CLIP && kind == PT_FACE_CURVED) {
      nr = bezier_clip_roots<G>(X64, X32, fs, xl, td, n1, n2, k, L, rs, rt, ra, MR);
    } else {
      const double* Bf = m.bil + 72 * (size_t)es + 12 * fs;
      double Bl[12];
#pragma unroll
      for (int i = 0; i < 12; ++i) Bl[i] = __ldg(Bf + i);
      nr = bilinear_roots(Bl, xl, td, n1, n2, rs, rt, ra);
      if (kind == PT_FACE_CURVED) {
        int kk = 0;
#pragma unroll 1
        for (int i = 0; i < nr; ++i) {
          double s = rs[i], t = rt[i], al = ra[i];
          if (!(fabs(s) < 2.0 && fabs(t) < 2.0)) continue;
          if (curved_refine<G>(X64, X32, fs, xl, td, k, s, t, al, L)) {
            rs[kk] = s;
            rt[kk] = t;
            ra[kk] = al;
            kk++;
          }
        }
        nr = kk;
      }
    }
#pragma unroll 1
    for (int i = 0; i < nr; ++i) {
      const double mm = fmax(fabs(rs[i]), fabs(rt[i]));
      if (mm > 1.0 + k.band_ref) continue;
      if (ra[i] < a0 - k.band_x || ra[i] > L + k.band_x) continue;
      const double dd = fabs(ra[i] - best);
      if (dd < db) {
        db = dd;
        kb = q;
        ka = ra[i];
        km = mm;
      }
    }
  }
  if (kb < 0) {
    const int is = bs > 0.0, it = bt > 0.0;
    kb = type == PT_MORTAR_FOUR ? is + 2 * it : (type == PT_MORTAR_S ? is : it);
    ka = best;
    km = 1.0;
  }
  if (fabs(km - 1.0) < k.band_ref) st |= PT_ST_NEAR_FACE;
  e = __ldg(mt + 1 + kb);
  fin = __ldg(mt + 5 + kb);
  anew = ka;
}

// CLIP: curved faces by Bezier clipping (a separate instantiation, so that the
// default path carries none of its code)
template <int G, typename R, bool CLIP>
__device__ __noinline__ void track_slow(const DevMesh& m, const DevConsts& k, int& e, double* x,
                                        double* xe, R* v, R* kx, R* kv, int& hits, unsigned& st,
                                        TrackCounters& tc) {
  tc.slow++;
  double xs[3] = {x[0], x[1], x[2]};
  double td[3] = {xe[0] - xs[0], xe[1] - xs[1], xe[2] - xs[2]};
  double L = sqrt(dot3d(td, td));
  if (!(L > 0.0)) {
#pragma unroll
    for (int r = 0; r < 3; ++r) x[r] = xe[r];
    return;
  }
  {
    const double iL = 1.0 / L;
#pragma unroll
    for (int r = 0; r < 3; ++r) td[r] *= iL;
  }
  float tdf[3] = {(float)td[0], (float)td[1], (float)td[2]};
  float Lf = (float)L;
  float n1f[3], n2f[3];
  double n1[3], n2[3];
  {
    double ax[3] = {0, 0, 0};
    int im = 0;
    if (fabs(td[1]) < fabs(td[im])) im = 1;
    if (fabs(td[2]) < fabs(td[im])) im = 2;
    ax[im] = 1.0;
    cross3d(td, ax, n1);
    const double inn = 1.0 / sqrt(dot3d(n1, n1));
#pragma unroll
    for (int r = 0; r < 3; ++r) n1[r] *= inn;
    cross3d(td, n1, n2);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      n1f[r] = (float)n1[r];
      n2f[r] = (float)n2[r];
    }
  }
  double a0 = 0.0;
  int fin = -1;
  int ncr;
  for (ncr = 0; ncr < k.max_cross; ++ncr) {
    const double* ce = m.ce + 3 * (size_t)e;
    double xl[3] = {xs[0] - __ldg(ce), xs[1] - __ldg(ce + 1), xs[2] - __ldg(ce + 2)};
    const double* X64 = m.xg64 + (size_t)e * 3 * G * G * G;
    const float xlf[3] = {(float)xl[0], (float)xl[1], (float)xl[2]};
    double best = 1e300, bs = 0.0, bt = 0.0;
    int bf = -1;
    // FP32 decision (FP32 mode): when exactly one face survives the screen,
    // it is internal or periodic, and its only FP32 crossing lies clearly
    // inside the face (max(|s|,|t|) < 1 - dl) and clearly inside the segment
    // (by the screen's margin ta, ~100x the FP32 error) while its other roots
    // are clearly outside, that crossing decides the exit face without the
    // FP64 solve: the owner follows from the face alone, the position is the
    // stage end point, and no near-face band can be met.  Otherwise the
    // provisional faces are solved exactly in a second pass.
    constexpr bool kFast = PT_FP32_DECIDE && PT_FACE_SCREEN && std::is_same<R, float>::value;
    int pf = -1, npro = 0;
    bool exact_seen = false;
    float pa32 = 0.f, ps32 = 0.f, pt32 = 0.f;
    unsigned redo = 0u;
#pragma unroll 1
    for (int pass = 0; pass < (kFast ? 2 : 1); ++pass) {
      if (pass == 1 && (pf < 0 || (npro == 1 && !exact_seen))) break;
#pragma unroll 1
      for (int f = 0; f < 6; ++f) {
        if (f == fin) continue;
        if (pass == 1 && !((redo >> f) & 1u)) continue;
        // slab prefilter (FP32, conservative: the margins cover its rounding)
        const float* sl = m.slab + 48 * (size_t)e + 8 * f;
        const float cosf_ = __ldg(sl) * tdf[0] + __ldg(sl + 1) * tdf[1] + __ldg(sl + 2) * tdf[2];
        const float pa = __ldg(sl) * xlf[0] + __ldg(sl + 1) * xlf[1] + __ldg(sl + 2) * xlf[2];
        const float pb = pa + Lf * cosf_;
        if (fmaxf(pa, pb) < __ldg(sl + 3) || fminf(pa, pb) > __ldg(sl + 4)) continue;
        const int info = __ldg(m.finfo + 6 * (size_t)e + f);
        const int kind = finfo_kind(info);
        // FP32 screen: skip the exact solve when every FP32 root is clearly
        // outside the segment or the face (margins ~100x the FP32 error)
        float fs[2], ft[2], fa[2];
        bool ill = fabsf(cosf_) < 1e-2f;
        if (PT_FACE_SCREEN) {
          const float* Bf32 = m.bil32 + 72 * (size_t)e + 12 * f;
          float B32[12];
#pragma unroll
          for (int q = 0; q < 12; ++q) B32[q] = __ldg(Bf32 + q);
          const int n32 = bilinear_roots_f32(B32, xlf, tdf, n1f, n2f, fs, ft, fa, ill);
          const float ta = 1e-4f * (__ldg(sl + 5) + Lf) / fmaxf(fabsf(cosf_), 1e-2f) +
                           4.f * (float)k.band_x;
          const float a0f = (float)a0;
          const float dl = fmaxf(1e-3f, 2.f * (float)k.band_ref);
          bool any = ill, amb = ill;
          int nin = 0, iin = 0;
          #pragma unroll 1
          for (int i = 0; i < n32 && !ill; ++i) {
            if (kind == PT_FACE_CURVED &&
                !curved_newton_f32<G>(m.xg32 + (size_t)e * 3 * G * G * G, f, xlf, tdf, k, fs[i],
                                      ft[i], fa[i])) {
              any = true;
              amb = true;
              break;
            }
            const float mm = fmaxf(fabsf(fs[i]), fabsf(ft[i]));
            if (!(fa[i] < a0f - ta || fa[i] > Lf + ta || mm > 1.f + 1e-3f)) any = true;
            if constexpr (kFast) {
              const bool out = fa[i] < a0f - ta || fa[i] > Lf + ta || mm > 1.f + dl;
              if (mm < 1.f - dl && fa[i] > a0f + ta && fa[i] < Lf - ta) {
                ++nin;
                iin = i;
              } else if (!out) {
                amb = true;
              }
            }
          }
          if (!any) continue;
          if constexpr (kFast) {
            const int bcf = finfo_bc(info);
            if (pass == 0 && !amb && nin == 1 && !(CLIP && kind == PT_FACE_CURVED) &&
                (bcf == PT_BC_INTERNAL || bcf == PT_BC_PERIODIC)) {
              ++npro;
              pf = f;
              pa32 = fa[iin];
              ps32 = fs[iin];
              pt32 = ft[iin];
              redo |= 1u << f;
              continue;
            }
          }
        }
        exact_seen = true;
        const double* Bf = m.bil + 72 * (size_t)e + 12 * f;
        double Bl[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) Bl[q] = __ldg(Bf + q);
        constexpr int MR = CLIP ? 4 : 2;
        double rs[MR], rt[MR], ra[MR];
        int nr = 0;
        const bool clip_all = CLIP && kind == PT_FACE_CURVED;
        if constexpr (CLIP) {
          if (clip_all)
            nr = bezier_clip_roots<G>(X64, m.xg32 + (size_t)e * 3 * G * G * G, f, xl, td, n1, n2,
                                      k, L, rs, rt, ra, MR);
          else
            nr = bilinear_roots(Bl, xl, td, n1, n2, rs, rt, ra);
        } else {
          nr = bilinear_roots(Bl, xl, td, n1, n2, rs, rt, ra);
        }
        if (kind == PT_FACE_CURVED && !clip_all) {
          // the curved face lies within dev of its bilinear patch: a bilinear
          // crossing far beyond the segment cannot refine into one inside it
          const double dev = (double)__ldg(sl + 6);
          const double reach = 4.0 * dev / fmax((double)fabsf(cosf_), 0.05) + 2.0 * k.band_x;
          int kk = 0;
          #pragma unroll 1
          for (int i = 0; i < nr; ++i) {
            double s = rs[i], t = rt[i], al = ra[i];
            if (!(fabs(s) < 2.0 && fabs(t) < 2.0)) continue;
            if (al > L + reach || al < a0 - reach) continue;
            if (curved_refine<G>(X64, m.xg32 + (size_t)e * 3 * G * G * G, f, xl, td, k, s, t,
                                 al, L)) {
              bool dup = false;
              for (int j = 0; j < kk; ++j)
                if (fabs(rs[j] - s) < 1e-10 && fabs(rt[j] - t) < 1e-10) dup = true;
              if (!dup) {
                rs[kk] = s;
                rt[kk] = t;
                ra[kk] = al;
                kk++;
              }
            }
          }
          nr = kk;
        }
        #pragma unroll 1
        for (int i = 0; i < nr; ++i) {
          double al = ra[i], s = rs[i], t = rt[i];
          double mm = fmax(fabs(s), fabs(t));
          if (mm > 1.0 + k.band_ref) continue;
          if (al < a0 - k.band_x || al > L + k.band_x) continue;
          if (fabs(mm - 1.0) < k.band_ref || fabs(al - a0) < k.band_x ||
              fabs(L - al) < k.band_x) {
            const int bcf = finfo_bc(info);
            st |= PT_ST_NEAR_FACE |
                  ((bcf == PT_BC_WALL || bcf == PT_BC_OPEN) ? (unsigned)PT_ST_NEAR_WALL : 0u);
          }
          if (mm <= 1.0 && al > a0 && al <= L && al < best) {
            best = al;
            bf = f;
            bs = s;
            bt = t;
          }
        }
      }
    }
    if (kFast && pf >= 0 && npro == 1 && !exact_seen) {
      best = (double)pa32;
      bf = pf;
      bs = (double)ps32;
      bt = (double)pt32;
    }
    if (bf < 0) break;
    const int info = __ldg(m.finfo + 6 * (size_t)e + bf);
    const int bc = finfo_bc(info);
    if (bc == PT_BC_MORTAR) {
      mortar_enter<G, CLIP>(m, k, __ldg(m.fnbr + 6 * (size_t)e + bf), bs, bt, xs, td, n1, n2, L,
                            a0, best, e, fin, a0, st);
      tc.cross++;
    } else if (bc == PT_BC_INTERNAL || bc == PT_BC_PERIODIC) {
      if (bc == PT_BC_PERIODIC) {
        const double* sh = m.shift + 18 * (size_t)e + 3 * bf;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          xs[r] += __ldg(sh + r);
          xe[r] += __ldg(sh + r);
        }
      }
      fin = finfo_nf(info);
      e = __ldg(m.fnbr + 6 * (size_t)e + bf);
      a0 = best;
      tc.cross++;
    } else if (bc == PT_BC_WALL) {
      double ps[3], pt[3], nrm[3];
      const int kind = finfo_kind(info);
      if (kind == PT_FACE_CURVED) {
        double p[3];
        face_eval<G>(X64, bf, bs, bt, k, p, ps, pt);
      } else {
        const double* Bf = m.bil + 72 * (size_t)e + 12 * bf;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          ps[r] = __ldg(Bf + r) * bt + __ldg(Bf + 3 + r);
          pt[r] = __ldg(Bf + r) * bs + __ldg(Bf + 6 + r);
        }
      }
      cross3d(ps, pt, nrm);
      const double inn = 1.0 / sqrt(dot3d(nrm, nrm));
#pragma unroll
      for (int r = 0; r < 3; ++r) nrm[r] *= inn;
      double xh[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) xh[r] = xs[r] + best * td[r];
      double Lr = L - best;
      double sdt = 2.0 * dot3d(td, nrm);
#pragma unroll
      for (int r = 0; r < 3; ++r) td[r] -= sdt * nrm[r];
      reflect3(v, nrm);
      reflect3(kx, nrm);
      reflect3(kv, nrm);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        xs[r] = xh[r];
        xe[r] = xs[r] + Lr * td[r];
      }
      L = Lr;
      a0 = 0.0;
      fin = bf;
      hits++;
      tc.hits++;
      // the frame follows the new direction
      double ax[3] = {0, 0, 0};
      int im = 0;
      if (fabs(td[1]) < fabs(td[im])) im = 1;
      if (fabs(td[2]) < fabs(td[im])) im = 2;
      ax[im] = 1.0;
      cross3d(td, ax, n1);
      const double in1 = 1.0 / sqrt(dot3d(n1, n1));
#pragma unroll
      for (int r = 0; r < 3; ++r) n1[r] *= in1;
      cross3d(td, n1, n2);
      // and so do the FP32 copies that the slab test and the screen use
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        tdf[r] = (float)td[r];
        n1f[r] = (float)n1[r];
        n2f[r] = (float)n2[r];
      }
      Lf = (float)L;
      if (!(L > 0.0)) break;
    } else {
#pragma unroll
      for (int r = 0; r < 3; ++r) x[r] = xs[r] + best * td[r];
      st |= PT_ST_OPEN;
      return;
    }
  }
  if (ncr >= k.max_cross) st |= PT_ST_CROSS_CAP;
#pragma unroll
  for (int r = 0; r < 3; ++r) x[r] = xe[r];
}

}  // namespace pt
