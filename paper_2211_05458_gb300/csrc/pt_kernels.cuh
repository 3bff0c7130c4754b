// pt_kernels.cuh -- the push, inverse-map and deposition kernels, templated on
// G = NGeo+1, NP = N+1 and the precision mode.  Each translation unit
// pt_push_g<G>_<mode>.cu instantiates one (G, mode) family for NP = 2..8.
#pragma once
#include "pt_device.cuh"
#include "pt_mlp_infer.cuh"

// minimum resident blocks of 128 threads per SM for the push kernel (sets the
// register budget: 2 -> 255 registers per thread, 3 -> 168, 4 -> 128).  At the
// 64^3 NGeo=3 workload 2 measured best (FP32: +1-2 % over 3, 3 +8-14 % over 4):
// spills cost more than the lower occupancy
#ifndef PT_PUSH_MINB
#define PT_PUSH_MINB 2
#endif
#define PT_PUSH_MINB_F64 2
// 1: the staged schedule evaluates the learned start on the tensor cores
// (tcgen05, k_guess_tc); 0: with the warp-level mma.sync form (k_guess_mlp)
#ifndef PT_MLP_TC
#define PT_MLP_TC 1
#endif

namespace pt {

template <bool F64>
struct RealOf {
  using type = float;
};
template <>
struct RealOf<true> {
  using type = double;
};

__device__ __forceinline__ void count_add(unsigned long long* stats, int slot,
                                          unsigned long long v) {
  // warp-aggregated: one atomic per warp and counter
  unsigned long long s = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(stats + slot, s);
}

// Inverse map of one particle with the context's precision and start guess.
template <int G, bool F64>
__device__ __forceinline__ bool locate_one(const DevMesh& m, const DevConsts& k, int e,
                                           const double* x, const float* guess, double* xi,
                                           int& it32, int& it64) {
  const double* ce = m.ce + 3 * (size_t)e;
  double xl[3] = {x[0] - __ldg(ce), x[1] - __ldg(ce + 1), x[2] - __ldg(ce + 2)};
  if (F64) {
    xi[0] = guess[0];
    xi[1] = guess[1];
    xi[2] = guess[2];
    return newton64<G>(m.xg64 + (size_t)e * 3 * G * G * G, xl, xi, k, k.max_newton, it64);
  }
  return newton_mixed<G>(m, k, e, xl, guess, xi, it32, it64);
}

// As locate_one, with x already relative to the element centre.
template <int G, bool F64>
__device__ __forceinline__ bool locate_local(const DevMesh& m, const DevConsts& k, int e,
                                             const double* xl, const float* guess, double* xi,
                                             int& it32, int& it64) {
  if (F64) {
    xi[0] = guess[0];
    xi[1] = guess[1];
    xi[2] = guess[2];
    return newton64<G>(m.xg64 + (size_t)e * 3 * G * G * G, xl, xi, k, k.max_newton, it64);
  }
  return newton_mixed<G>(m, k, e, xl, guess, xi, it32, it64);
}

// Start guess: trilinear, optionally corrected by the learned network (warp-
// collective: every lane of the warp must call it).
template <int G, bool MLP>
__device__ __forceinline__ void start_guess(const DevMesh& m, const DevConsts& k, MlpSmem* sm,
                                            const DevMLP* mlpp, int e, const double* x, bool live,
                                            float* guess) {
  const double* ce = m.ce + 3 * (size_t)e;
  float xf[3] = {(float)(x[0] - __ldg(ce)), (float)(x[1] - __ldg(ce + 1)),
                 (float)(x[2] - __ldg(ce + 2))};
  trilinear_guess(m, e, xf, guess);
  if constexpr (MLP) mlp_correct_smem(*sm, *mlpp, m, e, live, guess);
}

// As start_guess, with x already relative to the element centre (FP32).
template <int G, bool MLP>
__device__ __forceinline__ void start_guess_local(const DevMesh& m, const DevConsts& k,
                                                  MlpSmem* sm, const DevMLP* mlpp, int e,
                                                  const float* xf, bool live,
                                                  float* guess) {
  trilinear_guess(m, e, xf, guess);
  if constexpr (MLP) mlp_correct_smem(*sm, *mlpp, m, e, live, guess);
}

// The block's copy of the network weights (NGeo = 3 kernels only); must be
// reached by every thread of the block.
#define PT_MLP_PROLOGUE(USE, P)                       \
  MlpSmem* sm = nullptr;                              \
  if constexpr (USE) {                                \
    __shared__ MlpSmem s_mlp;                         \
    sm = &s_mlp;                                      \
    mlp_load(s_mlp, P);                               \
    __syncthreads();                                  \
  }

// Saffman lift with Mei's correction (Sec. 2.2): the force
//   F_S = 6.46/4 C_S d^2 sqrt(rho mu / |w|) (u - v) x w,   w = curl u,
// C_S = (1 - 0.3314 sqrt(th)) exp(-Re_p/10) + 0.3314 sqrt(th) for Re_p <= 40,
// 0.0524 sqrt(th Re_p) above, th = d |w| / (2 |u - v|) held within
// [0.005, 0.4]; zero when w or u - v vanishes.  The velocity gradient
// differentiates the Lagrange interpolant of rho and rho u (sum-factorised,
// Eq. part_interpolation): du_i/dxi_q = (d(rho u_i)/dxi_q - u_i drho/dxi_q)/rho,
// mapped to physical space with the inverse Jacobian of the element map at xi.
// Out of line: only runs with the lift enabled.
template <int G, int NP, typename T>
__device__ __noinline__ void saffman_force(const DevMesh& m, const DevConsts& k,
                                           const T* __restrict__ Ue, int e, const double* xi,
                                           const T* v, T d, T* F) {
  constexpr int N3 = NP * NP * NP;
  constexpr int G3 = G * G * G;
  T l[3][NP], dl[3][NP];
#pragma unroll
  for (int q = 0; q < 3; ++q) lagr_d<NP, T>((T)xi[q], Nodes<T>::sol(k), Nodes<T>::solw(k), l[q], dl[q]);
  // value and d/dxi_1..3 of rho, rho u, rho v, rho w
  T val[4], der[4][3];
#pragma unroll 1
  for (int w = 0; w < 4; ++w) {
    const T* Uw = Ue + w * N3;
    T s = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll 1
    for (int kk = 0; kk < NP; ++kk) {
      T b0 = 0, b1 = 0, b2 = 0;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        T a0 = 0, a1 = 0;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          const T u = Uw[i + NP * (j + NP * kk)];
          a0 = tfma(u, l[0][i], a0);
          a1 = tfma(u, dl[0][i], a1);
        }
        b0 = tfma(a0, l[1][j], b0);
        b1 = tfma(a1, l[1][j], b1);
        b2 = tfma(a0, dl[1][j], b2);
      }
      T lk = T(0), dk = T(0);
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c == kk) {
          lk = l[2][c];
          dk = dl[2][c];
        }
      s = tfma(b0, lk, s);
      s1 = tfma(b1, lk, s1);
      s2 = tfma(b2, lk, s2);
      s3 = tfma(b0, dk, s3);
    }
    val[w] = s;
    der[w][0] = s1;
    der[w][1] = s2;
    der[w][2] = s3;
  }
  // Jacobian of the element map at xi and its inverse
  T J[9], Ji[9];
  if constexpr (std::is_same<T, float>::value) {
    const float xf[3] = {(float)xi[0], (float)xi[1], (float)xi[2]};
    float chi[3];
    map_j32<G>(m.xg32 + (size_t)e * 3 * G3, xf, __ldg(m.tmask + e), k, chi, J);
  } else {
    double chi[3];
    map64<G, true>(m.xg64 + (size_t)e * 3 * G3, xi, k, chi, J);
  }
  F[0] = F[1] = F[2] = T(0);
  if (!inv3(J, Ji)) return;
  const T rho = val[0], irho = T(1) / rho;
  T u[3], rel[3], Gd[9];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    u[i] = val[1 + i] * irho;
    rel[i] = u[i] - v[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T dxi[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) dxi[q] = (der[1 + i][q] - u[i] * der[0][q]) * irho;
#pragma unroll
    for (int j = 0; j < 3; ++j) Gd[3 * i + j] = dxi[0] * Ji[j] + dxi[1] * Ji[3 + j] + dxi[2] * Ji[6 + j];
  }
  const T w[3] = {Gd[7] - Gd[5], Gd[2] - Gd[6], Gd[3] - Gd[1]};
  const T wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  const T rn = sqrt(rel[0] * rel[0] + rel[1] * rel[1] + rel[2] * rel[2]);
  if (!(wn > T(0)) || !(rn > T(0))) return;
  const T mu = (T)k.mu;
  const T re = rho * rn * d / mu;
  T th = d * wn / (T(2) * rn);
  th = th < T(0.005) ? T(0.005) : (th > T(0.4) ? T(0.4) : th);
  const T sth = sqrt(th);
  const T cs = re <= T(40) ? (T(1) - T(0.3314) * sth) * exp(T(-0.1) * re) + T(0.3314) * sth
                           : T(0.0524) * sqrt(th * re);
  const T kf = T(6.46 / 4.0) * cs * d * d * sqrt(rho * mu / wn);
  F[0] = kf * (rel[1] * w[2] - rel[2] * w[1]);
  F[1] = kf * (rel[2] * w[0] - rel[0] * w[2]);
  F[2] = kf * (rel[0] * w[1] - rel[1] * w[0]);
}

// Near-face band at a stage start (R8): max |xi_d| > 1 - band_ref sets
// PT_ST_NEAR_FACE; where the face of such a component (2d + (xi_d > 0)) is a
// wall or open face, PT_ST_NEAR_WALL as well.
template <typename T>
__device__ __forceinline__ unsigned near_bits(const DevMesh& m, int e, const T* xi, double band) {
  unsigned b = 0u;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (fabs((double)xi[d]) > 1.0 - band) {
      b |= PT_ST_NEAR_FACE;
      const int bc = finfo_bc(__ldg(m.finfo + 6 * (size_t)e + 2 * d + (xi[d] > T(0) ? 1 : 0)));
      if (bc == PT_BC_WALL || bc == PT_BC_OPEN) b |= PT_ST_NEAR_WALL;
    }
  }
  return b;
}

// Acceleration of a particle (Sec. 2.2, Eqs. dragforce, dragfactor, Eq.
// theory:maxey): a = m_d f_D (u - v) / tau_p + g (1 - rho / rho_p with
// buoyancy) + F_S / m_p with the lift; m_d the per-axis drag mask.  Uv holds
// rho, rho u at xi (interpolated by the caller).  Sets PT_ST_REP800 for the
// Schiller-Naumann law beyond its range.
template <int G, int NP, typename R>
__device__ __forceinline__ void particle_accel(const DevMesh& m, const DevConsts& k,
                                               const R* __restrict__ Ue, int e, const double* xi,
                                               const R* Uv, const R* v, R d, R tau, unsigned& st,
                                               R* acc) {
  const R mu = (R)k.mu;
  R irho = R(1) / Uv[0], rel[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) rel[r] = Uv[1 + r] * irho - v[r];
  R fD = R(1);
  if (k.drag_law) {
    R re = Uv[0] * sqrt(rel[0] * rel[0] + rel[1] * rel[1] + rel[2] * rel[2]) * d / mu;
    if (k.drag_law == 1 && re >= R(800)) st |= PT_ST_REP800;
    fD = drag_factor<R>(k, re);
  }
  const R coef = fD / tau;
  R al[3] = {R(0), R(0), R(0)};
  if (k.lift) {
    saffman_force<G, NP, R>(m, k, Ue, e, xi, v, d, al);
    const R imp = R(6) / (R(3.14159265358979323846) * (R)k.rho_p * d * d * d);
#pragma unroll
    for (int r = 0; r < 3; ++r) al[r] *= imp;
  }
  const R gf = k.buoyancy ? R(1) - Uv[0] / (R)k.rho_p : R(1);
#pragma unroll
  for (int r = 0; r < 3; ++r) acc[r] = (R)k.mask[r] * coef * rel[r] + (R)k.g[r] * gf + al[r];
}

// FP32 mode: as particle_accel, xi as a double-float (used by the lift only)
template <int G, int NP>
__device__ __forceinline__ void particle_accel_f32(const DevMesh& m, const DevConsts& k,
                                                   const float* __restrict__ Ue, int e,
                                                   const df* zd, const float* Uv, const float* v,
                                                   float d, float tau, unsigned& st, float* acc) {
  const float mu = (float)k.mu;
  float irho = 1.f / Uv[0], rel[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) rel[r] = Uv[1 + r] * irho - v[r];
  float fD = 1.f;
  if (k.drag_law) {
    float re = Uv[0] * sqrtf(rel[0] * rel[0] + rel[1] * rel[1] + rel[2] * rel[2]) * d / mu;
    if (k.drag_law == 1 && re >= 800.f) st |= PT_ST_REP800;
    fD = drag_factor<float>(k, re);
  }
  const float coef = fD / tau;
  float al[3] = {0.f, 0.f, 0.f};
  if (k.lift) {
    const double xid[3] = {df_to_double(zd[0]), df_to_double(zd[1]), df_to_double(zd[2])};
    saffman_force<G, NP, float>(m, k, Ue, e, xid, v, d, al);
    const float imp = 6.f / (3.14159265358979323846f * (float)k.rho_p * d * d * d);
#pragma unroll
    for (int r = 0; r < 3; ++r) al[r] *= imp;
  }
  const float gf = k.buoyancy ? 1.f - Uv[0] / (float)k.rho_p : 1.f;
#pragma unroll
  for (int r = 0; r < 3; ++r)
    acc[r] = (float)k.mask[r] * coef * rel[r] + (float)k.g[r] * gf + al[r];
}

struct PushCounters {
  unsigned long long steps, it32, it64;
  TrackCounters tc;
};

// Missed-crossing repair.  Curved faces are intersected by Newton from the
// roots of their bilinear patch, which can miss a near-tangential crossing
// (the ray leaves through the curved face where the patch has no nearby
// root).  Such a particle is found outside its element by the next inverse map
// (max |xi| > 1 + lost_tol).  It is then moved across the face of its largest
// |xi_d| -- translated on a periodic face -- and mapped again, until it lands
// inside, across at most 4 faces; a wall or open face ends the walk and the
// particle is lost as before.  Only a stage that took the exact tracking path
// can leave a particle outside: the walk runs only after such a stage (a
// particle found outside otherwise, e.g. given outside its element, is lost),
// and the push checks the final position of such a stage as well.  Returns 0 (inside), 1 (inverse map failed) or 2 (lost).
// Out of line: it is rare.
__device__ __forceinline__ int settle_face(const double* z) {
  const double a0 = fabs(z[0]), a1 = fabs(z[1]), a2 = fabs(z[2]);
  const int d = (a0 >= a1 && a0 >= a2) ? 0 : (a1 >= a2 ? 1 : 2);
  return 2 * d + (z[d] > 0.0 ? 1 : 0);
}

// The walk across a mortar's big face enters the small element whose part of
// the big face holds the point's face parameters (the two xi components other
// than the crossed one, in order).
__device__ __forceinline__ int mortar_small(const DevMesh& m, int row, int f, const double* z) {
  const int* mt = m.mort + 9 * (size_t)row;
  const int d = f >> 1;
  const double s = z[d == 0 ? 1 : 0], t = z[d == 2 ? 1 : 2];
  const int type = __ldg(mt), is = s > 0.0, it = t > 0.0;
  const int q = type == PT_MORTAR_FOUR ? is + 2 * it : (type == PT_MORTAR_S ? is : it);
  return __ldg(mt + 1 + q);
}

// Walk threshold: with physical tracking a position up to lost_tol outside is
// accepted (the tracking decided the owner); with reference-space localisation
// the owner is decided here, to the near-face band.
__device__ __forceinline__ double settle_tol(const DevConsts& k) {
  return k.track == PT_TRACK_REFERENCE ? fmin(k.band_ref, k.lost_tol) : k.lost_tol;
}

// FP64 mode: x global, xi valid on entry if have.
template <int G>
__device__ __noinline__ int settle64(const DevMesh& m, const DevConsts& k, int& e, double* x,
                                     double* xi, bool have, int& it64, int& cross) {
  const double wtol = settle_tol(k);
#pragma unroll 1
  for (int w = 0; w <= 4; ++w) {
    if (!have) {
      const double* ce = m.ce + 3 * (size_t)e;
      const double xl[3] = {x[0] - __ldg(ce), x[1] - __ldg(ce + 1), x[2] - __ldg(ce + 2)};
      const float xf[3] = {(float)xl[0], (float)xl[1], (float)xl[2]};
      float g[3];
      trilinear_guess(m, e, xf, g);
      xi[0] = g[0];
      xi[1] = g[1];
      xi[2] = g[2];
      if (!newton64<G>(m.xg64 + (size_t)e * 3 * G * G * G, xl, xi, k, k.max_newton, it64))
        return 1;
    }
    have = false;
    if (tmax3(xi[0], xi[1], xi[2]) <= 1.0 + wtol) return 0;
    if (w == 4) return tmax3(xi[0], xi[1], xi[2]) <= 1.0 + k.lost_tol ? 0 : 2;
    const int f = settle_face(xi);
    const int bc = finfo_bc(__ldg(m.finfo + 6 * (size_t)e + f));
    if (bc != PT_BC_INTERNAL && bc != PT_BC_PERIODIC && bc != PT_BC_MORTAR) break;
    if (bc == PT_BC_PERIODIC) {
      const double* sh = m.shift + 18 * (size_t)e + 3 * f;
#pragma unroll
      for (int r = 0; r < 3; ++r) x[r] += __ldg(sh + r);
    }
    e = bc == PT_BC_MORTAR ? mortar_small(m, __ldg(m.fnbr + 6 * (size_t)e + f), f, xi)
                           : __ldg(m.fnbr + 6 * (size_t)e + f);
    ++cross;
  }
  return 2;
}

// FP32 mode: xd local double-float position in element e, zd its xi (valid
// on entry if have).
template <int G>
__device__ __noinline__ int settle_f32(const DevMesh& m, const DevConsts& k, int& e, df* xd,
                                       df* zd, bool have, int& it32, int& it64, int& cross) {
  const double wtol = settle_tol(k);
#pragma unroll 1
  for (int w = 0; w <= 4; ++w) {
    if (!have) {
      const float xf[3] = {xd[0].hi, xd[1].hi, xd[2].hi};
      float g[3];
      trilinear_guess(m, e, xf, g);
      if (!newton_df<G>(m, k, e, xd, g, zd, it32, it64)) return 1;
    }
    have = false;
    const double z[3] = {df_to_double(zd[0]), df_to_double(zd[1]), df_to_double(zd[2])};
    if (tmax3(z[0], z[1], z[2]) <= 1.0 + wtol) return 0;
    if (w == 4) return tmax3(z[0], z[1], z[2]) <= 1.0 + k.lost_tol ? 0 : 2;
    const int f = settle_face(z);
    const int bc = finfo_bc(__ldg(m.finfo + 6 * (size_t)e + f));
    if (bc != PT_BC_INTERNAL && bc != PT_BC_PERIODIC && bc != PT_BC_MORTAR) break;
    const double* ce = m.ce + 3 * (size_t)e;
    double xg[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) xg[r] = __ldg(ce + r) + df_to_double(xd[r]);
    if (bc == PT_BC_PERIODIC) {
      const double* sh = m.shift + 18 * (size_t)e + 3 * f;
#pragma unroll
      for (int r = 0; r < 3; ++r) xg[r] += __ldg(sh + r);
    }
    e = bc == PT_BC_MORTAR ? mortar_small(m, __ldg(m.fnbr + 6 * (size_t)e + f), f, z)
                           : __ldg(m.fnbr + 6 * (size_t)e + f);
    const double* cn = m.ce + 3 * (size_t)e;
#pragma unroll
    for (int r = 0; r < 3; ++r) xd[r] = df_from_double(xg[r] - __ldg(cn + r));
    ++cross;
  }
  return 2;
}

// Advances particle ip of p by nsteps RK steps: per stage the inverse map,
// interpolation of rho and rho u, drag + gravity, the low-storage RK update of
// x and v, and tracking of the stage segment.  State lives in registers for
// the whole call (the fluid state is constant during it).  Every lane of a
// warp must call it (the learned start is warp-collective); lanes without a
// particle pass inrange = false.
template <int G, int NP, bool F64, bool MLP, bool CLIP = false>
__device__ __forceinline__ void push_particle(const DevMesh& m, const DevConsts& k, MlpSmem* sm,
                                              const DevMLP* mlpp,
                                              const typename RealOf<F64>::type* __restrict__ U,
                                              const DevParticles& p, int64_t ip, bool inrange,
                                              int nsteps, double dtd, PushCounters& c) {
  using R = typename RealOf<F64>::type;
  constexpr int N3 = NP * NP * NP;
  const int64_t n = p.n;
  const R dt = (R)dtd;
  const R mu = (R)k.mu;
  R* vg = reinterpret_cast<R*>(p.v);
  const R* dg = reinterpret_cast<const R*>(p.d);
  unsigned st = inrange ? p.status[ip] : PT_ST_FROZEN;
  bool live = !(st & PT_ST_FROZEN);
  double x[3] = {0, 0, 0};
  R v[3] = {0, 0, 0}, d = R(1);
  int e = 0, hits = 0;
  if (inrange) {
    x[0] = p.x[ip];
    x[1] = p.x[n + ip];
    x[2] = p.x[2 * n + ip];
    v[0] = vg[ip];
    v[1] = vg[n + ip];
    v[2] = vg[2 * n + ip];
    d = dg[ip];
    e = p.elem[ip];
    hits = p.hits[ip];
  }
  if (e < 0 || e >= m.nelem) {
    if (live) st |= PT_ST_LOST;
    live = false;
  }
  const R tau = (R)k.rho_p * d * d / (R(18) * mu);
  bool pending = false;  // the last stage took the exact tracking path
  for (int step = 0; step < nsteps; ++step) {
    R kx[3] = {0, 0, 0}, kv[3] = {0, 0, 0};
    for (int s = 0; s < 5; ++s) {
      const R As = F64 ? (R)k.A[s] : (R)k.A32[s];
      const R Bs = F64 ? (R)k.B[s] : (R)k.B32[s];
      const int eg = live ? e : 0;
      const double* ce = m.ce + 3 * (size_t)eg;
      double xl[3] = {x[0] - __ldg(ce), x[1] - __ldg(ce + 1), x[2] - __ldg(ce + 2)};
      float xf[3] = {(float)xl[0], (float)xl[1], (float)xl[2]};
      float guess[3];
      start_guess_local<G, MLP>(m, k, sm, mlpp, eg, xf, live, guess);
      if (!live) continue;
      double xi[3];
      int i32 = 0, i64 = 0;
      bool ok = locate_local<G, F64>(m, k, e, xl, guess, xi, i32, i64);
      c.it32 += i32;
      c.it64 += i64;
      if (!ok) {
        st |= PT_ST_NEWTON_FAIL;
        live = false;
        continue;
      }
      double mx = tmax3(xi[0], xi[1], xi[2]);
      if (mx > 1.0 + k.lost_tol && !pending) {  // outside without having moved: lost
        st |= PT_ST_LOST;
        live = false;
        continue;
      }
      if (mx > 1.0 + settle_tol(k) && pending) {
        int cr = 0, j64 = 0;
        const int rc = settle64<G>(m, k, e, x, xi, true, j64, cr);
        c.it64 += j64;
        c.tc.cross += cr;
        if (rc) {
          st |= rc == 1 ? PT_ST_NEWTON_FAIL : PT_ST_LOST;
          live = false;
          continue;
        }
        mx = tmax3(xi[0], xi[1], xi[2]);
        // the stage segment's slab test below works in the new element's frame
        const double* cn = m.ce + 3 * (size_t)e;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          xl[r] = x[r] - __ldg(cn + r);
          xf[r] = (float)xl[r];
        }
      }
      pending = false;
      if (mx > 1.0 - k.band_ref) st |= near_bits(m, e, xi, k.band_ref);
      // interpolation of rho, rho u at xi
      R l1[NP], l2[NP], l3[NP], Uv[4];
      lagr<NP, R>((R)xi[0], Nodes<R>::sol(k), Nodes<R>::solw(k), l1);
      lagr<NP, R>((R)xi[1], Nodes<R>::sol(k), Nodes<R>::solw(k), l2);
      lagr<NP, R>((R)xi[2], Nodes<R>::sol(k), Nodes<R>::solw(k), l3);
      interp4<NP, R>(U + (size_t)e * 5 * N3, l1, l2, l3, Uv);
      // drag + gravity
      R acc[3];
      particle_accel<G, NP, R>(m, k, U + (size_t)e * 5 * N3, e, xi, Uv, v, d, tau, st, acc);
      double xe[3];
      float bf[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        kx[r] = As * kx[r] + dt * v[r];
        kv[r] = As * kv[r] + dt * acc[r];
        const R dx = Bs * kx[r];
        xe[r] = x[r] + (double)dx;
        bf[r] = F64 ? (float)(xl[r] + (double)dx) : xf[r] + (float)dx;
        v[r] = v[r] + Bs * kv[r];
      }
      const int touch = slab_touch(m, e, xf, bf);
      if (!(touch & (k.track == PT_TRACK_REFERENCE ? 2 : 1))) {
        // no face reachable, or (localisation) no wall or open face: the end
        // point's owner is found by the next inverse map
#pragma unroll
        for (int r = 0; r < 3; ++r) x[r] = xe[r];
        pending = touch != 0;
      } else {
        track_slow<G, R, CLIP>(m, k, e, x, xe, v, kx, kv, hits, st, c.tc);
        pending = true;
      }
      if (st & PT_ST_FROZEN) live = false;
    }
    if (live) ++c.steps;
  }
  if (live && pending) {
    double xi[3];
    int cr = 0, j64 = 0;
    const int rc = settle64<G>(m, k, e, x, xi, false, j64, cr);
    c.it64 += j64;
    c.tc.cross += cr;
    if (rc) st |= rc == 1 ? PT_ST_NEWTON_FAIL : PT_ST_LOST;
  }
  if (inrange && !(p.status[ip] & PT_ST_FROZEN)) {
    p.x[ip] = x[0];
    p.x[n + ip] = x[1];
    p.x[2 * n + ip] = x[2];
    vg[ip] = v[0];
    vg[n + ip] = v[1];
    vg[2 * n + ip] = v[2];
    p.elem[ip] = e;
    p.hits[ip] = hits;
    p.status[ip] = st;
  }
}

// FP32 mode: as push_particle, with the position held during the call as a
// double-float offset from the owning element's centre, so that a stage issues
// no FP64 instruction except in the exact face-intersection path (the FP64
// position is formed again at the end and around that path).
template <int G, int NP, bool MLP, bool CLIP = false>
__device__ __forceinline__ void push_particle_f32(const DevMesh& m, const DevConsts& k,
                                                  MlpSmem* sm, const DevMLP* mlpp,
                                                  const float* __restrict__ U,
                                                  const DevParticles& p, int64_t ip, bool inrange,
                                                  int nsteps, double dtd, PushCounters& c) {
  constexpr int N3 = NP * NP * NP;
  const int64_t n = p.n;
  const float dt = (float)dtd;
  const float mu = (float)k.mu;
  float* vg = reinterpret_cast<float*>(p.v);
  const float* dg = reinterpret_cast<const float*>(p.d);
  unsigned st = inrange ? p.status[ip] : PT_ST_FROZEN;
  bool live = !(st & PT_ST_FROZEN);
  double x[3] = {0, 0, 0};
  float v[3] = {0, 0, 0}, d = 1.f;
  int e = 0, hits = 0;
  if (inrange) {
    x[0] = p.x[ip];
    x[1] = p.x[n + ip];
    x[2] = p.x[2 * n + ip];
    v[0] = vg[ip];
    v[1] = vg[n + ip];
    v[2] = vg[2 * n + ip];
    d = dg[ip];
    e = p.elem[ip];
    hits = p.hits[ip];
  }
  if (e < 0 || e >= m.nelem) {
    if (live) st |= PT_ST_LOST;
    live = false;
  }
  // local double-float position
  df xd[3];
  {
    const double* ce = m.ce + 3 * (size_t)(live ? e : 0);
#pragma unroll
    for (int r = 0; r < 3; ++r) xd[r] = df_from_double(x[r] - __ldg(ce + r));
  }
  bool moved = false;
  bool pending = false;  // the last stage took the exact tracking path
  const float tau = (float)k.rho_p * d * d / (18.f * mu);
  for (int step = 0; step < nsteps; ++step) {
    float kx[3] = {0, 0, 0}, kv[3] = {0, 0, 0};
    for (int s = 0; s < 5; ++s) {
      const float As = k.A32[s];
      const float Bs = k.B32[s];
      const int eg = live ? e : 0;
      float xf[3] = {xd[0].hi, xd[1].hi, xd[2].hi};
      float guess[3];
      start_guess_local<G, MLP>(m, k, sm, mlpp, eg, xf, live, guess);
      if (!live) continue;
      df zd[3];
      int i32 = 0, i64 = 0;
      bool ok = newton_df<G>(m, k, e, xd, guess, zd, i32, i64);
      c.it32 += i32;
      c.it64 += i64;
      if (!ok) {
        st |= PT_ST_NEWTON_FAIL;
        live = false;
        continue;
      }
      float xi[3] = {zd[0].hi + zd[0].lo, zd[1].hi + zd[1].lo, zd[2].hi + zd[2].lo};
      const float mx = tmax3(xi[0], xi[1], xi[2]);
      if (mx > 1.f - fmaxf(1e-5f, (float)k.band_ref)) {  // decide the bands exactly (rare)
        double md = fmax(fmax(fabs(df_to_double(zd[0])), fabs(df_to_double(zd[1]))),
                         fabs(df_to_double(zd[2])));
        if (md > 1.0 + k.lost_tol && !pending) {  // outside without having moved: lost
          st |= PT_ST_LOST;
          live = false;
          continue;
        }
        if (md > 1.0 + settle_tol(k) && pending) {
          int cr = 0, j32 = 0, j64 = 0;
          const int rc = settle_f32<G>(m, k, e, xd, zd, true, j32, j64, cr);
          c.it32 += j32;
          c.it64 += j64;
          c.tc.cross += cr;
          if (rc) {
            st |= rc == 1 ? PT_ST_NEWTON_FAIL : PT_ST_LOST;
            live = false;
            continue;
          }
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            xi[q] = zd[q].hi + zd[q].lo;
            xf[q] = xd[q].hi;  // the slab test below works in the new element's frame
          }
          md = fmax(fmax(fabs(df_to_double(zd[0])), fabs(df_to_double(zd[1]))),
                    fabs(df_to_double(zd[2])));
        }
        if (md > 1.0 - k.band_ref) {
          const double z[3] = {df_to_double(zd[0]), df_to_double(zd[1]), df_to_double(zd[2])};
          st |= near_bits(m, e, z, k.band_ref);
        }
      }
      pending = false;
      // interpolation of rho, rho u at xi
      float l1[NP], l2[NP], l3[NP], Uv[4];
      lagr<NP, float>(xi[0], k.sn32, k.sw32, l1);
      lagr<NP, float>(xi[1], k.sn32, k.sw32, l2);
      lagr<NP, float>(xi[2], k.sn32, k.sw32, l3);
      interp4<NP, float>(U + (size_t)e * 5 * N3, l1, l2, l3, Uv);
      // drag + gravity
      float acc[3];
      particle_accel_f32<G, NP>(m, k, U + (size_t)e * 5 * N3, e, zd, Uv, v, d, tau, st, acc);
      df xe[3];
      float bf[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        kx[r] = As * kx[r] + dt * v[r];
        kv[r] = As * kv[r] + dt * acc[r];
        xe[r] = df_add(xd[r], df_from(Bs * kx[r]));
        bf[r] = xe[r].hi;
        v[r] = v[r] + Bs * kv[r];
      }
      const int touch = slab_touch(m, e, xf, bf);
      if (!(touch & (k.track == PT_TRACK_REFERENCE ? 2 : 1))) {
        // no face reachable, or (localisation) no wall or open face: the end
        // point's owner is found by the next inverse map
#pragma unroll
        for (int r = 0; r < 3; ++r) xd[r] = xe[r];
        if (touch) pending = true;
      } else {
        // exact tracking in FP64 on global positions, then back to local
        const double* ce = m.ce + 3 * (size_t)e;
        double xs[3], xg[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const double cr = __ldg(ce + r);
          xs[r] = cr + df_to_double(xd[r]);
          xg[r] = cr + df_to_double(xe[r]);
        }
        track_slow<G, float, CLIP>(m, k, e, xs, xg, v, kx, kv, hits, st, c.tc);
        if (st & PT_ST_FROZEN) {
          live = false;
#pragma unroll
          for (int r = 0; r < 3; ++r) x[r] = xs[r];
          moved = true;
          continue;
        }
        const double* cn = m.ce + 3 * (size_t)e;
#pragma unroll
        for (int r = 0; r < 3; ++r) xd[r] = df_from_double(xs[r] - __ldg(cn + r));
        pending = true;
      }
    }
    if (live) ++c.steps;
  }
  if (live && pending) {
    df zd[3];
    int cr = 0, j32 = 0, j64 = 0;
    const int rc = settle_f32<G>(m, k, e, xd, zd, false, j32, j64, cr);
    c.it32 += j32;
    c.it64 += j64;
    c.tc.cross += cr;
    if (rc) {
      st |= rc == 1 ? PT_ST_NEWTON_FAIL : PT_ST_LOST;
      live = false;
    }
  }
  if (inrange && !(p.status[ip] & PT_ST_FROZEN)) {
    if (live || !moved) {
      const double* ce = m.ce + 3 * (size_t)(e >= 0 && e < m.nelem ? e : 0);
      if (e >= 0 && e < m.nelem) {
#pragma unroll
        for (int r = 0; r < 3; ++r) x[r] = __ldg(ce + r) + df_to_double(xd[r]);
      }
    }
    p.x[ip] = x[0];
    p.x[n + ip] = x[1];
    p.x[2 * n + ip] = x[2];
    vg[ip] = v[0];
    vg[n + ip] = v[1];
    vg[2 * n + ip] = v[2];
    p.elem[ip] = e;
    p.hits[ip] = hits;
    p.status[ip] = st;
  }
}

// One thread per particle, visiting particles in element-sorted order (perm)
// so that a warp shares its element's data through L1.  Persistent grid.
template <int G, int NP, bool F64, bool MLP, bool CLIP = false>
__global__ void __launch_bounds__(128, F64 ? PT_PUSH_MINB_F64 : PT_PUSH_MINB)
    k_push(const __grid_constant__ PushArgs a) {
  using R = typename RealOf<F64>::type;
  PT_MLP_PROLOGUE(MLP, a.mlp);
  const R* __restrict__ U = reinterpret_cast<const R*>(a.U);
  PushCounters c = {0, 0, 0, {0, 0, 0}};
  const int64_t n = a.p.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nround = (n + stride - 1) / stride * stride;  // uniform trip count per warp
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nround; t += stride) {
    const bool inrange = t < n;
    const int64_t ip = inrange ? (a.perm ? (int64_t)a.perm[t] : t) : 0;
    if constexpr (F64)
      push_particle<G, NP, true, false, CLIP>(a.m, a.k, sm, &a.mlp, U, a.p, ip, inrange, a.nsteps, a.dt,
                                        c);
    else
      push_particle_f32<G, NP, MLP, CLIP>(a.m, a.k, sm, &a.mlp, (const float*)U, a.p, ip, inrange, a.nsteps,
                               a.dt, c);
  }
  count_add(a.stats, PT_C_STEPS, c.steps);
  count_add(a.stats, PT_C_IT32, c.it32);
  count_add(a.stats, PT_C_IT64, c.it64);
  count_add(a.stats, PT_C_CROSS, (unsigned long long)c.tc.cross);
  count_add(a.stats, PT_C_HITS, (unsigned long long)c.tc.hits);
  count_add(a.stats, PT_C_SLOW, (unsigned long long)c.tc.slow);
}

template <int G, bool F64, bool MLP>
__global__ void __launch_bounds__(256) k_locate(const __grid_constant__ LocateArgs a) {
  PT_MLP_PROLOGUE(MLP, a.mlp);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nround = (a.n + stride - 1) / stride * stride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nround; i += stride) {
    const bool inrange = i < a.n;
    double x[3] = {0, 0, 0};
    int e = 0;
    if (inrange) {
      x[0] = a.x[i];
      x[1] = a.x[a.n + i];
      x[2] = a.x[2 * a.n + i];
      e = a.elem[i];
    }
    bool live = inrange && e >= 0 && e < a.m.nelem;
    if (!live) e = 0;
    float guess[3];
    start_guess<G, MLP>(a.m, a.k, sm, &a.mlp, e, x, live, guess);
    if (!inrange) continue;
    double xi[3] = {0, 0, 0};
    int i32 = 0, i64 = 0;
    bool ok = live && locate_one<G, F64>(a.m, a.k, e, x, guess, xi, i32, i64);
    a.xi[i] = xi[0];
    a.xi[a.n + i] = xi[1];
    a.xi[2 * a.n + i] = xi[2];
    if (a.iters) a.iters[i] = i32 + i64;
    if (a.status) a.status[i] = ok ? 0u : (unsigned)PT_ST_NEWTON_FAIL;
  }
}

// Point location without a known element (localisation in reference space,
// Sec. 3.2.3): the candidates are the elements listed in x's cell of a uniform
// background grid, tried closest centre first; the first whose inverse map
// puts x inside (max |xi| <= 1 + lost_tol) owns it.  At most 64 candidates per
// cell (the grid builder guarantees it).
template <int G, bool F64>
__global__ void __launch_bounds__(128) k_find(const __grid_constant__ FindArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const double x[3] = {a.x[i], a.x[a.n + i], a.x[2 * a.n + i]};
    int cidx[3];
    bool inside = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double u = (x[d] - a.lo[d]) * a.ih[d];
      inside = inside && u >= 0.0 && u < (double)a.dims[d];
      cidx[d] = inside ? (int)u : 0;
    }
    int found = -1;
    double xi[3] = {0.0, 0.0, 0.0};
    if (inside) {
      const int cell = cidx[0] + a.dims[0] * (cidx[1] + a.dims[1] * cidx[2]);
      const int beg = a.cell_start[cell];
      const int cnt = min(a.cell_start[cell + 1] - beg, PT_FIND_MAXC);
      unsigned long long done = 0ull;
#pragma unroll 1
      for (int t = 0; t < cnt && found < 0; ++t) {
        int best = -1;
        double bd = 1e300;
#pragma unroll 1
        for (int j = 0; j < cnt; ++j) {
          if ((done >> j) & 1ull) continue;
          const double* ce = a.m.ce + 3 * (size_t)a.cell_elem[beg + j];
          const double dx = x[0] - ce[0], dy = x[1] - ce[1], dz = x[2] - ce[2];
          const double d2 = dx * dx + dy * dy + dz * dz;
          if (d2 < bd) {
            bd = d2;
            best = j;
          }
        }
        done |= 1ull << best;
        const int e = a.cell_elem[beg + best];
        float guess[3];
        start_guess<G, false>(a.m, a.k, nullptr, nullptr, e, x, true, guess);
        double z[3];
        int i32 = 0, i64 = 0;
        if (locate_one<G, F64>(a.m, a.k, e, x, guess, z, i32, i64) &&
            tmax3(z[0], z[1], z[2]) <= 1.0 + a.k.lost_tol) {
          found = e;
          xi[0] = z[0];
          xi[1] = z[1];
          xi[2] = z[2];
        }
      }
    }
    a.elem[i] = found;
    a.xi[i] = xi[0];
    a.xi[a.n + i] = xi[1];
    a.xi[2 * a.n + i] = xi[2];
    if (a.status) a.status[i] = found >= 0 ? 0u : (unsigned)PT_ST_LOST;
  }
}

// Per-particle source of Eq. theory:source: returns the element and fills
// f[4] = (-F, -F.v) and three 1-D weight vectors whose outer product spreads f
// over the element's nodes; false if the particle is frozen or its inverse map
// fails.  Lagrange projection: the bases l(xi).  Nearest-node projection
// (NEAR): one-hot vectors at the node nearest to xi per direction (lower node
// on a tie), with f divided by that node's volume V_ijk = w_i w_j w_k |det J|;
// node[0] receives the node's index within the element.
template <int G, int NP, bool F64, bool NEAR>
__device__ __forceinline__ bool particle_source(const DepositArgs& a, int64_t ip, int& e,
                                                float* f, float* l1, float* l2, float* l3,
                                                int* node, float* xi_out = nullptr) {
  using R = typename RealOf<F64>::type;
  constexpr int N3 = NP * NP * NP;
  const int64_t n = a.p.n;
  if (a.p.status[ip] & PT_ST_FROZEN) return false;
  e = a.p.elem[ip];
  if (e < 0 || e >= a.m.nelem) return false;
  double x[3] = {a.p.x[ip], a.p.x[n + ip], a.p.x[2 * n + ip]};
  const R* vg = reinterpret_cast<const R*>(a.p.v);
  R v[3] = {vg[ip], vg[n + ip], vg[2 * n + ip]};
  R d = reinterpret_cast<const R*>(a.p.d)[ip];
  const double* ce = a.m.ce + 3 * (size_t)e;
  float xf[3] = {(float)(x[0] - __ldg(ce)), (float)(x[1] - __ldg(ce + 1)),
                 (float)(x[2] - __ldg(ce + 2))};
  float guess[3];
  trilinear_guess(a.m, e, xf, guess);
  double xi[3];
  int i32 = 0, i64 = 0;
  if (!locate_one<G, F64>(a.m, a.k, e, x, guess, xi, i32, i64)) return false;
  if (xi_out) {
    xi_out[0] = (float)xi[0];
    xi_out[1] = (float)xi[1];
    xi_out[2] = (float)xi[2];
  }
  R lr1[NP], lr2[NP], lr3[NP], Uv[4];
  lagr<NP, R>((R)xi[0], Nodes<R>::sol(a.k), Nodes<R>::solw(a.k), lr1);
  lagr<NP, R>((R)xi[1], Nodes<R>::sol(a.k), Nodes<R>::solw(a.k), lr2);
  lagr<NP, R>((R)xi[2], Nodes<R>::sol(a.k), Nodes<R>::solw(a.k), lr3);
  interp4<NP, R>(reinterpret_cast<const R*>(a.U) + (size_t)e * 5 * N3, lr1, lr2, lr3, Uv);
  const R mu = (R)a.k.mu;
  R rel[3];
  R irho = R(1) / Uv[0];
#pragma unroll
  for (int r = 0; r < 3; ++r) rel[r] = Uv[1 + r] * irho - v[r];
  R fD = R(1);
  if (a.k.drag_law) {
    R re = Uv[0] * sqrt(rel[0] * rel[0] + rel[1] * rel[1] + rel[2] * rel[2]) * d / mu;
    fD = drag_factor<R>(a.k, re);
  }
  // F = m_p f_D (u - v) / tau_p with m_p / tau_p = 3 pi mu d, plus the lift
  const R c = R(3.14159265358979323846) * R(3) * mu * d * fD;
  R FS[3] = {R(0), R(0), R(0)};
  if (a.k.lift)
    saffman_force<G, NP, R>(a.m, a.k, reinterpret_cast<const R*>(a.U) + (size_t)e * 5 * N3, e, xi,
                            v, d, FS);
  R Fv[3], Fe = R(0);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    Fv[r] = c * rel[r] + FS[r];
    f[r] = (float)(-Fv[r]);
    Fe -= Fv[r] * v[r];
  }
  if constexpr (NEAR) {
    int id[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      int best = 0;
      double bd = fabs(xi[q] - a.k.sn[0]);
#pragma unroll
      for (int i = 1; i < NP; ++i) {
        const double di = fabs(xi[q] - a.k.sn[i]);
        if (di < bd) {
          bd = di;
          best = i;
        }
      }
      id[q] = best;
    }
    const double xn[3] = {a.k.sn[id[0]], a.k.sn[id[1]], a.k.sn[id[2]]};
    double chi[3], J[9];
    map64<G, true>(a.m.xg64 + (size_t)e * G * G * G * 3, xn, a.k, chi, J);
    const double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                       J[2] * (J[3] * J[7] - J[4] * J[6]);
    const R iv = R(1) / (R)(a.k.sq[id[0]] * a.k.sq[id[1]] * a.k.sq[id[2]] * fabs(det));
#pragma unroll
    for (int r = 0; r < 3; ++r) f[r] = (float)(-Fv[r] * iv);
    f[3] = (float)(Fe * iv);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      l1[i] = i == id[0] ? 1.f : 0.f;
      l2[i] = i == id[1] ? 1.f : 0.f;
      l3[i] = i == id[2] ? 1.f : 0.f;
    }
    *node = id[0] + NP * (id[1] + NP * id[2]);
    return true;
  }
  f[3] = (float)Fe;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    l1[i] = (float)lr1[i];
    l2[i] = (float)lr2[i];
    l3[i] = (float)lr3[i];
  }
  *node = 0;
  return true;
}

// FP32 atomics straight into S (S cleared beforehand)
template <int G, int NP, bool F64, bool NEAR>
__global__ void __launch_bounds__(256) k_deposit_atomic(const DepositArgs a) {
  constexpr int N3 = NP * NP * NP;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.p.n; t += stride) {
    const int64_t ip = a.perm ? (int64_t)a.perm[t] : t;
    int e, node;
    float f[4], l1[NP], l2[NP], l3[NP];
    if (!particle_source<G, NP, F64, NEAR>(a, ip, e, f, l1, l2, l3, &node)) continue;
    float* Se = a.S + (size_t)e * 4 * N3;
    if constexpr (NEAR) {
#pragma unroll
      for (int q = 0; q < 4; ++q) atomicAdd(Se + q * N3 + node, f[q]);
    } else {
#pragma unroll 1
      for (int q = 0; q < 4; ++q)
#pragma unroll 1
        for (int kk = 0; kk < NP; ++kk)
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            const float w = f[q] * l3[kk] * l2[j];
#pragma unroll
            for (int i = 0; i < NP; ++i)
              atomicAdd(Se + q * N3 + i + NP * (j + NP * kk), w * l1[i]);
          }
    }
  }
}

// Deterministic segmented reduction in one pass: one block per element; the
// element's particles (a segment of the element-sorted order, each segment in
// particle-index order) are taken CH at a time, their sources computed by one
// thread each and staged as the two factors of
//   S_e[q][i,j,k] = sum_p (f_q l3_k)(p) (l1_i l2_j)(p),
// and every output node sums them in that fixed order -- bitwise reproducible,
// and in FP32 mode bitwise equal to the two-pass form below (same factors,
// same order).
template <int G, int NP, bool F64, bool NEAR>
__global__ void __launch_bounds__(256) k_deposit_segmented(const DepositArgs a) {
  constexpr int N3 = NP * NP * NP;
  constexpr int CH = 64;
  constexpr int NO = (4 * N3 + 255) / 256;
  __shared__ float sA[CH][4 * NP];
  __shared__ float sB[CH][NP * NP];
  for (int e = blockIdx.x; e < a.m.nelem; e += gridDim.x) {
    const int beg = a.offs[e], end = a.offs[e + 1];
    const int total = end - beg;
    float acc[NO];
#pragma unroll
    for (int r = 0; r < NO; ++r) acc[r] = 0.f;
    for (int base = 0; base < total; base += CH) {
      const int cnt = min(CH, total - base);
      __syncthreads();
      if (threadIdx.x < cnt) {
        int ee, node;
        float f[4], l1[NP], l2[NP], l3[NP];
        const bool ok = particle_source<G, NP, F64, NEAR>(a, a.perm[beg + base + threadIdx.x],
                                                          ee, f, l1, l2, l3, &node);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int k = 0; k < NP; ++k) sA[threadIdx.x][q * NP + k] = ok ? f[q] * l3[k] : 0.f;
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
          for (int i = 0; i < NP; ++i) sB[threadIdx.x][i + NP * j] = ok ? l1[i] * l2[j] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < NO; ++r) {
        const int o = threadIdx.x + 256 * r;
        if (o < 4 * N3) {
          const int q = o / N3, node = o - q * N3;
          const int row = q * NP + node / (NP * NP), col = node % (NP * NP);
          float s = acc[r];
          for (int p = 0; p < cnt; ++p) s = fmaf(sA[p][row], sB[p][col], s);
          acc[r] = s;
        }
      }
    }
    float* Se = a.S + (size_t)e * 4 * N3;
#pragma unroll
    for (int r = 0; r < NO; ++r) {
      const int o = threadIdx.x + 256 * r;
      if (o < 4 * N3) Se[o] = acc[r];
    }
  }
}

// Two-pass deterministic deposition.  Pass 1: one thread per particle (in the
// element-sorted order t) computes its source and writes src[2t] = f (or f/V),
// src[2t+1] = (xi, flag): flag 1 live, 0 skipped; for the nearest-node
// projection the node index instead, -1 when skipped.  All threads do the
// expensive part (inverse map, interpolation, drag) instead of one per
// particle of the element being reduced.
template <int G, int NP, bool F64, bool NEAR>
__global__ void __launch_bounds__(128) k_deposit_src(const DepositArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.p.n; t += stride) {
    const int64_t ip = a.perm[t];
    int e, node;
    float f[4], l1[NP], l2[NP], l3[NP], xi[3] = {0.f, 0.f, 0.f};
    const bool ok = particle_source<G, NP, F64, NEAR>(a, ip, e, f, l1, l2, l3, &node, xi);
    float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = make_float4(xi[0], xi[1], xi[2], 0.f);
    if (ok) w0 = make_float4(f[0], f[1], f[2], f[3]);
    if (NEAR)
      w1.w = __int_as_float(ok ? node : -1);
    else
      w1.w = ok ? 1.f : 0.f;
    a.src[2 * t] = w0;
    a.src[2 * t + 1] = w1;
  }
}

// Pass 2: one block per element.  The element's particles are taken in index
// order (the segments of the sorted order are in index order, so the sums are
// bitwise reproducible), CH at a time; each particle's
// weights are staged as the two factors of S[q][i,j,k] = sum_p (f_q l_k)(l_i l_j):
// A[p][q NP + k] = f_q l3_k and B[p][i + NP j] = l1_i l2_j, so every output
// needs two shared loads and one FMA per particle.  Nearest-node projection:
// each output adds the densities of the particles whose node it is.
template <int NP, bool NEAR>
__global__ void __launch_bounds__(256) k_deposit_seg2(const DepositArgs a) {
  constexpr int N3 = NP * NP * NP;
  constexpr int CH = 64;
  constexpr int NO = (4 * N3 + 255) / 256;
  __shared__ float sA[CH][4 * NP];
  __shared__ float sB[CH][NP * NP];
  __shared__ int snode[CH];
  for (int e = blockIdx.x; e < a.m.nelem; e += gridDim.x) {
    const int beg = a.offs[e], end = a.offs[e + 1];
    const int total = end - beg;
    float acc[NO];
#pragma unroll
    for (int r = 0; r < NO; ++r) acc[r] = 0.f;
    for (int base = 0; base < total; base += CH) {
      const int cnt = min(CH, total - base);
      __syncthreads();
      if (threadIdx.x < cnt) {
        const int t = beg + base + threadIdx.x;
        const float4 w0 = a.src[2 * (int64_t)t], w1 = a.src[2 * (int64_t)t + 1];
        const float f[4] = {w0.x, w0.y, w0.z, w0.w};
        if (NEAR) {
          snode[threadIdx.x] = __float_as_int(w1.w);
#pragma unroll
          for (int q = 0; q < 4; ++q) sA[threadIdx.x][q] = f[q];
        } else {
          const bool ok = w1.w != 0.f;
          float l1[NP], l2[NP], l3[NP];
          lagr<NP, float>(w1.x, a.k.sn32, a.k.sw32, l1);
          lagr<NP, float>(w1.y, a.k.sn32, a.k.sw32, l2);
          lagr<NP, float>(w1.z, a.k.sn32, a.k.sw32, l3);
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < NP; ++k) sA[threadIdx.x][q * NP + k] = ok ? f[q] * l3[k] : 0.f;
#pragma unroll
          for (int j = 0; j < NP; ++j)
#pragma unroll
            for (int i = 0; i < NP; ++i) sB[threadIdx.x][i + NP * j] = l1[i] * l2[j];
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < NO; ++r) {
        const int o = threadIdx.x + 256 * r;
        if (o < 4 * N3) {
          const int q = o / N3, node = o - q * N3;
          float sacc = acc[r];
          if (NEAR) {
            for (int p = 0; p < cnt; ++p)
              if (snode[p] == node) sacc += sA[p][q];
          } else {
            const int row = q * NP + node / (NP * NP), col = node % (NP * NP);
            for (int p = 0; p < cnt; ++p) sacc = fmaf(sA[p][row], sB[p][col], sacc);
          }
          acc[r] = sacc;
        }
      }
    }
    float* Se = a.S + (size_t)e * 4 * N3;
#pragma unroll
    for (int r = 0; r < NO; ++r) {
      const int o = threadIdx.x + 256 * r;
      if (o < 4 * N3) Se[o] = acc[r];
    }
  }
}

// First RK stage of each particle without tracking, by the push's own code:
// inverse map (trilinear start, the mode's Newton), interpolation of rho and
// rho u, the acceleration, and the stage increments B_1 k_x, B_1 k_v with
// k_x = dt v, k_v = dt a (the registers start at zero in a step).  Reports each
// result of the precision split separately, for comparison with FP64 values.
template <int G, int NP, bool F64>
__global__ void __launch_bounds__(128) k_terms(const __grid_constant__ TermsArgs a) {
  using R = typename RealOf<F64>::type;
  constexpr int N3 = NP * NP * NP;
  const int64_t n = a.p.n;
  const R* vg = reinterpret_cast<const R*>(a.p.v);
  const R* dg = reinterpret_cast<const R*>(a.p.d);
  const R* U = reinterpret_cast<const R*>(a.U);
  R* Uo = reinterpret_cast<R*>(a.Uo);
  R* ao = reinterpret_cast<R*>(a.acc);
  R* xo = reinterpret_cast<R*>(a.dx);
  R* vo = reinterpret_cast<R*>(a.dv);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int e = a.p.elem[i];
    unsigned st = 0u;
    if (e < 0 || e >= a.m.nelem) {
      a.p.status[i] = PT_ST_LOST;
      continue;
    }
    const R v[3] = {vg[i], vg[n + i], vg[2 * n + i]};
    const R d = dg[i];
    const double* ce = a.m.ce + 3 * (size_t)e;
    const double xl[3] = {a.p.x[i] - __ldg(ce), a.p.x[n + i] - __ldg(ce + 1),
                          a.p.x[2 * n + i] - __ldg(ce + 2)};
    double xi[3];
    R Uv[4], acc[3];
    int i32 = 0, i64 = 0;
    const R tau = (R)a.k.rho_p * d * d / (R(18) * (R)a.k.mu);
    if constexpr (F64) {
      const float xf[3] = {(float)xl[0], (float)xl[1], (float)xl[2]};
      float guess[3];
      trilinear_guess(a.m, e, xf, guess);
      if (!locate_local<G, true>(a.m, a.k, e, xl, guess, xi, i32, i64)) {
        a.p.status[i] = PT_ST_NEWTON_FAIL;
        continue;
      }
      R l1[NP], l2[NP], l3[NP];
      lagr<NP, R>((R)xi[0], Nodes<R>::sol(a.k), Nodes<R>::solw(a.k), l1);
      lagr<NP, R>((R)xi[1], Nodes<R>::sol(a.k), Nodes<R>::solw(a.k), l2);
      lagr<NP, R>((R)xi[2], Nodes<R>::sol(a.k), Nodes<R>::solw(a.k), l3);
      interp4<NP, R>(U + (size_t)e * 5 * N3, l1, l2, l3, Uv);
      particle_accel<G, NP, R>(a.m, a.k, U + (size_t)e * 5 * N3, e, xi, Uv, v, d, tau, st, acc);
    } else {
      df xd[3], zd[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) xd[r] = df_from_double(xl[r]);
      const float xf[3] = {xd[0].hi, xd[1].hi, xd[2].hi};
      float guess[3];
      trilinear_guess(a.m, e, xf, guess);
      if (!newton_df<G>(a.m, a.k, e, xd, guess, zd, i32, i64)) {
        a.p.status[i] = PT_ST_NEWTON_FAIL;
        continue;
      }
      const float xs[3] = {zd[0].hi + zd[0].lo, zd[1].hi + zd[1].lo, zd[2].hi + zd[2].lo};
      float l1[NP], l2[NP], l3[NP];
      lagr<NP, float>(xs[0], a.k.sn32, a.k.sw32, l1);
      lagr<NP, float>(xs[1], a.k.sn32, a.k.sw32, l2);
      lagr<NP, float>(xs[2], a.k.sn32, a.k.sw32, l3);
      interp4<NP, float>(reinterpret_cast<const float*>(U) + (size_t)e * 5 * N3, l1, l2, l3,
                         reinterpret_cast<float*>(Uv));
      particle_accel_f32<G, NP>(a.m, a.k, reinterpret_cast<const float*>(U) + (size_t)e * 5 * N3,
                                e, zd, reinterpret_cast<const float*>(Uv),
                                reinterpret_cast<const float*>(v), (float)d, (float)tau, st,
                                reinterpret_cast<float*>(acc));
#pragma unroll
      for (int r = 0; r < 3; ++r) xi[r] = df_to_double(zd[r]);
    }
    const R dt = (R)a.dt;
    const R B1 = F64 ? (R)a.k.B[0] : (R)a.k.B32[0];
    const R A1 = F64 ? (R)a.k.A[0] : (R)a.k.A32[0];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      a.xi[r * n + i] = xi[r];
      ao[r * n + i] = acc[r];
      // the push's register update with the registers at zero (first stage)
      const R kx = A1 * R(0) + dt * v[r], kv = A1 * R(0) + dt * acc[r];
      xo[r * n + i] = B1 * kx;
      vo[r * n + i] = B1 * kv;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) Uo[q * n + i] = Uv[q];
    a.p.status[i] = st;
  }
}

}  // namespace pt
#include "pt_staged.cuh"
namespace pt {

// launch helpers for one (G, mode) family
template <int G, bool F64>
struct Family {
  // the learned start exists only for NGeo = 3 in FP32 mode
  static constexpr bool kMlp = (G == 4) && !F64;
  template <int NP>
  static int push(const PushArgs& a, int grid, int block, cudaStream_t s) {
    // curved faces by Bezier clipping: separate instantiations, so that the
    // default kernels carry none of its code
    const bool mlp = kMlp && a.k.guess == PT_GUESS_MLP;
    if (a.k.curved_clip) {
      if (mlp)
        k_push<G, NP, F64, kMlp, true><<<grid, block, 0, s>>>(a);
      else
        k_push<G, NP, F64, false, true><<<grid, block, 0, s>>>(a);
    } else if (mlp) {
      k_push<G, NP, F64, kMlp><<<grid, block, 0, s>>>(a);
    } else {
      k_push<G, NP, F64, false><<<grid, block, 0, s>>>(a);
    }
    return (int)cudaGetLastError();
  }
  // mode bit 0: segmented summation, bit 1: nearest-node projection
  template <int NP>
  static int dep(int mode, const DepositArgs& a, int grid, int block, cudaStream_t s) {
    switch (mode) {
      case 0: k_deposit_atomic<G, NP, F64, false><<<grid, block, 0, s>>>(a); break;
      case 1: k_deposit_segmented<G, NP, F64, false><<<grid, 256, 0, s>>>(a); break;
      case 2: k_deposit_atomic<G, NP, F64, true><<<grid, block, 0, s>>>(a); break;
      case 3: k_deposit_segmented<G, NP, F64, true><<<grid, 256, 0, s>>>(a); break;
      // bit 2: two-pass segmented summation with the sources in a.src
      case 5:
      case 7: {
        const int g1 = (int)std::min<int64_t>((a.p.n + 127) / 128, (int64_t)grid * 8);
        if (a.p.n > 0) {
          if (mode == 5)
            k_deposit_src<G, NP, F64, false><<<std::max(g1, 1), 128, 0, s>>>(a);
          else
            k_deposit_src<G, NP, F64, true><<<std::max(g1, 1), 128, 0, s>>>(a);
        }
        if (mode == 5)
          k_deposit_seg2<NP, false><<<grid, 256, 0, s>>>(a);
        else
          k_deposit_seg2<NP, true><<<grid, 256, 0, s>>>(a);
        break;
      }
      default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
  }
  template <int NP>
  static int occ(int block) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push<G, NP, F64, false>, block, 0);
    return nb;
  }
  static int push_np(int np, const PushArgs& a, int grid, int block, cudaStream_t s) {
    switch (np) {
      case 2: return push<2>(a, grid, block, s);
      case 3: return push<3>(a, grid, block, s);
      case 4: return push<4>(a, grid, block, s);
      case 5: return push<5>(a, grid, block, s);
      case 6: return push<6>(a, grid, block, s);
      case 7: return push<7>(a, grid, block, s);
      case 8: return push<8>(a, grid, block, s);
    }
    return (int)cudaErrorInvalidValue;
  }
  static int dep_np(int np, int mode, const DepositArgs& a, int grid, int block, cudaStream_t s) {
    switch (np) {
      case 2: return dep<2>(mode, a, grid, block, s);
      case 3: return dep<3>(mode, a, grid, block, s);
      case 4: return dep<4>(mode, a, grid, block, s);
      case 5: return dep<5>(mode, a, grid, block, s);
      case 6: return dep<6>(mode, a, grid, block, s);
      case 7: return dep<7>(mode, a, grid, block, s);
      case 8: return dep<8>(mode, a, grid, block, s);
    }
    return (int)cudaErrorInvalidValue;
  }
  static int occ_np(int np, int block) {
    switch (np) {
      case 2: return occ<2>(block);
      case 3: return occ<3>(block);
      case 4: return occ<4>(block);
      case 5: return occ<5>(block);
      case 6: return occ<6>(block);
      case 7: return occ<7>(block);
      case 8: return occ<8>(block);
    }
    return 0;
  }
  static int terms_np(int np, const TermsArgs& a, int grid, int block, cudaStream_t s) {
    switch (np) {
      case 2: k_terms<G, 2, F64><<<grid, block, 0, s>>>(a); break;
      case 3: k_terms<G, 3, F64><<<grid, block, 0, s>>>(a); break;
      case 4: k_terms<G, 4, F64><<<grid, block, 0, s>>>(a); break;
      case 5: k_terms<G, 5, F64><<<grid, block, 0, s>>>(a); break;
      case 6: k_terms<G, 6, F64><<<grid, block, 0, s>>>(a); break;
      case 7: k_terms<G, 7, F64><<<grid, block, 0, s>>>(a); break;
      case 8: k_terms<G, 8, F64><<<grid, block, 0, s>>>(a); break;
      default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
  }
  // dynamic shared memory of k_stage_f32: the warp slots (blocks of 128 threads)
  template <int NP>
  static constexpr int stage_dyn_smem() {
    if constexpr (F64)
      return 0;
    else
      return UStage<NP>::ok ? 0 : WSlot<G, NP>::bytes;
  }
  // allows the dynamic shared memory above 48 KB per block; set once per
  // instantiation, before the first occupancy query or launch
  template <int NP>
  static void stage_smem_attr() {
    constexpr int dyn = stage_dyn_smem<NP>();
    if constexpr (dyn > 0) {
      static bool attr = false;
      if (!attr) {
        cudaFuncSetAttribute(k_stage_f32<G, NP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             dyn);
        cudaFuncSetAttribute(k_stage_f32<G, NP, kMlp>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             dyn);
        attr = true;
      }
    }
  }
  template <int NP>
  static int staged(int op, const StageArgs& a, const DevParticles& p, const int* perm, int grid,
                    int block, cudaStream_t s) {
    const bool clip = a.k.curved_clip != 0;
    switch (op) {
      case PT_SOP_GATHER: k_gather<F64><<<grid, block, 0, s>>>(a, p, perm); break;
      case PT_SOP_SCATTER: k_scatter_back<F64><<<grid, block, 0, s>>>(a, p, perm); break;
      case PT_SOP_STAGE:
        if constexpr (F64) {
          k_stage_f64<G, NP><<<grid, block, 0, s>>>(a);
        } else if (PT_STAGE_SPLIT && !UStage<NP>::ok) {
          if (kMlp && a.k.guess == PT_GUESS_MLP)
            k_locate_f32<G, kMlp><<<grid, block, 0, s>>>(a);
          else
            k_locate_f32<G, false><<<grid, block, 0, s>>>(a);
          k_advance_f32<G, NP><<<grid, block, 0, s>>>(a);
        } else {
          constexpr int dyn = stage_dyn_smem<NP>();
          stage_smem_attr<NP>();
          if (kMlp && a.k.guess == PT_GUESS_MLP)
            k_stage_f32<G, NP, kMlp><<<grid, block, dyn, s>>>(a);
          else
            k_stage_f32<G, NP, false><<<grid, block, dyn, s>>>(a);
        }
        break;
      case PT_SOP_TRACK:
        if constexpr (F64) {
          if (clip)
            k_track_f64<G, true><<<grid, block, 0, s>>>(a);
          else
            k_track_f64<G, false><<<grid, block, 0, s>>>(a);
        } else {
          if (clip)
            k_track_f32<G, true><<<grid, block, 0, s>>>(a);
          else
            k_track_f32<G, false><<<grid, block, 0, s>>>(a);
        }
        break;
      case PT_SOP_GUESS:
      case PT_SOP_GUESS_X_TC:
      case PT_SOP_GUESS_X_WARP:
        if constexpr (kMlp) {
          const bool tc = op == PT_SOP_GUESS_X_TC || (op == PT_SOP_GUESS && PT_MLP_TC);
          if (tc) {
            static bool attr = false;  // dynamic shared memory above 48 KB, set once
            if (!attr) {
              cudaFuncSetAttribute(k_guess_tc<G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kMlpTcSmem);
              cudaFuncSetAttribute(k_guess_tc<G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kMlpTcSmem);
              attr = true;
            }
            if (op == PT_SOP_GUESS)
              k_guess_tc<G, false><<<grid, 128, kMlpTcSmem, s>>>(a);
            else
              k_guess_tc<G, true><<<grid, 128, kMlpTcSmem, s>>>(a);
          } else if (op == PT_SOP_GUESS) {
            k_guess_mlp<G, false><<<grid, block, 0, s>>>(a);
          } else {
            k_guess_mlp<G, true><<<grid, block, 0, s>>>(a);
          }
          break;
        } else {
          return (int)cudaErrorInvalidValue;
        }
      default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
  }
  template <int NP>
  static int occ_stage(int block) {
    int nb = 0;
    if constexpr (F64) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage_f64<G, NP>, block, 0);
    } else if (PT_STAGE_SPLIT && !UStage<NP>::ok) {
      int nl = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_advance_f32<G, NP>, block, 0);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nl, k_locate_f32<G, false>, block, 0);
      nb = nb < nl ? nb : nl;
    } else {
      stage_smem_attr<NP>();
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage_f32<G, NP, false>, block,
                                                    stage_dyn_smem<NP>());
    }
    return nb;
  }
  static int staged_np(int np, int op, const StageArgs& a, const DevParticles& p, const int* perm,
                       int grid, int block, cudaStream_t s) {
    switch (np) {
      case 2: return staged<2>(op, a, p, perm, grid, block, s);
      case 3: return staged<3>(op, a, p, perm, grid, block, s);
      case 4: return staged<4>(op, a, p, perm, grid, block, s);
      case 5: return staged<5>(op, a, p, perm, grid, block, s);
      case 6: return staged<6>(op, a, p, perm, grid, block, s);
      case 7: return staged<7>(op, a, p, perm, grid, block, s);
      case 8: return staged<8>(op, a, p, perm, grid, block, s);
    }
    return (int)cudaErrorInvalidValue;
  }
  static int occ_stage_np(int np, int block) {
    switch (np) {
      case 2: return occ_stage<2>(block);
      case 3: return occ_stage<3>(block);
      case 4: return occ_stage<4>(block);
      case 5: return occ_stage<5>(block);
      case 6: return occ_stage<6>(block);
      case 7: return occ_stage<7>(block);
      case 8: return occ_stage<8>(block);
    }
    return 0;
  }
  static int find(const FindArgs& a, int grid, int block, cudaStream_t s) {
    k_find<G, F64><<<grid, block, 0, s>>>(a);
    return (int)cudaGetLastError();
  }
  static int locate(const LocateArgs& a, int grid, int block, cudaStream_t s) {
    if (kMlp && a.k.guess == PT_GUESS_MLP)
      k_locate<G, F64, kMlp><<<grid, block, 0, s>>>(a);
    else
      k_locate<G, F64, false><<<grid, block, 0, s>>>(a);
    return (int)cudaGetLastError();
  }
};

}  // namespace pt

#define PT_DEFINE_FAMILY(G, F64, NAME)                                                       \
  namespace pt {                                                                             \
  int NAME##_push(int np, const PushArgs& a, int grid, int block, void* s) {                 \
    return Family<G, F64>::push_np(np, a, grid, block, (cudaStream_t)s);                     \
  }                                                                                          \
  int NAME##_dep(int np, int mode, const DepositArgs& a, int grid, int block, void* s) {     \
    return Family<G, F64>::dep_np(np, mode, a, grid, block, (cudaStream_t)s);                \
  }                                                                                          \
  int NAME##_occ(int np, int block) { return Family<G, F64>::occ_np(np, block); }            \
  int NAME##_loc(const LocateArgs& a, int grid, int block, void* s) {                        \
    return Family<G, F64>::locate(a, grid, block, (cudaStream_t)s);                          \
  }                                                                                          \
  int NAME##_find(const FindArgs& a, int grid, int block, void* s) {                         \
    return Family<G, F64>::find(a, grid, block, (cudaStream_t)s);                            \
  }                                                                                          \
  int NAME##_terms(int np, const TermsArgs& a, int grid, int block, void* s) {              \
    return Family<G, F64>::terms_np(np, a, grid, block, (cudaStream_t)s);                    \
  }                                                                                          \
  int NAME##_staged(int np, int op, const StageArgs& a, const DevParticles& p, const int* perm,\
                    int grid, int block, void* s) {                                         \
    return Family<G, F64>::staged_np(np, op, a, p, perm, grid, block, (cudaStream_t)s);     \
  }                                                                                         \
  int NAME##_occs(int np, int block) { return Family<G, F64>::occ_stage_np(np, block); }    \
  }
