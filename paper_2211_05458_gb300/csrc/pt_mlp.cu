// pt_mlp.cu -- learned Newton start (no counterpart in the paper): geometry
// features, training pairs labelled by the FP64 Newton inverse, FP32 forward /
// backward kernels, Adam, and the export of the BF16 copy used by the push.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "pt_ctx.h"
#include "pt_device.cuh"
#include "pt_internal.h"

namespace {

constexpr int NPAR = PT_MLP_NP;  // 11843
constexpr int OFF_W1 = 0, OFF_B1 = 64 * 51, OFF_W2 = OFF_B1 + 64, OFF_B2 = OFF_W2 + 4096,
              OFF_W3 = OFF_B2 + 64, OFF_B3 = OFF_W3 + 4096, OFF_W4 = OFF_B3 + 64,
              OFF_B4 = OFF_W4 + 192;
static_assert(OFF_B4 + 3 == NPAR, "parameter layout");
constexpr int NNORM = 51 + 51 + 3;  // in_mean, in_std, out_scale

// SplitMix64 (Steele, Lea & Flood 2014): a counter-based 64-bit hash
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__host__ __device__ inline double u01(uint64_t h) { return (double)(h >> 11) * 0x1.0p-53; }

}  // namespace

struct pt_mlp_state {
  float* theta = nullptr;   // FP32 master parameters [NPAR]
  float* grad = nullptr;    // [NPAR]
  float* m = nullptr;       // Adam moments
  float* v = nullptr;
  float* norm = nullptr;    // [NNORM] device copy
  float* feat48 = nullptr;  // [E][48] per-element geometry deviations
  uint16_t* w2b = nullptr;  // BF16 export
  uint16_t* w3b = nullptr;
  float* w1x = nullptr;     // [64][3]
  float* b2 = nullptr;
  float* b3 = nullptr;
  float* w4s = nullptr;     // [3][64] scaled by out_scale
  float* b4s = nullptr;     // [3]
  double* dacc = nullptr;   // reductions scratch [64]
  float h_w1x[192], h_b2[64], h_b3[64], h_w4s[192], h_b4s[4];  // host copies for kernel params
  float hnorm[NNORM];
  bool have_theta = false;
};

static pt_status mfail(pt_ctx* c, pt_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define MCK(call)                                                                             \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return mfail(c, PT_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                   __LINE__);                                                                 \
  } while (0)

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------

// 48 deviations of element e (NGeo = 3): for the edge- and face-interior
// geometry nodes in node-index order, (y_node - y_trilinear) / h_y, where the
// trilinear map interpolates the 8 corner nodes and h_y is the mean y-length
// of the four xi2-edges.
__global__ void k_elem_features(const double* __restrict__ xg64, int nelem, float* feat48) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nelem) return;
  constexpr int G = 4, L = G - 1;
  const double* X = xg64 + (size_t)e * G * G * G * 3;
  double cy[8];
  for (int q = 0; q < 8; ++q) {
    int a = (q & 1) ? L : 0, b = (q & 2) ? L : 0, c = (q & 4) ? L : 0;
    cy[q] = X[3 * (a + G * (b + G * c)) + 1];
  }
  double hy = 0.0;
  for (int q = 0; q < 8; ++q)
    if (q & 2) hy += fabs(cy[q] - cy[q & ~2]) * 0.25;
  int k = 0;
  for (int c = 0; c < G; ++c)
    for (int b = 0; b < G; ++b)
      for (int a = 0; a < G; ++a) {
        int nb = (a == 0 || a == L) + (b == 0 || b == L) + (c == 0 || c == L);
        if (nb != 1 && nb != 2) continue;
        double xi[3] = {-1.0 + 2.0 * a / L, -1.0 + 2.0 * b / L, -1.0 + 2.0 * c / L};
        double yt = 0.0;
        for (int q = 0; q < 8; ++q) {
          double w = 1.0;
          for (int d = 0; d < 3; ++d) w *= 0.5 * (1.0 + (((q >> d) & 1) ? xi[d] : -xi[d]));
          yt += w * cy[q];
        }
        if (k < 48) feat48[48 * (size_t)e + k] = (float)((X[3 * (a + G * (b + G * c)) + 1] - yt) / hy);
        ++k;
      }
}

__global__ void k_particle_features(DevMesh m, int64_t n, const double* x, const int* elem,
                                    const float* feat48, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int e = elem[i];
  float* o = out + 51 * i;
  if (e < 0 || e >= m.nelem) {
    for (int q = 0; q < 51; ++q) o[q] = 0.f;
    return;
  }
  const double* ce = m.ce + 3 * (size_t)e;
  float xf[3] = {(float)(x[i] - ce[0]), (float)(x[n + i] - ce[1]), (float)(x[2 * n + i] - ce[2])};
  float g[3];
  pt::trilinear_guess(m, e, xf, g);
  o[0] = g[0];
  o[1] = g[1];
  o[2] = g[2];
  for (int q = 0; q < 48; ++q) o[3 + q] = feat48[48 * (size_t)e + q];
}

// Training pairs: element and reference point from the counter-based hash of
// (seed, i); x = chi(xi) in FP64; label = FP64 Newton inverse of x from the
// trilinear start (plain Newton measures the learned start's error).
__global__ void k_mlp_pairs(DevMesh m, DevConsts k, int64_t n, uint64_t seed, const float* feat48,
                            float* in, float* tgt, unsigned* nfail) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int G = 4;
  const uint64_t base = splitmix64(seed ^ splitmix64((uint64_t)i));
  const int e = (int)(splitmix64(base + 1) % (uint64_t)m.nelem);
  double xi_true[3];
  for (int q = 0; q < 3; ++q) xi_true[q] = 2.0 * u01(splitmix64(base + 2 + q)) - 1.0;
  const double* X64 = m.xg64 + (size_t)e * 3 * G * G * G;
  double xl[3];
  pt::map64<G, false>(X64, xi_true, k, xl, nullptr);
  float xf[3] = {(float)xl[0], (float)xl[1], (float)xl[2]}, g[3];
  pt::trilinear_guess(m, e, xf, g);
  double xi[3] = {g[0], g[1], g[2]};
  int it = 0;
  bool ok = pt::newton64<G>(X64, xl, xi, k, k.max_newton, it);
  if (!ok) {
    atomicAdd(nfail, 1u);
    for (int q = 0; q < 3; ++q) xi[q] = xi_true[q];
  }
  float* o = in + 51 * i;
  o[0] = g[0];
  o[1] = g[1];
  o[2] = g[2];
  for (int q = 0; q < 48; ++q) o[3 + q] = feat48[48 * (size_t)e + q];
  for (int q = 0; q < 3; ++q) tgt[3 * i + q] = (float)(xi[q] - (double)g[q]);
}

// column sums and sums of squares of in[n][51] and tgt[n][3] (double atomics)
__global__ void k_colstats(int64_t n, const float* in, const float* tgt, double* acc) {
  double s[54], s2[54];
  for (int q = 0; q < 54; ++q) s[q] = s2[q] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int q = 0; q < 51; ++q) {
      double v = in[51 * i + q];
      s[q] += v;
      s2[q] += v * v;
    }
    for (int q = 0; q < 3; ++q) {
      double v = tgt[3 * i + q];
      s[51 + q] += v;
      s2[51 + q] += v * v;
    }
  }
  for (int q = 0; q < 54; ++q) {
    double a = s[q], b = s2[q];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(acc + q, a);
      atomicAdd(acc + 54 + q, b);
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 forward / backward of a batch (one block = TB samples)
// ---------------------------------------------------------------------------

constexpr int TB = 32;
constexpr int NTH = 256;
constexpr int XLD = 52;
constexpr size_t FB_SMEM =
    sizeof(float) * ((size_t)(NPAR + 1) + TB * XLD + 6 * TB * 64 + 2 * TB * 64 + TB * 4);

__device__ __forceinline__ float gelu_ex(float z) {
  return 0.5f * z * (1.f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_dx(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) +
         z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

struct FBArgs {
  const float* theta;
  const float* in;
  const float* tgt;
  const float* norm;    // mean[51], std[51], oscale[3], or null (inputs already normalised)
  int64_t nrows;        // rows available
  int64_t row0;         // first batch row (position in the shuffled order)
  int B;                // batch rows
  uint64_t pa, pb;      // shuffle: row j -> (pa * j + pb) mod nrows (pa coprime with nrows)
  float* grad;          // accumulated (atomics) or null for forward only
  double* loss;         // accumulated or null
  float* out;           // forward output [B][3] or null
};

__global__ void __launch_bounds__(NTH) k_mlp_fb(const FBArgs a) {
  extern __shared__ float sm[];
  float* W = sm;
  float* X = W + NPAR + 1;
  float* Z1 = X + TB * XLD;
  float* H1 = Z1 + TB * 64;
  float* Z2 = H1 + TB * 64;
  float* H2 = Z2 + TB * 64;
  float* Z3 = H2 + TB * 64;
  float* H3 = Z3 + TB * 64;
  float* dA = H3 + TB * 64;
  float* dZ = dA + TB * 64;
  float* dY = dZ + TB * 64;
  const int tid = threadIdx.x;
  for (int i = tid; i < NPAR; i += NTH) W[i] = a.theta[i];
  __shared__ int valid[TB];
  for (int idx = tid; idx < TB * XLD; idx += NTH) {
    const int s = idx / XLD, q = idx % XLD;
    const int64_t gi = a.row0 + (int64_t)blockIdx.x * TB + s;
    const bool ok = gi < a.row0 + a.B && gi < a.nrows;
    if (q == 0) valid[s] = ok;
    float v = 0.f;
    if (ok && q < 51) {
      const int64_t j = (int64_t)((a.pa * (uint64_t)gi + a.pb) % (uint64_t)a.nrows);
      v = a.in[51 * j + q];
      if (a.norm) v = (v - a.norm[q]) / a.norm[51 + q];
    }
    X[s * XLD + q] = v;
  }
  __syncthreads();
  // forward
  const float* Hin[3] = {X, H1, H2};
  float* Zo[3] = {Z1, Z2, Z3};
  float* Ho[3] = {H1, H2, H3};
  const int offW[3] = {OFF_W1, OFF_W2, OFF_W3}, offB[3] = {OFF_B1, OFF_B2, OFF_B3};
  for (int l = 0; l < 3; ++l) {
    const int nin = l == 0 ? 51 : 64, ld = l == 0 ? XLD : 64;
    for (int idx = tid; idx < TB * 64; idx += NTH) {
      const int s = idx >> 6, o = idx & 63;
      float z = W[offB[l] + o];
      const float* w = W + offW[l] + o * nin;
      const float* h = Hin[l] + s * ld;
      for (int i = 0; i < nin; ++i) z = fmaf(w[i], h[i], z);
      Zo[l][idx] = z;
      Ho[l][idx] = gelu_ex(z);
    }
    __syncthreads();
  }
  double lsum = 0.0;
  for (int idx = tid; idx < TB * 3; idx += NTH) {
    const int s = idx / 3, q = idx % 3;
    float y = W[OFF_B4 + q];
    for (int i = 0; i < 64; ++i) y = fmaf(W[OFF_W4 + 64 * q + i], H3[s * 64 + i], y);
    float d = 0.f;
    if (valid[s]) {
      const int64_t gi = a.row0 + (int64_t)blockIdx.x * TB + s;
      if (a.out) a.out[3 * (gi - a.row0) + q] = y;
      if (a.tgt) {
        const int64_t j = (int64_t)((a.pa * (uint64_t)gi + a.pb) % (uint64_t)a.nrows);
        float t = a.tgt[3 * j + q];
        if (a.norm) t /= a.norm[102 + q];
        const float r = y - t;
        lsum += (double)r * r / (3.0 * a.B);
        d = 2.f * r / (3.f * a.B);
      }
    }
    dY[s * 4 + q] = d;
  }
  if (a.loss) {
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0 && lsum != 0.0) atomicAdd(a.loss, lsum);
  }
  if (!a.grad) return;
  __syncthreads();
  // output layer gradients
  for (int idx = tid; idx < 3 * 64 + 3; idx += NTH) {
    float g = 0.f;
    if (idx < 192) {
      const int q = idx >> 6, i = idx & 63;
      for (int s = 0; s < TB; ++s) g = fmaf(dY[s * 4 + q], H3[s * 64 + i], g);
      atomicAdd(a.grad + OFF_W4 + idx, g);
    } else {
      const int q = idx - 192;
      for (int s = 0; s < TB; ++s) g += dY[s * 4 + q];
      atomicAdd(a.grad + OFF_B4 + q, g);
    }
  }
  for (int idx = tid; idx < TB * 64; idx += NTH) {
    const int s = idx >> 6, i = idx & 63;
    float g = 0.f;
    for (int q = 0; q < 3; ++q) g = fmaf(W[OFF_W4 + 64 * q + i], dY[s * 4 + q], g);
    dZ[idx] = g * gelu_dx(Z3[idx]);
  }
  __syncthreads();
  for (int l = 2; l >= 0; --l) {
    const int nin = l == 0 ? 51 : 64, ld = l == 0 ? XLD : 64;
    const float* Hp = Hin[l];
    // weight and bias gradients of layer l: dW[o][i] = sum_s dZ[s][o] Hp[s][i]
    for (int idx = tid; idx < 64 * nin + 64; idx += NTH) {
      float g = 0.f;
      if (idx < 64 * nin) {
        const int o = idx / nin, i = idx % nin;
        for (int s = 0; s < TB; ++s) g = fmaf(dZ[s * 64 + o], Hp[s * ld + i], g);
        atomicAdd(a.grad + offW[l] + idx, g);
      } else {
        const int o = idx - 64 * nin;
        for (int s = 0; s < TB; ++s) g += dZ[s * 64 + o];
        atomicAdd(a.grad + offB[l] + o, g);
      }
    }
    if (l == 0) break;
    // dZ of the layer below: (W^T dZ) * GELU'(Z_{l-1})
    for (int idx = tid; idx < TB * 64; idx += NTH) {
      const int s = idx >> 6, i = idx & 63;
      float g = 0.f;
      for (int o = 0; o < 64; ++o) g = fmaf(W[offW[l] + 64 * o + i], dZ[s * 64 + o], g);
      dA[idx] = g * gelu_dx(Zo[l - 1][idx]);
    }
    __syncthreads();
    for (int idx = tid; idx < TB * 64; idx += NTH) dZ[idx] = dA[idx];
    __syncthreads();
  }
}

__global__ void k_adam(float* th, float* g, float* m, float* v, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  g[i] = 0.f;
}

// Element part of layer 1 after folding the input normalisation:
// pre_e[o] = b1[o] + sum_j W1[o][3+j] (f_ej - mean_j)/std_j - sum_q W1[o][q] mean_q / std_q
__global__ void k_mlp_pre(const float* th, const float* norm, const float* feat48, int nelem,
                          float* pre) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nelem * 64) return;
  const int e = (int)(idx >> 6), o = (int)(idx & 63);
  float z = th[OFF_B1 + o];
  for (int q = 0; q < 3; ++q) z -= th[OFF_W1 + 51 * o + q] * norm[q] / norm[51 + q];
  for (int j = 0; j < 48; ++j)
    z += th[OFF_W1 + 51 * o + 3 + j] * (feat48[48 * (size_t)e + j] - norm[3 + j]) / norm[54 + j];
  pre[idx] = z;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

DevMLP pt_dev_mlp(const pt_ctx* c) {
  DevMLP m;
  std::memset(&m, 0, sizeof m);
  if (!c->mlp || !c->mlp_ready) return m;
  m.w2 = c->mlp->w2b;
  m.w3 = c->mlp->w3b;
  std::memcpy(m.w1x, c->mlp->h_w1x, sizeof m.w1x);
  std::memcpy(m.b2, c->mlp->h_b2, sizeof m.b2);
  std::memcpy(m.b3, c->mlp->h_b3, sizeof m.b3);
  std::memcpy(m.w4, c->mlp->h_w4s, sizeof m.w4);
  std::memcpy(m.b4, c->mlp->h_b4s, sizeof m.b4);
  return m;
}

void pt_mlp_release(pt_ctx* c) {
  if (!c->mlp) return;
  pt_mlp_state* s = c->mlp;
  void* ptrs[] = {s->theta, s->grad, s->m, s->v, s->norm, s->feat48, s->w2b, s->w3b,
                  s->w1x,   s->b2,   s->b3, s->w4s, s->b4s, s->dacc};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->d_mlp_pre) cudaFree(c->d_mlp_pre);
  c->d_mlp_pre = nullptr;
  delete s;
  c->mlp = nullptr;
  c->mlp_ready = false;
}

void pt_fill_consts(const pt_ctx* c, DevConsts& k);
DevMesh pt_dev_mesh(const pt_ctx* c);

static pt_status ensure_state(pt_ctx* c) {
  if (c->g != 4) return mfail(c, PT_ERR_STATE, "the learned guess needs ngeo = 3");
  if (c->mlp) return PT_OK;
  pt_mlp_state* s = new pt_mlp_state();
  c->mlp = s;
  MCK(cudaMalloc(&s->theta, NPAR * 4));
  MCK(cudaMalloc(&s->grad, NPAR * 4));
  MCK(cudaMalloc(&s->m, NPAR * 4));
  MCK(cudaMalloc(&s->v, NPAR * 4));
  MCK(cudaMalloc(&s->norm, NNORM * 4));
  MCK(cudaMalloc(&s->feat48, (size_t)c->nelem * 48 * 4));
  MCK(cudaMalloc(&s->w2b, 4096 * 2));
  MCK(cudaMalloc(&s->w3b, 4096 * 2));
  MCK(cudaMalloc(&s->w1x, 192 * 4));
  MCK(cudaMalloc(&s->b2, 64 * 4));
  MCK(cudaMalloc(&s->b3, 64 * 4));
  MCK(cudaMalloc(&s->w4s, 192 * 4));
  MCK(cudaMalloc(&s->b4s, 4 * 4));
  MCK(cudaMalloc(&s->dacc, 128 * 8));
  MCK(cudaMalloc(&c->d_mlp_pre, (size_t)c->nelem * 64 * 4));
  k_elem_features<<<(c->nelem + 127) / 128, 128, 0, c->stream>>>(c->d_xg64, c->nelem, s->feat48);
  MCK(cudaGetLastError());
  MCK(cudaFuncSetAttribute(k_mlp_fb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FB_SMEM));
  return PT_OK;
}

// BF16 export and folding of normalisation into the push-side tables
static pt_status export_bf16(pt_ctx* c) {
  pt_mlp_state* s = c->mlp;
  std::vector<float> th(NPAR);
  MCK(cudaMemcpyAsync(th.data(), s->theta, NPAR * 4, cudaMemcpyDeviceToHost, c->stream));
  MCK(cudaMemcpyAsync(s->norm, s->hnorm, NNORM * 4, cudaMemcpyHostToDevice, c->stream));
  MCK(cudaStreamSynchronize(c->stream));
  // the input means are folded into the per-element layer-1 table (k_mlp_pre)
  const float* sd = s->hnorm + 51;
  const float* osc = s->hnorm + 102;
  std::vector<uint16_t> w2(4096), w3(4096);
  for (int i = 0; i < 4096; ++i) {
    __nv_bfloat16 a = __float2bfloat16_rn(th[OFF_W2 + i]), b = __float2bfloat16_rn(th[OFF_W3 + i]);
    std::memcpy(&w2[i], &a, 2);
    std::memcpy(&w3[i], &b, 2);
  }
  std::vector<float> w1x(192), w4s(192), b4s(4, 0.f);
  for (int o = 0; o < 64; ++o)
    for (int q = 0; q < 3; ++q) w1x[3 * o + q] = th[OFF_W1 + 51 * o + q] / sd[q];
  for (int q = 0; q < 3; ++q) {
    for (int i = 0; i < 64; ++i) w4s[64 * q + i] = th[OFF_W4 + 64 * q + i] * osc[q];
    b4s[q] = th[OFF_B4 + q] * osc[q];
  }
  MCK(cudaMemcpy(s->w2b, w2.data(), 4096 * 2, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(s->w3b, w3.data(), 4096 * 2, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(s->w1x, w1x.data(), 192 * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(s->b2, th.data() + OFF_B2, 64 * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(s->b3, th.data() + OFF_B3, 64 * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(s->w4s, w4s.data(), 192 * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(s->b4s, b4s.data(), 4 * 4, cudaMemcpyHostToDevice));
  std::memcpy(s->h_w1x, w1x.data(), sizeof s->h_w1x);
  std::memcpy(s->h_b2, th.data() + OFF_B2, sizeof s->h_b2);
  std::memcpy(s->h_b3, th.data() + OFF_B3, sizeof s->h_b3);
  std::memcpy(s->h_w4s, w4s.data(), sizeof s->h_w4s);
  std::memcpy(s->h_b4s, b4s.data(), sizeof s->h_b4s);
  const int64_t tot = (int64_t)c->nelem * 64;
  k_mlp_pre<<<(int)((tot + 255) / 256), 256, 0, c->stream>>>(s->theta, s->norm, s->feat48,
                                                              c->nelem, c->d_mlp_pre);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(c->stream));
  c->mlp_ready = true;
  return PT_OK;
}

static void init_theta(uint64_t seed, std::vector<float>& th) {
  th.assign(NPAR, 0.f);
  const int offW[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4}, offB[4] = {OFF_B1, OFF_B2, OFF_B3, OFF_B4};
  const int nin[4] = {51, 64, 64, 64}, nout[4] = {64, 64, 64, 3};
  uint64_t ctr = splitmix64(seed);
  for (int l = 0; l < 4; ++l) {
    const float bound = 1.f / std::sqrt((float)nin[l]);
    for (int i = 0; i < nin[l] * nout[l]; ++i)
      th[offW[l] + i] = (float)((2.0 * u01(splitmix64(ctr++)) - 1.0) * bound);
    for (int i = 0; i < nout[l]; ++i)
      th[offB[l] + i] = (float)((2.0 * u01(splitmix64(ctr++)) - 1.0) * bound);
  }
}

static uint64_t gcd64(uint64_t a, uint64_t b) {
  while (b) {
    uint64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

extern "C" {

int32_t pt_mlp_nparams(void) { return NPAR; }

pt_status pt_mlp_features(pt_ctx* c, int64_t n, const double* x, const int32_t* elem, float* f) {
  if (!c) return PT_ERR_ARG;
  if (n < 0 || (n > 0 && (!x || !elem || !f))) return mfail(c, PT_ERR_ARG, "bad arguments");
  pt_status st = ensure_state(c);
  if (st) return st;
  if (n == 0) return PT_OK;
  k_particle_features<<<(int)((n + 127) / 128), 128, 0, c->stream>>>(pt_dev_mesh(c), n, x, elem,
                                                                    c->mlp->feat48, f);
  MCK(cudaGetLastError());
  return PT_OK;
}

pt_status pt_mlp_make_pairs(pt_ctx* c, int64_t n, uint64_t seed, float* in, float* tgt) {
  if (!c) return PT_ERR_ARG;
  if (n <= 0 || !in || !tgt) return mfail(c, PT_ERR_ARG, "bad arguments");
  pt_status st = ensure_state(c);
  if (st) return st;
  DevConsts k;
  pt_fill_consts(c, k);
  unsigned* nf = reinterpret_cast<unsigned*>(c->mlp->dacc);
  MCK(cudaMemsetAsync(nf, 0, 4, c->stream));
  k_mlp_pairs<<<(int)((n + 127) / 128), 128, 0, c->stream>>>(pt_dev_mesh(c), k, n, seed,
                                                              c->mlp->feat48, in, tgt, nf);
  MCK(cudaGetLastError());
  unsigned h = 0;
  MCK(cudaMemcpyAsync(&h, nf, 4, cudaMemcpyDeviceToHost, c->stream));
  MCK(cudaStreamSynchronize(c->stream));
  if (h) return mfail(c, PT_ERR_NEWTON, "%u training labels: FP64 Newton did not converge", h);
  return PT_OK;
}

pt_status pt_mlp_set(pt_ctx* c, const float* theta, const float* norm) {
  if (!c) return PT_ERR_ARG;
  if (!theta || !norm) return mfail(c, PT_ERR_ARG, "NULL theta or norm");
  for (int q = 0; q < 51; ++q)
    if (!(norm[51 + q] > 0)) return mfail(c, PT_ERR_ARG, "in_std must be > 0");
  pt_status st = ensure_state(c);
  if (st) return st;
  MCK(cudaMemcpy(c->mlp->theta, theta, NPAR * 4, cudaMemcpyHostToDevice));
  std::memcpy(c->mlp->hnorm, norm, sizeof(float) * NNORM);
  c->mlp->have_theta = true;
  return export_bf16(c);
}

pt_status pt_mlp_get(pt_ctx* c, float* theta, float* norm) {
  if (!c) return PT_ERR_ARG;
  if (!c->mlp || !c->mlp->have_theta) return mfail(c, PT_ERR_STATE, "no network");
  if (theta) MCK(cudaMemcpy(theta, c->mlp->theta, NPAR * 4, cudaMemcpyDeviceToHost));
  if (norm) std::memcpy(norm, c->mlp->hnorm, sizeof(float) * NNORM);
  return PT_OK;
}

pt_status pt_mlp_forward(pt_ctx* c, int32_t B, const float* in, float* out) {
  if (!c) return PT_ERR_ARG;
  if (B <= 0 || !in || !out) return mfail(c, PT_ERR_ARG, "bad arguments");
  if (!c->mlp || !c->mlp->have_theta) return mfail(c, PT_ERR_STATE, "no network");
  FBArgs a{c->mlp->theta, in, nullptr, nullptr, B, 0, B, 1, 0, nullptr, nullptr, out};
  k_mlp_fb<<<(B + TB - 1) / TB, NTH, FB_SMEM, c->stream>>>(a);
  MCK(cudaGetLastError());
  return PT_OK;
}

pt_status pt_mlp_grad(pt_ctx* c, int32_t B, const float* in, const float* tgt, float* grad,
                      float* loss) {
  if (!c) return PT_ERR_ARG;
  if (B <= 0 || !in || !tgt || !grad) return mfail(c, PT_ERR_ARG, "bad arguments");
  if (!c->mlp || !c->mlp->have_theta) return mfail(c, PT_ERR_STATE, "no network");
  MCK(cudaMemsetAsync(grad, 0, NPAR * 4, c->stream));
  MCK(cudaMemsetAsync(c->mlp->dacc, 0, 8, c->stream));
  FBArgs a{c->mlp->theta, in, tgt, nullptr, B, 0, B, 1, 0, grad, c->mlp->dacc, nullptr};
  k_mlp_fb<<<(B + TB - 1) / TB, NTH, FB_SMEM, c->stream>>>(a);
  MCK(cudaGetLastError());
  double h = 0.0;
  MCK(cudaMemcpyAsync(&h, c->mlp->dacc, 8, cudaMemcpyDeviceToHost, c->stream));
  MCK(cudaStreamSynchronize(c->stream));
  if (loss) *loss = (float)h;
  return PT_OK;
}

pt_status pt_mlp_train(pt_ctx* c, int64_t n, const float* in, const float* tgt, int32_t epochs,
                       int32_t batch, float lr, uint64_t seed, float* loss_host) {
  if (!c) return PT_ERR_ARG;
  if (n <= 1 || !in || !tgt || epochs < 1 || batch < 1 || !(lr > 0))
    return mfail(c, PT_ERR_ARG, "bad arguments");
  pt_status st = ensure_state(c);
  if (st) return st;
  pt_mlp_state* s = c->mlp;
  // normalisation statistics
  MCK(cudaMemsetAsync(s->dacc, 0, 128 * 8, c->stream));
  k_colstats<<<c->nsm * 4, 256, 0, c->stream>>>(n, in, tgt, s->dacc);
  MCK(cudaGetLastError());
  double acc[108];
  MCK(cudaMemcpyAsync(acc, s->dacc, sizeof acc, cudaMemcpyDeviceToHost, c->stream));
  MCK(cudaStreamSynchronize(c->stream));
  for (int q = 0; q < 51; ++q) {
    double mean = acc[q] / n, var = acc[54 + q] / n - mean * mean;
    s->hnorm[q] = (float)mean;
    s->hnorm[51 + q] = (float)std::sqrt(std::max(var, 1e-24));
  }
  for (int q = 0; q < 3; ++q) s->hnorm[102 + q] = (float)std::sqrt(std::max(acc[105 + q] / n, 1e-30));
  MCK(cudaMemcpy(s->norm, s->hnorm, NNORM * 4, cudaMemcpyHostToDevice));
  std::vector<float> th;
  init_theta(seed, th);
  MCK(cudaMemcpy(s->theta, th.data(), NPAR * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemsetAsync(s->grad, 0, NPAR * 4, c->stream));
  MCK(cudaMemsetAsync(s->m, 0, NPAR * 4, c->stream));
  MCK(cudaMemsetAsync(s->v, 0, NPAR * 4, c->stream));
  const int64_t steps = std::max<int64_t>(1, n / batch);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  int t = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    // epoch order: row j -> (pa j + pb) mod n with pa coprime to n
    uint64_t h = splitmix64(seed * 1000003ull + ep);
    uint64_t pa = 1 + h % (uint64_t)(n - 1);
    while (gcd64(pa, (uint64_t)n) != 1) pa = 1 + (pa % (uint64_t)(n - 1));
    uint64_t pb = splitmix64(h) % (uint64_t)n;
    MCK(cudaMemsetAsync(s->dacc, 0, 8, c->stream));
    for (int64_t stp = 0; stp < steps; ++stp) {
      FBArgs a{s->theta, in, tgt, s->norm, n, stp * batch, batch, pa, pb, s->grad, s->dacc,
               nullptr};
      k_mlp_fb<<<(batch + TB - 1) / TB, NTH, FB_SMEM, c->stream>>>(a);
      ++t;
      const float c1 = 1.f - std::pow(b1, (float)t), c2 = 1.f - std::pow(b2, (float)t);
      k_adam<<<(NPAR + 255) / 256, 256, 0, c->stream>>>(s->theta, s->grad, s->m, s->v, NPAR, lr,
                                                         b1, b2, eps, c1, c2);
    }
    MCK(cudaGetLastError());
    double lsum = 0.0;
    MCK(cudaMemcpyAsync(&lsum, s->dacc, 8, cudaMemcpyDeviceToHost, c->stream));
    MCK(cudaStreamSynchronize(c->stream));
    if (loss_host) loss_host[ep] = (float)(lsum / steps);
  }
  s->have_theta = true;
  return export_bf16(c);
}

}  // extern "C"
