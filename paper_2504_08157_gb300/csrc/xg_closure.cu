// xg_closure.cu -- learned subgrid closure (include/xg_closure.h).
//
// Kernels:
//   * features of a state: q, assembled gradients, heating (k_features);
//   * restriction of fine fields to coarse nodes, one axis at a time
//     (k_interp_axis);
//   * training in FP32 on the CUDA cores: forward and back-propagation over
//     chunks of samples with the weights, activations and per-block gradient
//     sums in shared memory (k_mlp_grad, each gradient entry owned by one
//     thread so the sums are deterministic), the fixed-order reduction of
//     the block partials (k_mlp_reduce), Adam (k_adam), column statistics
//     (k_col_stats);
//   * inference on the fifth-generation tensor cores (tcgen05.mma, bfloat16
//     operands in shared memory, FP32 accumulators in TMEM): persistent CTAs
//     of 128 threads take 128 samples per tile, one row of every product per
//     thread; bias, SiLU and the bfloat16 rounding of the hidden activations
//     run on the CUDA cores between the layers.  k_closure computes the
//     features of each tile's nodes straight from the state and runs the
//     network on them; k_mlp_bf16 runs it on given features.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/xg_closure.h"
#include "xg_ctx.h"
#include "xg_setup.h"
#include "xg_tc.cuh"

namespace xg {

constexpr int kIn = XG_CLOSURE_IN, kHid = XG_CLOSURE_HIDDEN, kOut = XG_CLOSURE_OUT;
constexpr int kParams = XG_CLOSURE_PARAMS;
// Normalised inputs are clamped to [-kClampIn, kClampIn]: a state outside
// the training distribution cannot drive the network's output without bound.
constexpr float kClampIn = 8.0f;
__device__ __forceinline__ float norm_in(float x, float mean, float scale) {
  return fminf(fmaxf((x - mean) * scale, -kClampIn), kClampIn);
}
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid;
static_assert(kOffB3 + kOut == kParams, "parameter layout");

// ------------------------------------------------------------------ features

// The stencil of the assembled derivative along direction d at global
// index g of a line starting at offset base (stride sd): the node's segment
// (row a of the scaled matrix Dm = -(2/h) D, rows 0 and N halved), at a
// shared face also the segment before (its row N), at a wall the one
// segment's row doubled.  Built once per direction and applied to all five
// variables.
template <int N>
struct LineStencil {
  int off[2 * (N + 1)];   // within one variable's array (np < 2^31)
  float r0[N + 1], r1[N + 1];
  bool two;
  float scale;
};

template <int N>
__device__ __forceinline__ void line_stencil(const FParams& P, int d, long long base, long long sd, int g,
                                             LineStencil<N>& L) {
  const int nd = P.n[d], nseg = P.nseg[d];
  int s = g / N;
  if (s >= nseg) s = nseg - 1;
  const int a = g - s * N;
#pragma unroll
  for (int l = 0; l <= N; ++l) {
    int k = s * N + l;
    if (k >= nd) k -= nd;
    L.off[l] = (int)(base + sd * k);
    L.r0[l] = P.Dm[d][a][l];
  }
  L.two = a == 0 && (s > 0 || P.per[d]);
  L.scale = (a == N || (a == 0 && !L.two)) ? -2.0f : -1.0f;   // the sign undoes Dm's minus
  const int s2 = s > 0 ? s - 1 : nseg - 1;
#pragma unroll
  for (int l = 0; l <= N; ++l) {
    int k = s2 * N + l;
    if (k >= nd) k -= nd;
    L.off[N + 1 + l] = L.two ? (int)(base + sd * k) : L.off[l];
    L.r1[l] = L.two ? P.Dm[d][N][l] : 0.0f;
  }
}

template <int N>
__device__ __forceinline__ float line_apply(const LineStencil<N>& L, const float* __restrict__ f) {
  float acc = 0.0f;
#pragma unroll
  for (int l = 0; l <= N; ++l) acc = fmaf(L.r0[l], f[L.off[l]], acc);
  if (L.two) {
#pragma unroll
    for (int l = 0; l <= N; ++l) acc = fmaf(L.r1[l], f[L.off[N + 1 + l]], acc);
  }
  return L.scale * acc;
}

// The 21 features of node I, handed to emit(f, value): per direction the
// stencil once, then that direction's derivative of all five variables.
template <int N, typename Emit>
__device__ __forceinline__ void node_features(const FParams& P, const float* __restrict__ q,
                                              const float* __restrict__ S, long long I, Emit emit) {
  const long long np = P.np;
  const int nx = P.n[0], ny = P.n[1];
  const int gx = (int)(I % nx);
  const long long r = I / nx;
  const int gy = (int)(r % ny), gz = (int)(r / ny);
#pragma unroll
  for (int v = 0; v < 5; ++v) emit(v, q[v * np + I]);
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    LineStencil<N> L;
    if (d == 0) line_stencil<N>(P, 0, I - gx, 1, gx, L);
    else if (d == 1) line_stencil<N>(P, 1, I - (long long)gy * nx, nx, gy, L);
    else line_stencil<N>(P, 2, I - (long long)gz * nx * ny, (long long)nx * ny, gz, L);
#pragma unroll
    for (int v = 0; v < 5; ++v) emit(5 + 3 * v + d, line_apply<N>(L, q + v * np));
  }
  emit(20, S ? S[I] : 0.0f);
}

template <int N>
__global__ void __launch_bounds__(128) k_features(const FParams P, const float* __restrict__ q,
                                                  const float* __restrict__ S, float* __restrict__ X) {
  const long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (I >= P.np) return;
  const long long np = P.np;
  node_features<N>(P, q, S, I, [&](int f, float v) { X[f * np + I] = v; });
}

// ------------------------------------------------------------------ restriction

// out[o][c][i] = sum_a w[c][a] in[o][(start[c] + a) mod n_in][i]
__global__ void k_interp_axis(const double* __restrict__ in, double* __restrict__ out, long long outer,
                              int n_in, int n_out, long long inner, const int* __restrict__ start,
                              const double* __restrict__ w, int npts) {
  const long long total = outer * n_out * inner;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t % inner;
    const long long rest = t / inner;
    const int c = (int)(rest % n_out);
    const long long o = rest / n_out;
    double acc = 0.0;
    for (int a = 0; a < npts; ++a) {
      int k = start[c] + a;
      if (k >= n_in) k -= n_in;
      acc = fma(w[c * npts + a], in[(o * n_in + k) * inner + i], acc);
    }
    out[t] = acc;
  }
}

// ------------------------------------------------------------------ training (FP32)

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_prime_f(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

constexpr int kTrainThreads = 256;
constexpr int kChunk = 32;   // samples per pass through the network

struct TrainSmem {
  float W[kParams];
  float G[kParams];
  float x[kIn][kChunk];
  float t[kOut][kChunk];
  float z1[kHid][kChunk];
  float h1[kHid][kChunk];    // silu(z1)
  float z2[kHid][kChunk];    // later the first layer's delta
  float h2[kHid][kChunk];    // silu(z2)
  float d2[kHid][kChunk];
  float d3[kOut][kChunk];
  float stat[2 * kIn + kOut];
  double red[kTrainThreads];
};

// Samples [begin, end) of this block; writes the block's gradient sums and
// loss partial.  scale = 2 / (5 n) (the derivative of the mean square).
__global__ void __launch_bounds__(kTrainThreads) k_mlp_grad(const float* __restrict__ params,
                                                           const float* __restrict__ X,
                                                           const float* __restrict__ T, long long ld,
                                                           long long n, const float* __restrict__ in_mean,
                                                           const float* __restrict__ in_scale,
                                                           const float* __restrict__ out_scale,
                                                           float* __restrict__ partial,
                                                           double* __restrict__ lossp, float scale) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smraw);
  const int tid = threadIdx.x;
  for (int k = tid; k < kParams; k += blockDim.x) {
    S.W[k] = params[k];
    S.G[k] = 0.0f;
  }
  if (tid < kIn) {
    S.stat[tid] = in_mean[tid];
    S.stat[kIn + tid] = in_scale[tid];
  }
  if (tid < kOut) S.stat[2 * kIn + tid] = 1.0f / out_scale[tid];
  const long long begin = n * blockIdx.x / gridDim.x, end = n * (blockIdx.x + 1) / gridDim.x;
  double lacc = 0.0;
  const float* W1 = S.W + kOffW1;
  const float* b1 = S.W + kOffB1;
  const float* W2 = S.W + kOffW2;
  const float* b2 = S.W + kOffB2;
  const float* W3 = S.W + kOffW3;
  const float* b3 = S.W + kOffB3;
  __syncthreads();
  for (long long c0 = begin; c0 < end; c0 += kChunk) {
    const int cn = (int)min((long long)kChunk, end - c0);
    for (int k = tid; k < kIn * kChunk; k += blockDim.x) {
      const int f = k / kChunk, s = k % kChunk;
      S.x[f][s] = s < cn ? norm_in(X[f * ld + c0 + s], S.stat[f], S.stat[kIn + f]) : 0.0f;
    }
    for (int k = tid; k < kOut * kChunk; k += blockDim.x) {
      const int o = k / kChunk, s = k % kChunk;
      S.t[o][s] = s < cn ? T[o * ld + c0 + s] * S.stat[2 * kIn + o] : 0.0f;
    }
    __syncthreads();
    for (int k = tid; k < kHid * kChunk; k += blockDim.x) {   // z1 = W1 x + b1
      const int o = k / kChunk, s = k % kChunk;
      float a = b1[o];
      for (int i = 0; i < kIn; ++i) a = fmaf(W1[o * kIn + i], S.x[i][s], a);
      S.z1[o][s] = a;
      S.h1[o][s] = silu_f(a);
    }
    __syncthreads();
    for (int k = tid; k < kHid * kChunk; k += blockDim.x) {   // z2 = W2 silu(z1) + b2
      const int o = k / kChunk, s = k % kChunk;
      float a = b2[o];
      for (int i = 0; i < kHid; ++i) a = fmaf(W2[o * kHid + i], S.h1[i][s], a);
      S.z2[o][s] = a;
      S.h2[o][s] = silu_f(a);
    }
    __syncthreads();
    for (int k = tid; k < kOut * kChunk; k += blockDim.x) {   // y, residual, output delta
      const int o = k / kChunk, s = k % kChunk;
      float a = b3[o];
      for (int i = 0; i < kHid; ++i) a = fmaf(W3[o * kHid + i], S.h2[i][s], a);
      const float r = s < cn ? a - S.t[o][s] : 0.0f;
      lacc += (double)r * r;
      S.d3[o][s] = scale * r;
    }
    __syncthreads();
    for (int k = tid; k < kOut * kHid + kOut; k += blockDim.x) {   // W3, b3 gradients
      float a = 0.0f;
      if (k < kOut * kHid) {
        const int o = k / kHid, i = k % kHid;
        for (int s = 0; s < cn; ++s) a = fmaf(S.d3[o][s], S.h2[i][s], a);
      } else {
        for (int s = 0; s < cn; ++s) a += S.d3[k - kOut * kHid][s];
      }
      S.G[kOffW3 + k] += a;
    }
    for (int k = tid; k < kHid * kChunk; k += blockDim.x) {   // second hidden layer's delta
      const int i = k / kChunk, s = k % kChunk;
      float a = 0.0f;
      for (int o = 0; o < kOut; ++o) a = fmaf(W3[o * kHid + i], S.d3[o][s], a);
      S.d2[i][s] = a * silu_prime_f(S.z2[i][s]);
    }
    __syncthreads();
    for (int k = tid; k < kHid * kHid + kHid; k += blockDim.x) {   // W2, b2 gradients
      float a = 0.0f;
      if (k < kHid * kHid) {
        const int o = k / kHid, i = k % kHid;
        for (int s = 0; s < cn; ++s) a = fmaf(S.d2[o][s], S.h1[i][s], a);
      } else {
        for (int s = 0; s < cn; ++s) a += S.d2[k - kHid * kHid][s];
      }
      S.G[kOffW2 + k] += a;
    }
    __syncthreads();
    for (int k = tid; k < kHid * kChunk; k += blockDim.x) {   // first hidden layer's delta (into z2)
      const int i = k / kChunk, s = k % kChunk;
      float a = 0.0f;
      for (int o = 0; o < kHid; ++o) a = fmaf(W2[o * kHid + i], S.d2[o][s], a);
      S.z2[i][s] = a * silu_prime_f(S.z1[i][s]);
    }
    __syncthreads();
    for (int k = tid; k < kHid * kIn + kHid; k += blockDim.x) {   // W1, b1 gradients
      float a = 0.0f;
      if (k < kHid * kIn) {
        const int o = k / kIn, i = k % kIn;
        for (int s = 0; s < cn; ++s) a = fmaf(S.z2[o][s], S.x[i][s], a);
      } else {
        for (int s = 0; s < cn; ++s) a += S.z2[k - kHid * kIn][s];
      }
      S.G[kOffW1 + k] += a;
    }
    __syncthreads();
  }
  for (int k = tid; k < kParams; k += blockDim.x) partial[(long long)blockIdx.x * kParams + k] = S.G[k];
  S.red[tid] = lacc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (tid < h) S.red[tid] += S.red[tid + h];
    __syncthreads();
  }
  if (tid == 0) lossp[blockIdx.x] = S.red[0];
}

__global__ void k_mlp_reduce(const float* __restrict__ partial, int nblocks, float* __restrict__ grad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kParams) return;
  float a = 0.0f;
  for (int b = 0; b < nblocks; ++b) a += partial[(long long)b * kParams + k];
  grad[k] = a;
}

// Adam; 1 - beta1 and 1 - beta2 come from the host in double precision
// (1.0f - 0.999f would carry a 5e-5 relative error into v).
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int n, float lr, float b1, float b2, float omb1,
                       float omb2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + omb1 * gk;
  const float vk = b2 * v[k] + omb2 * gk * gk;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

__global__ void k_col_stats(const float* __restrict__ X, long long ld, long long n, double* __restrict__ out) {
  __shared__ double red[256];
  const int c = blockIdx.x, tid = threadIdx.x;
  const float* x = X + c * ld;
  double s = 0.0;
  for (long long i = tid; i < n; i += blockDim.x) s += x[i];
  red[tid] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (tid < h) red[tid] += red[tid + h];
    __syncthreads();
  }
  const double mean = red[0] / (double)n;
  __syncthreads();
  double q = 0.0;
  for (long long i = tid; i < n; i += blockDim.x) {
    const double d = x[i] - mean;
    q += d * d;
  }
  red[tid] = q;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (tid < h) red[tid] += red[tid + h];
    __syncthreads();
  }
  if (tid == 0) {
    out[2 * c] = mean;
    out[2 * c + 1] = sqrt(red[0] / (double)n);
  }
}

__global__ void k_mlp_fp32(const float* __restrict__ params, const float* __restrict__ X, long long ld,
                           long long n, const float* __restrict__ in_mean, const float* __restrict__ in_scale,
                           const float* __restrict__ out_scale, float* __restrict__ Y, long long ldy) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[kIn], h1[kHid], h2[kHid];
  for (int f = 0; f < kIn; ++f) x[f] = norm_in(X[f * ld + s], in_mean[f], in_scale[f]);
  for (int o = 0; o < kHid; ++o) {
    float a = params[kOffB1 + o];
    for (int i = 0; i < kIn; ++i) a = fmaf(params[kOffW1 + o * kIn + i], x[i], a);
    h1[o] = silu_f(a);
  }
  for (int o = 0; o < kHid; ++o) {
    float a = params[kOffB2 + o];
    for (int i = 0; i < kHid; ++i) a = fmaf(params[kOffW2 + o * kHid + i], h1[i], a);
    h2[o] = silu_f(a);
  }
  for (int o = 0; o < kOut; ++o) {
    float a = params[kOffB3 + o];
    for (int i = 0; i < kHid; ++i) a = fmaf(params[kOffW3 + o * kHid + i], h2[i], a);
    Y[o * ldy + s] = a * out_scale[o];
  }
}

// ------------------------------------------------------------------ inference (tcgen05)
//
// Inference runs on the fifth-generation tensor cores.  A persistent CTA of
// 128 threads takes 128 samples at a time: they are the M = 128 rows of every
// product, one row per thread and per TMEM lane.  Per tile:
//   features -> A (bfloat16, shared memory)              all threads
//   D = A W1h^T   (K 32, N 64)                           one thread issues tcgen05.mma
//   A <- bf16(SiLU(2 (D + b1/2)))                        all threads: tcgen05.ld, FP32
//   D = A W2h^T   (K 64, N 64)
//   A <- bf16(SiLU(2 (D + b2/2)))
//   D = A W3^T    (K 64, N 16; outputs 5..15 are zero rows of W3)
//   y = (D + b3) * out_scale                             all threads, coalesced stores
// W1h and W2h are the bfloat16 weights halved (exact), so the accumulator
// holds h = z / 2 and SiLU(z) = h + h tanh(h) needs no further scaling.  The
// accumulator takes 64 TMEM columns; shared memory (31.5 KB per CTA) lets at
// most 7 CTAs share an SM (448 of its 512 columns), the launch bound 4.
constexpr int kTcRows = 128;             // samples per tile, the MMA's M
constexpr int kK1 = 32;                  // layer-1 K: 21 features, zero padded
constexpr int kN3 = 16;                  // layer-3 N: 5 outputs, zero padded
constexpr int kTcCols = 64;              // TMEM columns per CTA

// Packed inference constants (one device blob, copied to shared memory):
// the bfloat16 weights in the canonical K-major layout (tc::kmajor), then
// FP32 b1/2, b2/2, b3, in_mean, in_scale, out_scale.
struct InferPack {
  __nv_bfloat16 W1[kHid * kK1];
  __nv_bfloat16 W2[kHid * kHid];
  __nv_bfloat16 W3[kN3 * kHid];
  float hb1[kHid], hb2[kHid], b3[8];
  float mean[24], scale[24], oscale[8];
};
static_assert(sizeof(InferPack) % 16 == 0, "InferPack is copied as int4");

__global__ void k_pack(const float* __restrict__ p, const float* __restrict__ mean,
                       const float* __restrict__ scale, const float* __restrict__ oscale,
                       InferPack* __restrict__ out) {
  for (int k = threadIdx.x; k < kHid * kK1; k += blockDim.x) {
    const int o = k / kK1, i = k % kK1;
    out->W1[tc::kmajor(kHid, o, i)] = __float2bfloat16_rn(i < kIn ? 0.5f * p[kOffW1 + o * kIn + i] : 0.0f);
  }
  for (int k = threadIdx.x; k < kHid * kHid; k += blockDim.x) {
    const int o = k / kHid, i = k % kHid;
    out->W2[tc::kmajor(kHid, o, i)] = __float2bfloat16_rn(0.5f * p[kOffW2 + o * kHid + i]);
  }
  for (int k = threadIdx.x; k < kN3 * kHid; k += blockDim.x) {
    const int o = k / kHid, i = k % kHid;
    out->W3[tc::kmajor(kN3, o, i)] = __float2bfloat16_rn(o < kOut ? p[kOffW3 + o * kHid + i] : 0.0f);
  }
  for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
    out->hb1[k] = 0.5f * p[kOffB1 + k];
    out->hb2[k] = 0.5f * p[kOffB2 + k];
  }
  for (int k = threadIdx.x; k < 24; k += blockDim.x) {
    out->mean[k] = k < kIn ? mean[k] : 0.0f;
    out->scale[k] = k < kIn ? scale[k] : 0.0f;
  }
  for (int k = threadIdx.x; k < 8; k += blockDim.x) {
    out->b3[k] = k < kOut ? p[kOffB3 + k] : 0.0f;
    out->oscale[k] = k < kOut ? oscale[k] : 0.0f;
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// SiLU(2h) = h (1 + tanh h) with the hardware tanh approximation (relative
// error ~2^-11), below the bfloat16 rounding that follows it.
__device__ __forceinline__ float silu_of_half(float h) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
  return fmaf(h, t, h);
}

struct TcSmem {
  InferPack K;
  __nv_bfloat16 A[kTcRows * kHid];   // features (first 4 K-chunks) or hidden activations
  unsigned long long bar;            // mbarrier: MMA completion
  uint32_t tmem;                     // TMEM base address
};

__device__ __forceinline__ void load_pack(InferPack& dst, const InferPack* src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(InferPack) / 16); k += blockDim.x) d[k] = s[k];
}

// One layer's products: makes this thread's writes of A visible to the
// tensor cores, synchronises the CTA, issues the K/16 MMAs from thread 0 and
// waits for them.  False (on every thread) when a wait ran out; the kernel
// then reports XG_ERR_TIMEOUT through the flag and stops.
__device__ __forceinline__ bool tc_layer(TcSmem& S, uint32_t w_addr, uint32_t w_lbo, int ksteps,
                                         uint32_t idesc, uint32_t& phase) {
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t bar = tc::smem_addr(&S.bar);
  if (threadIdx.x == 0) {
    const uint32_t a_addr = tc::smem_addr(S.A);
    constexpr uint32_t a_lbo = kTcRows * 16;
    for (int k = 0; k < ksteps; ++k) {
      tc::mma_bf16(S.tmem, tc::smem_desc(a_addr + 2 * k * a_lbo, a_lbo, 128),
                   tc::smem_desc(w_addr + 2 * k * w_lbo, w_lbo, 128), idesc, k > 0);
    }
    tc::commit(bar);
  }
  const bool ok = tc::mbar_wait(bar, phase, tc::kWaitNs);
  phase ^= 1u;
  const int bad = __syncthreads_or(!ok);
  tc::fence_after_sync();
  return !bad;
}

// The hidden layer's epilogue: this thread's row of D (64 columns) plus the
// halved bias, SiLU, bfloat16 into its row of A.
__device__ __forceinline__ void tc_hidden(TcSmem& S, uint32_t lane_addr, const float* hb) {
  char* A = reinterpret_cast<char*>(S.A);
#pragma unroll
  for (int c0 = 0; c0 < kHid; c0 += 16) {
    uint32_t r[16];
    tc::tmem_ld16(lane_addr + c0, r);
    tc::tmem_wait_ld();
    uint32_t pk[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      pk[j] = pack_bf16(silu_of_half(__uint_as_float(r[2 * j]) + hb[c0 + 2 * j]),
                        silu_of_half(__uint_as_float(r[2 * j + 1]) + hb[c0 + 2 * j + 1]));
    const int off = (c0 >> 3) * (kTcRows * 16) + threadIdx.x * 16;
    *reinterpret_cast<uint4*>(A + off) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4*>(A + off + kTcRows * 16) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
  }
}

// The persistent inference loop over the tiles of n samples: feat(s, emit)
// hands the raw features f = 0..20 of sample s < n to emit(f, value);
// Y[o * ldy + s] = out_scale_o * y_o.  On a wait that runs out, sets bit 1
// (value 2) of *flag and returns after freeing its TMEM.  blockDim.x = kTcRows.
template <typename Feat>
__device__ __forceinline__ void tc_infer(TcSmem& S, const InferPack* __restrict__ pack, long long n,
                                         float* __restrict__ Y, long long ldy, int* flag, Feat feat) {
  const int tid = threadIdx.x, warp = tid >> 5;
  load_pack(S.K, pack);
#pragma unroll
  for (int k = kIn; k < kK1; ++k) S.A[tc::kmajor(kTcRows, tid, k)] = __float2bfloat16_rn(0.0f);
  if (tid == 0) tc::mbar_init(tc::smem_addr(&S.bar), 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(&S.tmem), kTcCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t lane_addr = S.tmem + ((uint32_t)(32 * warp) << 16);
  const uint32_t w1 = tc::smem_addr(S.K.W1), w2 = tc::smem_addr(S.K.W2), w3 = tc::smem_addr(S.K.W3);
  uint32_t phase = 0;
  bool ok = true;
  const long long ntiles = (n + kTcRows - 1) / kTcRows;
  for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const long long s = t * kTcRows + tid;
    if (s < n) {
      feat(s, [&](int f, float v) {
        S.A[tc::kmajor(kTcRows, tid, f)] = __float2bfloat16_rn(norm_in(v, S.K.mean[f], S.K.scale[f]));
      });
    } else {
#pragma unroll
      for (int f = 0; f < kIn; ++f) S.A[tc::kmajor(kTcRows, tid, f)] = __float2bfloat16_rn(0.0f);
    }
    ok = tc_layer(S, w1, kHid * 16, kK1 / 16, tc::idesc_bf16(kTcRows, kHid), phase);
    if (!ok) break;
    tc_hidden(S, lane_addr, S.K.hb1);
    ok = tc_layer(S, w2, kHid * 16, kHid / 16, tc::idesc_bf16(kTcRows, kHid), phase);
    if (!ok) break;
    tc_hidden(S, lane_addr, S.K.hb2);
    ok = tc_layer(S, w3, kN3 * 16, kHid / 16, tc::idesc_bf16(kTcRows, kN3), phase);
    if (!ok) break;
    uint32_t r[8];
    tc::tmem_ld8(lane_addr, r);
    tc::tmem_wait_ld();
    if (s < n) {
#pragma unroll
      for (int o = 0; o < kOut; ++o) Y[o * ldy + s] = (__uint_as_float(r[o]) + S.K.b3[o]) * S.K.oscale[o];
    }
  }
  if (!ok && tid == 0) {
    // the products whose completion was not seen may still write tensor
    // memory: wait (bounded) once more for their commit before freeing it
    atomicOr(flag, 2);
    tc::mbar_wait(tc::smem_addr(&S.bar), phase ^ 1u, tc::kWaitNs);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(S.tmem, kTcCols);
  }
}

constexpr int kTcCtasPerSm = 4;

__global__ void __launch_bounds__(kTcRows, kTcCtasPerSm)
    k_mlp_bf16(const InferPack* __restrict__ pack, const float* __restrict__ X, long long ld, long long n,
               float* __restrict__ Y, long long ldy, int* flag) {
  __shared__ __align__(128) TcSmem S;
  tc_infer(S, pack, n, Y, ldy, flag, [&](long long s, auto&& emit) {
#pragma unroll
    for (int f = 0; f < kIn; ++f) emit(f, X[f * ld + s]);
  });
}

// The closure correction C [5][np]: the features of each tile's 128 nodes
// straight from the state, then the network.
template <int N>
__global__ void __launch_bounds__(kTcRows, kTcCtasPerSm)
    k_closure(const FParams P, const InferPack* __restrict__ pack, const float* __restrict__ q,
              const float* __restrict__ Sth, float* __restrict__ C, int* flag) {
  __shared__ __align__(128) TcSmem S;
  tc_infer(S, pack, P.np, C, P.np, flag,
           [&](long long I, auto&& emit) { node_features<N>(P, q, Sth, I, emit); });
}

// The bounded wait of the tensor-core kernels, made to run out: one CTA
// allocates TMEM, initialises an mbarrier that nothing will complete, waits
// for it with the limit, records the timeout in *status and frees its TMEM
// (the path every tcgen05 kernel here takes when a wait gives up).
__global__ void k_tc_wait_selftest(unsigned long long limit_ns, int* status) {
  __shared__ unsigned long long bar;
  __shared__ uint32_t tmem;
  const int warp = threadIdx.x >> 5;
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(&tmem), 32);
  if (threadIdx.x == 0) tc::mbar_init(tc::smem_addr(&bar), 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const bool ok = tc::mbar_wait(tc::smem_addr(&bar), 0, limit_ns);
  const int bad = __syncthreads_or(!ok);
  if (threadIdx.x == 0) *status = bad ? 2 : 0;
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 32);
  }
}

// Persistent grid: kTcCtasPerSm CTAs per SM, at most one per tile.  (The
// occupancy calculator reports one CTA per SM for these kernels, although
// their registers and shared memory admit kTcCtasPerSm, and the hardware
// does co-schedule them; the grid is therefore sized from the launch bound.)
inline int tc_grid(long long n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (n + kTcRows - 1) / kTcRows;
  return (int)std::max(1LL, std::min(tiles, (long long)kTcCtasPerSm * std::max(sms, 1)));
}

}  // namespace xg

using xg::InferPack;

// ------------------------------------------------------------------ stage hook

// Called by the FP32 stage before its passes when the closure is on:
// C = correction of the stage's input state.
cudaError_t closure_launch(xg_ctx* c, const float* q, cudaStream_t st) {
  const float* S = c->has_forcing ? (const float*)c->S : nullptr;
  const InferPack* K = (const InferPack*)c->cl_pack;
  const long long np = c->np;
  switch (c->d.order) {
#define XG_CLOSURE_CASE(n)                                                                              \
  case n: {                                                                                             \
    if (!c->cl_grid) c->cl_grid = xg::tc_grid(np);                                                      \
    const unsigned g = (unsigned)c->cl_grid;                                                            \
    xg::k_closure<n><<<g, xg::kTcRows, 0, st>>>(c->Pf, K, q, S, c->cl_C, c->flag);                       \
    break;                                                                                              \
  }
    XG_CLOSURE_CASE(1) XG_CLOSURE_CASE(2) XG_CLOSURE_CASE(3) XG_CLOSURE_CASE(4)
    XG_CLOSURE_CASE(5) XG_CLOSURE_CASE(6) XG_CLOSURE_CASE(7) XG_CLOSURE_CASE(8)
#undef XG_CLOSURE_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

void closure_free(xg_ctx* c) {
  cudaFree(c->cl_pack);
  cudaFree(c->cl_C);
  c->cl_pack = nullptr;
  c->cl_C = nullptr;
  c->closure = false;
  c->cl_fixed = false;
}

namespace xg {

// out = s (a - b), FP64 (out may alias a or b: each element is read before it is written)
__global__ void k_scaled_difference(const double* a, const double* b, double s, long long n, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = s * (a[i] - b[i]);
}

// dst = (float) src, rounded to nearest
__global__ void k_round_to_f32(const double* __restrict__ src, long long n, float* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = __double2float_rn(src[i]);
}

inline unsigned stream_grid(long long n) {
  return (unsigned)std::max(1LL, std::min((n + 255) / 256, 152LL * 16));
}

}  // namespace xg

namespace {

xg_status cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return XG_OK;
  fprintf(stderr, "xg_closure: %s: %s\n", where, cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? XG_ERR_OOM : XG_ERR_CUDA;
}

// 1-D restriction table: for each coarse node its fine element's first
// global node and the N_f + 1 Lagrange weights of the fine element's LGL
// points at the coarse node's position.
void axis_table(const xg_ctx* f, const xg_ctx* c, int d, std::vector<int>& start, std::vector<double>& w) {
  const int Nf = f->d.order, Nc = c->d.order;
  long double xf[xg::kMaxOrder + 1], xc[xg::kMaxOrder + 1];
  xg::lgl_nodes(Nf, xf);
  xg::lgl_nodes(Nc, xc);
  const double lo = f->d.lo[d], hi = f->d.hi[d];
  const int nelf = f->d.nel[d], nelc = c->d.nel[d];
  const int nf = f->n[d], ncn = c->n[d];
  start.assign(ncn, 0);
  w.assign((size_t)ncn * (Nf + 1), 0.0);
  for (int g = 0; g < ncn; ++g) {
    int e = std::min(g / Nc, nelc - 1);
    const int a = g - Nc * e;
    // position as a fraction of the box, then in fine element units
    const long double frac = ((long double)e + (xc[a] + 1.0L) / 2.0L) / nelc;
    const long double sf = frac * nelf;
    int ef = (int)floorl(sf);
    ef = std::max(0, std::min(ef, nelf - 1));
    const long double loc = 2.0L * (sf - ef) - 1.0L;
    start[g] = (Nf * ef) % nf;
    for (int l = 0; l <= Nf; ++l) {
      long double L = 1.0L;
      for (int k = 0; k <= Nf; ++k)
        if (k != l) L *= (loc - xf[k]) / (xf[l] - xf[k]);
      w[(size_t)g * (Nf + 1) + l] = (double)L;
    }
  }
  (void)lo;
  (void)hi;
}

}  // namespace

extern "C" {

xg_status xg_features(xg_ctx* c, float* X, void* stream) {
  if (!c || !X) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (!c->f32) return XG_ERR_UNSUPPORTED;
  if (!c->has_state) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)((c->np + 127) / 128);
  const float* q = (const float*)c->A;
  const float* S = c->has_forcing ? (const float*)c->S : nullptr;
  switch (c->d.order) {
    case 1: xg::k_features<1><<<blocks, 128, 0, st>>>(c->Pf, q, S, X); break;
    case 2: xg::k_features<2><<<blocks, 128, 0, st>>>(c->Pf, q, S, X); break;
    case 3: xg::k_features<3><<<blocks, 128, 0, st>>>(c->Pf, q, S, X); break;
    case 4: xg::k_features<4><<<blocks, 128, 0, st>>>(c->Pf, q, S, X); break;
    case 5: xg::k_features<5><<<blocks, 128, 0, st>>>(c->Pf, q, S, X); break;
    case 6: xg::k_features<6><<<blocks, 128, 0, st>>>(c->Pf, q, S, X); break;
    case 7: xg::k_features<7><<<blocks, 128, 0, st>>>(c->Pf, q, S, X); break;
    case 8: xg::k_features<8><<<blocks, 128, 0, st>>>(c->Pf, q, S, X); break;
    default: return XG_ERR_ARG;
  }
  return cuda_status(cudaGetLastError(), "xg_features");
}

xg_status xg_restrict(const xg_ctx* f, const xg_ctx* c, const double* src, int nvar, double* dst,
                      void* stream) {
  if (!f || !c || !src || !dst || nvar < 1) return XG_ERR_ARG;
  for (int d = 0; d < 3; ++d) {
    if (f->d.lo[d] != c->d.lo[d] || f->d.hi[d] != c->d.hi[d]) return XG_ERR_ARG;
    if ((f->d.periodic[d] != 0) != (c->d.periodic[d] != 0)) return XG_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int Nf = f->d.order;
  std::vector<int> start[3];
  std::vector<double> w[3];
  for (int d = 0; d < 3; ++d) axis_table(f, c, d, start[d], w[d]);
  const int* nf = f->n;
  const int* nc = c->n;
  const long long s1 = (long long)nvar * nf[2] * nf[1] * nc[0];
  const long long s2 = (long long)nvar * nf[2] * nc[1] * nc[0];
  double *t1 = nullptr, *t2 = nullptr, *dw = nullptr;
  int* ds = nullptr;
  size_t nw = 0, ns = 0;
  for (int d = 0; d < 3; ++d) {
    nw += w[d].size();
    ns += start[d].size();
  }
  cudaError_t e = cudaMalloc((void**)&t1, sizeof(double) * s1);
  if (e == cudaSuccess) e = cudaMalloc((void**)&t2, sizeof(double) * s2);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dw, sizeof(double) * nw);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ds, sizeof(int) * ns);
  size_t ow[3], os[3];
  if (e == cudaSuccess) {
    size_t a = 0, b = 0;
    for (int d = 0; d < 3; ++d) {
      ow[d] = a;
      os[d] = b;
      e = cudaMemcpy(dw + a, w[d].data(), sizeof(double) * w[d].size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(ds + b, start[d].data(), sizeof(int) * start[d].size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) break;
      a += w[d].size();
      b += start[d].size();
    }
  }
  if (e == cudaSuccess) {
    auto grid = [](long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 65535); };
    // x: [v][z_f][y_f] x (x_f -> x_c)
    xg::k_interp_axis<<<grid(s1), 256, 0, st>>>(src, t1, (long long)nvar * nf[2] * nf[1], nf[0], nc[0], 1,
                                                ds + os[0], dw + ow[0], Nf + 1);
    // y: [v][z_f] x (y_f -> y_c) x [x_c]
    xg::k_interp_axis<<<grid(s2), 256, 0, st>>>(t1, t2, (long long)nvar * nf[2], nf[1], nc[1], nc[0],
                                                ds + os[1], dw + ow[1], Nf + 1);
    // z: [v] x (z_f -> z_c) x [y_c x_c]
    const long long s3 = (long long)nvar * nc[2] * nc[1] * nc[0];
    xg::k_interp_axis<<<grid(s3), 256, 0, st>>>(t2, dst, nvar, nf[2], nc[2], (long long)nc[1] * nc[0],
                                                ds + os[2], dw + ow[2], Nf + 1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(t1);
  cudaFree(t2);
  cudaFree(dw);
  cudaFree(ds);
  return cuda_status(e, "xg_restrict");
}

xg_status xg_column_stats(const float* X, int ncol, long long ld, long long n, double* mean,
                          double* stdev, void* stream) {
  if (!X || ncol < 1 || n < 1 || ld < n || !mean || !stdev) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  double* d = nullptr;
  cudaError_t e = cudaMalloc((void**)&d, sizeof(double) * 2 * ncol);
  if (e == cudaSuccess) {
    xg::k_col_stats<<<ncol, 256, 0, st>>>(X, ld, n, d);
    e = cudaGetLastError();
  }
  std::vector<double> h(2 * (size_t)ncol);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(double) * 2 * ncol, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_status(e, "xg_column_stats");
  for (int k = 0; k < ncol; ++k) {
    mean[k] = h[2 * k];
    stdev[k] = h[2 * k + 1];
  }
  return XG_OK;
}

xg_status xg_mlp_loss_grad(const float* params, const float* X, const float* T, long long ld,
                           long long n, const float* in_mean, const float* in_scale,
                           const float* out_scale, float* grad, double* loss, void* stream) {
  if (!params || !X || !T || !in_mean || !in_scale || !out_scale || !grad || !loss) return XG_ERR_ARG;
  if (n < 1 || ld < n) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)std::min<long long>((n + xg::kChunk - 1) / xg::kChunk, 2LL * sms);
  const size_t smem = sizeof(xg::TrainSmem);
  float* partial = nullptr;
  double* lossp = nullptr;
  cudaError_t e = xg::raise_dynamic_smem(xg::k_mlp_grad, smem);
  if (e == cudaSuccess) e = cudaMalloc((void**)&partial, sizeof(float) * (size_t)blocks * xg::kParams);
  if (e == cudaSuccess) e = cudaMalloc((void**)&lossp, sizeof(double) * blocks);
  if (e == cudaSuccess) {
    xg::k_mlp_grad<<<blocks, xg::kTrainThreads, smem, st>>>(params, X, T, ld, n, in_mean, in_scale, out_scale,
                                                           partial, lossp, (float)(2.0 / (5.0 * (double)n)));
    xg::k_mlp_reduce<<<(xg::kParams + 255) / 256, 256, 0, st>>>(partial, blocks, grad);
    e = cudaGetLastError();
  }
  std::vector<double> h(blocks);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), lossp, sizeof(double) * blocks, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(partial);
  cudaFree(lossp);
  if (e != cudaSuccess) return cuda_status(e, "xg_mlp_loss_grad");
  double s = 0.0;
  for (double v : h) s += v;
  *loss = s / (5.0 * (double)n);
  return XG_OK;
}

xg_status xg_mlp_adam(float* params, float* m, float* v, const float* grad, int nparams, int t,
                      double lr, double beta1, double beta2, double eps, void* stream) {
  if (!params || !m || !v || !grad || nparams < 1 || t < 1) return XG_ERR_ARG;
  if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps >= 0.0))
    return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
  xg::k_adam<<<(nparams + 255) / 256, 256, 0, st>>>(params, m, v, grad, nparams, (float)lr, (float)beta1,
                                                    (float)beta2, (float)(1.0 - beta1), (float)(1.0 - beta2),
                                                    (float)eps, (float)c1, (float)c2);
  return cuda_status(cudaGetLastError(), "xg_mlp_adam");
}

xg_status xg_mlp_forward(const float* params, const float* X, long long ld, long long n,
                         const float* in_mean, const float* in_scale, const float* out_scale, float* Y,
                         long long ldy, int precision, void* stream) {
  if (!params || !X || !in_mean || !in_scale || !out_scale || !Y) return XG_ERR_ARG;
  if (n < 1 || ld < n || ldy < n) return XG_ERR_ARG;
  if (precision != XG_MLP_FP32 && precision != XG_MLP_BF16) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == XG_MLP_FP32) {
    xg::k_mlp_fp32<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(params, X, ld, n, in_mean, in_scale,
                                                                 out_scale, Y, ldy);
    return cuda_status(cudaGetLastError(), "xg_mlp_forward");
  }
  // the packed network, then the timeout flag
  char* blob = nullptr;
  cudaError_t e = cudaMalloc((void**)&blob, sizeof(InferPack) + 16);
  int hflag = 0;
  if (e == cudaSuccess) {
    InferPack* K = (InferPack*)blob;
    int* flag = (int*)(blob + sizeof(InferPack));
    e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess) {
      xg::k_pack<<<1, 256, 0, st>>>(params, in_mean, in_scale, out_scale, K);
      xg::k_mlp_bf16<<<xg::tc_grid(n), xg::kTcRows, 0, st>>>(K, X, ld, n, Y, ldy, flag);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(blob);
  if (e == cudaSuccess && hflag) return XG_ERR_TIMEOUT;
  return cuda_status(e, "xg_mlp_forward");
}

xg_status xg_tc_wait_selftest(long long limit_ns, void* stream) {
  if (limit_ns < 1 || limit_ns > 1000000000LL) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* d = nullptr;
  int h = -1;
  cudaError_t e = cudaMalloc((void**)&d, sizeof(int));
  if (e == cudaSuccess) {
    xg::k_tc_wait_selftest<<<1, 128, 0, st>>>((unsigned long long)limit_ns, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(d);
  if (e != cudaSuccess) return cuda_status(e, "xg_tc_wait_selftest");
  return h == 2 ? XG_ERR_TIMEOUT : XG_OK;
}

xg_status xg_closure_set(xg_ctx* c, const float* params, const float* in_mean, const float* in_scale,
                         const float* out_scale, void* stream) {
  if (!c) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (!params) {
    c->closure = false;
    return XG_OK;
  }
  if (!in_mean || !in_scale || !out_scale) return XG_ERR_ARG;
  if (!c->f32) return XG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!c->cl_pack) e = cudaMalloc(&c->cl_pack, sizeof(InferPack));
  if (e == cudaSuccess && !c->cl_C) e = cudaMalloc((void**)&c->cl_C, sizeof(float) * 5 * (size_t)c->np);
  if (e == cudaSuccess) {
    xg::k_pack<<<1, 256, 0, st>>>(params, in_mean, in_scale, out_scale, (InferPack*)c->cl_pack);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    closure_free(c);
    return cuda_status(e, "xg_closure_set");
  }
  c->closure = true;
  c->cl_fixed = false;
  return XG_OK;
}

xg_status xg_correction_set(xg_ctx* c, const double* C, void* stream) {
  if (!c) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (!C) {
    if (c->cl_fixed) c->closure = c->cl_fixed = false;
    return XG_OK;
  }
  if (!c->f32) return XG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const long long n = 5 * c->np;
  cudaError_t e = cudaSuccess;
  if (!c->cl_C) e = cudaMalloc((void**)&c->cl_C, sizeof(float) * (size_t)n);
  if (e == cudaSuccess) {
    xg::k_round_to_f32<<<xg::stream_grid(n), 256, 0, st>>>(C, n, c->cl_C);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    closure_free(c);
    return cuda_status(e, "xg_correction_set");
  }
  c->closure = true;
  c->cl_fixed = true;
  return XG_OK;
}

xg_status xg_closure_target(const double* a, const double* b, double s, long long n, double* out,
                            void* stream) {
  if (!a || !b || !out || n < 0) return XG_ERR_ARG;
  if (n == 0) return XG_OK;
  xg::k_scaled_difference<<<xg::stream_grid(n), 256, 0, (cudaStream_t)stream>>>(a, b, s, n, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? XG_OK : cuda_status(e, "xg_closure_target");
}

}  // extern "C"
