// xg_kernels_f32.cuh -- the precision form: FP32 state and volume arithmetic.
//
// Same method as xg_kernels.cuh in two passes per stage: the x and y parts
// in the plane kernel of xg_plane_f32.cuh, then the tiled z pass here (z
// part, sources, closure correction, walls, stage store).  The state
// perturbations (rho', rho u, rho v, rho w, Theta'), the fluxes, the LGL
// contractions, the assembly, the sources and the SSP-RK combination are
// FP32 (4 bytes per value, FMA on the FP32 pipes).  The pressure
// perturbation p' = p(Theta_0 + Theta') - p(Theta_0) of Eq. 3 is evaluated
// FP64-accurately (double-float, xg_df.cuh) from the FP64 reference state,
// so the hydrostatic reference is subtracted analytically and never from
// rounded FP32 totals; conservation sums are FP64 (xg_diagnostics).
#pragma once

#include <cuda_runtime.h>

#include "xg_df.cuh"
#include "xg_kernels.cuh"
#include "xg_kernels_df.cuh"

namespace xg {

struct FParams {
  int n[3];
  int nseg[3];
  int per[3];
  long long np;
  float Dm[3][kMaxOrder + 1][kMaxOrder + 1];   // -(2/h_d) D, rows 0 and N halved
  df eos_c[3];                                 // C(gamma,1..3)
  float eos_g[kEosTerms - 3];                  // C(gamma,4..8)
  float eos_xmax;
  double gamma;
  float f, g;
};

struct FBufs {
  const float* q;
  const float* qn;
  float* out;
  float* W;          // [3][np] v, w, p'
  float* T;          // [5][np]
  const float* S;    // [np] or null
  const df* base;    // [4][nz] rho0, Theta0, p0, 1/Theta0 (FP64-accurate pairs)
  const float* C;    // [5][np] closure correction added to the tendency, or null
  int* flag;
  float dt, alpha, beta;
  int rhs_only;
};

__device__ __forceinline__ bool f_nonfinite(float v) {
  return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u;
}

// p' = p0 ((1 + x)^gamma - 1), x = Theta'/Theta0, in double-float.
__device__ __forceinline__ float f_pressure_pert(const FParams& P, float tp, df p0, df iTh0) {
  const df x = df_mul_f(iTh0, tp);
  df phi;
  if (fabsf(x.h) < P.eos_xmax) {
    float g = P.eos_g[kEosTerms - 4];
#pragma unroll
    for (int k = kEosTerms - 5; k >= 0; --k) g = __fmaf_rn(g, x.h, P.eos_g[k]);
    df a = df_add_nc(P.eos_c[2], df_mul_f(x, g));
    a = df_add_nc(P.eos_c[1], df_mul(x, a));
    a = df_add_nc(P.eos_c[0], df_mul(x, a));
    phi = df_mul(x, a);
  } else {
    phi = df_from_double(expm1(P.gamma * log1p(df_to_double(x))));
  }
  const df pp = df_mul(p0, phi);
  return __fadd_rn(pp.h, pp.l);
}

template <int N, int D>
__device__ __forceinline__ float f_row_from(const FParams& P, int a, const float (&f)[N + 1], float acc) {
#pragma unroll
  for (int l = 0; l <= N; ++l) acc = fmaf(P.Dm[D][a][l], f[l], acc);
  return acc;
}

// Row a of the rho' and Theta' contractions in difference form, added to r0
// and r4, from the segment's rho' fluxes m_l = rho u_D and theta_l:
//   sum_{l>=1} Dm[a][l] (m_l - m_0)  and  sum_{l>=1} Dm[a][l] (F_l - F_0),
//   F_l - F_0 = theta_l (m_l - m_0) + (theta_l - theta_0) m_0.
// Equal to the plain rows because each row of the derivative matrix sums to
// zero; the roundings scale with the fluxes' variation across the segment
// instead of the fluxes themselves, which matters where the two tendencies
// are residuals of cancelling x, y and z parts (the difference form is
// described in full beside df_seg_diffs).
template <int N, int D>
__device__ __forceinline__ void f_drows(const FParams& P, int a, const float (&m)[N + 1],
                                        const float (&th)[N + 1], float& r0, float& r4) {
#pragma unroll
  for (int l = 1; l <= N; ++l) {
    const float dm = m[l] - m[0];
    const float dF = fmaf(th[l], dm, (th[l] - th[0]) * m[0]);
    r0 = fmaf(P.Dm[D][a][l], dm, r0);
    r4 = fmaf(P.Dm[D][a][l], dF, r4);
  }
}

// start + sum_{l>=1} Dm[D][a][l] d[l-1] (differences against the segment start)
template <int N, int D>
__device__ __forceinline__ float f_drow_from(const FParams& P, int a, const float (&d)[N], float acc) {
#pragma unroll
  for (int l = 1; l <= N; ++l) acc = fmaf(P.Dm[D][a][l], d[l - 1], acc);
  return acc;
}

// Shared floats of one y/z tile of K segments: the fluxes [5][NS][32] and the
// rho' and Theta' flux differences [2][NS][32], NS = K N + N + 1.
__host__ __device__ constexpr int tline_smem_floats(int N, int K) { return 7 * (K * N + N + 1) * kTileCols; }

// ---------------------------------------------------------------- y and z lines, tiled
// One thread per node over (32 x-columns) x (K segments along DIR) tiles, as
// k_df_tline; DIR = 1 adds the y part into T, DIR = 2 finishes the node.
// Slot 4 holds theta = Theta / rho: the Theta' flux theta (rho u_DIR) is taken
// in difference form with slot 0.
template <int DIR>
__device__ __forceinline__ void f_flux_vals(const float (&qv)[5], float vel, float pp, float rho0,
                                            float Th0, float (&f)[5]) {
  f[0] = qv[DIR + 1];
  f[1] = qv[1] * vel;
  f[2] = DIR == 1 ? fmaf(qv[2], vel, pp) : qv[2] * vel;
  f[3] = DIR == 1 ? qv[3] * vel : fmaf(qv[3], vel, pp);
  f[4] = (Th0 + qv[4]) * __frcp_rn(rho0 + qv[0]);
}

__device__ __forceinline__ void f_finish_vals(const FParams& P, const FBufs& B,
                                              const float (&qv)[5], const float (&qnv)[5],
                                              float sv, float rho0, float* __restrict__ out,
                                              long long I, int x, int y, int gz, float (&L)[5],
                                              bool& bad, const float (&cv)[5]) {
  const long long np = P.np;
  if (B.C) {
#pragma unroll
    for (int c = 0; c < 5; ++c) L[c] += cv[c];
  }
  L[1] = fmaf(P.f, qv[2], L[1]);
  L[2] = fmaf(-P.f, qv[1], L[2]);
  L[3] = fmaf(-P.g, qv[0], L[3]);
  if (B.S) L[4] = fmaf(rho0 + qv[0], sv, L[4]);
  if (!P.per[0] && (x == 0 || x == P.n[0] - 1)) L[1] = 0.0f;
  if (!P.per[1] && (y == 0 || y == P.n[1] - 1)) L[2] = 0.0f;
  if (!P.per[2] && (gz == 0 || gz == P.n[2] - 1)) L[3] = 0.0f;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    float o;
    if (B.rhs_only) o = L[c];
    else if (B.alpha == 0.0f) o = fmaf(B.dt, L[c], qv[c]);
    else o = fmaf(B.alpha, qnv[c], B.beta * fmaf(B.dt, L[c], qv[c]));
    out[c * np + I] = o;
    bad |= f_nonfinite(o);
  }
}

// One thread per node over (32 x-columns) x (K segments along DIR) tiles, as
// k_df_tline: every global load first, fluxes to shared memory, then each
// thread assembles its node (DIR = 1 adds the y part into T, DIR = 2
// finishes the node).
//
// f_tline_tile is the body of one tile (bx: 32-column block, by: K-segment
// block, other: the y index for DIR = 2, the z index for DIR = 1) for the
// thread (tx, ty), ty < K N + 1 (larger ty own nothing, but every thread of
// the block calls it: it synchronises the block twice); Fsm holds the tile's
// tline_smem_floats(N, K) shared floats.
// CG selects L2-only loads (ld.global.cg) for every array a launch may
// itself have written, which a persistent launch that runs several passes
// needs; the per-pass kernels use ordinary loads.
template <bool CG>
__device__ __forceinline__ float ldf(const float* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

template <int N, int DIR, bool CG, int K = tile_segments(N)>
__device__ __forceinline__ void f_tline_tile(const FParams& P, const FBufs& B, int bx, int by,
                                             int other, int tx, int ty, float* Fsm) {
  constexpr int NS = K * N + N + 1;
  auto Fs = reinterpret_cast<float(*)[NS][kTileCols]>(Fsm);
  // rho' and Theta' flux differences of slot j against the first slot of its
  // segment, N floor((j - 1) / N) (slot j >= 1 is an interior node or the end)
  auto Ds = reinterpret_cast<float(*)[NS][kTileCols]>(Fsm + 5 * NS * kTileCols);
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const int nd = P.n[DIR];
  const int nseg = P.nseg[DIR];
  const bool per = P.per[DIR] != 0;
  const int x = bx * kTileCols + tx;
  const bool xin = x < nx;
  const int s0 = by * K;
  const int kc = min(K, nseg - s0);
  const long long np = P.np;
  const long long sd = DIR == 1 ? (long long)nx : (long long)nx * ny;
  const long long base = DIR == 1 ? x + (long long)nx * ny * other : x + (long long)nx * other;
  const bool has_left = s0 > 0 || per;
  auto plane = [&](int g) -> int { return g >= nd ? g - nd : (g < 0 ? g + nd : g); };
  auto th0 = [&](int g) -> float {
    const df t = B.base[nz + (DIR == 2 ? g : other)];
    return t.h + t.l;
  };
  auto rh0 = [&](int g) -> float {
    const df t = B.base[DIR == 2 ? g : other];
    return t.h + t.l;
  };
  const int vslot = DIR == 1 ? 0 : 1;

  const int own = s0 * N + ty;
  const bool owns = xin && (ty < kc * N || (ty == kc * N && s0 + kc == nseg && !per));
  const bool main_plane = xin && ty <= kc * N;
  const bool halo = xin && has_left && ty < N;
  const int g = plane(own);
  const int gh = plane((s0 - 1) * N + ty);
  const long long I = base + sd * (main_plane ? g : 0);
  const long long Ih = base + sd * (halo ? gh : 0);

  float qv[5], vel = 0.0f, pp = 0.0f, hq[5] = {0, 0, 0, 0, 0}, hvel = 0.0f, hpp = 0.0f;
  float t[5], qnv[5] = {0, 0, 0, 0, 0}, sv = 0.0f, cv[5] = {0, 0, 0, 0, 0};
  if (main_plane) {
#pragma unroll
    for (int c = 0; c < 5; ++c) qv[c] = ldf<CG>(B.q + c * np + I);
    vel = ldf<CG>(B.W + vslot * np + I);
    pp = ldf<CG>(B.W + 2 * np + I);
  }
  if (halo) {
#pragma unroll
    for (int c = 0; c < 5; ++c) hq[c] = ldf<CG>(B.q + c * np + Ih);
    hvel = ldf<CG>(B.W + vslot * np + Ih);
    hpp = ldf<CG>(B.W + 2 * np + Ih);
  }
  if (owns) {
#pragma unroll
    for (int c = 0; c < 5; ++c) t[c] = ldf<CG>(B.T + c * np + I);
    if (DIR == 2) {
      if (!B.rhs_only && B.alpha != 0.0f) {
#pragma unroll
        for (int c = 0; c < 5; ++c) qnv[c] = ldf<CG>(B.qn + c * np + I);
      }
      if (B.S) sv = B.S[I];
      if (B.C) {
#pragma unroll
        for (int c = 0; c < 5; ++c) cv[c] = ldf<CG>(B.C + c * np + I);
      }
    }
  }
  if (main_plane) {
    float f[5];
    f_flux_vals<DIR>(qv, vel, pp, rh0(g), th0(g), f);
#pragma unroll
    for (int c = 0; c < 5; ++c) Fs[c][N + ty][tx] = f[c];
  }
  if (halo) {
    float f[5];
    f_flux_vals<DIR>(hq, hvel, hpp, rh0(gh), th0(gh), f);
#pragma unroll
    for (int c = 0; c < 5; ++c) Fs[c][ty][tx] = f[c];
  }
  __syncthreads();
  // difference form of the rho' and Theta' fluxes, slot by slot (every
  // thread of the block reaches both barriers)
  auto diff_slot = [&](int j) {
    const int b = N * ((j - 1) / N);
    const float mb = Fs[0][b][tx], thb = Fs[4][b][tx], thj = Fs[4][j][tx];
    const float dm = Fs[0][j][tx] - mb;
    Ds[0][j][tx] = dm;
    Ds[1][j][tx] = fmaf(thj, dm, (thj - thb) * mb);
  };
  if (main_plane && (ty > 0 || has_left)) diff_slot(N + ty);   // slot N closes the halo segment
  if (halo && ty > 0) diff_slot(ty);
  __syncthreads();
  if (!owns) return;   // no barrier follows: the caller synchronises before reusing Fs

  const int k = ty < kc * N ? ty / N : kc - 1;
  const int a = ty < kc * N ? ty - k * N : N;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int c = e == 0 ? 0 : 4;
    float d[N];
#pragma unroll
    for (int l = 1; l <= N; ++l) d[l - 1] = Ds[e][N + k * N + l][tx];
    if (a == N) {
      t[c] = fmaf(2.0f, f_drow_from<N, DIR>(P, N, d, 0.0f), t[c]);
    } else if (a > 0) {
      t[c] = f_drow_from<N, DIR>(P, a, d, t[c]);
    } else if (k > 0 || has_left) {
      float dl[N];
#pragma unroll
      for (int l = 1; l <= N; ++l) dl[l - 1] = Ds[e][k * N + l][tx];
      t[c] = f_drow_from<N, DIR>(P, 0, d, t[c]);
      t[c] = f_drow_from<N, DIR>(P, N, dl, t[c]);
    } else {
      t[c] = f_drow_from<N, DIR>(P, 0, d, t[c]);
      t[c] = f_drow_from<N, DIR>(P, 0, d, t[c]);
    }
  }
#pragma unroll
  for (int c = 1; c < 4; ++c) {
    float f[N + 1];
#pragma unroll
    for (int l = 0; l <= N; ++l) f[l] = Fs[c][N + k * N + l][tx];
    if (a == N) {
      t[c] = fmaf(2.0f, f_row_from<N, DIR>(P, N, f, 0.0f), t[c]);
    } else if (a > 0) {
      t[c] = f_row_from<N, DIR>(P, a, f, t[c]);
    } else if (k > 0 || has_left) {
      float fl[N + 1];
#pragma unroll
      for (int l = 0; l <= N; ++l) fl[l] = Fs[c][k * N + l][tx];
      t[c] = f_row_from<N, DIR>(P, 0, f, t[c]);
      t[c] = f_row_from<N, DIR>(P, N, fl, t[c]);
    } else {
      t[c] = f_row_from<N, DIR>(P, 0, f, t[c]);
      t[c] = f_row_from<N, DIR>(P, 0, f, t[c]);
    }
  }
  if (DIR == 1) {
#pragma unroll
    for (int c = 0; c < 5; ++c) B.T[c * np + I] = t[c];
  } else {
    bool bad = false;
    const df r0 = B.base[g];
    f_finish_vals(P, B, qv, qnv, sv, r0.h, B.out, I, x, other, g, t, bad, cv);
    if (bad) atomicOr(B.flag, 1);   // bit 0; the closure kernel reports a timeout in bit 1
  }
}

// The single-context z tiles hold at most 9 planes: 4 CTAs of 288 threads
// per SM (measured: 0.297 vs 0.338 ms per launch on the 128x128x16 order-4
// box against 17-plane tiles).
__host__ __device__ constexpr int f32_tile_segments(int N) { return N >= 8 ? 1 : 8 / N; }

template <int N, int DIR>
__global__ void __launch_bounds__(kTileCols * (8 + 1), 4) k_f_tline(const FParams P, const FBufs B) {
  constexpr int K = f32_tile_segments(N);
  __shared__ float Fs[tline_smem_floats(N, K)];
  f_tline_tile<N, DIR, false, K>(P, B, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, threadIdx.y, Fs);
}

// FP64 <-> FP32 conversion of n values (data entering or leaving).
__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, long long n);
__global__ void k_from_f32(const float* __restrict__ in, double* __restrict__ out, long long n);

}  // namespace xg
