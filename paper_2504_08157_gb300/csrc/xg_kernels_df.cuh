// xg_kernels_df.cuh -- the line kernels of xg_kernels.cuh in double-float
// arithmetic (xg_df.cuh) on the FP32 pipes.
//
// Same method, same three-kernel stage (x lines with primitives, y lines,
// z lines with sources, walls and the SSP-RK stage), same data layout: every
// [5][Np] array holds double-float pairs (8 bytes per value, like FP64).
// The contractions are compensated dot products (Dot2) seeded with the
// running tendency; additions that can cancel use the accurate double-word
// sum; the equation of state keeps the binomial series, its tail in float
// and its first three terms in double-float.  The FP64 pipe is used only by
// the rare equation-of-state fallback (|Theta'/Theta_0| >= x_max).
#pragma once

#include <cuda_runtime.h>

#include "xg_df.cuh"
#include "xg_kernels.cuh"

namespace xg {

struct DfParams {
  int n[3];
  int nseg[3];
  int per[3];
  long long np;
  df Dm[3][kMaxOrder + 1][kMaxOrder + 1];   // -(2/h_d) D, rows 0 and N halved
  df eos_c[3];                              // C(gamma,1..3)
  float eos_g[kEosTerms - 3];               // C(gamma,4..8)
  float eos_xmax;
  double gamma;
  df f, g;
};

struct DfBufs {
  const df* q;
  const df* qn;
  df* out;
  df* W;          // [3][np] v, w, p'
  df* T;          // [5][np]
  const df* S;    // [np] or null
  const df* base; // [4][nz] rho0, Theta0, p0, 1/Theta0
  int* flag;
  df dt, alpha, beta, bdt;   // bdt = beta dt
  int rhs_only;
};

// (1+x)^gamma - 1 = x (c1 + x (c2 + x (c3 + x g(x)))), g = c4 + ... + c8 x^4
// in float (its rounding enters at relative size x^3 2^-24).
__device__ __forceinline__ df df_eos_phi(const DfParams& P, df x) {
  if (fabsf(x.h) < P.eos_xmax) {
    float g = P.eos_g[kEosTerms - 4];
#pragma unroll
    for (int k = kEosTerms - 5; k >= 0; --k) g = __fmaf_rn(g, x.h, P.eos_g[k]);
    df a = df_add_nc(P.eos_c[2], df_mul_f(x, g));
    a = df_add_nc(P.eos_c[1], df_mul(x, a));
    a = df_add_nc(P.eos_c[0], df_mul(x, a));
    return df_mul(x, a);
  }
  const double xd = df_to_double(x);
  return df_from_double(expm1(P.gamma * log1p(xd)));
}

// start + sum_l Dm[d][a][l] f[l] (Dot2)
template <int N, int D>
__device__ __forceinline__ df df_row_from(const DfParams& P, int a, const df (&f)[N + 1], df start) {
  dacc A = dacc_from(start);
#pragma unroll
  for (int l = 0; l <= N; ++l) dacc_fma(A, P.Dm[D][a][l], f[l]);
  return dacc_value(A);
}

template <int N, int D>
__device__ __forceinline__ df df_row(const DfParams& P, int a, const df (&f)[N + 1]) {
  dacc A = dacc_prod(P.Dm[D][a][0], f[0]);
#pragma unroll
  for (int l = 1; l <= N; ++l) dacc_fma(A, P.Dm[D][a][l], f[l]);
  return dacc_value(A);
}

// ---------------------------------------------------------------- x lines
template <int N>
__global__ void __launch_bounds__(kXThreads) k_df_line_x(const DfParams P, const DfBufs B) {
  extern __shared__ df smd[];
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const int nseg = P.nseg[0];
  const int y = blockIdx.x, z = blockIdx.y;
  const long long np = P.np;
  const long long row = (long long)nx * (y + (long long)ny * z);
  const int ld = nx + 1;
  df* F = smd;             // [5][ld], later rows 0..N-1 of every segment in place
  df* RN = smd + 5 * ld;   // [5][nseg] row N
  const df rho0 = B.base[z], Th0 = B.base[nz + z], p0 = B.base[2 * nz + z];
  const df iTh0 = B.base[3 * nz + z];
  const df* __restrict__ q = B.q;

  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const long long I = row + i;
    const df rp = q[I], mu = q[np + I], mv = q[2 * np + I], mw = q[3 * np + I];
    const df tp = q[4 * np + I];
    const df ir = df_rcp(df_add(rho0, rp));
    const df u = df_mul(mu, ir), v = df_mul(mv, ir), w = df_mul(mw, ir);
    const df pp = df_mul(p0, df_eos_phi(P, df_mul(tp, iTh0)));
    const df Th = df_add(Th0, tp);
    B.W[I] = v;
    B.W[np + I] = w;
    B.W[2 * np + I] = pp;
    F[i] = mu;
    F[ld + i] = df_add(df_mul(mu, u), pp);
    F[2 * ld + i] = df_mul(mv, u);
    F[3 * ld + i] = df_mul(mw, u);
    F[4 * ld + i] = df_mul(Th, u);
    if (P.per[0] && i == 0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) F[c * ld + nx] = F[c * ld];
    }
  }
  __syncthreads();

  for (int s0 = 0; s0 < nseg; s0 += blockDim.x) {
    const int s = s0 + threadIdx.x;
    df rows[5][N + 1];
    if (s < nseg) {
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        df f[N + 1];
#pragma unroll
        for (int l = 0; l <= N; ++l) f[l] = F[c * ld + s * N + l];
#pragma unroll
        for (int a = 0; a <= N; ++a) rows[c][a] = df_row<N, 0>(P, a, f);
      }
    }
    __syncthreads();
    if (s < nseg) {
#pragma unroll
      for (int c = 0; c < 5; ++c) {
#pragma unroll
        for (int a = 0; a < N; ++a) F[c * ld + s * N + a] = rows[c][a];
        RN[c * nseg + s] = rows[c][N];
      }
    }
    __syncthreads();
  }

  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const int s = i / N, a = i - s * N;
    const long long I = row + i;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      df v;
      if (s == nseg) {
        v = df_scale2(RN[c * nseg + nseg - 1], 2.0f);
      } else if (a != 0) {
        v = F[c * ld + i];
      } else {
        const df r0 = F[c * ld + i];
        const int left = s > 0 ? s - 1 : (P.per[0] ? nseg - 1 : -1);
        v = left >= 0 ? df_add(r0, RN[c * nseg + left]) : df_scale2(r0, 2.0f);
      }
      B.T[c * np + I] = v;
    }
  }
}

// ---------------------------------------------------------------- y lines
__device__ __forceinline__ void df_flux_y(const df* __restrict__ q, const df* __restrict__ W,
                                          long long np, long long I, df Th0, df (&f)[5]) {
  const df mu = q[np + I], mv = q[2 * np + I], mw = q[3 * np + I], tp = q[4 * np + I];
  const df v = W[I], pp = W[2 * np + I];
  f[0] = mv;
  f[1] = df_mul(mu, v);
  f[2] = df_add(df_mul(mv, v), pp);
  f[3] = df_mul(mw, v);
  f[4] = df_mul(df_add(Th0, tp), v);
}

template <int N>
__global__ void __launch_bounds__(128, 4) k_df_line_y(const DfParams P, const DfBufs B, int chunk) {
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const int nseg = P.nseg[1];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int z = blockIdx.z;
  const int s0 = blockIdx.y * chunk;
  const int s1 = min(nseg, s0 + chunk);
  if (s0 >= s1) return;
  const long long np = P.np;
  const long long col = x + (long long)nx * ny * z;
  const df Th0 = B.base[nz + z];
  const df* __restrict__ q = B.q;
  const df* __restrict__ W = B.W;
  df* __restrict__ T = B.T;
  auto nodeI = [&](int gy) -> long long { return col + (long long)nx * (gy == ny ? 0 : gy); };

  df carry[5];
  bool has_left = (s0 > 0) || P.per[1];
  if (has_left) {
    const int sp = s0 > 0 ? s0 - 1 : nseg - 1;
    df fl[5][N + 1];
#pragma unroll
    for (int l = 0; l <= N; ++l) {
      df f[5];
      df_flux_y(q, W, np, nodeI(sp * N + l), Th0, f);
#pragma unroll
      for (int c = 0; c < 5; ++c) fl[c][l] = f[c];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) carry[c] = df_row<N, 1>(P, N, fl[c]);
  }

  df fc[5][N + 1];
  {
    df f[5];
    df_flux_y(q, W, np, nodeI(s0 * N), Th0, f);
#pragma unroll
    for (int c = 0; c < 5; ++c) fc[c][0] = f[c];
  }
  for (int s = s0; s < s1; ++s) {
#pragma unroll
    for (int l = 1; l <= N; ++l) {
      df f[5];
      df_flux_y(q, W, np, nodeI(s * N + l), Th0, f);
#pragma unroll
      for (int c = 0; c < 5; ++c) fc[c][l] = f[c];
    }
    df tv[5][N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const long long I = nodeI(s * N + a);
#pragma unroll
      for (int c = 0; c < 5; ++c) tv[c][a] = T[c * np + I];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      df t0 = tv[c][0];
      if (!has_left) t0 = df_row_from<N, 1>(P, 0, fc[c], t0);   // wall: the row counts twice
      t0 = df_row_from<N, 1>(P, 0, fc[c], t0);
      T[c * np + nodeI(s * N)] = has_left ? df_add(t0, carry[c]) : t0;
#pragma unroll
      for (int a = 1; a < N; ++a) T[c * np + nodeI(s * N + a)] = df_row_from<N, 1>(P, a, fc[c], tv[c][a]);
      carry[c] = df_row<N, 1>(P, N, fc[c]);
      fc[c][0] = fc[c][N];
    }
    has_left = true;
  }
  if (!P.per[1] && s1 == nseg) {
    const long long I = nodeI(nseg * N);
#pragma unroll
    for (int c = 0; c < 5; ++c) T[c * np + I] = df_add(T[c * np + I], df_scale2(carry[c], 2.0f));
  }
}

// ---------------------------------------------------------------- z lines + sources + stage
__device__ __forceinline__ void df_flux_z(const df* __restrict__ q, const df* __restrict__ W,
                                          long long np, long long I, df Th0, df (&f)[5]) {
  const df mu = q[np + I], mv = q[2 * np + I], mw = q[3 * np + I], tp = q[4 * np + I];
  const df w = W[np + I], pp = W[2 * np + I];
  f[0] = mw;
  f[1] = df_mul(mu, w);
  f[2] = df_mul(mv, w);
  f[3] = df_add(df_mul(mw, w), pp);
  f[4] = df_mul(df_add(Th0, tp), w);
}

__device__ __forceinline__ void df_finish_node(const DfParams& P, const DfBufs& B, long long I,
                                               int x, int y, int gz, df (&L)[5], bool& bad) {
  const long long np = P.np;
  const df* __restrict__ q = B.q;
  const df rp = q[I], mu = q[np + I], mv = q[2 * np + I];
  {
    dacc A = dacc_from(L[1]);
    dacc_fma(A, P.f, mv);                        // +f rho v
    L[1] = dacc_value(A);
    A = dacc_from(L[2]);
    dacc_fma(A, df_neg(P.f), mu);                // -f rho u
    L[2] = dacc_value(A);
    A = dacc_from(L[3]);
    dacc_fma(A, df_neg(P.g), rp);                // -rho' g
    L[3] = dacc_value(A);
    if (B.S) {
      A = dacc_from(L[4]);
      dacc_fma(A, df_add(B.base[gz], rp), B.S[I]);   // rho S_theta
      L[4] = dacc_value(A);
    }
  }
  const df zero = {0.0f, 0.0f};
  if (!P.per[0] && (x == 0 || x == P.n[0] - 1)) L[1] = zero;
  if (!P.per[1] && (y == 0 || y == P.n[1] - 1)) L[2] = zero;
  if (!P.per[2] && (gz == 0 || gz == P.n[2] - 1)) L[3] = zero;
  if (B.rhs_only) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      B.out[c * np + I] = L[c];
      bad |= df_nonfinite(L[c]);
    }
  } else if (B.alpha.h == 0.0f) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      dacc A = dacc_from(q[c * np + I]);
      dacc_fma(A, B.dt, L[c]);
      const df o = dacc_value(A);
      B.out[c * np + I] = o;
      bad |= df_nonfinite(o);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      dacc A = dacc_prod(B.alpha, B.qn[c * np + I]);
      dacc_fma(A, B.beta, q[c * np + I]);
      dacc_fma(A, B.bdt, L[c]);
      const df o = dacc_value(A);
      B.out[c * np + I] = o;
      bad |= df_nonfinite(o);
    }
  }
}

template <int N>
__global__ void __launch_bounds__(128) k_df_line_z(const DfParams P, const DfBufs B, int chunk) {
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const int nseg = P.nseg[2];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int y = blockIdx.z;
  const int s0 = blockIdx.y * chunk;
  const int s1 = min(nseg, s0 + chunk);
  if (s0 >= s1) return;
  const long long np = P.np;
  const long long nxy = (long long)nx * ny;
  const long long col = x + (long long)nx * y;
  const df* __restrict__ q = B.q;
  const df* __restrict__ W = B.W;
  const df* __restrict__ T = B.T;
  auto lev = [&](int gz) -> int { return gz == nz ? 0 : gz; };
  bool bad = false;

  df carry[5];
  bool has_left = (s0 > 0) || P.per[2];
  if (has_left) {
    const int sp = s0 > 0 ? s0 - 1 : nseg - 1;
    df fl[5][N + 1];
#pragma unroll
    for (int l = 0; l <= N; ++l) {
      const int gz = lev(sp * N + l);
      df f[5];
      df_flux_z(q, W, np, col + nxy * gz, B.base[nz + gz], f);
#pragma unroll
      for (int c = 0; c < 5; ++c) fl[c][l] = f[c];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) carry[c] = df_row<N, 2>(P, N, fl[c]);
  }

  df fc[5][N + 1];
  {
    const int gz = s0 * N;
    df f[5];
    df_flux_z(q, W, np, col + nxy * gz, B.base[nz + gz], f);
#pragma unroll
    for (int c = 0; c < 5; ++c) fc[c][0] = f[c];
  }
  for (int s = s0; s < s1; ++s) {
#pragma unroll
    for (int l = 1; l <= N; ++l) {
      const int gz = lev(s * N + l);
      df f[5];
      df_flux_z(q, W, np, col + nxy * gz, B.base[nz + gz], f);
#pragma unroll
      for (int c = 0; c < 5; ++c) fc[c][l] = f[c];
    }
    df tv[5][N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const long long I = col + nxy * (s * N + a);
#pragma unroll
      for (int c = 0; c < 5; ++c) tv[c][a] = T[c * np + I];
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const int gz = s * N + a;
      const long long I = col + nxy * gz;
      df L[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        df t = tv[c][a];
        if (a == 0 && !has_left) t = df_row_from<N, 2>(P, 0, fc[c], t);
        t = df_row_from<N, 2>(P, a, fc[c], t);
        L[c] = (a == 0 && has_left) ? df_add(t, carry[c]) : t;
      }
      df_finish_node(P, B, I, x, y, gz, L, bad);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      carry[c] = df_row<N, 2>(P, N, fc[c]);
      fc[c][0] = fc[c][N];
    }
    has_left = true;
  }
  if (!P.per[2] && s1 == nseg) {
    const int gz = nseg * N;
    const long long I = col + nxy * gz;
    df L[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) L[c] = df_add(T[c * np + I], df_scale2(carry[c], 2.0f));
    df_finish_node(P, B, I, x, y, gz, L, bad);
  }
  if (bad) *B.flag = 1;
}

// FP64 <-> double-float conversion of n values (data entering or leaving).
__global__ void k_to_df(const double* __restrict__ in, df* __restrict__ out, long long n);
__global__ void k_from_df(const df* __restrict__ in, double* __restrict__ out, long long n);

}  // namespace xg
