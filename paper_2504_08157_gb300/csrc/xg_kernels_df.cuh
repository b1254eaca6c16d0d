// xg_kernels_df.cuh -- the line kernels of xg_kernels.cuh in double-float
// arithmetic (xg_df.cuh) on the FP32 pipes.
//
// Same method, same three-kernel stage (x lines with primitives, y lines,
// z lines with sources, walls and the SSP-RK stage; the z kernel is tiled
// instead of marching, see k_df_tline), same data layout: every
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
  int open_y[2];   // partition faces at the y ends (see LineParams)
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
  df* W;          // [4][np] v, w, p', theta = Theta / rho
  df* T;          // [5][np]
  const df* S;    // [np] or null
  const df* base; // [4][nz] rho0, Theta0, p0, 1/Theta0
  int* flag;
  df dt, alpha, beta, bdt;   // bdt = beta dt
  int rhs_only;
  df* face_hi;    // [5][n_z][n_x] one-sided row N at an open y end (see StageBufs)
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

// ---------------------------------------------------------------- difference form
// The rho' and Theta' tendencies are small residuals of cancelling flux
// derivatives wherever the flow is nearly non-divergent (a vortex: the x and
// y parts nearly cancel), so their absolute error must stay far below the
// size of each part.  A compensated dot product's error is proportional to
// the sum of |Dm[a][l] f_l|, which for a smooth flux is many times the
// derivative itself.  Each row of the LGL derivative matrix sums to zero
// (D 1 = 0: the derivative of a constant), so
//     sum_l Dm[a][l] f_l = sum_{l>=1} Dm[a][l] (f_l - f_0),
// whose terms scale with the flux's variation across the element segment
// instead of with the flux itself.  The Theta' flux Theta u_d is written as
// theta (rho u_d) with theta = Theta / rho, and its differences as
//     F_l - F_0 = theta_l (m_l - m_0) + (theta_l - theta_0) m_0,
// so that the rounding of the product also scales with the variation (for a
// level-uniform theta, as in a balanced vortex, the second part vanishes).
// The exact value is unchanged; only the rounding is.

// differences of one element segment: dm[l-1] = m_l - m_0 (the rho' flux)
// and dF[l-1] = theta_l m_l - theta_0 m_0 (the Theta' flux), l = 1..N
template <int N>
__device__ __forceinline__ void df_seg_diffs(const df (&m)[N + 1], const df (&th)[N + 1],
                                             df (&dm)[N], df (&dF)[N]) {
#pragma unroll
  for (int l = 1; l <= N; ++l) {
    dm[l - 1] = df_sub(m[l], m[0]);
    dF[l - 1] = df_add_nc(df_mul(th[l], dm[l - 1]), df_mul(df_sub(th[l], th[0]), m[0]));
  }
}

// start + sum_{l>=1} Dm[d][a][l] d[l-1] (Dot2)
template <int N, int D>
__device__ __forceinline__ df df_drow_from(const DfParams& P, int a, const df (&d)[N], df start) {
  dacc A = dacc_from(start);
#pragma unroll
  for (int l = 1; l <= N; ++l) dacc_fma(A, P.Dm[D][a][l], d[l - 1]);
  return dacc_value(A);
}

template <int N, int D>
__device__ __forceinline__ df df_drow(const DfParams& P, int a, const df (&d)[N]) {
  dacc A = dacc_prod(P.Dm[D][a][1], d[0]);
#pragma unroll
  for (int l = 2; l <= N; ++l) dacc_fma(A, P.Dm[D][a][l], d[l - 1]);
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
  df* __restrict__ Wo = B.W;
  df* __restrict__ To = B.T;

  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const long long I = row + i;
    const df rp = q[I], mu = q[np + I], mv = q[2 * np + I], mw = q[3 * np + I];
    const df tp = q[4 * np + I];
    const df ir = df_rcp(df_add(rho0, rp));
    const df u = df_mul(mu, ir), v = df_mul(mv, ir), w = df_mul(mw, ir);
    const df pp = df_mul(p0, df_eos_phi(P, df_mul(tp, iTh0)));
    const df Th = df_add(Th0, tp);
    const df th = df_mul(Th, ir);
    Wo[I] = v;
    Wo[np + I] = w;
    Wo[2 * np + I] = pp;
    Wo[3 * np + I] = th;
    F[i] = mu;
    F[ld + i] = df_add(df_mul(mu, u), pp);
    F[2 * ld + i] = df_mul(mv, u);
    F[3 * ld + i] = df_mul(mw, u);
    F[4 * ld + i] = th;               // theta: the Theta' flux is theta (rho u)
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
      {
        df m[N + 1], th[N + 1], dm[N], dF[N];
#pragma unroll
        for (int l = 0; l <= N; ++l) {
          m[l] = F[s * N + l];
          th[l] = F[4 * ld + s * N + l];
        }
        df_seg_diffs<N>(m, th, dm, dF);
#pragma unroll
        for (int a = 0; a <= N; ++a) {
          rows[0][a] = df_drow<N, 0>(P, a, dm);
          rows[4][a] = df_drow<N, 0>(P, a, dF);
        }
      }
#pragma unroll
      for (int c = 1; c < 4; ++c) {
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
      To[c * np + I] = v;
    }
  }
}

// ---------------------------------------------------------------- y lines
// y-fluxes at one node; slot 4 holds theta = Theta / rho from W (the Theta'
// flux is theta (rho v), taken in difference form)
__device__ __forceinline__ void df_flux_y(const df* __restrict__ q, const df* __restrict__ W,
                                          long long np, long long I, df (&f)[5]) {
  const df mu = q[np + I], mv = q[2 * np + I], mw = q[3 * np + I];
  const df v = W[I], pp = W[2 * np + I];
  f[0] = mv;
  f[1] = df_mul(mu, v);
  f[2] = df_add(df_mul(mv, v), pp);
  f[3] = df_mul(mw, v);
  f[4] = W[3 * np + I];
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
      df_flux_y(q, W, np, nodeI(sp * N + l), f);
#pragma unroll
      for (int c = 0; c < 5; ++c) fl[c][l] = f[c];
    }
    df dm[N], dF[N];
    df_seg_diffs<N>(fl[0], fl[4], dm, dF);
    carry[0] = df_drow<N, 1>(P, N, dm);
    carry[4] = df_drow<N, 1>(P, N, dF);
#pragma unroll
    for (int c = 1; c < 4; ++c) carry[c] = df_row<N, 1>(P, N, fl[c]);
  }

  df fc[5][N + 1];
  {
    df f[5];
    df_flux_y(q, W, np, nodeI(s0 * N), f);
#pragma unroll
    for (int c = 0; c < 5; ++c) fc[c][0] = f[c];
  }
  for (int s = s0; s < s1; ++s) {
#pragma unroll
    for (int l = 1; l <= N; ++l) {
      df f[5];
      df_flux_y(q, W, np, nodeI(s * N + l), f);
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
    df dm[N], dF[N];
    df_seg_diffs<N>(fc[0], fc[4], dm, dF);
    // row a of variable c seeded with start: rho' and Theta' in difference form
    auto rowc = [&](int c, int a, df start) -> df {
      if (c == 0) return df_drow_from<N, 1>(P, a, dm, start);
      if (c == 4) return df_drow_from<N, 1>(P, a, dF, start);
      return df_row_from<N, 1>(P, a, fc[c], start);
    };
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      df t0 = tv[c][0];
      if (!has_left && !P.open_y[0]) t0 = rowc(c, 0, t0);   // wall: the row counts twice
      t0 = rowc(c, 0, t0);
      T[c * np + nodeI(s * N)] = has_left ? df_add(t0, carry[c]) : t0;
#pragma unroll
      for (int a = 1; a < N; ++a) T[c * np + nodeI(s * N + a)] = rowc(c, a, tv[c][a]);
      carry[c] = c == 0 ? df_drow<N, 1>(P, N, dm)
                        : (c == 4 ? df_drow<N, 1>(P, N, dF) : df_row<N, 1>(P, N, fc[c]));
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) fc[c][0] = fc[c][N];
    has_left = true;
  }
  if (!P.per[1] && s1 == nseg) {
    const long long I = nodeI(nseg * N);
    if (P.open_y[1]) {   // partition face: the row goes to the neighbour
      const long long Fo = x + (long long)nx * z;
#pragma unroll
      for (int c = 0; c < 5; ++c) B.face_hi[c * (long long)nx * nz + Fo] = carry[c];
    } else {
#pragma unroll
      for (int c = 0; c < 5; ++c) T[c * np + I] = df_add(T[c * np + I], df_scale2(carry[c], 2.0f));
    }
  }
}

// ---------------------------------------------------------------- z lines + sources + stage

// FP64 <-> double-float conversion of n values (data entering or leaving).
__global__ void k_to_df(const double* __restrict__ in, df* __restrict__ out, long long n);
__global__ void k_from_df(const df* __restrict__ in, double* __restrict__ out, long long n);

}  // namespace xg

namespace xg {

// ---------------------------------------------------------------- z lines, tiled
// (The template also covers y lines; the marching k_df_line_y measured faster
// there, so only DIR = 2 is launched.)
// One CTA per (32 x-columns) x (a chunk of K element segments along the line
// direction DIR: 1 = y, 2 = z) x (the remaining coordinate), one thread per
// node: block (32, K N + 1), warp = one plane of 32 columns, so every warp
// does the same kind of work.  All loads of the chunk are issued up front
// (high memory-level parallelism), the fluxes along DIR go to shared memory
// -- the chunk's K N + 1 planes plus the N planes of the segment before it
// (whose last row completes the chunk's first face node) -- and each thread
// then assembles its own node: y adds its part into T, z adds its part,
// the sources, walls and the stage store.  Thread row K N handles the
// chunk's end face: its fluxes close the last segment, and at a wall it
// also owns the wall node.
// Fluxes along DIR at one node from loaded values: qv = (rho', rho u,
// rho v, rho w, Theta'), vel = v (DIR 1) or w (DIR 2), pp = p'.
// Slot 4 holds theta = Theta / rho: the Theta' flux theta (rho u_DIR) is
// taken in difference form with slot 0.
template <int DIR>
__device__ __forceinline__ void df_flux_vals(const df (&qv)[5], df vel, df pp, df th, df (&f)[5]) {
  f[0] = qv[DIR + 1];
  f[1] = DIR == 1 ? df_mul(qv[1], vel) : df_mul(qv[1], vel);
  f[2] = DIR == 1 ? df_add(df_mul(qv[2], vel), pp) : df_mul(qv[2], vel);
  f[3] = DIR == 1 ? df_mul(qv[3], vel) : df_add(df_mul(qv[3], vel), pp);
  f[4] = th;
}

// Sources, walls and the stage store of one node from loaded values.
__device__ __forceinline__ void df_finish_vals(const DfParams& P, const DfBufs& B,
                                               const df (&qv)[5], const df (&qnv)[5], df sv,
                                               df rho0, df* __restrict__ out, long long I, int x,
                                               int y, int gz, df (&L)[5], bool& bad) {
  const long long np = P.np;
  dacc A = dacc_from(L[1]);
  dacc_fma(A, P.f, qv[2]);                       // +f rho v
  L[1] = dacc_value(A);
  A = dacc_from(L[2]);
  dacc_fma(A, df_neg(P.f), qv[1]);               // -f rho u
  L[2] = dacc_value(A);
  A = dacc_from(L[3]);
  dacc_fma(A, df_neg(P.g), qv[0]);               // -rho' g
  L[3] = dacc_value(A);
  if (B.S) {
    A = dacc_from(L[4]);
    dacc_fma(A, df_add(rho0, qv[0]), sv);        // rho S_theta
    L[4] = dacc_value(A);
  }
  const df zero = {0.0f, 0.0f};
  if (!P.per[0] && (x == 0 || x == P.n[0] - 1)) L[1] = zero;
  if (!P.per[1] && ((y == 0 && !P.open_y[0]) || (y == P.n[1] - 1 && !P.open_y[1]))) L[2] = zero;
  if (!P.per[2] && (gz == 0 || gz == P.n[2] - 1)) L[3] = zero;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    df o;
    if (B.rhs_only) {
      o = L[c];
    } else if (B.alpha.h == 0.0f) {
      dacc R = dacc_from(qv[c]);
      dacc_fma(R, B.dt, L[c]);
      o = dacc_value(R);
    } else {
      dacc R = dacc_prod(B.alpha, qnv[c]);
      dacc_fma(R, B.beta, qv[c]);
      dacc_fma(R, B.bdt, L[c]);
      o = dacc_value(R);
    }
    out[c * np + I] = o;
    bad |= df_nonfinite(o);
  }
}

constexpr int kTileCols = 32;

__host__ __device__ constexpr int tile_segments(int N) { return N >= 16 ? 1 : 16 / N; }
// The double-float z tiles hold half as many segments (at most 9 planes):
// 3 CTAs of 288 threads fit an SM without spills (measured: 0.76 vs 0.84 ms
// per launch on the 128x128x16 order-4 box against 16-plane tiles).
__host__ __device__ constexpr int df_tile_segments(int N) { return N >= 8 ? 1 : 8 / N; }

template <int N, int DIR>
__global__ void __launch_bounds__(kTileCols * (8 + 1), 3) k_df_tline(const DfParams P, const DfBufs B) {
  constexpr int K = df_tile_segments(N);
  constexpr int NS = K * N + N + 1;            // flux slots: N halo planes + K N + 1
  __shared__ df Fs[5][NS][kTileCols];
  // rho' and Theta' flux differences of slot j against its segment's first
  // slot (difference form); slot j >= 1 lies in the segment that starts at
  // slot N floor((j - 1) / N), of which it is an interior node or the end
  __shared__ df Ds[2][NS][kTileCols];
  const int nx = P.n[0], ny = P.n[1];
  const int nd = P.n[DIR];                      // nodes along the line
  const int nseg = P.nseg[DIR];
  const bool per = P.per[DIR] != 0;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = blockIdx.x * kTileCols + tx;
  const bool xin = x < nx;
  const int s0 = blockIdx.y * K;
  const int kc = min(K, nseg - s0);             // segments in this chunk
  const int other = blockIdx.z;                  // z for y-lines, y for z-lines
  const long long np = P.np;
  const long long sd = DIR == 1 ? (long long)nx : (long long)nx * ny;
  const long long base = DIR == 1 ? x + (long long)nx * ny * other : x + (long long)nx * other;
  const bool has_left = s0 > 0 || per;
  auto plane = [&](int g) -> int { return g >= nd ? g - nd : (g < 0 ? g + nd : g); };
  const int vslot = DIR == 1 ? 0 : 1;            // v or w in W

  // the node this thread owns: planes s0 N + ty for ty < kc N, and the end
  // wall plane for the extra row of the last chunk of a walled line
  const int own = s0 * N + ty;
  const bool owns = xin && (ty < kc * N || (ty == kc * N && s0 + kc == nseg && !per));
  const bool main_plane = xin && ty <= kc * N;   // the extra row fills the end face
  const bool halo = xin && has_left && ty < N;   // the N planes before the chunk
  const int g = plane(own);
  const int gh = plane((s0 - 1) * N + ty);
  const long long I = base + sd * (main_plane ? g : 0);
  const long long Ih = base + sd * (halo ? gh : 0);
  // every global load of the thread first: one memory round trip
  df qv[5], vel, pp, th, hq[5], hvel, hpp, hth, t[5], qnv[5], sv = {0.0f, 0.0f};
  hq[0] = sv;
  if (main_plane) {
#pragma unroll
    for (int c = 0; c < 5; ++c) qv[c] = B.q[c * np + I];
    vel = B.W[vslot * np + I];
    pp = B.W[2 * np + I];
    th = B.W[3 * np + I];
  }
  if (halo) {
#pragma unroll
    for (int c = 1; c < 5; ++c) hq[c] = B.q[c * np + Ih];
    hvel = B.W[vslot * np + Ih];
    hpp = B.W[2 * np + Ih];
    hth = B.W[3 * np + Ih];
  }
  if (owns) {
#pragma unroll
    for (int c = 0; c < 5; ++c) t[c] = B.T[c * np + I];
    if (DIR == 2) {
      if (!B.rhs_only && B.alpha.h != 0.0f) {
#pragma unroll
        for (int c = 0; c < 5; ++c) qnv[c] = B.qn[c * np + I];
      }
      if (B.S) sv = B.S[I];
    }
  }
  if (main_plane) {
    df f[5];
    df_flux_vals<DIR>(qv, vel, pp, th, f);
#pragma unroll
    for (int c = 0; c < 5; ++c) Fs[c][N + ty][tx] = f[c];
  }
  if (halo) {
    df f[5];
    df_flux_vals<DIR>(hq, hvel, hpp, hth, f);
#pragma unroll
    for (int c = 0; c < 5; ++c) Fs[c][ty][tx] = f[c];
  }
  __syncthreads();

  // difference form of the rho' and Theta' fluxes, slot by slot
  auto diff_slot = [&](int j) {
    const int b = N * ((j - 1) / N);
    const df mj = Fs[0][j][tx], mb = Fs[0][b][tx];
    const df thj = Fs[4][j][tx], thb = Fs[4][b][tx];
    const df dm = df_sub(mj, mb);
    Ds[0][j][tx] = dm;
    Ds[1][j][tx] = df_add_nc(df_mul(thj, dm), df_mul(df_sub(thj, thb), mb));
  };
  if (main_plane && (ty > 0 || has_left)) diff_slot(N + ty);   // slot N closes the halo segment
  if (halo && ty > 0) diff_slot(ty);
  __syncthreads();
  if (!owns) return;

  // the node's segment k and local index a; the wall node is row N of the last
  const int k = ty < kc * N ? ty / N : kc - 1;
  const int a = ty < kc * N ? ty - k * N : N;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    if (c == 0 || c == 4) {
      const int e = c == 0 ? 0 : 1;
      df d[N];
#pragma unroll
      for (int l = 1; l <= N; ++l) d[l - 1] = Ds[e][N + k * N + l][tx];
      if (a == N) {                                 // wall node: its one-sided row counts twice
        const df r = df_drow<N, DIR>(P, N, d);
        t[c] = df_add(t[c], df_scale2(r, 2.0f));
      } else if (a > 0) {
        t[c] = df_drow_from<N, DIR>(P, a, d, t[c]);
      } else {
        // a face: both one-sided rows in one compensated sum (the segment
        // before, or the same row twice at the wall at the line start)
        df dl[N];
        const bool left = k > 0 || has_left;
#pragma unroll
        for (int l = 1; l <= N; ++l) dl[l - 1] = left ? Ds[e][k * N + l][tx] : d[l - 1];
        dacc A = dacc_from(t[c]);
#pragma unroll
        for (int l = 1; l <= N; ++l) dacc_fma(A, P.Dm[DIR][0][l], d[l - 1]);
#pragma unroll
        for (int l = 1; l <= N; ++l) dacc_fma(A, P.Dm[DIR][left ? N : 0][l], dl[l - 1]);
        t[c] = dacc_value(A);
      }
      continue;
    }
    df f[N + 1];
#pragma unroll
    for (int l = 0; l <= N; ++l) f[l] = Fs[c][N + k * N + l][tx];
    if (a == N) {                                   // wall node: its one-sided row counts twice
      const df r = df_row<N, DIR>(P, N, f);
      t[c] = df_add(t[c], df_scale2(r, 2.0f));
    } else if (a > 0) {
      t[c] = df_row_from<N, DIR>(P, a, f, t[c]);
    } else if (k > 0 || has_left) {                 // shared face: both one-sided halves
      df fl[N + 1];
#pragma unroll
      for (int l = 0; l <= N; ++l) fl[l] = Fs[c][k * N + l][tx];
      t[c] = df_row_from<N, DIR>(P, 0, f, t[c]);
      t[c] = df_add(t[c], df_row<N, DIR>(P, N, fl));
    } else {                                        // wall at the line start
      t[c] = df_row_from<N, DIR>(P, 0, f, t[c]);
      t[c] = df_row_from<N, DIR>(P, 0, f, t[c]);
    }
  }
  if (DIR == 1) {
#pragma unroll
    for (int c = 0; c < 5; ++c) B.T[c * np + I] = t[c];
  } else {
    bool bad = false;
    df_finish_vals(P, B, qv, qnv, sv, B.base[g], B.out, I, x, other, g, t, bad);
    if (bad) *B.flag = 1;
  }
}

}  // namespace xg
