// xg_kernels_df.cuh -- the FP64-accurate fast path (XG_DF64): the line
// kernels of xg_kernels.cuh with the work split between the FP64 and the
// FP32 pipes.
//
// GB300 runs 2 FP64 FMAs per clock per SM against 128 FP32 FMAs.  The state
// stays in FP64 (every [5][Np] array holds doubles, the ABI's own format), and
// each equation is computed in the arithmetic its conditioning needs:
//   * rho' and Theta' (Eq. 1a, 1c) -- their tendencies are residuals of
//     cancelling flux derivatives where the flow is nearly non-divergent, so
//     their whole path is native FP64: theta = Theta/rho, the fluxes' segment
//     differences (difference form, xg_kernels.cuh), the contractions, the
//     face sums, the partial tendency T, the heating source and the stage
//     update.  These are the only FP64 instructions of the stage (~60 per
//     node), which bound it.
//   * the momentum (Eq. 1b) -- its tendency does not cancel; primitives,
//     the equation of state, fluxes, contractions (compensated Dot2), face
//     sums, Coriolis and gravity and the stage update run in double-float
//     arithmetic (xg_df.cuh, unit roundoff 2^-48) on the FP32 pipes, from the
//     FP64 state split into float pairs with integer operations only (FP64
//     conversions run at the FP64 rate), and the results are widened back
//     to FP64 for storage.
// The partial tendency T holds doubles for rho' and Theta' and double-float
// pairs for the momentum (8 bytes each); W holds v, w, p' as pairs and theta
// as a double.
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
  LineParams P64;  // the FP64 constants of the rho' and Theta' path
};

struct DfBufs {
  const double* q;
  const double* qn;
  double* out;
  df* W;            // [3][np] v, w, p' (pairs); theta follows as doubles (W64)
  double* W64;      // [np] theta = Theta / rho
  double* T;        // [5][np]: slots 0 and 4 doubles, slots 1..3 pairs (Tm)
  df* Tm;           // the same array seen as pairs
  const double* S;  // [np] heating or null
  const df* base;   // [4][nz] rho0, Theta0, p0, 1/Theta0 as pairs
  const double* base64;  // the same table in FP64
  int* flag;
  df dt, alpha, beta, bdt;      // momentum stage coefficients (bdt = beta dt)
  double dt64, alpha64, beta64; // rho' and Theta' stage coefficients
  int rhs_only;
  double* face_hi;  // [5][n_z][n_x] row N at an open y end (slot types as T)
  // [5][nseg_y][n_z][n_x] row N of the y segment that ends at each y face,
  // written by the y pass and added by the z pass (slot types as T)
  double* Fy;
};

// ---------------------------------------------------------------- FP64 <-> pairs
// x = h + l with h the leading 24 significand bits of x (truncated) and l the
// next ones rounded to a float, then renormalised (|l| <= ulp(h)/2): unit
// roundoff 2^-48, integer and FP32 operations only.  |x| < 2^-100 gives 0 (far
// below any state value's significance); |x| >= 2^128 gives +-inf, so a
// non-finite value stays non-finite.
__device__ __forceinline__ df df_of_double(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned sign = hi & 0x80000000u;
  if (e < 1023 - 100) return {__uint_as_float(sign), 0.0f};
  if (e > 1023 + 127) return {__uint_as_float(sign | 0x7f800000u), 0.0f};
  const unsigned top = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const float h = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | top);
  float l = 0.0f;
  if (e >= 949) {   // the remainder's scale 2^(e - 1075) is a normal float
    l = __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), __uint_as_float((unsigned)(e - 948) << 23));
    if (sign) l = -l;
  }
  float s, t;
  fast_two_sum(h, l, s, t);
  return {s, t};
}

// A float widened to a double exactly, with integer operations (subnormal
// floats, below 2^-126, give 0; inf/nan stay non-finite).
__device__ __forceinline__ double dbl_of_float(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xffu;
  if (ef == 0) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (ef == 255) return __hiloint2double((int)((u & 0x80000000u) | 0x7ff00000u | ((u >> 3) & 0xfffffu)), 0);
  const unsigned hi = (u & 0x80000000u) | ((ef + 896u) << 20) | ((u >> 3) & 0xfffffu);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// h + l as an FP64 value, with integer operations only (no FP64 add): h's
// 24-bit significand becomes the top of a 53-bit one and l's is added or
// subtracted at its place, truncated below the last bit (an error below one
// unit in the last place of the double, far below the pair's own 2^-48).
// Expects a normalised pair (|l| <= ulp(h)/2, as every double-float
// operation returns).
__device__ __forceinline__ double dbl_of_df(df a) {
  const unsigned uh = __float_as_uint(a.h), ul = __float_as_uint(a.l);
  const int eh = (int)((uh >> 23) & 0xffu), el = (int)((ul >> 23) & 0xffu);
  if (eh == 0 || eh == 255 || el == 0) return dbl_of_float(a.h);
  unsigned long long M = (unsigned long long)((uh & 0x7fffffu) | 0x800000u) << 29;
  const unsigned long long ml = (unsigned long long)((ul & 0x7fffffu) | 0x800000u);
  const int d = eh - el;                      // >= 24 for a normalised pair
  const unsigned long long L = d >= 29 ? (d - 29 < 64 ? ml >> (d - 29) : 0ull) : ml << (29 - d);
  int e = eh;
  if ((uh ^ ul) & 0x80000000u) {
    M -= L;
    if (M < (1ull << 52)) { M <<= 1; --e; }
  } else {
    M += L;
    if (M >= (1ull << 53)) { M >>= 1; ++e; }
  }
  const unsigned long long bits = ((unsigned long long)(uh & 0x80000000u) << 32) |
                                  ((unsigned long long)(e + 896) << 52) | (M & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

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
// Orders up to 4 at 8 CTAs per SM (64 registers): 0.691 against 0.722 ms per
// launch with no bound (71 registers, 7 CTAs) and 0.706 at 10 (spilling), on
// the 128 x 128 x 16 order-4 box; higher orders would spill at 8
__host__ __device__ constexpr int df_x_min_blocks(int N) { return N <= 4 ? 8 : 1; }
template <int N>
__global__ void __launch_bounds__(kXThreads, df_x_min_blocks(N)) k_df_line_x(const DfParams P, const DfBufs B) {
  extern __shared__ df smd[];
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const int nseg = P.nseg[0];
  const int y = blockIdx.x, z = blockIdx.y;
  const long long np = P.np;
  const long long row = (long long)nx * (y + (long long)ny * z);
  const int ld = nx + 1;
  // [5][ld] fluxes (slots 0 and 4 doubles: rho u and theta; 1..3 pairs), later
  // rows 0..N-1 of every segment in place; RN [5][nseg] row N (same types)
  df* F = smd;
  double* F64 = reinterpret_cast<double*>(smd);
  df* RN = smd + 5 * ld;
  double* RN64 = reinterpret_cast<double*>(RN);
  const df p0 = B.base[2 * nz + z], iTh0 = B.base[3 * nz + z];
  const double rho0 = B.base64[z], Th0 = B.base64[nz + z];
  const double* __restrict__ q = B.q;

  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const long long I = row + i;
    const double rp = q[I], mu = q[np + I], mv = q[2 * np + I], mw = q[3 * np + I];
    const double tp = q[4 * np + I];
    // theta = Theta / rho in FP64 from a double-float estimate and one Newton
    // correction (t1 = t0 + (Theta - t0 rho) / rho: the estimate's 2^-47
    // error squares away, leaving FP64 rounding), 2 FP64 adds and 2 FMAs
    const double rho = rho0 + rp, Th = Th0 + tp;
    const df ir = df_rcp(df_of_double(rho));
    const double t0 = dbl_of_df(df_mul(df_of_double(Th), ir));
    const double th = fma(fma(-t0, rho, Th), dbl_of_df(ir), t0);
    const df muD = df_of_double(mu), mvD = df_of_double(mv), mwD = df_of_double(mw);
    const df u = df_mul(muD, ir), v = df_mul(mvD, ir), w = df_mul(mwD, ir);
    const df pp = df_mul(p0, df_eos_phi(P, df_mul(df_of_double(tp), iTh0)));
    B.W[I] = v;
    B.W[np + I] = w;
    B.W[2 * np + I] = pp;
    B.W64[I] = th;
    F64[i] = mu;
    F[ld + i] = df_add(df_mul(muD, u), pp);
    F[2 * ld + i] = df_mul(mvD, u);
    F[3 * ld + i] = df_mul(mwD, u);
    F64[4 * ld + i] = th;                 // the Theta' flux is theta (rho u)
    if (P.per[0] && i == 0) {
      F64[nx] = mu;
#pragma unroll
      for (int c = 1; c < 4; ++c) F[c * ld + nx] = F[c * ld];
      F64[4 * ld + nx] = th;
    }
  }
  __syncthreads();

  for (int s0 = 0; s0 < nseg; s0 += blockDim.x) {
    const int s = s0 + threadIdx.x;
    double r64[2][N + 1];
    df rows[3][N + 1];
    if (s < nseg) {
      {   // rho' and Theta': FP64, difference form
        double m[N + 1], th[N + 1], dm[N + 1], dF[N + 1];
#pragma unroll
        for (int l = 0; l <= N; ++l) {
          m[l] = F64[s * N + l];
          th[l] = F64[4 * ld + s * N + l];
        }
        seg_diffs<N>(m, th, dm, dF);
        contract_eo<N, 0>(P.P64, dm, r64[0]);
        contract_eo<N, 0>(P.P64, dF, r64[1]);
      }
#pragma unroll
      for (int c = 1; c < 4; ++c) {
        df f[N + 1];
#pragma unroll
        for (int l = 0; l <= N; ++l) f[l] = F[c * ld + s * N + l];
#pragma unroll
        for (int a = 0; a <= N; ++a) rows[c - 1][a] = df_row<N, 0>(P, a, f);
      }
    }
    __syncthreads();
    if (s < nseg) {
#pragma unroll
      for (int a = 0; a < N; ++a) {
        F64[s * N + a] = r64[0][a];
        F64[4 * ld + s * N + a] = r64[1][a];
      }
      RN64[s] = r64[0][N];
      RN64[4 * nseg + s] = r64[1][N];
#pragma unroll
      for (int c = 1; c < 4; ++c) {
#pragma unroll
        for (int a = 0; a < N; ++a) F[c * ld + s * N + a] = rows[c - 1][a];
        RN[c * nseg + s] = rows[c - 1][N];
      }
    }
    __syncthreads();
  }

  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const int s = i / N, a = i - s * N;
    const long long I = row + i;
    const int left = s > 0 ? s - 1 : (P.per[0] ? nseg - 1 : -1);
#pragma unroll
    for (int c = 0; c < 5; c += 4) {
      double v;
      if (s == nseg) {
        v = RN64[c * nseg + nseg - 1];
        v = v + v;
      } else if (a != 0) {
        v = F64[c * ld + i];
      } else {
        const double r0 = F64[c * ld + i];
        v = r0 + (left >= 0 ? RN64[c * nseg + left] : r0);
      }
      B.T[c * np + I] = v;
    }
#pragma unroll
    for (int c = 1; c < 4; ++c) {
      df v;
      if (s == nseg) {
        v = df_scale2(RN[c * nseg + nseg - 1], 2.0f);
      } else if (a != 0) {
        v = F[c * ld + i];
      } else {
        const df r0 = F[c * ld + i];
        v = left >= 0 ? df_add(r0, RN[c * nseg + left]) : df_scale2(r0, 2.0f);
      }
      B.Tm[c * np + I] = v;
    }
  }
}

// ---------------------------------------------------------------- z lines + sources + stage

// Momentum fluxes along DIR (1 = y, 2 = z) at one node from its momentum as
// pairs, vel = v or w and pp = p'.
template <int DIR>
__device__ __forceinline__ void df_flux_mom(const df (&m)[3], df vel, df pp, df (&f)[3]) {
  f[0] = df_mul(m[0], vel);
  f[1] = DIR == 1 ? df_add(df_mul(m[1], vel), pp) : df_mul(m[1], vel);
  f[2] = DIR == 1 ? df_mul(m[2], vel) : df_add(df_mul(m[2], vel), pp);
}

// Sources, walls and the stage store of one node: L64 = the rho' and Theta'
// tendencies (FP64), Lm = the momentum tendencies (pairs); qv the node's
// FP64 state, qm its momentum as pairs, qnv the FP64 q^n (stages 2-3).
__device__ __forceinline__ void df_finish(const DfParams& P, const DfBufs& B, const double (&qv)[5],
                                          const df (&qm)[3], const double (&qnv)[5], double sv,
                                          double rho0, double* __restrict__ out, long long I, int x,
                                          int y, int gz, double (&L64)[2], df (&Lm)[3], bool& bad) {
  const long long np = P.np;
  dacc A = dacc_from(Lm[0]);
  dacc_fma(A, P.f, qm[1]);                       // +f rho v
  Lm[0] = dacc_value(A);
  A = dacc_from(Lm[1]);
  dacc_fma(A, df_neg(P.f), qm[0]);               // -f rho u
  Lm[1] = dacc_value(A);
  A = dacc_from(Lm[2]);
  dacc_fma(A, df_neg(P.g), df_of_double(qv[0])); // -rho' g
  Lm[2] = dacc_value(A);
  if (B.S) L64[1] = fma(rho0 + qv[0], sv, L64[1]);   // rho S_theta
  const df zero = {0.0f, 0.0f};
  if (!P.per[0] && (x == 0 || x == P.n[0] - 1)) Lm[0] = zero;
  if (!P.per[1] && ((y == 0 && !P.open_y[0]) || (y == P.n[1] - 1 && !P.open_y[1]))) Lm[1] = zero;
  if (!P.per[2] && (gz == 0 || gz == P.n[2] - 1)) Lm[2] = zero;
  const bool stage1 = B.alpha64 == 0.0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int c = e == 0 ? 0 : 4;
    double o;
    if (B.rhs_only) o = L64[e];
    else if (stage1) o = fma(B.dt64, L64[e], qv[c]);
    else o = fma(B.alpha64, qnv[c], B.beta64 * fma(B.dt64, L64[e], qv[c]));
    out[c * np + I] = o;
    bad |= is_nonfinite(o);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    df o;
    if (B.rhs_only) {
      o = Lm[c];
    } else if (stage1) {
      dacc R = dacc_from(qm[c]);
      dacc_fma(R, B.dt, Lm[c]);
      o = dacc_value(R);
    } else {
      dacc R = dacc_prod(B.alpha, df_of_double(qnv[c + 1]));
      dacc_fma(R, B.beta, qm[c]);
      dacc_fma(R, B.bdt, Lm[c]);
      o = dacc_value(R);
    }
    bad |= df_nonfinite(o);
    out[(c + 1) * np + I] = dbl_of_df(o);
  }
}

constexpr int kTileCols = 32;

__host__ __device__ constexpr int tile_segments(int N) { return N >= 16 ? 1 : 16 / N; }
// Segments per tile and launch bounds of the y (DIR = 1) and z (DIR = 2)
// tile kernels.  A sweep on the 128 x 128 x 16 order-4 box: y tiles of one
// segment (160 threads) at 8 CTAs per SM (48 registers) took 0.692 ms per
// launch, against 0.853 with two segments at 3 CTAs and 0.748 at 4; z tiles
// of two segments at 4 CTAs per SM (56 registers) 1.054 ms, against 1.100 at
// 3, 1.106 at 5 and 1.096 with one segment at 6.  Other orders keep about the
// same threads per SM.
__host__ __device__ constexpr int df_tile_segments(int N, int DIR) {
  return DIR == 1 ? (N >= 4 ? 1 : 4 / N) : (N >= 8 ? 1 : 8 / N);
}
__host__ __device__ constexpr int df_tile_threads(int N, int DIR) {
  return kTileCols * (df_tile_segments(N, DIR) * N + 1);
}
__host__ __device__ constexpr int df_tile_min_blocks(int N, int DIR) {
  return (DIR == 1 ? 1280 : 1152) / df_tile_threads(N, DIR) > 1
             ? (DIR == 1 ? 1280 : 1152) / df_tile_threads(N, DIR) : 1;
}

// ---------------------------------------------------------------- y and z lines, tiled
// One CTA per (32 x-columns) x (a chunk of K element segments along DIR) x
// the remaining coordinate, one thread per node: block (32, K N + 1), warp =
// one plane of 32 columns.  All loads of the chunk are issued up front, the
// fluxes go to shared memory -- the chunk's K N + 1 planes plus the N planes
// of the segment before it (whose last row completes the chunk's first face
// node) -- and each thread then assembles its own node: DIR = 1 adds the y
// part into T, DIR = 2 the z part, the sources, walls and the stage store.
// Thread row K N handles the chunk's end face: its fluxes close the last
// segment, and at a wall it also owns the wall node.  y tiles (DIR = 1)
// load no halo: the end-face thread of a y tile writes its last segment's
// row N to Fy, and the z pass adds it to the next tile's first node (t0 +
// row N, the same two operands as a tile that loads the halo).  This saves
// the halo's FP64 differences (y: 0.692 -> 0.546 ms per launch on the
// 128 x 128 x 16 order-4 box, z: 1.054 -> 1.135 for the extra reads).  A shared face node
// takes its two one-sided rows as t0 + row N (t0: the running tendency plus
// row 0), the order a partition face is completed in (xg_partition_stage),
// so partitioned runs match single domains bit for bit.  At a partition face
// (open_y, DIR = 1) the slab's first node takes row 0 once, and the end node
// hands its one-sided row N to face_hi instead of doubling it.
template <int N, int DIR>
__global__ void __launch_bounds__(df_tile_threads(N, DIR), df_tile_min_blocks(N, DIR))
    k_df_tline(const DfParams P, const DfBufs B) {
  constexpr int K = df_tile_segments(N, DIR);
  // z tiles load the N planes of the segment before them; y tiles load none:
  // the row N of that segment at a y tile's first node is written to Fy by
  // the tile it belongs to and added by the z pass (t0 + row N, as above)
  constexpr int H = DIR == 1 ? 0 : N;
  constexpr int NS = K * N + H + 1;            // flux slots: H halo planes + K N + 1
  __shared__ df Fm[3][NS][kTileCols];          // momentum fluxes (pairs)
  __shared__ double Fs[2][NS][kTileCols];      // rho u_DIR and theta
  // rho' and Theta' flux differences of slot j against its segment's first
  // slot (difference form); slot j >= 1 lies in the segment that starts at
  // slot N floor((j - 1) / N), of which it is an interior node or the end
  __shared__ double Ds[2][NS][kTileCols];
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
  const LineParams& P64 = P.P64;

  const bool open_lo = DIR == 1 && P.open_y[0], open_hi = DIR == 1 && P.open_y[1];
  const int own = s0 * N + ty;
  const bool owns = xin && (ty < kc * N || (ty == kc * N && s0 + kc == nseg && !per));
  const bool main_plane = xin && ty <= kc * N;   // the extra row fills the end face
  const bool halo = H > 0 && xin && has_left && ty < N;   // the N planes before the chunk
  const int g = plane(own);
  const int gh = plane((s0 - 1) * N + ty);
  const long long I = base + sd * (main_plane ? g : 0);
  const long long Ih = base + sd * (halo ? gh : 0);

  // the global loads the fluxes and rows need first (one memory round trip);
  // q^n and S, needed only by the stage at the end, are loaded there: kept
  // live across the rows they spilled 56 bytes per thread, and z launches
  // took 1.136 ms against 0.980 (128 x 128 x 16 order-4 box)
  double qv[5], hq[3], th = 0.0, hth = 0.0, t64[2], qnv[5], sv = 0.0;
  df vel, pp, hvel, hpp, tm[3];
  if (main_plane) {
#pragma unroll
    for (int c = 0; c < 5; ++c) qv[c] = B.q[c * np + I];
    vel = B.W[vslot * np + I];
    pp = B.W[2 * np + I];
    th = B.W64[I];
  }
  if (halo) {
#pragma unroll
    for (int c = 0; c < 3; ++c) hq[c] = B.q[(c + 1) * np + Ih];
    hvel = B.W[vslot * np + Ih];
    hpp = B.W[2 * np + Ih];
    hth = B.W64[Ih];
  }
  if (owns) {
    t64[0] = B.T[I];
    t64[1] = B.T[4 * np + I];
#pragma unroll
    for (int c = 0; c < 3; ++c) tm[c] = B.Tm[(c + 1) * np + I];
  }
  df qm[3];
  if (main_plane) {
#pragma unroll
    for (int c = 0; c < 3; ++c) qm[c] = df_of_double(qv[c + 1]);
    df f[3];
    df_flux_mom<DIR>(qm, vel, pp, f);
#pragma unroll
    for (int c = 0; c < 3; ++c) Fm[c][H + ty][tx] = f[c];
    Fs[0][H + ty][tx] = qv[DIR + 1];
    Fs[1][H + ty][tx] = th;
  }
  if (halo) {
    df hm[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) hm[c] = df_of_double(hq[c]);
    df f[3];
    df_flux_mom<DIR>(hm, hvel, hpp, f);
#pragma unroll
    for (int c = 0; c < 3; ++c) Fm[c][ty][tx] = f[c];
    Fs[0][ty][tx] = hq[DIR];
    Fs[1][ty][tx] = hth;
  }
  __syncthreads();

  // difference form of the rho' and Theta' fluxes, slot by slot (FP64)
  auto diff_slot = [&](int j) {
    const int b = N * ((j - 1) / N);
    const double mb = Fs[0][b][tx], thb = Fs[1][b][tx], thj = Fs[1][j][tx];
    const double dm = Fs[0][j][tx] - mb;
    Ds[0][j][tx] = dm;
    Ds[1][j][tx] = fma(thj, dm, (thj - thb) * mb);
  };
  if (main_plane && (ty > 0 || (H > 0 && has_left))) diff_slot(H + ty);   // slot N closes the halo
  if (halo && ty > 0) diff_slot(ty);
  __syncthreads();
  const long long nfy = (long long)P.nseg[1] * P.n[2] * P.n[0];   // one variable of Fy
  if (DIR == 1 && xin && ty == kc * N && !owns && B.Fy) {
    // the end face, owned by the next tile (or, periodic, the first): row N
    // of this tile's last segment for it
    const long long Io = ((s0 + kc) % nseg) * (long long)P.n[2] * P.n[0] + (long long)P.n[0] * other + x;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      double d[N + 1];
      d[0] = -0.0;
#pragma unroll
      for (int l = 1; l <= N; ++l) d[l] = Ds[e][H + (kc - 1) * N + l][tx];
      B.Fy[(e == 0 ? 0 : 4) * nfy + Io] = drow_N<N, DIR>(P64, d);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      df f[N + 1];
#pragma unroll
      for (int l = 0; l <= N; ++l) f[l] = Fm[c][H + (kc - 1) * N + l][tx];
      reinterpret_cast<df*>(B.Fy)[(c + 1) * nfy + Io] = df_row<N, DIR>(P, N, f);
    }
  }
  if (!owns) return;
  if (DIR == 2 && B.Fy) {   // the first node of a y tile: t0 + row N of the tile before
    constexpr int KY = df_tile_segments(N, 1);
    if (other % (KY * N) == 0 && (P.per[1] || (other > 0 && other < ny - 1))) {
      const long long If = (other / N) * (long long)P.n[2] * P.n[0] + (long long)P.n[0] * g + x;
      t64[0] = t64[0] + B.Fy[If];
      t64[1] = t64[1] + B.Fy[4 * nfy + If];
#pragma unroll
      for (int c = 0; c < 3; ++c) tm[c] = df_add(tm[c], reinterpret_cast<const df*>(B.Fy)[(c + 1) * nfy + If]);
    }
  }

  // the node's segment k and local index a; the wall node is row N of the last
  const int k = ty < kc * N ? ty / N : kc - 1;
  const int a = ty < kc * N ? ty - k * N : N;
  // the end node of an open slab end: its rows go to the neighbour
  const bool hand = open_hi && a == N;
  const long long Fo = x + (long long)P.n[0] * other, nf = (long long)P.n[0] * P.n[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    double d[N + 1];
    d[0] = -0.0;
#pragma unroll
    for (int l = 1; l <= N; ++l) d[l] = Ds[e][H + k * N + l][tx];
    double t = t64[e];
    if (a == N) {                                 // wall node: its one-sided row counts twice
      const double r = drow_N<N, DIR>(P64, d);
      if (hand) B.face_hi[(e == 0 ? 0 : 4) * nf + Fo] = r;
      t = t + (r + r);
    } else if (a > 0) {
      t = drow_from<N, DIR>(P64, a, d, t);
    } else if (DIR == 1 && k == 0 && has_left) {  // shared face: t0 here, row N via Fy
      t = drow_from<N, DIR>(P64, 0, d, t);
    } else if (k > 0 || has_left) {               // shared face: t0 + row N of the left
      double dl[N + 1];
      dl[0] = -0.0;
#pragma unroll
      for (int l = 1; l <= N; ++l) dl[l] = Ds[e][H + (k - 1) * N + l][tx];
      t = drow_from<N, DIR>(P64, 0, d, t) + drow_N<N, DIR>(P64, dl);
    } else {                                      // line start: a wall (twice) or open (once)
      if (!open_lo) t = drow_from<N, DIR>(P64, 0, d, t);
      t = drow_from<N, DIR>(P64, 0, d, t);
    }
    t64[e] = t;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    df f[N + 1];
#pragma unroll
    for (int l = 0; l <= N; ++l) f[l] = Fm[c][H + k * N + l][tx];
    if (a == N) {
      const df r = df_row<N, DIR>(P, N, f);
      if (hand) reinterpret_cast<df*>(B.face_hi)[(c + 1) * nf + Fo] = r;
      tm[c] = df_add(tm[c], df_scale2(r, 2.0f));
    } else if (a > 0) {
      tm[c] = df_row_from<N, DIR>(P, a, f, tm[c]);
    } else if (DIR == 1 && k == 0 && has_left) {
      tm[c] = df_row_from<N, DIR>(P, 0, f, tm[c]);
    } else if (k > 0 || has_left) {
      df fl[N + 1];
#pragma unroll
      for (int l = 0; l <= N; ++l) fl[l] = Fm[c][H + (k - 1) * N + l][tx];
      tm[c] = df_row_from<N, DIR>(P, 0, f, tm[c]);
      tm[c] = df_add(tm[c], df_row<N, DIR>(P, N, fl));
    } else {
      if (!open_lo) tm[c] = df_row_from<N, DIR>(P, 0, f, tm[c]);
      tm[c] = df_row_from<N, DIR>(P, 0, f, tm[c]);
    }
  }
  if (DIR == 1) {
    if (hand) return;                             // completed after the exchange
    B.T[I] = t64[0];
    B.T[4 * np + I] = t64[1];
#pragma unroll
    for (int c = 0; c < 3; ++c) B.Tm[(c + 1) * np + I] = tm[c];
  } else {
    if (!B.rhs_only && B.alpha64 != 0.0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) qnv[c] = B.qn[c * np + I];
    }
    if (B.S) sv = B.S[I];
    bool bad = false;
    df_finish(P, B, qv, qm, qnv, sv, B.base64[g], B.out, I, x, other, g, t64, tm, bad);
    if (bad) *B.flag = 1;
  }
}

}  // namespace xg
