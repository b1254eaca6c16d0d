// xg_kernels.cuh -- FP64 line kernels of the explicit CG Euler path (sm_103a).
//
// The right-hand side of Sec. 2.1 (Eq. 1 restated for q = (rho', rho u,
// rho v, rho w, Theta'), pressure from Eq. 3) is evaluated by the collocated
// strong form of Sec. 2.2 (Eqs. 7-8) with DSS (Eqs. 9-11, Alg. 3) and the
// inverse diagonal mass (Eq. 12).  On an axis-aligned box of equal elements
// the metric is the same constant diagonal in every element, and the mass
// is the tensor product M_I = J W_x(gx) W_y(gy) W_z(gz) of assembled 1-D LGL
// weights.  The assembled divergence then splits into three 1-D operators:
// along each grid line, a node interior to an element takes that element's
// derivative (D F)_a, and a node on a shared face takes
// (w_N (D F^left)_N + w_0 (D F^right)_0) / (w_N + w_0) =
// ((D F^left)_N + (D F^right)_0) / 2 (w_0 = w_N); the transverse weights
// cancel against M.  This is the paper's gather/assembly/scatter of
// Alg. 1-3, reached without element-local storage and without atomics.
//
// One stage = three kernels over the SoA state:
//   k_line_x  one CTA per x-line: pointwise primitives (u, v, w, p') of every
//             node, x-fluxes staged in shared memory, one thread per element
//             segment for the 1-D contraction (Alg. 2), face averaging;
//             writes the x part of the tendency to T and (v, w, p', theta =
//             Theta/rho) to W.
//   k_line_y  one thread per (x, z) column marching along y over a chunk of
//             element segments, carrying the shared face node's flux and
//             one-sided derivative; adds the y part into T.
//   k_line_z  one thread per (x, y) column marching along z; adds the z part,
//             the sources (-rho' g k, -f k x rho u, rho S_theta), applies
//             no-flux walls and either stores dq/dt or the fused SSP-RK
//             stage combination out = alpha q^n + beta (q + dt L(q)) into a
//             buffer distinct from every input.
//
// Every arithmetic step is FP64.  The derivative matrices come pre-scaled by
// -2/h_d (chain rule of the affine map, sign of the divergence) with rows 0
// and N halved for the face average; wall nodes undo the halving.  The FP64
// pipe (2 DFMA/clk/SM on GB300) bounds these kernels, so the arithmetic is
// arranged to spend few FP64 instructions: the running tendency is the
// starting value of each contraction's FMA chain (no separate additions), the
// x contraction uses the even/odd split of the centro-antisymmetric LGL
// derivative matrix, 1/rho is one hardware reciprocal estimate refined by
// two Newton steps, and the equation of state is a short binomial series.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace xg {

constexpr int kMaxOrder = 8;
constexpr int kMaxPairs = (kMaxOrder + 1) / 2;
constexpr int kEosTerms = 8;

// Launch-time constants of one mesh (passed by value as a kernel parameter).
struct LineParams {
  int n[3];       // global nodes per direction
  int nseg[3];    // elements per direction
  int per[3];     // 1 = periodic
  // y ends that are faces of an element partition (a domain split into
  // y-slabs, Sec. 3.1): the face node's y part is completed by the
  // neighbouring partition's one-sided row (xg_partition_*) instead of the
  // wall's doubled row, and no wall condition applies there
  int open_y[2];
  long long np;   // n[0] n[1] n[2]
  // Dm[d][a][l] = -(2/h_d) D[a][l] (x 1/2 for a = 0 and a = N)
  double Dm[3][kMaxOrder + 1][kMaxOrder + 1];
  // even/odd split of Dm (pairs l < N-l):  for i < (N+1)/2
  //   (Dm f)_i   = sum_l EA[i][l] o_l + (sum_l EB[i][l] e_l + EBm[i] f_mid)
  //   (Dm f)_N-i = sum_l EA[i][l] o_l - (...)
  // with e_l = f_l + f_{N-l}, o_l = f_l - f_{N-l}; for even N the middle row
  //   (Dm f)_{N/2} = sum_l EM[l] o_l.
  double EA[3][kMaxPairs][kMaxPairs];
  double EB[3][kMaxPairs][kMaxPairs];
  double EBm[3][kMaxPairs];
  double EM[3][kMaxPairs];
  // (1 + x)^gamma - 1 = sum_{k=1..8} eos_c[k-1] x^k for |x| < eos_xmax
  double eos_c[kEosTerms];
  double eos_xmax;
  double gamma;
  double f, g;    // Coriolis parameter, gravity
};

// Buffers and stage coefficients of one launch.
struct StageBufs {
  const double* q;      // [5][np] state the tendency is taken of
  const double* qn;     // [5][np] q^n of the RK combination (alpha != 0)
  double* out;          // [5][np] new state, or dq/dt when rhs_only
  double* W;            // [4][np] v, w, p', theta = Theta/rho (written by k_line_x)
  double* T;            // [5][np] x + y parts of the tendency
  const double* S;      // [np] heating S_theta (K/s)
  const double* base;   // [4][nz]: rho0, Theta0, p0, 1/Theta0 per level
  int* flag;            // set to 1 when a non-finite value is stored
  double dt, alpha, beta;
  int rhs_only;
  const double* E = nullptr;  // [5][np] extra tendency (hyper-diffusion, sponge) or null
  // open_y[1]: the one-sided row N of the slab's last y segment at every
  // (x, z) of the end face, [5][n_z][n_x] (written by k_line_y instead of the
  // wall's doubled row)
  double* face_hi = nullptr;
};

// (1 + x)^gamma - 1: the binomial series (Horner) for small |x|, where the
// truncation error after 8 terms is below 2^-56 relative (bound checked on
// the host), else expm1(gamma log1p(x)).
__device__ __forceinline__ double eos_phi(const LineParams& P, double x) {
  if (fabs(x) < P.eos_xmax) {
    double acc = P.eos_c[kEosTerms - 1];
#pragma unroll
    for (int k = kEosTerms - 2; k >= 0; --k) acc = fma(acc, x, P.eos_c[k]);
    return acc * x;
  }
  return expm1(P.gamma * log1p(x));
}

// 1/a for positive normal a: the hardware reciprocal estimate refined by two
// Newton-Raphson steps r <- r + r (1 - a r) (quadratic convergence; the
// estimate's error squared twice is far below the FP64 rounding, and the
// last FMA step leaves the result within an ulp).
__device__ __forceinline__ double rcp_newton(double a) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a));
  double e = fma(-a, r, 1.0);
  r = fma(r, e, r);
  e = fma(-a, r, 1.0);
  return fma(r, e, r);
}

__device__ __forceinline__ bool is_nonfinite(double v) {
  return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
}

// rows[a] = sum_l Dm[d][a][l] f[l], a = 0..N, by the even/odd split
// (2P + P (2P + [N even] + 2) + [N even] P FP64 operations, P = (N+1)/2:
// 20 instead of 25 at N = 4).
template <int N, int D>
__device__ __forceinline__ void contract_eo(const LineParams& P, const double (&f)[N + 1],
                                            double (&rows)[N + 1]) {
  constexpr int Pp = (N + 1) / 2;
  double e[Pp], o[Pp];
#pragma unroll
  for (int l = 0; l < Pp; ++l) {
    e[l] = f[l] + f[N - l];
    o[l] = f[l] - f[N - l];
  }
#pragma unroll
  for (int i = 0; i < Pp; ++i) {
    double s = P.EA[D][i][0] * o[0];
#pragma unroll
    for (int l = 1; l < Pp; ++l) s = fma(P.EA[D][i][l], o[l], s);
    double t = P.EB[D][i][0] * e[0];
#pragma unroll
    for (int l = 1; l < Pp; ++l) t = fma(P.EB[D][i][l], e[l], t);
    if (N % 2 == 0) t = fma(P.EBm[D][i], f[N / 2], t);
    rows[i] = s + t;
    rows[N - i] = s - t;
  }
  if (N % 2 == 0) {
    double m = P.EM[D][0] * o[0];
#pragma unroll
    for (int l = 1; l < Pp; ++l) m = fma(P.EM[D][l], o[l], m);
    rows[N / 2] = m;
  }
}

// start + sum_l Dm[d][a][l] f[l] as one FMA chain (N+1 operations).
template <int N, int D>
__device__ __forceinline__ double row_from(const LineParams& P, int a, const double (&f)[N + 1],
                                           double start) {
  double acc = start;
#pragma unroll
  for (int l = 0; l <= N; ++l) acc = fma(P.Dm[D][a][l], f[l], acc);
  return acc;
}

template <int N, int D>
__device__ __forceinline__ double row_N(const LineParams& P, const double (&f)[N + 1]) {
  double acc = P.Dm[D][N][0] * f[0];
#pragma unroll
  for (int l = 1; l <= N; ++l) acc = fma(P.Dm[D][N][l], f[l], acc);
  return acc;
}

// ---------------------------------------------------------------- difference form
// The rho' and Theta' tendencies are residuals of cancelling flux
// derivatives where the flow is nearly non-divergent (in a vortex the x and
// y parts nearly cancel), so their rounding must stay far below the size of
// each part.  Every row of the LGL derivative matrix sums to zero (D 1 = 0,
// the derivative of a constant), so a row may be applied to the flux minus
// its value at the segment's first node:
//     sum_l Dm[a][l] f_l = sum_{l>=1} Dm[a][l] (f_l - f_0);
// the roundings then scale with the flux's variation across the segment
// instead of the flux.  The Theta' flux Theta u_d is written theta (rho u_d)
// with theta = Theta / rho (W[3]), and its differences as
//     F_l - F_0 = theta_l (m_l - m_0) + (theta_l - theta_0) m_0,
// so the product's rounding scales with the variation as well.  The exact
// value is unchanged.
//
// diffs(m, th, dm, dF): dm[l] = m_l - m_0 and dF[l] = theta_l m_l - theta_0
// m_0 in that form, l = 0..N (dm[0] = dF[0] = -0, the additive identity, so
// the even/odd contraction's sums with them need no instruction).
template <int N>
__device__ __forceinline__ void seg_diffs(const double (&m)[N + 1], const double (&th)[N + 1],
                                          double (&dm)[N + 1], double (&dF)[N + 1]) {
  dm[0] = -0.0;
  dF[0] = -0.0;
#pragma unroll
  for (int l = 1; l <= N; ++l) {
    dm[l] = m[l] - m[0];
    dF[l] = fma(th[l], dm[l], (th[l] - th[0]) * m[0]);
  }
}

// start + sum_{l>=1} Dm[d][a][l] d[l] (d[0] = 0 is not used)
template <int N, int D>
__device__ __forceinline__ double drow_from(const LineParams& P, int a, const double (&d)[N + 1],
                                            double start) {
  double acc = start;
#pragma unroll
  for (int l = 1; l <= N; ++l) acc = fma(P.Dm[D][a][l], d[l], acc);
  return acc;
}

template <int N, int D>
__device__ __forceinline__ double drow_N(const LineParams& P, const double (&d)[N + 1]) {
  double acc = P.Dm[D][N][1] * d[1];
#pragma unroll
  for (int l = 2; l <= N; ++l) acc = fma(P.Dm[D][N][l], d[l], acc);
  return acc;
}

// ---------------------------------------------------------------- x lines
// grid (n_y, n_z), block kXThreads, dynamic shared memory
// 8 * (5 (n_x + 1) + 5 nseg_x) bytes.
constexpr int kXThreads = 128;

template <int N>
__global__ void __launch_bounds__(kXThreads) k_line_x(const LineParams P, const StageBufs B) {
  extern __shared__ double sm[];
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const int nseg = P.nseg[0];
  const int y = blockIdx.x, z = blockIdx.y;
  const long long np = P.np;
  const long long row = (long long)nx * (y + (long long)ny * z);
  const int ld = nx + 1;
  // F [5][ld]: x-fluxes of the line's nodes (+ periodic wrap slot); later
  // each segment's one-sided rows 0..N-1 in place.  RN [5][nseg]: row N.
  double* F = sm;
  double* RN = sm + 5 * ld;
  const double rho0 = __ldg(B.base + z);
  const double Th0 = __ldg(B.base + nz + z);
  const double p0 = __ldg(B.base + 2 * nz + z);
  const double iTh0 = __ldg(B.base + 3 * nz + z);
  const double* __restrict__ q = B.q;
  double* __restrict__ Wo = B.W;
  double* __restrict__ To = B.T;

  // pointwise primitives and x-fluxes, one node per thread (coalesced)
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const long long I = row + i;
    const double rp = q[I], mu = q[np + I], mv = q[2 * np + I], mw = q[3 * np + I];
    const double tp = q[4 * np + I];
    const double ir = rcp_newton(rho0 + rp);
    const double u = mu * ir, v = mv * ir, w = mw * ir;
    const double pp = p0 * eos_phi(P, tp * iTh0);
    const double Th = Th0 + tp;
    const double th = Th * ir;
    Wo[I] = v;
    Wo[np + I] = w;
    Wo[2 * np + I] = pp;
    Wo[3 * np + I] = th;
    F[i] = mu;
    F[ld + i] = fma(mu, u, pp);
    F[2 * ld + i] = mv * u;
    F[3 * ld + i] = mw * u;
    F[4 * ld + i] = th;              // theta: the Theta' flux is theta (rho u)
    if (P.per[0] && i == 0) {
      F[nx] = F[0];
      F[ld + nx] = F[ld];
      F[2 * ld + nx] = F[2 * ld];
      F[3 * ld + nx] = F[3 * ld];
      F[4 * ld + nx] = F[4 * ld];
    }
  }
  __syncthreads();

  // one element segment per thread: even/odd contraction per flux component;
  // every segment is read before any is overwritten (the loop below keeps
  // each thread's segments in registers when nseg <= blockDim, the usual
  // case; otherwise segments are processed in rounds with a barrier)
  for (int s0 = 0; s0 < nseg; s0 += blockDim.x) {
    const int s = s0 + threadIdx.x;
    double rows[5][N + 1];
    if (s < nseg) {
      {   // rho' and Theta' in difference form
        double m[N + 1], th[N + 1], dm[N + 1], dF[N + 1];
#pragma unroll
        for (int l = 0; l <= N; ++l) {
          m[l] = F[s * N + l];
          th[l] = F[4 * ld + s * N + l];
        }
        seg_diffs<N>(m, th, dm, dF);
        contract_eo<N, 0>(P, dm, rows[0]);
        contract_eo<N, 0>(P, dF, rows[4]);
      }
#pragma unroll
      for (int c = 1; c < 4; ++c) {
        double f[N + 1];
#pragma unroll
        for (int l = 0; l <= N; ++l) f[l] = F[c * ld + s * N + l];
        contract_eo<N, 0>(P, f, rows[c]);
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

  // assemble: face nodes add both one-sided halves, wall nodes double theirs
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const int s = i / N, a = i - s * N;
    const long long I = row + i;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      double v;
      if (s == nseg) {                     // last wall node
        v = RN[c * nseg + nseg - 1];
        v = v + v;
      } else if (a != 0) {
        v = F[c * ld + i];
      } else {
        const double r0 = F[c * ld + i];
        const int left = s > 0 ? s - 1 : (P.per[0] ? nseg - 1 : -1);
        v = r0 + (left >= 0 ? RN[c * nseg + left] : r0);
      }
      To[c * np + I] = v;
    }
  }
}

// ---------------------------------------------------------------- y lines
// grid (ceil(n_x / blockDim), nchunk, n_z); each thread marches `chunk`
// element segments along y at its (x, z).
// y-fluxes at one node; slot 4 holds theta (the Theta' flux theta (rho v)
// is taken in difference form with slot 0)
__device__ __forceinline__ void flux_y(const double* __restrict__ q, const double* __restrict__ W,
                                       long long np, long long I, double (&f)[5]) {
  const double mu = q[np + I], mv = q[2 * np + I], mw = q[3 * np + I];
  const double v = W[I], pp = W[2 * np + I];
  f[0] = mv;
  f[1] = mu * v;
  f[2] = fma(mv, v, pp);
  f[3] = mw * v;
  f[4] = W[3 * np + I];
}

template <int N>
__global__ void __launch_bounds__(128) k_line_y(const LineParams P, const StageBufs B, int chunk) {
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
  const double* __restrict__ q = B.q;
  const double* __restrict__ W = B.W;
  auto nodeI = [&](int gy) -> long long { return col + (long long)nx * (gy == ny ? 0 : gy); };

  double carry[5];
  bool has_left = (s0 > 0) || P.per[1];
  if (has_left) {
    const int sp = s0 > 0 ? s0 - 1 : nseg - 1;
    double fl[5][N + 1];
#pragma unroll
    for (int l = 0; l <= N; ++l) {
      double f[5];
      flux_y(q, W, np, nodeI(sp * N + l), f);
#pragma unroll
      for (int c = 0; c < 5; ++c) fl[c][l] = f[c];
    }
    double dm[N + 1], dF[N + 1];
    seg_diffs<N>(fl[0], fl[4], dm, dF);
    carry[0] = drow_N<N, 1>(P, dm);
    carry[4] = drow_N<N, 1>(P, dF);
#pragma unroll
    for (int c = 1; c < 4; ++c) carry[c] = row_N<N, 1>(P, fl[c]);
  }

  double fc[5][N + 1];
  {
    double f[5];
    flux_y(q, W, np, nodeI(s0 * N), f);
#pragma unroll
    for (int c = 0; c < 5; ++c) fc[c][0] = f[c];
  }
  double* __restrict__ T = B.T;
  for (int s = s0; s < s1; ++s) {
#pragma unroll
    for (int l = 1; l <= N; ++l) {
      double f[5];
      flux_y(q, W, np, nodeI(s * N + l), f);
#pragma unroll
      for (int c = 0; c < 5; ++c) fc[c][l] = f[c];
    }
    double dm[N + 1], dF[N + 1];
    seg_diffs<N>(fc[0], fc[4], dm, dF);
    // row a of variable c from start (rho' and Theta' in difference form)
    auto rowc = [&](int c, int a, double start) -> double {
      if (c == 0) return drow_from<N, 1>(P, a, dm, start);
      if (c == 4) return drow_from<N, 1>(P, a, dF, start);
      return row_from<N, 1>(P, a, fc[c], start);
    };
    // the segment's running x parts, all loaded before any store
    double tv[5][N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const long long I = nodeI(s * N + a);
#pragma unroll
      for (int c = 0; c < 5; ++c) tv[c][a] = T[c * np + I];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      // the running x part is the start of each row's FMA chain
      double t0 = tv[c][0];
      if (!has_left && !P.open_y[0]) t0 = rowc(c, 0, t0);   // wall: the row counts twice
      t0 = rowc(c, 0, t0);
      T[c * np + nodeI(s * N)] = has_left ? t0 + carry[c] : t0;
#pragma unroll
      for (int a = 1; a < N; ++a) T[c * np + nodeI(s * N + a)] = rowc(c, a, tv[c][a]);
      carry[c] = c == 0 ? drow_N<N, 1>(P, dm) : (c == 4 ? drow_N<N, 1>(P, dF) : row_N<N, 1>(P, fc[c]));
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
      for (int c = 0; c < 5; ++c) T[c * np + I] += carry[c] + carry[c];
    }
  }
}

// ---------------------------------------------------------------- z lines + sources + stage
// z-fluxes at one node; slot 4 holds theta (see flux_y)
__device__ __forceinline__ void flux_z(const double* __restrict__ q, const double* __restrict__ W,
                                       long long np, long long I, double (&f)[5]) {
  const double mu = q[np + I], mv = q[2 * np + I], mw = q[3 * np + I];
  const double w = W[np + I], pp = W[2 * np + I];
  f[0] = mw;
  f[1] = mu * w;
  f[2] = mv * w;
  f[3] = fma(mw, w, pp);
  f[4] = W[3 * np + I];
}

// Completes node I at level gz given L[5] = T + z part (the assembled flux
// divergence): sources, no-flux walls, then the stage store.  Every array of
// a launch is distinct (the stage output never overwrites an input), which
// the __restrict__ qualifiers state so loads can be issued ahead of stores.
__device__ __forceinline__ void finish_node(const LineParams& P, const StageBufs& B,
                                            const double* __restrict__ q,
                                            const double* __restrict__ qn,
                                            double* __restrict__ out, long long I, int x, int y,
                                            int gz, double (&L)[5], bool& bad) {
  const long long np = P.np;
  const double rp = q[I], mu = q[np + I], mv = q[2 * np + I];
  if (B.E) {
#pragma unroll
    for (int c = 0; c < 5; ++c) L[c] += B.E[c * np + I];
  }
  L[1] = fma(P.f, mv, L[1]);                     // -f k x (rho u): +f rho v
  L[2] = fma(-P.f, mu, L[2]);                    //                 -f rho u
  L[3] = fma(-P.g, rp, L[3]);                    // -rho' g
  if (B.S) L[4] = fma(__ldg(B.base + gz) + rp, __ldg(B.S + I), L[4]);  // rho S_theta
  if (!P.per[0] && (x == 0 || x == P.n[0] - 1)) L[1] = 0.0;
  if (!P.per[1] && ((y == 0 && !P.open_y[0]) || (y == P.n[1] - 1 && !P.open_y[1]))) L[2] = 0.0;
  if (!P.per[2] && (gz == 0 || gz == P.n[2] - 1)) L[3] = 0.0;
  if (B.rhs_only) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      out[c * np + I] = L[c];
      bad |= is_nonfinite(L[c]);
    }
  } else if (B.alpha == 0.0) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const double o = fma(B.dt, L[c], q[c * np + I]);
      out[c * np + I] = o;
      bad |= is_nonfinite(o);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const double o = fma(B.alpha, qn[c * np + I], B.beta * fma(B.dt, L[c], q[c * np + I]));
      out[c * np + I] = o;
      bad |= is_nonfinite(o);
    }
  }
}

// grid (ceil(n_x / blockDim), nchunk, n_y); each thread marches `chunk`
// element segments along z at its (x, y).
template <int N>
__global__ void __launch_bounds__(128) k_line_z(const LineParams P, const StageBufs B, int chunk) {
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
  const double* __restrict__ q = B.q;
  const double* __restrict__ W = B.W;
  const double* __restrict__ T = B.T;
  const double* __restrict__ qn = B.qn;
  double* __restrict__ out = B.out;
  auto lev = [&](int gz) -> int { return gz == nz ? 0 : gz; };
  bool bad = false;

  double carry[5];
  bool has_left = (s0 > 0) || P.per[2];
  if (has_left) {
    const int sp = s0 > 0 ? s0 - 1 : nseg - 1;
    double fl[5][N + 1];
#pragma unroll
    for (int l = 0; l <= N; ++l) {
      const int gz = lev(sp * N + l);
      double f[5];
      flux_z(q, W, np, col + nxy * gz, f);
#pragma unroll
      for (int c = 0; c < 5; ++c) fl[c][l] = f[c];
    }
    double dm[N + 1], dF[N + 1];
    seg_diffs<N>(fl[0], fl[4], dm, dF);
    carry[0] = drow_N<N, 2>(P, dm);
    carry[4] = drow_N<N, 2>(P, dF);
#pragma unroll
    for (int c = 1; c < 4; ++c) carry[c] = row_N<N, 2>(P, fl[c]);
  }

  double fc[5][N + 1];
  {
    const int gz = s0 * N;
    double f[5];
    flux_z(q, W, np, col + nxy * gz, f);
#pragma unroll
    for (int c = 0; c < 5; ++c) fc[c][0] = f[c];
  }
  for (int s = s0; s < s1; ++s) {
#pragma unroll
    for (int l = 1; l <= N; ++l) {
      const int gz = lev(s * N + l);
      double f[5];
      flux_z(q, W, np, col + nxy * gz, f);
#pragma unroll
      for (int c = 0; c < 5; ++c) fc[c][l] = f[c];
    }
    double dm[N + 1], dF[N + 1];
    seg_diffs<N>(fc[0], fc[4], dm, dF);
    auto rowc = [&](int c, int a, double start) -> double {
      if (c == 0) return drow_from<N, 2>(P, a, dm, start);
      if (c == 4) return drow_from<N, 2>(P, a, dF, start);
      return row_from<N, 2>(P, a, fc[c], start);
    };
    // the segment's x + y parts, all loaded before any store
    double tv[5][N];
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
      double L[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        double t = tv[c][a];
        if (a == 0 && !has_left) t = rowc(c, 0, t);  // wall: the row counts twice
        t = rowc(c, a, t);
        L[c] = (a == 0 && has_left) ? t + carry[c] : t;
      }
      finish_node(P, B, q, qn, out, I, x, y, gz, L, bad);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c)
      carry[c] = c == 0 ? drow_N<N, 2>(P, dm) : (c == 4 ? drow_N<N, 2>(P, dF) : row_N<N, 2>(P, fc[c]));
#pragma unroll
    for (int c = 0; c < 5; ++c) fc[c][0] = fc[c][N];
    has_left = true;
  }
  if (!P.per[2] && s1 == nseg) {
    const int gz = nseg * N;
    const long long I = col + nxy * gz;
    double L[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) L[c] = T[c * np + I] + (carry[c] + carry[c]);
    finish_node(P, B, q, qn, out, I, x, y, gz, L, bad);
  }
  if (bad) *B.flag = 1;
}

}  // namespace xg
