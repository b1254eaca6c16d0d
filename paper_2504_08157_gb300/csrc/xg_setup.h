// xg_setup.h -- host-side mesh checks and launch constants shared by the
// entry points: the LGL derivative matrix (Sec. 2.2, Eq. 5), the binomial
// series of the equation of state (Eq. 3), the pre-scaled per-direction
// derivative matrices, and the marching-chunk choice of the line kernels.
#pragma once

#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/xg.h"
#include "xg_kernels.cuh"
#include "xg_kernels_df.cuh"
#include "xg_kernels_f32.cuh"
#include "xg_plane_f32.cuh"

namespace xg {

inline bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Legendre P_N and P_{N-1} at x by the three-term recurrence.
inline void legendre2(int N, long double x, long double* pN, long double* pN1) {
  long double p0 = 1.0L, p1 = x;
  if (N == 0) { *pN = 1.0L; *pN1 = 0.0L; return; }
  for (int k = 1; k < N; ++k) {
    long double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  *pN = p1;
  *pN1 = p0;
}

// LGL points: the zeros of x P_N - P_{N-1} = -(1 - x^2) P_N' / N, found by
// Newton's method (its derivative is (N+1) P_N) from the Chebyshev-Lobatto
// points; then the derivative matrix of the Lagrange basis,
// D[i][j] = P_N(x_i) / (P_N(x_j) (x_i - x_j)) for i != j,
// D[0][0] = -N(N+1)/4, D[N][N] = N(N+1)/4, else 0 on the diagonal.
inline void lgl_nodes(int N, long double* x) {
  const long double pi = 3.14159265358979323846264338327950288L;
  for (int j = 0; j <= N; ++j) {
    long double xj = -cosl(pi * j / N);
    for (int it = 0; it < 100; ++it) {
      long double pn, pn1;
      legendre2(N, xj, &pn, &pn1);
      long double dx = (xj * pn - pn1) / ((N + 1) * pn);
      xj -= dx;
      if (fabsl(dx) < 1e-30L) break;
    }
    x[j] = xj;
  }
  x[0] = -1.0L;
  x[N] = 1.0L;
}

inline void lgl_derivative(int N, double D[kMaxOrder + 1][kMaxOrder + 1]) {
  long double x[kMaxOrder + 1], PN[kMaxOrder + 1];
  lgl_nodes(N, x);
  for (int j = 0; j <= N; ++j) {
    long double pn1;
    legendre2(N, x[j], &PN[j], &pn1);
  }
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N; ++j) {
      long double v;
      if (i != j) v = PN[i] / (PN[j] * (x[i] - x[j]));
      else if (i == 0) v = -(long double)N * (N + 1) / 4.0L;
      else if (i == N) v = (long double)N * (N + 1) / 4.0L;
      else v = 0.0L;
      D[i][j] = (double)v;
    }
}

// LGL weights w_j = 2 / (N (N+1) P_N(x_j)^2) at the points of lgl_derivative.
inline void lgl_weights(int N, double* w) {
  const long double pi = 3.14159265358979323846264338327950288L;
  for (int j = 0; j <= N; ++j) {
    long double xj = -cosl(pi * j / N);
    for (int it = 0; it < 100; ++it) {
      long double pn, pn1;
      legendre2(N, xj, &pn, &pn1);
      long double dx = (xj * pn - pn1) / ((N + 1) * pn);
      xj -= dx;
      if (fabsl(dx) < 1e-30L) break;
    }
    if (j == 0) xj = -1.0L;
    if (j == N) xj = 1.0L;
    long double pn, pn1;
    legendre2(N, xj, &pn, &pn1);
    w[j] = (double)(2.0L / ((long double)N * (N + 1) * pn * pn));
  }
}

// Binomial coefficients C(gamma, k), k = 1..K (K = kEosTerms), of
// (1+x)^gamma - 1 and the largest |x| (<= 0.1) for which the truncation
// error after K terms stays below 2^-56 of the sum:
// |R| <= |C(gamma,K+1)| |x|^(K+1) / (1 - |x|) (the coefficients decrease in
// magnitude for 1 < gamma < 2) against a sum of at least 0.9 gamma |x|.
inline void eos_series(double gamma, double* c, double* xmax) {
  long double ck = 1.0L;
  for (int k = 1; k <= kEosTerms; ++k) {
    ck = ck * ((long double)gamma - (k - 1)) / k;
    c[k - 1] = (double)ck;
  }
  long double cK1 = fabsl(ck * ((long double)gamma - kEosTerms) / (kEosTerms + 1));
  long double bound = ldexpl(1.0L, -56) * 0.9L * gamma * 0.9L / (cK1 > 0 ? cK1 : 1e-300L);
  long double xm = powl(bound, 1.0L / kEosTerms);
  *xmax = (double)(xm < 0.1L ? xm : 0.1L);
}

// Sizes a mesh description implies.
struct MeshGeom {
  int n[3];        // global nodes per direction
  long long np;    // n[0] n[1] n[2]
  size_t xsmem;    // dynamic shared memory of k_line_x
};

// Host-side checks of a mesh description (no GPU work).  XG_ERR_ARG for
// invalid values, XG_ERR_UNSUPPORTED for valid ones this build cannot run.
inline xg_status check_desc(const xg_mesh_desc* d, MeshGeom* g) {
  if (!d) return XG_ERR_ARG;
  for (int k = 0; k < 3; ++k) {
    if (d->nel[k] < 1) return XG_ERR_ARG;
    if (!(std::isfinite(d->lo[k]) && std::isfinite(d->hi[k]) && d->hi[k] > d->lo[k])) return XG_ERR_ARG;
    if (d->periodic[k] != 0 && d->periodic[k] != 1) return XG_ERR_ARG;
  }
  if (d->order < 1 || d->order > kMaxOrder) return XG_ERR_ARG;
  if (!(finite_pos(d->R) && finite_pos(d->cp) && finite_pos(d->cv) && finite_pos(d->p_a))) return XG_ERR_ARG;
  if (!(std::isfinite(d->g) && d->g >= 0.0 && std::isfinite(d->f_coriolis))) return XG_ERR_ARG;
  const double gamma = d->cp / d->cv;
  if (!(gamma > 1.0 && gamma < 2.0)) return XG_ERR_ARG;
  if (d->precision != XG_FP64 && d->precision != XG_DF64 && d->precision != XG_FP32)
    return XG_ERR_UNSUPPORTED;
  const int N = d->order;
  for (int k = 0; k < 3; ++k) {
    long long nk = (long long)N * d->nel[k] + (d->periodic[k] ? 0 : 1);
    if (nk > (1 << 24)) return XG_ERR_UNSUPPORTED;
    g->n[k] = (int)nk;
  }
  g->np = (long long)g->n[0] * g->n[1] * g->n[2];
  // one x-line per CTA: its fluxes and segment derivatives in shared memory
  g->xsmem = sizeof(double) * (5 * (size_t)(g->n[0] + 1) + 5 * (size_t)d->nel[0]);
  if (g->xsmem > 220 * 1024) return XG_ERR_UNSUPPORTED;
  if (g->n[1] > 65535 || g->n[2] > 65535) return XG_ERR_UNSUPPORTED;  // grid y/z limits
  return XG_OK;
}

// Launch constants of the line kernels for a checked description.
inline void fill_line_params(const xg_mesh_desc* d, const MeshGeom& g, LineParams* P) {
  memset(P, 0, sizeof(*P));
  const int N = d->order;
  double D[kMaxOrder + 1][kMaxOrder + 1];
  lgl_derivative(N, D);
  for (int k = 0; k < 3; ++k) {
    P->n[k] = g.n[k];
    P->nseg[k] = d->nel[k];
    P->per[k] = d->periodic[k];
    const double h = (d->hi[k] - d->lo[k]) / d->nel[k];
    for (int a = 0; a <= N; ++a) {
      const double face = (a == 0 || a == N) ? 0.5 : 1.0;
      for (int l = 0; l <= N; ++l) P->Dm[k][a][l] = -(2.0 / h) * face * D[a][l];
    }
    // even/odd split (the LGL matrix is centro-antisymmetric,
    // D[N-i][N-l] = -D[i][l]; the halved rows 0 and N keep that property)
    const int Pp = (N + 1) / 2;
    for (int i = 0; i < Pp; ++i) {
      for (int l = 0; l < Pp; ++l) {
        P->EA[k][i][l] = 0.5 * (P->Dm[k][i][l] - P->Dm[k][i][N - l]);
        P->EB[k][i][l] = 0.5 * (P->Dm[k][i][l] + P->Dm[k][i][N - l]);
      }
      P->EBm[k][i] = (N % 2 == 0) ? P->Dm[k][i][N / 2] : 0.0;
      P->EM[k][i] = (N % 2 == 0) ? P->Dm[k][N / 2][i] : 0.0;
    }
  }
  P->np = g.np;
  const double gamma = d->cp / d->cv;
  eos_series(gamma, P->eos_c, &P->eos_xmax);
  P->gamma = gamma;
  P->f = d->f_coriolis;
  P->g = d->g;
}

// A double split into a double-float pair (host).
inline df split_df(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

// Launch constants of the double-float line kernels, from the FP64 ones.
inline void fill_df_params(const LineParams& P, DfParams* Q) {
  memset(Q, 0, sizeof(*Q));
  for (int k = 0; k < 3; ++k) {
    Q->n[k] = P.n[k];
    Q->nseg[k] = P.nseg[k];
    Q->per[k] = P.per[k];
    for (int a = 0; a <= kMaxOrder; ++a)
      for (int l = 0; l <= kMaxOrder; ++l) Q->Dm[k][a][l] = split_df(P.Dm[k][a][l]);
  }
  Q->np = P.np;
  for (int k = 0; k < 3; ++k) Q->eos_c[k] = split_df(P.eos_c[k]);
  for (int k = 3; k < kEosTerms; ++k) Q->eos_g[k - 3] = (float)P.eos_c[k];
  Q->eos_xmax = (float)P.eos_xmax;
  Q->gamma = P.gamma;
  Q->f = split_df(P.f);
  Q->g = split_df(P.g);
  Q->P64 = P;
}

// Launch constants of the FP32 line kernels, from the FP64 ones.
inline void fill_f32_params(const LineParams& P, FParams* Q) {
  memset(Q, 0, sizeof(*Q));
  for (int k = 0; k < 3; ++k) {
    Q->n[k] = P.n[k];
    Q->nseg[k] = P.nseg[k];
    Q->per[k] = P.per[k];
    for (int a = 0; a <= kMaxOrder; ++a)
      for (int l = 0; l <= kMaxOrder; ++l) Q->Dm[k][a][l] = (float)P.Dm[k][a][l];
  }
  Q->np = P.np;
  for (int k = 0; k < 3; ++k) Q->eos_c[k] = split_df(P.eos_c[k]);
  for (int k = 3; k < kEosTerms; ++k) Q->eos_g[k - 3] = (float)P.eos_c[k];
  Q->eos_xmax = (float)P.eos_xmax;
  Q->gamma = P.gamma;
  Q->f = (float)P.f;
  Q->g = (float)P.g;
}

// Element segments per marching thread of k_line_y / k_line_z.  A launch
// has items_per_chunk CTAs for every chunk of the line.  The kernels are
// bound by the FP64 pipe of each SM, which its resident CTAs share, so the
// launch lasts about as long as the SM given the most CTAs: ceil(items /
// SMs) chunks, each one chunk of segments plus the halo segment a chunk
// start recomputes (about a fifth of a segment's work).  The chunk count with
// the smallest such makespan wins.
inline void choose_chunks(int nseg, long long items_per_chunk, long long sms, bool periodic,
                          int* chunk, int* nchunk) {
  if (sms < 1) sms = 1;
  double best = 1e300;
  *chunk = nseg;
  *nchunk = 1;
  for (int k = 1; k <= nseg; ++k) {
    const int c = (nseg + k - 1) / k;
    const int nk = (nseg + c - 1) / c;
    if (nk != k) continue;
    const long long per_sm = (items_per_chunk * nk + sms - 1) / sms;
    const double cost = (double)per_sm * (c + ((nk > 1 || periodic) ? 0.2 : 0.0));
    if (cost < best - 1e-9) {
      best = cost;
      *chunk = c;
      *nchunk = nk;
    }
  }
}

// Chunking of both marching kernels for a mesh on a device with `sms` SMs.
inline void plan_marches(const xg_mesh_desc* d, const MeshGeom& g, int sms, int* chunk_y,
                         int* nchunk_y, int* chunk_z, int* nchunk_z) {
  const long long xblocks = (g.n[0] + 127) / 128;
  choose_chunks(d->nel[1], xblocks * g.n[2], sms, d->periodic[1] != 0, chunk_y, nchunk_y);
  choose_chunks(d->nel[2], xblocks * g.n[1], sms, d->periodic[2] != 0, chunk_z, nchunk_z);
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes`.  The
// limit is an attribute of the kernel function on the device, shared by
// every context (and every translation unit that launches the kernel), so
// it is only ever raised: lowering it for one mesh would break the launches
// of a larger mesh that is still alive.
template <typename F>
inline cudaError_t raise_dynamic_smem(F* func, size_t bytes) {
  static std::mutex m;
  std::lock_guard<std::mutex> lock(m);
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, (const void*)func);
  if (e != cudaSuccess) return e;
  if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute((const void*)func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace xg
