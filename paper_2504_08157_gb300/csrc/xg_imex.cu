// xg_imex.cu -- IMEX ARK2 time integration with matrix-free GMRES
// (include/xg_imex.h).
//
// The linear operator is evaluated node by node: for each node the
// assembled derivatives it needs (rho u along x, rho v along y, rho w and
// theta_0 rho w along z, Theta' along x and y, p'_lin along z) are sums of
// the pre-scaled derivative rows Dm over the node's segments (a face node
// adds the segment before, a wall node doubles its row), exactly the
// structure of the right-hand side's contractions.  One kernel returns
// c0 v + c1 L(v), so a GMRES product (I - dt g L) v is a single pass.
//
// GMRES (restarted; one classical Gram-Schmidt pass, a second only where the
// first cancels severely) runs on the host with the device vectors; the
// inner products are deterministic (fixed grid, per-block and per-variable
// partial sums added on the host in block order) and weight variable v by
// 1/rms(b_v)^2.  The explicit part is the context's own stage in
// right-hand-side mode (FP64, or the mixed XG_DF64 stage); L, the inner
// products and the combinations are FP64, and all of them are bound by
// GB300's FP64 pipe.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/xg_imex.h"
#include "xg_ctx.h"
#include "xg_setup.h"

namespace xg {

constexpr int kDotBlocksMax = 2048;   // partial-sum slots; a launch uses 4 blocks per SM
constexpr int kDotThreads = 256;
constexpr int kDotBatch = 16;   // vectors per multi-dot launch
constexpr int kCombMax = 17;    // terms per combination launch

// sum over the node's segment(s) along d of Dm rows times f: -d/dx_d of the
// assembled field.  With tab (z only) the coefficients are tab's, the rows
// of Dm already multiplied by a per-level factor of the loaded node:
// tab[(s (N + 1) + a) (N + 1) + l] = Dm[2][a][l] lev[s N + l] (k_lin_tables).
template <int N>
__device__ __forceinline__ double line_sum(const LineParams& P, int d, const double* __restrict__ f,
                                           long long base, long long sd, int g,
                                           const double* __restrict__ tab) {
  const int nd = P.n[d], nseg = P.nseg[d];
  int s = g / N;
  if (s >= nseg) s = nseg - 1;
  const int a = g - s * N;
  const double* t = tab ? tab + (s * (N + 1) + a) * (N + 1) : nullptr;
  double acc = 0.0;
#pragma unroll
  for (int l = 0; l <= N; ++l) {
    int k = s * N + l;
    if (k >= nd) k -= nd;
    acc = fma(t ? t[l] : P.Dm[d][a][l], f[base + sd * k], acc);
  }
  if (a == 0) {
    if (s > 0 || P.per[d]) {
      const int s2 = s > 0 ? s - 1 : nseg - 1;
      const double* t2 = tab ? tab + (s2 * (N + 1) + N) * (N + 1) : nullptr;
#pragma unroll
      for (int l = 0; l <= N; ++l) {
        int k = s2 * N + l;
        if (k >= nd) k -= nd;
        acc = fma(t2 ? t2[l] : P.Dm[d][N][l], f[base + sd * k], acc);
      }
    } else {
      acc = acc + acc;
    }
  } else if (a == N) {
    acc = acc + acc;
  }
  return acc;
}

// out = c0 v + c1 L(v) (out = L(v) for c0 = 0, c1 = 1); cpl = gamma p0 /
// Theta0 per level, tw and tp the z rows times theta0 = Theta0 / rho0 and
// times cpl (k_lin_tables).  FP64 work per node: the seven line sums' FMAs
// (N + 1 each, twice at a face node) and the assembly; the per-level factors
// of the z sums ride in their coefficients.
template <int N>
__global__ void __launch_bounds__(128) k_linear(const LineParams P, const double* __restrict__ v,
                                                const double* __restrict__ cpl,
                                                const double* __restrict__ th0,
                                                const double* __restrict__ tw,
                                                const double* __restrict__ tp, double c0, double c1,
                                                double* __restrict__ out) {
  const long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (I >= P.np) return;
  const long long np = P.np;
  const int nx = P.n[0], ny = P.n[1];
  const long long nxy = (long long)nx * ny;
  const int gx = (int)(I % nx);
  const long long r = I / nx;
  const int gy = (int)(r % ny), gz = (int)(r / ny);
  const long long bx = I - gx, by = I - (long long)gy * nx, bz = I - (long long)gz * nxy;
  const double* ru = v + np;
  const double* rv = v + 2 * np;
  const double* rw = v + 3 * np;
  const double* th = v + 4 * np;
  const double dxu = line_sum<N>(P, 0, ru, bx, 1, gx, nullptr);
  const double dyv = line_sum<N>(P, 1, rv, by, nx, gy, nullptr);
  const double dzw = line_sum<N>(P, 2, rw, bz, nxy, gz, nullptr);
  const double dzwt = line_sum<N>(P, 2, rw, bz, nxy, gz, tw);
  const double dxp = cpl[gz] * line_sum<N>(P, 0, th, bx, 1, gx, nullptr);
  const double dyp = cpl[gz] * line_sum<N>(P, 1, th, by, nx, gy, nullptr);
  const double dzp = line_sum<N>(P, 2, th, bz, nxy, gz, tp);
  double L[5];
  L[0] = dxu + dyv + dzw;
  L[1] = dxp;
  L[2] = dyp;
  L[3] = fma(-P.g, v[I], dzp);
  L[4] = fma(th0[gz], dxu + dyv, dzwt);
  if (!P.per[0] && (gx == 0 || gx == nx - 1)) L[1] = 0.0;
  if (!P.per[1] && (gy == 0 || gy == ny - 1)) L[2] = 0.0;
  if (!P.per[2] && (gz == 0 || gz == P.n[2] - 1)) L[3] = 0.0;
  if (c0 == 0.0 && c1 == 1.0) {
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c * np + I] = L[c];
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c * np + I] = c0 == 0.0 ? c1 * L[c] : fma(c1, L[c], c0 * v[c * np + I]);
  }
}

struct Comb {
  const double* x[kCombMax];
  double c[kCombMax];
  int k;
};

// out = sum_k c_k x_k over the first K terms of C (out may be one of the
// x_k); K fixed at compile time so that the K loads of an element are issued
// together.
template <int K>
__global__ void __launch_bounds__(256) k_comb(const Comb C, double* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double x[K];
#pragma unroll
    for (int k = 0; k < K; ++k) x[k] = C.x[k][i];
    double a = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) a = fma(C.c[k], x[k], a);
    out[i] = a;
  }
}

struct Dots {
  const double* v[kDotBatch];
  int k;
};

// partial[(b 5 + c) K + i] = sum over block b's nodes of variable c of
// w v_i, for the K vectors of D, in a fixed order (deterministic for a given
// grid); the host weights the variables.  One FP64 FMA per loaded value of
// the v_i: on GB300 a dot product is bound by the FP64 pipe, not by HBM, so
// the weights stay out of the loop.  The loads of two nodes (K <= 8) or of
// one are issued together; warps reduce by shuffles, the block's warps in
// order.  SELF (K = 1, v_0 = w): |w|^2 per variable from one read of w.
template <int K, bool SELF = false>
__global__ void __launch_bounds__(kDotThreads, 4) k_wdots(const double* __restrict__ w, const Dots D, long long np,
                                                       double* __restrict__ partial) {
  constexpr int U = K <= 8 ? 2 : 1;   // nodes per thread and iteration
  __shared__ double red[K][kDotThreads / 32];
  const long long per = (np + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * per, hi = min(np, lo + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long step = blockDim.x;
  for (int c = 0; c < 5; ++c) {
    const long long off = c * np;
    double acc[K];
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] = 0.0;
    long long I = lo + threadIdx.x;
    for (; I + (U - 1) * step < hi; I += U * step) {
      double wi[U], v[U][K];
#pragma unroll
      for (int u = 0; u < U; ++u) wi[u] = w[off + I + u * step];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int i = 0; i < K; ++i) v[u][i] = SELF ? wi[u] : D.v[i][off + I + u * step];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int i = 0; i < K; ++i) acc[i] = fma(wi[u], v[u][i], acc[i]);
    }
    if (U > 1 && I < hi) {             // the one node left over (I + step >= hi)
      const double wi = w[off + I];
#pragma unroll
      for (int i = 0; i < K; ++i) acc[i] = fma(wi, SELF ? wi : D.v[i][off + I], acc[i]);
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], o);
      if (lane == 0) red[i][warp] = acc[i];
    }
    __syncthreads();
    if (threadIdx.x < K) {
      double t = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
      partial[((long long)blockIdx.x * 5 + c) * K + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// tw[(s (N + 1) + a) (N + 1) + l] = Dm[2][a][l] theta0[k] and tp the same
// with cpl[k], k = s N + l (wrapped when z is periodic): the z rows of the
// linear operator with their per-level factor
template <int N>
__global__ void k_lin_tables(const LineParams P, const double* __restrict__ cpl, const double* __restrict__ th0,
                             double* __restrict__ tw, double* __restrict__ tp) {
  const int nseg = P.nseg[2], nd = P.n[2];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nseg * (N + 1) * (N + 1)) return;
  const int l = e % (N + 1), a = (e / (N + 1)) % (N + 1), s = e / ((N + 1) * (N + 1));
  int k = s * N + l;
  if (k >= nd) k -= nd;
  tw[e] = P.Dm[2][a][l] * th0[k];
  tp[e] = P.Dm[2][a][l] * cpl[k];
}

__global__ void k_lin_levels(const double* __restrict__ base, int nz, double gamma, double* __restrict__ cpl,
                             double* __restrict__ th0) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nz) return;
  const double rho0 = base[k], Th0 = base[nz + k], p0 = base[2 * nz + k], iTh0 = base[3 * nz + k];
  cpl[k] = gamma * p0 * iTh0;
  th0[k] = Th0 / rho0;
}

}  // namespace xg

namespace {

using xg::LineParams;

struct Imex {
  int m = 0;
  long long n = 0;             // 5 np
  double* V = nullptr;         // m + 1 Krylov vectors
  double* x = nullptr;         // stage solution
  double* b = nullptr;         // stage right-hand side
  double* w = nullptr;         // work
  double* S[3] = {nullptr, nullptr, nullptr};
  double* L[2] = {nullptr, nullptr};
  double* q1 = nullptr;        // q^{n+1}
  double* cpl = nullptr;       // [nz]
  double* th0 = nullptr;       // [nz]
  double* tw = nullptr;        // [nseg_z][N + 1][N + 1] z rows times theta0
  double* tp = nullptr;        // [nseg_z][N + 1][N + 1] z rows times cpl
  double wt[5] = {1.0, 1.0, 1.0, 1.0, 1.0};   // inner-product weights per variable
  double* partial = nullptr;   // [kDotBlocksMax][5][kDotBatch]
  int dot_blocks = 512;        // blocks of the reductions: 4 per SM
  std::vector<double> hpart;
  long long reorth = 0;        // Arnoldi steps that took a second Gram-Schmidt pass
};

cudaError_t launch_linear(xg_ctx* c, const Imex& X, const double* v, double c0, double c1, double* out,
                          cudaStream_t st) {
  const LineParams& P = c->P;
  const unsigned blocks = (unsigned)((c->np + 127) / 128);
  switch (c->d.order) {
    case 1: xg::k_linear<1><<<blocks, 128, 0, st>>>(P, v, X.cpl, X.th0, X.tw, X.tp, c0, c1, out); break;
    case 2: xg::k_linear<2><<<blocks, 128, 0, st>>>(P, v, X.cpl, X.th0, X.tw, X.tp, c0, c1, out); break;
    case 3: xg::k_linear<3><<<blocks, 128, 0, st>>>(P, v, X.cpl, X.th0, X.tw, X.tp, c0, c1, out); break;
    case 4: xg::k_linear<4><<<blocks, 128, 0, st>>>(P, v, X.cpl, X.th0, X.tw, X.tp, c0, c1, out); break;
    case 5: xg::k_linear<5><<<blocks, 128, 0, st>>>(P, v, X.cpl, X.th0, X.tw, X.tp, c0, c1, out); break;
    case 6: xg::k_linear<6><<<blocks, 128, 0, st>>>(P, v, X.cpl, X.th0, X.tw, X.tp, c0, c1, out); break;
    case 7: xg::k_linear<7><<<blocks, 128, 0, st>>>(P, v, X.cpl, X.th0, X.tw, X.tp, c0, c1, out); break;
    case 8: xg::k_linear<8><<<blocks, 128, 0, st>>>(P, v, X.cpl, X.th0, X.tw, X.tp, c0, c1, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t comb(const std::vector<std::pair<double, const double*>>& terms, double* out, long long n,
                 cudaStream_t st) {
  // in chunks of kCombMax - 1 after the first, accumulating into out
  size_t k = 0;
  bool first = true;
  while (k < terms.size() || first) {
    xg::Comb C;
    memset(&C, 0, sizeof(C));
    int j = 0;
    if (!first) {
      C.x[j] = out;
      C.c[j++] = 1.0;
    }
    while (j < xg::kCombMax && k < terms.size()) {
      C.x[j] = terms[k].second;
      C.c[j++] = terms[k].first;
      ++k;
    }
    C.k = j;
    const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 8192);
    switch (C.k) {
#define XG_COMB_CASE(K) \
  case K: xg::k_comb<K><<<blocks, 256, 0, st>>>(C, out, n); break;
      XG_COMB_CASE(1) XG_COMB_CASE(2) XG_COMB_CASE(3) XG_COMB_CASE(4) XG_COMB_CASE(5) XG_COMB_CASE(6)
      XG_COMB_CASE(7) XG_COMB_CASE(8) XG_COMB_CASE(9) XG_COMB_CASE(10) XG_COMB_CASE(11) XG_COMB_CASE(12)
      XG_COMB_CASE(13) XG_COMB_CASE(14) XG_COMB_CASE(15) XG_COMB_CASE(16)
      default: xg::k_comb<xg::kCombMax><<<blocks, 256, 0, st>>>(C, out, n); break;
#undef XG_COMB_CASE
    }
    first = false;
  }
  return cudaGetLastError();
}

// unweighted per-variable inner products of w with vs[0..k-1] (k <= kDotBatch)
// into X.hpart[(b 5 + c) k + i]
cudaError_t var_dots(Imex& X, long long np, const double* w, const double* const* vs, int k, cudaStream_t st) {
  xg::Dots D;
  memset(&D, 0, sizeof(D));
  D.k = k;
  for (int i = 0; i < k; ++i) D.v[i] = vs[i];
  if (k == 1 && D.v[0] == w) {
    xg::k_wdots<1, true><<<X.dot_blocks, xg::kDotThreads, 0, st>>>(w, D, np, X.partial);
  } else switch (k) {
#define XG_WDOTS_CASE(K) \
  case K: xg::k_wdots<K><<<X.dot_blocks, xg::kDotThreads, 0, st>>>(w, D, np, X.partial); break;
    XG_WDOTS_CASE(1) XG_WDOTS_CASE(2) XG_WDOTS_CASE(3) XG_WDOTS_CASE(4) XG_WDOTS_CASE(5)
    XG_WDOTS_CASE(6) XG_WDOTS_CASE(7) XG_WDOTS_CASE(8) XG_WDOTS_CASE(9) XG_WDOTS_CASE(10)
    XG_WDOTS_CASE(11) XG_WDOTS_CASE(12) XG_WDOTS_CASE(13) XG_WDOTS_CASE(14) XG_WDOTS_CASE(15)
    XG_WDOTS_CASE(16)
    default: return cudaErrorInvalidValue;
#undef XG_WDOTS_CASE
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(X.hpart.data(), X.partial, sizeof(double) * X.dot_blocks * 5 * k, cudaMemcpyDeviceToHost,
                        st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

// weighted inner products of w with vs[0..k-1]: per variable the blocks'
// partials in block order, then the variables in order, each times its weight
cudaError_t wdots(Imex& X, long long np, const double* w, const double* const* vs, int k, double* out,
                  cudaStream_t st) {
  for (int i0 = 0; i0 < k; i0 += xg::kDotBatch) {
    const int kb = std::min(xg::kDotBatch, k - i0);
    const cudaError_t e = var_dots(X, np, w, vs + i0, kb, st);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < kb; ++i) {
      double t = 0.0;
      for (int c = 0; c < 5; ++c) {
        double s = 0.0;
        for (int b = 0; b < X.dot_blocks; ++b) s += X.hpart[((size_t)b * 5 + c) * kb + i];
        t = fma(X.wt[c], s, t);
      }
      out[i0 + i] = t;
    }
  }
  return cudaSuccess;
}

// per-variable weights 1 / mean(b_v^2) (1 where b_v vanishes), and the
// weighted |b|^2 from the same partials (the value wdots of b with itself
// returns, in the same order)
cudaError_t set_weights(Imex& X, long long np, const double* b, double* bn2, cudaStream_t st) {
  const cudaError_t e = var_dots(X, np, b, &b, 1, st);
  if (e != cudaSuccess) return e;
  double s[5];
  for (int c = 0; c < 5; ++c) {
    s[c] = 0.0;
    for (int blk = 0; blk < X.dot_blocks; ++blk) s[c] += X.hpart[(size_t)blk * 5 + c];
    const double ms = s[c] / (double)np;
    X.wt[c] = ms > 0.0 ? 1.0 / ms : 1.0;
  }
  double t = 0.0;
  for (int c = 0; c < 5; ++c) t = fma(X.wt[c], s[c], t);
  *bn2 = t;
  return cudaSuccess;
}

// Solve (I - h L) x = b, x holding the initial guess; returns XG_ERR_TIMEOUT
// when the relative residual stays above tol after the restarts.
xg_status gmres(xg_ctx* c, Imex& X, double h, double tol, int maxrs, int* iters, double* resid,
                cudaStream_t st, cudaError_t* err) {
  const long long np = c->np, n = X.n;
  const int m = X.m;
  auto vec = [&](int i) { return X.V + (size_t)i * n; };
  double bn2;
  *err = set_weights(X, np, X.b, &bn2, st);
  if (*err != cudaSuccess) return XG_ERR_CUDA;
  const double bnorm = std::sqrt(bn2);
  *iters = 0;
  *resid = 0.0;
  if (bnorm == 0.0) {
    *err = cudaMemsetAsync(X.x, 0, sizeof(double) * n, st);
    return *err == cudaSuccess ? XG_OK : XG_ERR_CUDA;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hcol(m + 1), h2(m + 1);
  std::vector<const double*> vp(m + 1);
  for (int rs = 0; rs < maxrs; ++rs) {
    // r = b - (x - h L x)  into V_0
    *err = launch_linear(c, X, X.x, 1.0, -h, X.w, st);
    if (*err == cudaSuccess) *err = comb({{1.0, X.b}, {-1.0, X.w}}, vec(0), n, st);
    double r2;
    const double* r0 = vec(0);
    if (*err == cudaSuccess) *err = wdots(X, np, vec(0), &r0, 1, &r2, st);
    if (*err != cudaSuccess) return XG_ERR_CUDA;
    const double beta = std::sqrt(r2);
    *resid = beta / bnorm;
    if (*resid <= tol) return XG_OK;
    *err = comb({{1.0 / beta, vec(0)}}, vec(0), n, st);
    if (*err != cudaSuccess) return XG_ERR_CUDA;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < m; ++j) {
      // The Arnoldi step runs on L: A = I - h L spans the same Krylov space,
      // and L V_m = V_{m+1} H_L gives A V_m = V_{m+1} (I~ - h H_L) exactly,
      // while L v_j -- unlike A v_j, which is mostly v_j -- is not largely
      // removed by its projection.  w = L v_j is orthogonalised against
      // v_0..v_j by one classical Gram-Schmidt pass.  The pass's multi-dot
      // includes <w, w>, and the norm after it follows from Pythagoras in the
      // weighted inner product (the v_i are orthonormal in it), so a pass is
      // one multi-dot and one combination that also normalises.  Only where
      // the pass removed more than 1 - 1e-4 of |w|^2 (a sharper form of the
      // criterion of Daniel, Gragg, Kaufman & Stewart, 1976, whose bound is
      // one half) a second pass runs, and the norm is then taken exactly.
      *err = launch_linear(c, X, vec(j), 0.0, 1.0, vec(j + 1), st);
      if (*err != cudaSuccess) return XG_ERR_CUDA;
      for (int i = 0; i <= j; ++i) vp[i] = vec(i);
      vp[j + 1] = vec(j + 1);
      std::fill(hcol.begin(), hcol.end(), 0.0);
      *err = wdots(X, np, vec(j + 1), vp.data(), j + 2, h2.data(), st);
      if (*err != cudaSuccess) return XG_ERR_CUDA;
      double w2 = h2[j + 1], s2 = 0.0;
      for (int i = 0; i <= j; ++i) {
        hcol[i] = h2[i];
        s2 += h2[i] * h2[i];
      }
      const double r2 = w2 - s2;
      std::vector<std::pair<double, const double*>> t;
      if (r2 > 1e-4 * w2) {
        // one pass: orthogonality to ~eps |w| / |w'| <= 1e2 eps; the norm by
        // Pythagoras, whose rounding (a few eps w2 in w2 and in s2) is
        // <= ~1e3 eps of r2 here, so v_{j+1} has norm 1 to ~1e-13, and the
        // combination normalises
        const double nrm = std::sqrt(r2), inv = 1.0 / nrm;
        t.push_back({inv, vec(j + 1)});
        for (int i = 0; i <= j; ++i) t.push_back({-h2[i] * inv, vec(i)});
        *err = comb(t, vec(j + 1), n, st);
        if (*err != cudaSuccess) return XG_ERR_CUDA;
        hcol[j + 1] = nrm;
      } else {
        // severe cancellation: subtract, orthogonalise once more, and take the norm exactly
        t.push_back({1.0, vec(j + 1)});
        for (int i = 0; i <= j; ++i) t.push_back({-h2[i], vec(i)});
        *err = comb(t, vec(j + 1), n, st);
        if (*err != cudaSuccess) return XG_ERR_CUDA;
        *err = wdots(X, np, vec(j + 1), vp.data(), j + 1, h2.data(), st);
        if (*err != cudaSuccess) return XG_ERR_CUDA;
        t.clear();
        t.push_back({1.0, vec(j + 1)});
        for (int i = 0; i <= j; ++i) {
          t.push_back({-h2[i], vec(i)});
          hcol[i] += h2[i];
        }
        *err = comb(t, vec(j + 1), n, st);
        if (*err != cudaSuccess) return XG_ERR_CUDA;
        const double* wp = vec(j + 1);
        *err = wdots(X, np, vec(j + 1), &wp, 1, &w2, st);
        if (*err != cudaSuccess) return XG_ERR_CUDA;
        hcol[j + 1] = std::sqrt(w2);
        if (hcol[j + 1] > 0.0) {
          *err = comb({{1.0 / hcol[j + 1], vec(j + 1)}}, vec(j + 1), n, st);
          if (*err != cudaSuccess) return XG_ERR_CUDA;
        }
        ++X.reorth;
      }
      ++*iters;
      // the column of I~ - h H_L
      for (int i = 0; i <= j + 1; ++i) hcol[i] *= -h;
      hcol[j] += 1.0;
      // Givens rotations
      for (int i = 0; i < j; ++i) {
        const double a = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
        hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
        hcol[i] = a;
      }
      const double den = std::hypot(hcol[j], hcol[j + 1]);
      cs[j] = den > 0.0 ? hcol[j] / den : 1.0;
      sn[j] = den > 0.0 ? hcol[j + 1] / den : 0.0;
      hcol[j] = den;
      hcol[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
      *resid = std::fabs(g[j + 1]) / bnorm;
      if (*resid <= tol || hcol[j] == 0.0) {
        ++j;
        break;
      }
    }
    // x += V y with H y = g (upper triangular, j columns)
    std::vector<double> y(j);
    for (int i = j - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * m + k] * y[k];
      y[i] = H[(size_t)i * m + i] != 0.0 ? s / H[(size_t)i * m + i] : 0.0;
    }
    std::vector<std::pair<double, const double*>> t;
    t.push_back({1.0, X.x});
    for (int i = 0; i < j; ++i) t.push_back({y[i], vec(i)});
    *err = comb(t, X.x, n, st);
    if (*err != cudaSuccess) return XG_ERR_CUDA;
    if (*resid <= tol) return XG_OK;
  }
  return XG_ERR_TIMEOUT;
}

void imex_free_buffers(Imex* X) {
  cudaFree(X->V);
  cudaFree(X->x);
  cudaFree(X->b);
  cudaFree(X->w);
  for (auto& p : X->S) cudaFree(p);
  for (auto& p : X->L) cudaFree(p);
  cudaFree(X->q1);
  cudaFree(X->cpl);
  cudaFree(X->th0);
  cudaFree(X->tw);
  cudaFree(X->tp);
  cudaFree(X->partial);
}

xg_status fail(xg_ctx* c, cudaError_t e, const char* where) {
  fprintf(stderr, "xg_imex: %s: %s\n", where, cudaGetErrorString(e));
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return XG_ERR_OOM;
  c->failed = true;
  return XG_ERR_CUDA;
}

// allocate (or keep) the work arrays for m Krylov vectors; refresh the
// per-level coefficients
cudaError_t prepare(xg_ctx* c, int m, cudaStream_t st) {
  Imex* X = static_cast<Imex*>(c->imex);
  if (X && X->m != m) {
    imex_free_buffers(X);
    delete X;
    X = nullptr;
    c->imex = nullptr;
  }
  const long long n = 5 * c->np;
  if (!X) {
    X = new (std::nothrow) Imex();
    if (!X) return cudaErrorMemoryAllocation;
    c->imex = X;
    X->m = m;
    X->n = n;
    X->hpart.resize((size_t)xg::kDotBlocksMax * 5 * xg::kDotBatch);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
    X->dot_blocks = std::min(xg::kDotBlocksMax, std::max(1, 4 * sms));
    const size_t vb = sizeof(double) * (size_t)n;
    cudaError_t e = cudaMalloc((void**)&X->V, vb * (m + 1));
    double** bufs[] = {&X->x, &X->b, &X->w, &X->S[0], &X->S[1], &X->S[2], &X->L[0], &X->L[1], &X->q1};
    for (double** p : bufs)
      if (e == cudaSuccess) e = cudaMalloc((void**)p, vb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&X->cpl, sizeof(double) * c->n[2]);
    if (e == cudaSuccess) e = cudaMalloc((void**)&X->th0, sizeof(double) * c->n[2]);
    const size_t tb = sizeof(double) * (size_t)c->P.nseg[2] * (c->d.order + 1) * (c->d.order + 1);
    if (e == cudaSuccess) e = cudaMalloc((void**)&X->tw, tb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&X->tp, tb);
    if (e == cudaSuccess)
      e = cudaMalloc((void**)&X->partial, sizeof(double) * xg::kDotBlocksMax * 5 * xg::kDotBatch);
    if (e != cudaSuccess) {
      imex_free_buffers(X);
      delete X;
      c->imex = nullptr;
      return e;
    }
  }
  xg::k_lin_levels<<<(c->n[2] + 127) / 128, 128, 0, st>>>(c->base64, c->n[2], c->P.gamma, X->cpl, X->th0);
  const int ne = c->P.nseg[2] * (c->d.order + 1) * (c->d.order + 1);
  const unsigned tblocks = (unsigned)((ne + 127) / 128);
  switch (c->d.order) {
#define XG_TABLES_CASE(N) \
  case N: xg::k_lin_tables<N><<<tblocks, 128, 0, st>>>(c->P, X->cpl, X->th0, X->tw, X->tp); break;
    XG_TABLES_CASE(1) XG_TABLES_CASE(2) XG_TABLES_CASE(3) XG_TABLES_CASE(4)
    XG_TABLES_CASE(5) XG_TABLES_CASE(6) XG_TABLES_CASE(7) XG_TABLES_CASE(8)
#undef XG_TABLES_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

void imex_free(xg_ctx* c) {
  Imex* X = static_cast<Imex*>(c->imex);
  if (!X) return;
  imex_free_buffers(X);
  delete X;
  c->imex = nullptr;
}

extern "C" {

xg_status xg_linear_operator(xg_ctx* c, const double* v, double* out, void* stream) {
  if (!c || !v || !out) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (c->f32) return XG_ERR_UNSUPPORTED;
  if (!c->has_base) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = prepare(c, c->imex ? static_cast<Imex*>(c->imex)->m : 20, st);
  if (e == cudaSuccess) e = launch_linear(c, *static_cast<Imex*>(c->imex), v, 0.0, 1.0, out, st);
  return e == cudaSuccess ? XG_OK : fail(c, e, "xg_linear_operator");
}

xg_status xg_step_imex(xg_ctx* c, double dt, int nsteps, const xg_imex_opts* opts, xg_imex_stats* stats,
                       void* stream) {
  if (!c) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (c->f32) return XG_ERR_UNSUPPORTED;
  if (c->part_open[0] || c->part_open[1]) return XG_ERR_UNSUPPORTED;   // partitioned: explicit only
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0 || !c->has_state) return XG_ERR_ARG;
  double tol = 1e-10;
  int m = 20, maxrs = 50;
  if (opts) {
    tol = opts->tol;
    m = opts->krylov;
    maxrs = opts->max_restarts;
    if (!(tol > 0.0 && tol < 1.0) || m < 1 || m > 64 || maxrs < 1) return XG_ERR_ARG;
  }
  if (stats) memset(stats, 0, sizeof(*stats));
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = prepare(c, m, st);
  if (e != cudaSuccess) return fail(c, e, "xg_step_imex");
  Imex& X = *static_cast<Imex*>(c->imex);
  const long long n = X.n;
  const double G = 1.0 - 1.0 / std::sqrt(2.0), Dl = 1.0 / (2.0 * std::sqrt(2.0));
  const double Al = (3.0 + 2.0 * std::sqrt(2.0)) / 6.0;
  const double ae[3][3] = {{0, 0, 0}, {2 * G, 0, 0}, {1 - Al, Al, 0}};
  const double ai[3][3] = {{0, 0, 0}, {G, G, 0}, {Dl, Dl, G}};
  const double bw[3] = {Dl, Dl, G};
  e = cudaMemsetAsync(c->flag, 0, sizeof(int), st);
  if (e != cudaSuccess) return fail(c, e, "xg_step_imex");
  for (int step = 0; step < nsteps; ++step) {
    const double* q = c->A;
    // stage 1 is explicit: Q1 = q
    e = rhs_f64_state(c, q, X.S[0], st);
    if (e == cudaSuccess) e = launch_linear(c, X, q, 0.0, 1.0, X.L[0], st);
    for (int i = 1; i < 3 && e == cudaSuccess; ++i) {
      // b = q + dt sum_j (ae_ij (S_j - L_j) + ai_ij L_j)
      std::vector<std::pair<double, const double*>> t;
      t.push_back({1.0, q});
      for (int j = 0; j < i; ++j) {
        t.push_back({dt * ae[i][j], X.S[j]});
        t.push_back({dt * (ai[i][j] - ae[i][j]), X.L[j]});
      }
      e = comb(t, X.b, n, st);
      // the first guess: q for the first solve; the second starts from the
      // first's solution, which X.x still holds
      if (e == cudaSuccess && i == 1)
        e = cudaMemcpyAsync(X.x, q, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) break;
      int it = 0;
      double res = 0.0;
      cudaError_t ge = cudaSuccess;
      const long long reorth0 = X.reorth;
      const xg_status s = gmres(c, X, dt * ai[i][i], tol, maxrs, &it, &res, st, &ge);
      if (stats) {
        stats->reorthogonalised += X.reorth - reorth0;
        stats->iterations += it;
        stats->max_iterations = std::max(stats->max_iterations, it);
        stats->solves += 1;
        stats->max_residual = std::max(stats->max_residual, res);
      }
      if (s == XG_ERR_CUDA) return fail(c, ge, "xg_step_imex gmres");
      if (s != XG_OK) return s;
      // S and L of the stage value
      e = rhs_f64_state(c, X.x, X.S[i], st);
      if (e == cudaSuccess && i < 2) e = launch_linear(c, X, X.x, 0.0, 1.0, X.L[i], st);
    }
    if (e == cudaSuccess)
      e = comb({{1.0, q}, {dt * bw[0], X.S[0]}, {dt * bw[1], X.S[1]}, {dt * bw[2], X.S[2]}}, c->Dq, n, st);
    if (e != cudaSuccess) return fail(c, e, "xg_step_imex");
    std::swap(c->A, c->Dq);
  }
  e = cudaMemcpyAsync(c->hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(c, e, "xg_step_imex");
  return *c->hflag ? XG_ERR_NONFINITE : XG_OK;
}

}  // extern "C"
