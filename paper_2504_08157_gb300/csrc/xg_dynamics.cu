// xg_dynamics.cu -- hyper-diffusion, sponge and the RI-velocity diagnostic
// (include/xg_dynamics.h).
//
// The weak Laplacian on the box is, per direction, a 1-D operator along grid
// lines: with the collocated LGL quadrature the transverse weights cancel
// against the diagonal mass (as for the right-hand side), leaving
//   (L_d q)_I = -nu_d (2/h_d)^2 / W_d(g) sum_{segments s of I} sum_l K[a_s][l] q_{s,l},
// K[a][l] = sum_k w_k D[k][a] D[k][l] the 1-D stiffness and W_d the assembled
// 1-D weight (w_a inside an element, 2 w_0 on a shared face, w_0 on a wall).
// The rows are pre-scaled by -nu_d (2/h_d)^2 / w_a, rows 0 and N by half of
// that over 2 w_0; a face node adds its two segments' rows and a wall node
// doubles its one row -- the same structure as the derivative rows of the
// right-hand side.  Hyper-diffusion applies it twice (FP64, one thread per
// node, loads along the three lines through the node) and the second pass
// adds the sponge, into the extra tendency E that the FP64 stage adds
// before the wall condition.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/xg_dynamics.h"
#include "xg_ctx.h"
#include "xg_setup.h"

namespace xg {

struct LapParams {
  int n[3], nseg[3], per[3];
  long long np;
  double Km[3][kMaxOrder + 1][kMaxOrder + 1];
};

template <int N>
__device__ __forceinline__ double line_apply(const LapParams& P, int d, const double* __restrict__ f,
                                             long long base, long long sd, int g) {
  const int nd = P.n[d], nseg = P.nseg[d];
  int s = g / N;
  if (s >= nseg) s = nseg - 1;
  const int a = g - s * N;
  double acc = 0.0;
#pragma unroll
  for (int l = 0; l <= N; ++l) {
    int k = s * N + l;
    if (k >= nd) k -= nd;
    acc = fma(P.Km[d][a][l], f[base + sd * k], acc);
  }
  if (a == 0) {
    if (s > 0 || P.per[d]) {
      const int s2 = s > 0 ? s - 1 : nseg - 1;
#pragma unroll
      for (int l = 0; l <= N; ++l) {
        int k = s2 * N + l;
        if (k >= nd) k -= nd;
        acc = fma(P.Km[d][N][l], f[base + sd * k], acc);
      }
    } else {
      acc = acc + acc;
    }
  } else if (a == N) {
    acc = acc + acc;
  }
  return acc;
}

// out = Laplacian(in) (FIRST), or out = -Laplacian(in) - gamma(z) rho w
// (second pass: in = the first pass's result, q = the state)
template <int N, bool SECOND>
__global__ void __launch_bounds__(128) k_laplace(const LapParams P, const double* __restrict__ in,
                                                 const double* __restrict__ q,
                                                 const double* __restrict__ gamma,
                                                 double* __restrict__ out) {
  const long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (I >= P.np) return;
  const long long np = P.np;
  const int nx = P.n[0], ny = P.n[1];
  const int gx = (int)(I % nx);
  const long long r = I / nx;
  const int gy = (int)(r % ny), gz = (int)(r / ny);
  const long long bx = I - gx, by = I - (long long)gy * nx, bz = I - (long long)gz * nx * ny;
#pragma unroll 1
  for (int v = 0; v < 5; ++v) {
    const double* f = in + v * np;
    double L = line_apply<N>(P, 0, f, bx, 1, gx);
    L += line_apply<N>(P, 1, f, by, nx, gy);
    L += line_apply<N>(P, 2, f, bz, (long long)nx * ny, gz);
    if (SECOND) {
      L = -L;
      if (v == 3 && gamma) L = fma(-gamma[gz], q[3 * np + I], L);
    }
    out[v * np + I] = L;
  }
}

// E = sponge only (no hyper-diffusion)
__global__ void k_sponge_only(long long np, int nxy, const double* __restrict__ q,
                              const double* __restrict__ gamma, double* __restrict__ out) {
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < 5 * np;
       I += (long long)gridDim.x * blockDim.x) {
    const long long v = I / np, J = I - v * np;
    out[I] = v == 3 ? -gamma[J / nxy] * q[I] : 0.0;
  }
}

// ------------------------------------------------------------------ RI velocity

constexpr int kRiThreads = 256;

__device__ __forceinline__ void velocity(const double* __restrict__ q, const double* __restrict__ rho0,
                                         long long np, long long I, int gz, double& u, double& v,
                                         double& w) {
  const double rho = rho0[gz] + q[I];
  u = q[np + I] / rho;
  v = q[2 * np + I] / rho;
  w = q[3 * np + I] / rho;
}

// one block per level: centroid of |u| (fixed-order tree sums)
__global__ void __launch_bounds__(kRiThreads) k_ri_centroid(const double* __restrict__ q,
                                                           const double* __restrict__ rho0,
                                                           const double* __restrict__ px,
                                                           const double* __restrict__ py, int nx,
                                                           int ny, long long np, double cx0, double cy0,
                                                           double* __restrict__ cent) {
  __shared__ double red[3][kRiThreads];
  const int gz = blockIdx.x, tid = threadIdx.x;
  const long long nxy = (long long)nx * ny;
  double s = 0.0, sx = 0.0, sy = 0.0;
  for (long long k = tid; k < nxy; k += blockDim.x) {
    const long long I = (long long)gz * nxy + k;
    double u, v, w;
    velocity(q, rho0, np, I, gz, u, v, w);
    const double sp = sqrt(u * u + v * v + w * w);
    s += sp;
    sx = fma(sp, px[k % nx], sx);
    sy = fma(sp, py[k / nx], sy);
  }
  red[0][tid] = s;
  red[1][tid] = sx;
  red[2][tid] = sy;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (tid < h)
      for (int c = 0; c < 3; ++c) red[c][tid] += red[c][tid + h];
    __syncthreads();
  }
  if (tid == 0) {
    const bool ok = red[0][0] > 0.0;
    cent[2 * gz] = ok ? red[1][0] / red[0][0] : cx0;
    cent[2 * gz + 1] = ok ? red[2][0] / red[0][0] : cy0;
  }
}

// one block per (level, strip): mean tangential speed over the strip's nodes
__global__ void __launch_bounds__(kRiThreads) k_ri_strip(const double* __restrict__ q,
                                                        const double* __restrict__ rho0,
                                                        const double* __restrict__ px,
                                                        const double* __restrict__ py, int nx, int ny,
                                                        long long np, const double* __restrict__ cent,
                                                        int nstrips, double eps,
                                                        double* __restrict__ means) {
  __shared__ double red[2][kRiThreads];
  const int gz = blockIdx.y, j = blockIdx.x, tid = threadIdx.x;
  const long long nxy = (long long)nx * ny;
  const double cx = cent[2 * gz], cy = cent[2 * gz + 1];
  double s = 0.0, cnt = 0.0;
  for (long long k = tid; k < nxy; k += blockDim.x) {
    const double rx = px[k % nx] - cx, ry = py[k / nx] - cy;
    const double r = sqrt(rx * rx + ry * ry);
    if ((long long)floor(r / eps) != j) continue;
    const long long I = (long long)gz * nxy + k;
    double u, v, w;
    velocity(q, rho0, np, I, gz, u, v, w);
    const double erx = r > 0.0 ? rx / r : 0.0, ery = r > 0.0 ? ry / r : 0.0;
    const double ur = u * erx + v * ery;
    const double tx = u - ur * erx, ty = v - ur * ery;
    s += sqrt(tx * tx + ty * ty);
    cnt += 1.0;
  }
  red[0][tid] = s;
  red[1][tid] = cnt;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (tid < h) {
      red[0][tid] += red[0][tid + h];
      red[1][tid] += red[1][tid + h];
    }
    __syncthreads();
  }
  if (tid == 0) means[(long long)gz * nstrips + j] = red[1][0] > 0.0 ? red[0][0] / red[1][0] : 0.0;
}

}  // namespace xg

using xg::LapParams;

namespace {

xg_status status_of(xg_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return XG_OK;
  fprintf(stderr, "xg_dynamics: %s: %s\n", where, cudaGetErrorString(e));
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return XG_ERR_OOM;
  c->failed = true;
  return XG_ERR_CUDA;
}

// Global node positions along direction d (the mesh's own formula).
std::vector<double> axis_positions(const xg_ctx* c, int d) {
  const int N = c->d.order;
  long double xi[xg::kMaxOrder + 1];
  xg::lgl_nodes(N, xi);
  const double h = (c->d.hi[d] - c->d.lo[d]) / c->d.nel[d];
  std::vector<double> p(c->n[d]);
  for (int g = 0; g < c->n[d]; ++g) {
    const int e = std::min(g / N, c->d.nel[d] - 1);
    const int a = g - N * e;
    p[g] = c->d.lo[d] + ((double)e + (double)((xi[a] + 1.0L) / 2.0L)) * h;
  }
  return p;
}

template <int N>
void launch_lap(const LapParams& P, const double* q, double* L1, const double* gamma, double* E,
                bool hyper, cudaStream_t st) {
  const unsigned blocks = (unsigned)((P.np + 127) / 128);
  if (hyper) {
    xg::k_laplace<N, false><<<blocks, 128, 0, st>>>(P, q, nullptr, nullptr, L1);
    xg::k_laplace<N, true><<<blocks, 128, 0, st>>>(P, L1, q, gamma, E);
  } else {
    const int nxy = P.n[0] * P.n[1];
    xg::k_sponge_only<<<(unsigned)std::min<long long>((5 * P.np + 255) / 256, 65535), 256, 0, st>>>(
        P.np, nxy, q, gamma, E);
  }
}

}  // namespace

// Called by the FP64 stage before its line kernels: E = H(q) + sponge(q).
cudaError_t dynamics_launch(xg_ctx* c, const double* q, cudaStream_t st) {
  const LapParams& P = *static_cast<const LapParams*>(c->dyn_params);
  const bool hyper = c->dyn_hyper;
  switch (c->d.order) {
    case 1: launch_lap<1>(P, q, c->dyn_L1, c->dyn_gamma, c->dyn_E, hyper, st); break;
    case 2: launch_lap<2>(P, q, c->dyn_L1, c->dyn_gamma, c->dyn_E, hyper, st); break;
    case 3: launch_lap<3>(P, q, c->dyn_L1, c->dyn_gamma, c->dyn_E, hyper, st); break;
    case 4: launch_lap<4>(P, q, c->dyn_L1, c->dyn_gamma, c->dyn_E, hyper, st); break;
    case 5: launch_lap<5>(P, q, c->dyn_L1, c->dyn_gamma, c->dyn_E, hyper, st); break;
    case 6: launch_lap<6>(P, q, c->dyn_L1, c->dyn_gamma, c->dyn_E, hyper, st); break;
    case 7: launch_lap<7>(P, q, c->dyn_L1, c->dyn_gamma, c->dyn_E, hyper, st); break;
    case 8: launch_lap<8>(P, q, c->dyn_L1, c->dyn_gamma, c->dyn_E, hyper, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

void dynamics_free(xg_ctx* c) {
  cudaFree(c->dyn_L1);
  cudaFree(c->dyn_E);
  cudaFree(c->dyn_gamma);
  delete static_cast<LapParams*>(c->dyn_params);
  c->dyn_L1 = c->dyn_E = c->dyn_gamma = nullptr;
  c->dyn_params = nullptr;
  c->dyn = c->dyn_hyper = false;
}

extern "C" {

xg_status xg_set_dynamics(xg_ctx* c, const xg_dynamics* dyn) {
  if (!c) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (!dyn) {
    c->dyn = false;
    return XG_OK;
  }
  if (c->dfm || c->f32) return XG_ERR_UNSUPPORTED;
  if (c->part_open[0] || c->part_open[1]) return XG_ERR_UNSUPPORTED;   // partitioned contexts
  const double H = c->d.hi[2] - c->d.lo[2];
  bool hyper = false;
  for (int k = 0; k < 3; ++k) {
    if (!(dyn->hyper_c[k] >= 0.0) || !std::isfinite(dyn->hyper_c[k])) return XG_ERR_ARG;
    hyper |= dyn->hyper_c[k] > 0.0;
  }
  if (hyper && !(dyn->hyper_dt > 0.0 && std::isfinite(dyn->hyper_dt))) return XG_ERR_ARG;
  if (!(dyn->sponge_depth >= 0.0 && dyn->sponge_depth <= H)) return XG_ERR_ARG;
  if (!(dyn->sponge_gamma >= 0.0 && std::isfinite(dyn->sponge_gamma))) return XG_ERR_ARG;
  const bool sponge = dyn->sponge_depth > 0.0 && dyn->sponge_gamma > 0.0;

  const int N = c->d.order;
  LapParams* P = static_cast<LapParams*>(c->dyn_params);
  if (!P) {
    P = new (std::nothrow) LapParams();
    if (!P) return XG_ERR_OOM;
    c->dyn_params = P;
  }
  memset(P, 0, sizeof(*P));
  for (int k = 0; k < 3; ++k) {
    P->n[k] = c->n[k];
    P->nseg[k] = c->d.nel[k];
    P->per[k] = c->d.periodic[k] ? 1 : 0;
  }
  P->np = c->np;
  // principal axes: descending element size, x, y, z on ties
  double h[3];
  int order[3] = {0, 1, 2};
  for (int k = 0; k < 3; ++k) h[k] = (c->d.hi[k] - c->d.lo[k]) / c->d.nel[k];
  std::stable_sort(order, order + 3, [&](int a, int b) { return h[a] > h[b]; });
  double nu[3];
  for (int i = 0; i < 3; ++i) {
    const int d = order[i];
    const double dx = h[d] / N;
    nu[d] = hyper ? std::sqrt(dyn->hyper_c[i]) * dx * dx / std::sqrt(dyn->hyper_dt) : 0.0;
  }
  double D[xg::kMaxOrder + 1][xg::kMaxOrder + 1], w[xg::kMaxOrder + 1];
  xg::lgl_derivative(N, D);
  xg::lgl_weights(N, w);
  for (int d = 0; d < 3; ++d) {
    const double s = -nu[d] * (2.0 / h[d]) * (2.0 / h[d]);
    for (int a = 0; a <= N; ++a) {
      const double wa = (a == 0 || a == N) ? 2.0 * w[0] : w[a];
      for (int l = 0; l <= N; ++l) {
        long double K = 0.0L;
        for (int k = 0; k <= N; ++k) K += (long double)w[k] * D[k][a] * D[k][l];
        P->Km[d][a][l] = (double)(s * (double)K / wa);
      }
    }
  }
  cudaError_t e = cudaSuccess;
  const size_t vec = sizeof(double) * 5 * (size_t)c->np;
  if (!c->dyn_L1) e = cudaMalloc((void**)&c->dyn_L1, vec);
  if (e == cudaSuccess && !c->dyn_E) e = cudaMalloc((void**)&c->dyn_E, vec);
  if (e == cudaSuccess && !c->dyn_gamma) e = cudaMalloc((void**)&c->dyn_gamma, sizeof(double) * c->n[2]);
  if (e == cudaSuccess) {
    const std::vector<double> z = axis_positions(c, 2);
    std::vector<double> g(c->n[2], 0.0);
    if (sponge) {
      const double zs = c->d.hi[2] - dyn->sponge_depth;
      const double pi = 3.14159265358979323846;
      for (int k = 0; k < c->n[2]; ++k) {
        if (z[k] > zs) {
          const double sn = std::sin(0.5 * pi * std::min(1.0, (z[k] - zs) / dyn->sponge_depth));
          g[k] = dyn->sponge_gamma * sn * sn;
        }
      }
    }
    e = cudaMemcpy(c->dyn_gamma, g.data(), sizeof(double) * c->n[2], cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    dynamics_free(c);
    return status_of(c, e, "xg_set_dynamics");
  }
  c->dyn_hyper = hyper;
  c->dyn = hyper || sponge;
  return XG_OK;
}

xg_status xg_dynamics_tendency(xg_ctx* c, double* out, int where, void* stream) {
  if (!c || !out) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (c->dfm || c->f32) return XG_ERR_UNSUPPORTED;
  if (!c->has_state || (where != XG_HOST && where != XG_DEVICE)) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * 5 * (size_t)c->np;
  cudaError_t e;
  if (!c->dyn) {
    e = where == XG_DEVICE ? cudaMemsetAsync(out, 0, bytes, st) : cudaSuccess;
    if (where == XG_HOST) memset(out, 0, bytes);
    return status_of(c, e, "xg_dynamics_tendency");
  }
  e = dynamics_launch(c, c->A, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, c->dyn_E, bytes, where == XG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        st);
  if (e == cudaSuccess && where == XG_HOST) e = cudaStreamSynchronize(st);
  return status_of(c, e, "xg_dynamics_tendency");
}

xg_status xg_ri_velocity(xg_ctx* c, int nstrips, double* u_ri, double* centroid, double* means,
                         void* stream) {
  if (!c || !u_ri || nstrips < 1 || nstrips > 1024) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (!c->has_state) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
  const long long np = c->np;
  double *q = nullptr, *px = nullptr, *py = nullptr, *r0 = nullptr, *cent = nullptr, *mn = nullptr;
  cudaError_t e = cudaMalloc((void**)&q, sizeof(double) * 5 * (size_t)np);
  if (e == cudaSuccess) e = cudaMalloc((void**)&px, sizeof(double) * (nx + ny + nz));
  if (e == cudaSuccess) e = cudaMalloc((void**)&cent, sizeof(double) * 2 * nz);
  if (e == cudaSuccess) e = cudaMalloc((void**)&mn, sizeof(double) * (size_t)nz * nstrips);
  std::vector<double> hcent(2 * (size_t)nz), hmean((size_t)nz * nstrips);
  if (e == cudaSuccess) {
    py = px + nx;
    r0 = py + ny;
    const std::vector<double> ax = axis_positions(c, 0), ay = axis_positions(c, 1);
    // rho_0 per level: the reference table's first row (FP64, or double-float pairs)
    std::vector<double> hb(4 * (size_t)nz), rho0(nz);
    e = cudaMemcpy(hb.data(), c->base, sizeof(double) * 4 * nz, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
      for (int k = 0; k < nz; ++k) {
        if (c->dfm || c->f32) {
          xg::df v;
          memcpy(&v, &hb[k], sizeof(v));
          rho0[k] = (double)v.h + (double)v.l;
        } else {
          rho0[k] = hb[k];
        }
      }
      e = cudaMemcpy(px, ax.data(), sizeof(double) * nx, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(py, ay.data(), sizeof(double) * ny, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r0, rho0.data(), sizeof(double) * nz, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    const xg_status s = xg_get_state(c, q, XG_DEVICE, stream);
    if (s != XG_OK) e = cudaErrorUnknown;
  }
  if (e == cudaSuccess) {
    const double cx0 = 0.5 * (c->d.lo[0] + c->d.hi[0]), cy0 = 0.5 * (c->d.lo[1] + c->d.hi[1]);
    const double R = 0.5 * std::min(c->d.hi[0] - c->d.lo[0], c->d.hi[1] - c->d.lo[1]);
    xg::k_ri_centroid<<<nz, xg::kRiThreads, 0, st>>>(q, r0, px, py, nx, ny, np, cx0, cy0, cent);
    xg::k_ri_strip<<<dim3(nstrips, nz), xg::kRiThreads, 0, st>>>(q, r0, px, py, nx, ny, np, cent, nstrips,
                                                                  R / nstrips, mn);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hcent.data(), cent, sizeof(double) * 2 * nz, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hmean.data(), mn, sizeof(double) * hmean.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(q);
  cudaFree(px);
  cudaFree(cent);
  cudaFree(mn);
  if (e != cudaSuccess) return status_of(c, e, "xg_ri_velocity");
  double best = 0.0;
  for (double v : hmean) best = std::max(best, v);
  *u_ri = best;
  if (centroid) memcpy(centroid, hcent.data(), sizeof(double) * hcent.size());
  if (means) memcpy(means, hmean.data(), sizeof(double) * hmean.size());
  return XG_OK;
}

}  // extern "C"
