// xg_plane_f32.cuh -- FP32 precision form: the x and y passes fused into one
// kernel over element-aligned tiles of one z-level.
//
// A CTA owns up to TS x TS nodes of a level (TS = N E: E elements per side;
// the last tile of a walled direction also owns the wall node).  It loads the
// state of a cross-shaped region -- its own rows extended by the N columns
// before them and the one after (the x segments), and its own columns
// extended likewise (the y segments) -- computes the primitives (u, v, w,
// p') once per loaded node and keeps the x-fluxes and y-fluxes in shared
// memory.  Each thread then evaluates its own nodes' x and y parts straight
// from those tiles: an element-interior node one row of its segment, a face
// node row 0 of its segment plus row N of the segment before (FP32 FMAs are
// cheap next to the HBM traffic this kernel moves), and writes T = x part +
// y part and W = (v, w, p') for the z pass.  Compared with separate x and y
// passes this saves the y pass's re-reads of q and W and its
// read-modify-write of T.
#pragma once

#include <cuda_runtime.h>

#include "xg_kernels_f32.cuh"

namespace xg {

__host__ __device__ constexpr int plane_elems_f32(int N) { return N >= 32 ? 1 : 32 / N; }
// 256 threads, 3 cross-region nodes per thread and pass (measured on the
// 128x128x16 order-4 box: 0.342 ms per launch, against 0.351 with 2 nodes and
// 0.365 / 0.422 / 0.496 ms with 384 / 512 / 128 threads)
constexpr int kPlaneThreads = 256;
constexpr int kPlaneBatch = 3;

// Shared-memory layout of a tile of E x E elements (floats), see f_plane_tile.
// a / b for 0 <= a < 2^22 and 1 <= b <= 64 from a float reciprocal (the
// tile index arithmetic; exact: the quotient estimate is corrected once)
__device__ __forceinline__ int small_div(int a, int b, float rb) {
  int q = (int)((float)a * rb);
  const int r = a - q * b;
  if (r < 0) --q;
  else if (r >= b) ++q;
  return q;
}

template <int N, int E_ = plane_elems_f32(N)>
struct PlaneLayoutF {
  static constexpr int E = E_;
  static constexpr int TS = E * N;
  static constexpr int LO = TS + 1;          // owned extent across the line (wall node included)
  static constexpr int LX = TS + N + 1;      // loaded extent along the line
  static constexpr int FX = 5 * LO * LX;     // x-fluxes [5][LO][LX]
  static constexpr int FY = 5 * LX * LO;     // y-fluxes [5][LX][LO]
  static constexpr int total = FX + FY;
  static constexpr size_t bytes = sizeof(float) * (size_t)total;
};

// Extent of tile (bx, by): its first element and node along x and y, the
// elements it owns, the owned node extents ox, oy (the wall node of a
// walled end included) and whether the segment before each direction's
// first node exists (interior tile, or periodic).
struct PlaneTile {
  int ekx, eky, x0, y0, ox, oy;
  bool wallx, wally, hxl, hyl;
  template <int N, int E>
  __device__ __forceinline__ void init(const FParams& P, int bx, int by) {
    const int ex0 = bx * E, ey0 = by * E;
    ekx = min(E, P.nseg[0] - ex0);
    eky = min(E, P.nseg[1] - ey0);
    x0 = ex0 * N;
    y0 = ey0 * N;
    wallx = !P.per[0] && ex0 + ekx == P.nseg[0];
    wally = !P.per[1] && ey0 + eky == P.nseg[1];
    ox = ekx * N + (wallx ? 1 : 0);
    oy = eky * N + (wally ? 1 : 0);
    hxl = ex0 > 0 || P.per[0];
    hyl = ey0 > 0 || P.per[1];
  }
};

// The pointwise phase of tile T of level z: the primitives of every node of
// the cross-shaped region, W = (v, w, p') of the owned nodes, and the fluxes
// handed to fxs(j, ii, F[5]) (x-fluxes of owned row j at ii = i + N) and
// fys(jj, i, F[5]) (y-fluxes of owned column i at jj = j + N).  With THETA,
// slot 4 holds theta = Theta / rho instead of the Theta' flux, for the
// difference form of the contraction (f_drows).
template <int N, int BATCH, bool CG, bool THETA, typename StoreX, typename StoreY>
__device__ __forceinline__ void f_plane_pointwise(const FParams& P, const FBufs& B, const PlaneTile& T, int z,
                                                  int tid, int nthr, StoreX fxs, StoreY fys) {
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const int ekx = T.ekx, eky = T.eky, x0 = T.x0, y0 = T.y0, ox = T.ox, oy = T.oy;
  const bool hxl = T.hxl, hyl = T.hyl;
  const long long np = P.np;
  const long long zoff = (long long)nx * ny * z;
  const df rho0d = B.base[z], Th0d = B.base[nz + z], p0 = B.base[2 * nz + z];
  const df iTh0 = B.base[3 * nz + z];
  const float rho0 = rho0d.h + rho0d.l, Th0 = Th0d.h + Th0d.l;
  const float* __restrict__ q = B.q;
  float* __restrict__ Wo = B.W;

  // ---- pointwise over the cross: local (i, j) with i in [-N, ekx N] and
  // j in [-N, eky N]; x-fluxes on owned rows (i extended by the segment
  // before and the end face), y-fluxes on owned columns (j likewise).  The
  // cross is enumerated as the owned rows at full width, then the owned
  // columns of the rows above and below them.
  // Each thread takes BATCH items per pass and issues all their loads
  // before any arithmetic, to keep enough bytes in flight.
  const int wx = ekx * N + N + 1, wy = eky * N + N + 1;
  const int nrow = oy * wx;                       // owned rows, full width
  const int nitem = nrow + ox * (wy - oy);        // + owned columns, remaining rows
  const float rwx = 1.0f / (float)wx, rox = 1.0f / (float)ox;
  for (int base = tid; base < nitem; base += BATCH * nthr) {
    int ib[BATCH], jb[BATCH];
    long long Ib[BATCH];
    float qb[BATCH][5];
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const int idx = base + u * nthr;
      int i = -N - 1, j = 0;                      // i = -N - 1 marks "nothing to do"
      if (idx < nrow) {
        j = small_div(idx, wx, rwx);
        i = idx - j * wx - N;
      } else if (idx < nitem) {
        const int r = small_div(idx - nrow, ox, rox);
        i = (idx - nrow) - r * ox;
        j = r < N ? r - N : oy + (r - N);          // N rows before, then the rows after
      }
      const bool needx = j >= 0 && j < oy && (i >= 0 || hxl) && i >= -N;
      const bool needy = i >= 0 && i < ox && (j >= 0 || hyl);
      if (!needx && !needy) i = -N - 1;
      ib[u] = i;
      jb[u] = j;
      int gx = x0 + i, gy = y0 + j;
      if (gx < 0) gx += nx;                       // only reached when periodic (hxl)
      if (gy < 0) gy += ny;
      if (gx >= nx) gx -= nx;                     // the periodic end face
      if (gy >= ny) gy -= ny;
      Ib[u] = zoff + gx + (long long)nx * gy;
      if (i >= -N) {
#pragma unroll
        for (int c = 0; c < 5; ++c) qb[u][c] = ldf<CG>(q + c * np + Ib[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const int i = ib[u], j = jb[u];
      if (i < -N) continue;
      const long long I = Ib[u];
      const float mu = qb[u][1], mv = qb[u][2], mw = qb[u][3], tp = qb[u][4];
      const float ir = __frcp_rn(rho0 + qb[u][0]);
      const float u_ = mu * ir, v = mv * ir, w = mw * ir;
      const float pp = f_pressure_pert(P, tp, p0, iTh0);
      const float Th = Th0 + tp;
      const bool inx = i >= 0 && i < ox;
      const bool iny = j >= 0 && j < oy;
      if (inx && iny) {
        Wo[I] = v;
        Wo[np + I] = w;
        Wo[2 * np + I] = pp;
      }
      const float th = Th * ir;
      if (iny) {                                  // x-fluxes on owned rows
        const float F[5] = {mu, fmaf(mu, u_, pp), mv * u_, mw * u_, THETA ? th : Th * u_};
        fxs(j, i + N, F);
      }
      if (inx) {                                  // y-fluxes on owned columns
        const float F[5] = {mv, mu * v, fmaf(mv, v, pp), mw * v, THETA ? th : Th * v};
        fys(j + N, i, F);
      }
    }
  }
}

// The x part + y part of the owned node (i, j) of tile T from its flux
// tiles, fx(c, j, i + N) and fy(c, j + N, i) (slot 4: theta): an element-
// interior node takes one row of its segment, a face node row 0 of its
// segment plus row N of the segment before, a wall node its one-sided row
// twice; rho' and Theta' in difference form (f_drows).
template <int N, typename FXs, typename FYs>
__device__ __forceinline__ void f_plane_node_xy(const FParams& P, const PlaneTile& T, FXs fx, FYs fy, int i, int j,
                                                float (&t)[5]) {
  const int ekx = T.ekx, eky = T.eky;
  const bool hxl = T.hxl, hyl = T.hyl;
  const int sx = min(i / N, ekx - 1), ax = i - sx * N;   // the wall node is row N of the last
  const int sy = min(j / N, eky - 1), ay = j - sy * N;
  {   // rho' and Theta' in difference form (slot 0: rho u_d, slot 4: theta)
    float m[N + 1], th[N + 1], v0 = 0.0f, v4 = 0.0f, w0 = 0.0f, w4 = 0.0f;
#pragma unroll
    for (int l = 0; l <= N; ++l) {
      m[l] = fx(0, j, N + sx * N + l);
      th[l] = fx(4, j, N + sx * N + l);
    }
    f_drows<N, 0>(P, ax, m, th, v0, v4);
    if (ax == 0 || ax == N) {
      if (ax == 0 && (sx > 0 || hxl)) {
#pragma unroll
        for (int l = 0; l <= N; ++l) {
          m[l] = fx(0, j, sx * N + l);
          th[l] = fx(4, j, sx * N + l);
        }
        f_drows<N, 0>(P, N, m, th, v0, v4);
      } else {
        v0 = v0 + v0;
        v4 = v4 + v4;
      }
    }
#pragma unroll
    for (int l = 0; l <= N; ++l) {
      m[l] = fy(0, N + sy * N + l, i);
      th[l] = fy(4, N + sy * N + l, i);
    }
    f_drows<N, 1>(P, ay, m, th, w0, w4);
    if (ay == 0 || ay == N) {
      if (ay == 0 && (sy > 0 || hyl)) {
#pragma unroll
        for (int l = 0; l <= N; ++l) {
          m[l] = fy(0, sy * N + l, i);
          th[l] = fy(4, sy * N + l, i);
        }
        f_drows<N, 1>(P, N, m, th, w0, w4);
      } else {
        w0 = w0 + w0;
        w4 = w4 + w4;
      }
    }
    t[0] = v0 + w0;
    t[4] = v4 + w4;
  }
#pragma unroll
  for (int c = 1; c < 4; ++c) {
    float f[N + 1], v = 0.0f;
#pragma unroll
    for (int l = 0; l <= N; ++l) f[l] = fx(c, j, N + sx * N + l);
    v = f_row_from<N, 0>(P, ax, f, v);
    if (ax == 0 || ax == N) {
      if (ax == 0 && (sx > 0 || hxl)) {
#pragma unroll
        for (int l = 0; l <= N; ++l) f[l] = fx(c, j, sx * N + l);
        v = f_row_from<N, 0>(P, N, f, v);
      } else {
        v = v + v;                                  // wall: the one-sided row counts twice
      }
    }
#pragma unroll
    for (int l = 0; l <= N; ++l) f[l] = fy(c, N + sy * N + l, i);
    float w = f_row_from<N, 1>(P, ay, f, 0.0f);
    if (ay == 0 || ay == N) {
      if (ay == 0 && (sy > 0 || hyl)) {
#pragma unroll
        for (int l = 0; l <= N; ++l) f[l] = fy(c, sy * N + l, i);
        w = f_row_from<N, 1>(P, N, f, w);
      } else {
        w = w + w;
      }
    }
    t[c] = v + w;
  }
}

// One tile (bx, by) of level z, run by threads tid = 0 .. nthr-1 of the
// block; sm holds PlaneLayoutF<N, E>::bytes.  CG: L2-only loads of q (see
// ldf).  The block synchronises once, between the pointwise and the
// contraction phases; the caller synchronises before reusing sm.
template <int N, int E, int BATCH, bool CG>
__device__ __forceinline__ void f_plane_tile(const FParams& P, const FBufs& B, int bx, int by, int z,
                                             float* sm_plane, int tid, int nthr) {
  using L = PlaneLayoutF<N, E>;
  constexpr int LO = L::LO, LX = L::LX;
  float* FX = sm_plane;                   // [c][j][i + N]
  float* FY = FX + L::FX;                 // [c][j + N][i]
  auto fx = [&](int c, int j, int ii) -> float& { return FX[(c * LO + j) * LX + ii]; };
  auto fy = [&](int c, int jj, int i) -> float& { return FY[(c * LX + jj) * LO + i]; };

  PlaneTile T;
  T.init<N, E>(P, bx, by);
  f_plane_pointwise<N, BATCH, CG, true>(
      P, B, T, z, tid, nthr,
      [&](int j, int ii, const float (&F)[5]) {
#pragma unroll
        for (int c = 0; c < 5; ++c) fx(c, j, ii) = F[c];
      },
      [&](int jj, int i, const float (&F)[5]) {
#pragma unroll
        for (int c = 0; c < 5; ++c) fy(c, jj, i) = F[c];
      });
  __syncthreads();

  const int nx = P.n[0], ny = P.n[1];
  const int x0 = T.x0, y0 = T.y0, ox = T.ox, oy = T.oy;
  const long long np = P.np;
  const long long zoff = (long long)nx * ny * z;
  const float rox = 1.0f / (float)ox;
  float* __restrict__ To = B.T;

  // ---- each owned node: x part + y part from the flux tiles
  for (int idx = tid; idx < ox * oy; idx += nthr) {
    const int j = small_div(idx, ox, rox), i = idx - j * ox;
    const long long I = zoff + (x0 + i) + (long long)nx * (y0 + j);
    float t[5];
    f_plane_node_xy<N>(P, T, fx, fy, i, j, t);
#pragma unroll
    for (int c = 0; c < 5; ++c) To[c * np + I] = t[c];
  }
}

template <int N>
__global__ void __launch_bounds__(kPlaneThreads) k_f_plane_xy(const FParams P, const FBufs B) {
  extern __shared__ float sm_plane[];
  f_plane_tile<N, plane_elems_f32(N), kPlaneBatch, false>(P, B, blockIdx.x, blockIdx.y, blockIdx.z,
                                                           sm_plane, threadIdx.x, blockDim.x);
}

}  // namespace xg
