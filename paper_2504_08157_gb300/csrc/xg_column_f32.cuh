// xg_column_f32.cuh -- FP32 precision form: the whole pass (x, y and z
// contractions, sources, walls, the SSP-RK3 stage) in one kernel that marches
// a column of E x E elements up through the levels, for order N = 4 on boxes
// with walls at the bottom and top.
//
// Per level z the CTA stages the state of its cross-shaped region (its own
// nodes, the N columns before them and the end face, in both x and y) in
// shared memory, computes the primitives once per staged node, the x- and
// y-fluxes and -- for its own nodes -- the z-fluxes, and assembles the x and
// y parts of every own node (f_plane_node_xy, the arithmetic of the plane
// kernel).  The z-fluxes and x + y parts of the N + 1 levels of the current
// z segment are kept in a ring of N + 1 level slots (level z in slot
// z mod (N + 1); consecutive segments share their face level, whose slot
// they share).  When a segment's last level is done, every own node of its
// levels gets its z part (difference form for rho' and Theta', as the z tile
// kernel), a face level adds row N of the segment below (kept per node from
// the previous segment), and the stage is finished and stored.  So W (v, w,
// p') and the partial tendency T never leave the chip: the pass reads q (and
// q^n, S, the closure correction C) and writes the stage output, its
// algorithmic traffic.
//
// Staging by TMA.  When the row pitch allows it (n_x a multiple of 4: every
// stride a multiple of 16 bytes), the state of a level is one
// cp.async.bulk.tensor load of a 24 x 21 x 1 x 5 box of the 4-D view
// [5][n_z][n_y][n_x] at (x0 - N, y0 - N, z, 0) -- x0 - N is a multiple of 4
// floats, so the innermost coordinate is 16-byte aligned -- into one of two
// buffers, issued one level ahead and completed on that buffer's mbarrier.
// Values across a periodic end (coordinates outside the array, which the
// load fills with zeros) are then fetched with ordinary loads.  Other pitches
// stage the same box with ordinary loads.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "xg_plane_f32.cuh"
#include "xg_tma.cuh"

namespace xg {

constexpr int kColThreads = 512;

struct ColLayout {
  static constexpr int N = 4, E = 4;
  static constexpr int TS = E * N;             // 16 nodes per tile side, the end face apart
  static constexpr int LO = TS + 1;            // own extent across a line (a wall node included)
  static constexpr int LX = TS + N + 1;        // staged extent along a line: 21
  static constexpr int OWN = LO * LO;          // own nodes of a level, at most: 289
  static constexpr int QX = 24;                // staged x extent (a multiple of 4 floats)
  static constexpr int QV = QX * LX;           // staged floats of one variable: 504
  static constexpr int QB = 5 * QV;            // staged floats of a level: 2520 (10,080 bytes)
  static constexpr int QBP = 2528;             // buffer pitch: 128-byte aligned
  static constexpr int SLOTS = N + 1;          // level slots of the ring
  // float offsets
  static constexpr int OFF_Q = 0;                          // [2][5][LX][QX]
  static constexpr int OFF_FX = 2 * QBP;                   // x-fluxes [5][LO][LX]
  static constexpr int OFF_FY = OFF_FX + 5 * LO * LX;      // y-fluxes [5][LX][LO]
  static constexpr int OFF_ZF = OFF_FY + 5 * LX * LO;      // z-fluxes [SLOTS][5][OWN]
  static constexpr int OFF_TX = OFF_ZF + SLOTS * 5 * OWN;  // x + y parts [SLOTS][5][OWN]
  static constexpr int OFF_PV = OFF_TX + SLOTS * 5 * OWN;  // row N of the segment below [2][5][OWN]
  static constexpr int OFF_BAR = OFF_PV + 2 * 5 * OWN;     // two mbarriers (8-byte aligned)
  static constexpr size_t bytes = sizeof(float) * (size_t)OFF_BAR + 16;
  static constexpr uint32_t TX_BYTES = sizeof(float) * QB; // one staged level
};
static_assert((ColLayout::QBP * 4) % 128 == 0 && ColLayout::QBP >= ColLayout::QB, "staging buffers 128-byte aligned");
static_assert((ColLayout::OFF_BAR * 4) % 8 == 0, "mbarrier alignment");
static_assert(ColLayout::QX >= ColLayout::LX && ColLayout::QX % 4 == 0, "staged rows cover the loaded extent");
static_assert(2 * (ColLayout::bytes + 1024) <= 233472, "two CTAs per SM");

// Staged value of variable c at local node (i, j) of the level in buffer st
// (i, j in [-N, TS]).
__device__ __forceinline__ float& col_q(float* st, int c, int i, int j) {
  using L = ColLayout;
  return st[c * L::QV + (j + L::N) * L::QX + (i + L::N)];
}

// Ordinary loads of the staged box of level z (all of it when `all`, else
// only the entries across a periodic end), wrapping periodic directions and
// skipping nodes outside the box of the mesh.
__device__ __forceinline__ void col_stage_plain(const FParams& P, const float* __restrict__ q, const PlaneTile& T,
                                                int z, float* st, bool all, int tid, int nthr) {
  using L = ColLayout;
  const int nx = P.n[0], ny = P.n[1];
  const long long np = P.np;
  const long long zoff = (long long)nx * ny * z;
  for (int k = tid; k < L::LX * L::LX; k += nthr) {
    const int jj = k / L::LX, ii = k - jj * L::LX;
    int gx = T.x0 - L::N + ii, gy = T.y0 - L::N + jj;
    const bool outx = gx < 0 || gx >= nx, outy = gy < 0 || gy >= ny;
    if (!all && !(outx && P.per[0]) && !(outy && P.per[1])) continue;
    if (outx) {
      if (!P.per[0]) continue;
      gx += gx < 0 ? nx : -nx;
    }
    if (outy) {
      if (!P.per[1]) continue;
      gy += gy < 0 ? ny : -ny;
    }
    const long long I = zoff + gx + (long long)nx * gy;
#pragma unroll
    for (int c = 0; c < 5; ++c) st[c * L::QV + jj * L::QX + ii] = q[c * np + I];
  }
}

// The pointwise phase of level z from the staged state: for every node of the
// cross-shaped region the primitives; the x-fluxes of own rows into FX, the
// y-fluxes of own columns into FY, and the z-fluxes of own nodes into ZS
// (slot 4 of each: theta = Theta / rho, for the difference form).
__device__ __forceinline__ void col_pointwise(const FParams& P, const FBufs& B, const PlaneTile& T, int z,
                                              const float* st, float* FX, float* FY, float* ZS, int tid,
                                              int nthr) {
  using L = ColLayout;
  constexpr int N = L::N, LO = L::LO, LX = L::LX;
  const int nz = P.n[2];
  const int ekx = T.ekx, eky = T.eky, ox = T.ox, oy = T.oy;
  const bool hxl = T.hxl, hyl = T.hyl;
  const df rho0d = B.base[z], Th0d = B.base[nz + z], p0 = B.base[2 * nz + z];
  const df iTh0 = B.base[3 * nz + z];
  const float rho0 = rho0d.h + rho0d.l, Th0 = Th0d.h + Th0d.l;
  const int wx = ekx * N + N + 1, wy = eky * N + N + 1;
  const int nrow = oy * wx;                       // own rows, full width
  const int nitem = nrow + ox * (wy - oy);        // + own columns, remaining rows
  const float rwx = 1.0f / (float)wx, rox = 1.0f / (float)ox;
  for (int idx = tid; idx < nitem; idx += nthr) {
    int i, j;
    if (idx < nrow) {
      j = small_div(idx, wx, rwx);
      i = idx - j * wx - N;
    } else {
      const int r = small_div(idx - nrow, ox, rox);
      i = (idx - nrow) - r * ox;
      j = r < N ? r - N : oy + (r - N);            // N rows before, then the rows after
    }
    const bool iny = j >= 0 && j < oy, inx = i >= 0 && i < ox;
    const bool needx = iny && (i >= 0 || hxl);
    const bool needy = inx && (j >= 0 || hyl);
    if (!needx && !needy) continue;
    const float* s = st + (j + N) * L::QX + (i + N);
    const float q0 = s[0], mu = s[L::QV], mv = s[2 * L::QV], mw = s[3 * L::QV], tp = s[4 * L::QV];
    const float ir = __frcp_rn(rho0 + q0);
    const float u_ = mu * ir, v = mv * ir, w = mw * ir;
    const float pp = f_pressure_pert(P, tp, p0, iTh0);
    const float th = (Th0 + tp) * ir;
    if (needx) {
      float* f = FX + j * LX + (i + N);
      f[0] = mu;
      f[LO * LX] = fmaf(mu, u_, pp);
      f[2 * LO * LX] = mv * u_;
      f[3 * LO * LX] = mw * u_;
      f[4 * LO * LX] = th;
    }
    if (needy) {
      float* f = FY + (j + N) * LO + i;
      f[0] = mv;
      f[LX * LO] = mu * v;
      f[2 * LX * LO] = fmaf(mv, v, pp);
      f[3 * LX * LO] = mw * v;
      f[4 * LX * LO] = th;
    }
    if (inx && iny) {
      float* f = ZS + j * LO + i;
      f[0] = mw;
      f[L::OWN] = mu * w;
      f[2 * L::OWN] = mv * w;
      f[3 * L::OWN] = fmaf(mw, w, pp);
      f[4 * L::OWN] = th;
    }
  }
}

// The z part and the stage of the own nodes of z segment s (levels s N ..
// s N + N - 1, and the top wall level s N + N when s is the last segment)
// from the ring: item (node, level) per thread.  A face level s N adds row N
// of segment s - 1 (PVo, kept from that segment's finish) to its row 0, or
// doubles row 0 at the bottom wall; the top wall level takes row N twice.
// Row N of this segment is kept in PVn for the next one.
__device__ __forceinline__ void col_finish_segment(const FParams& P, const FBufs& B, const PlaneTile& T, int s,
                                                   const float* ZF, const float* TX, const float* PVo, float* PVn,
                                                   int tid, int nthr) {
  using L = ColLayout;
  constexpr int N = L::N, OWN = L::OWN;
  const int nx = P.n[0], ny = P.n[1], nseg = P.nseg[2];
  const long long np = P.np;
  const int ox = T.ox, oy = T.oy, nown = ox * oy;
  const int nl = s == nseg - 1 ? N + 1 : N;      // levels finished here (the top wall in the last)
  const float rox = 1.0f / (float)ox;
  bool bad = false;
  for (int idx = tid; idx < nl * nown; idx += nthr) {
    const int a = idx / nown, node = idx - a * nown;
    const int j = small_div(node, ox, rox), i = node - j * ox;
    const int k = j * L::LO + i;
    const int zl = s * N + a;
    const float* zs[N + 1];
#pragma unroll
    for (int l = 0; l <= N; ++l) zs[l] = ZF + ((s * N + l) % L::SLOTS) * 5 * OWN + k;
    const float* tx = TX + (zl % L::SLOTS) * 5 * OWN + k;
    float t[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) t[c] = tx[c * OWN];
    // rho' and Theta' in difference form (slot 0: rho w, slot 4: theta)
    float d0[N], d4[N];
    {
      const float m0 = zs[0][0], th0 = zs[0][4 * OWN];
#pragma unroll
      for (int l = 1; l <= N; ++l) {
        const float thl = zs[l][4 * OWN];
        const float dm = zs[l][0] - m0;
        d0[l - 1] = dm;
        d4[l - 1] = fmaf(thl, dm, (thl - th0) * m0);
      }
    }
    // row N of this segment: the top wall's part, and kept for the next
    // segment's face level (by the item of level 0)
    const bool keep = a == 0 && s < nseg - 1;
    if (a == N || keep) {
      float rn[5];
      rn[0] = f_drow_from<N, 2>(P, N, d0, 0.0f);
      rn[4] = f_drow_from<N, 2>(P, N, d4, 0.0f);
#pragma unroll
      for (int c = 1; c < 4; ++c) {
        float f[N + 1];
#pragma unroll
        for (int l = 0; l <= N; ++l) f[l] = zs[l][c * OWN];
        rn[c] = f_row_from<N, 2>(P, N, f, 0.0f);
      }
      if (a == N) {
#pragma unroll
        for (int c = 0; c < 5; ++c) t[c] = fmaf(2.0f, rn[c], t[c]);
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c) PVn[c * OWN + k] = rn[c];
      }
    }
    if (a < N) {
      const int ar = a;
#pragma unroll
      for (int c = 1; c < 4; ++c) {
        float f[N + 1];
#pragma unroll
        for (int l = 0; l <= N; ++l) f[l] = zs[l][c * OWN];
        if (ar > 0) t[c] = f_row_from<N, 2>(P, ar, f, t[c]);
        else if (s > 0) t[c] = f_row_from<N, 2>(P, 0, f, t[c]) + PVo[c * OWN + k];
        else t[c] = f_row_from<N, 2>(P, 0, f, f_row_from<N, 2>(P, 0, f, t[c]));
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = e == 0 ? 0 : 4;
        const float (&d)[N] = e == 0 ? d0 : d4;
        if (ar > 0) t[c] = f_drow_from<N, 2>(P, ar, d, t[c]);
        else if (s > 0) t[c] = f_drow_from<N, 2>(P, 0, d, t[c]) + PVo[c * OWN + k];
        else t[c] = f_drow_from<N, 2>(P, 0, d, f_drow_from<N, 2>(P, 0, d, t[c]));
      }
    }
    // the stage: sources, walls, the SSP-RK3 combination
    const int gx = T.x0 + i, gy = T.y0 + j;
    const long long I = (long long)nx * ny * zl + gx + (long long)nx * gy;
    float qv[5], qnv[5] = {0, 0, 0, 0, 0}, cv[5] = {0, 0, 0, 0, 0}, sv = 0.0f;
#pragma unroll
    for (int c = 0; c < 5; ++c) qv[c] = B.q[c * np + I];
    if (!B.rhs_only && B.alpha != 0.0f) {
#pragma unroll
      for (int c = 0; c < 5; ++c) qnv[c] = B.qn[c * np + I];
    }
    if (B.S) sv = B.S[I];
    if (B.C) {
#pragma unroll
      for (int c = 0; c < 5; ++c) cv[c] = B.C[c * np + I];
    }
    const df r0 = B.base[zl];
    f_finish_vals(P, B, qv, qnv, sv, r0.h, B.out, I, gx, gy, zl, t, bad, cv);
  }
  if (bad) atomicOr(B.flag, 1);
}

// One CTA per column of E x E elements (grid ceil(nel_x / E) x
// ceil(nel_y / E)), kColThreads threads, ColLayout::bytes of dynamic shared memory;
// the mesh has walls at the bottom and top (P.per[2] == 0).  TMA: q is staged
// through qmap (a map of this launch's q, box 24 x 21 x 1 x 5); every wait
// for a staged level is bounded, and one that runs out sets bit 1 of the
// flag, waits (bounded) for the load once more and ends the CTA.
template <bool TMA>
__global__ void __launch_bounds__(kColThreads, 2)
    k_f_column(const FParams P, const FBufs B, const __grid_constant__ CUtensorMap qmap) {
  using L = ColLayout;
  constexpr int N = L::N;
  extern __shared__ __align__(128) float sm_col[];
  float* Q = sm_col + L::OFF_Q;
  float* FX = sm_col + L::OFF_FX;
  float* FY = sm_col + L::OFF_FY;
  float* ZF = sm_col + L::OFF_ZF;
  float* TX = sm_col + L::OFF_TX;
  float* PV = sm_col + L::OFF_PV;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm_col + L::OFF_BAR);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nz = P.n[2];

  PlaneTile T;
  T.init<N, L::E>(P, blockIdx.x, blockIdx.y);
  const bool wraps = (P.per[0] && (T.x0 == 0 || T.x0 + T.ekx * N >= P.n[0])) ||
                     (P.per[1] && (T.y0 == 0 || T.y0 + T.eky * N >= P.n[1]));
  const uint32_t bar0 = tc::smem_addr(bar), bar1 = tc::smem_addr(bar + 1);
  if (TMA) {
    if (tid == 0) {
      tc::mbar_init(bar0, 1);
      tc::mbar_init(bar1, 1);
      tma::arrive_expect_tx(bar0, L::TX_BYTES);
      tma::load_4d(tc::smem_addr(Q), &qmap, T.x0 - N, T.y0 - N, 0, 0, bar0);
    }
    __syncthreads();
  }
  auto fx = [&](int c, int j, int ii) -> float { return FX[(c * L::LO + j) * L::LX + ii]; };
  auto fy = [&](int c, int jj, int i) -> float { return FY[(c * L::LX + jj) * L::LO + i]; };
  const float rox = 1.0f / (float)T.ox;

#pragma unroll 1
  for (int z = 0; z < nz; ++z) {
    const int b = z & 1;
    float* st = Q + b * L::QBP;
    if (TMA) {
      const bool ok = tc::mbar_wait(b ? bar1 : bar0, (uint32_t)((z >> 1) & 1), tc::kWaitNs);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicOr(B.flag, 2);
          tc::mbar_wait(b ? bar1 : bar0, (uint32_t)((z >> 1) & 1), tc::kWaitNs);
        }
        return;
      }
      if (wraps) col_stage_plain(P, B.q, T, z, st, false, tid, nthr);
    } else {
      col_stage_plain(P, B.q, T, z, st, true, tid, nthr);
    }
    // every thread's generic accesses to the other buffer (level z - 1) come
    // before the load into it that thread 0 issues after the barrier
    if (TMA) tma::fence_proxy_async();
    __syncthreads();
    if (TMA && tid == 0 && z + 1 < nz) {         // the next level into the other buffer
      const uint32_t nb = b ? bar0 : bar1;
      tma::fence_proxy_async();
      tma::arrive_expect_tx(nb, L::TX_BYTES);
      tma::load_4d(tc::smem_addr(Q + (b ^ 1) * L::QBP), &qmap, T.x0 - N, T.y0 - N, z + 1, 0, nb);
    }
    const int slot = z % L::SLOTS;
    col_pointwise(P, B, T, z, st, FX, FY, ZF + slot * 5 * L::OWN, tid, nthr);
    __syncthreads();
    float* tx = TX + slot * 5 * L::OWN;
    for (int idx = tid; idx < T.ox * T.oy; idx += nthr) {
      const int j = small_div(idx, T.ox, rox), i = idx - j * T.ox;
      float t[5];
      f_plane_node_xy<N>(P, T, fx, fy, i, j, t);
#pragma unroll
      for (int c = 0; c < 5; ++c) tx[c * L::OWN + j * L::LO + i] = t[c];
    }
    if (z > 0 && z % N == 0) {
      __syncthreads();
      const int s = z / N - 1;
      col_finish_segment(P, B, T, s, ZF, TX, PV + (s & 1) * 5 * L::OWN, PV + ((s + 1) & 1) * 5 * L::OWN,
                         tid, nthr);
    }
    // the next level's staging barrier orders these reads before its writes
  }
}

}  // namespace xg
