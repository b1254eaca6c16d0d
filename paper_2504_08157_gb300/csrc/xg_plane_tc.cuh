// xg_plane_tc.cuh -- the FP32 plane kernel (x and y passes of one level)
// with the derivative contractions on the tensor cores: tcgen05.mma of kind
// tf32 in split form, for order N = 4.
//
// The contraction of a direction is one small GEMM per tile.  Its rows are
// the (variable, line, element segment) triples, its K index the N + 1 flux
// values of the segment, its columns the segment's N + 1 output rows a:
//   D[(c, line, s)][a] = sum_l F_c(line, s N + l) Dm[a][l]
// with Dm = -(2/h) D, rows 0 and N halved, of Eqs. 8-12 along the direction.
// The flux tiles are stored line by line with pitch 40 floats; with N = 4 the
// segments of a line start 16 bytes apart, so the A operand of a product is
// read in place: 8 consecutive segments of a line form a core matrix (rows 16
// bytes apart), the next line is the next 8-row group (stride 160 bytes) and
// the second K-chunk starts 16 bytes after the first (it runs into the next
// segment, whose values meet the zero rows 5..7 of B).  One product covers
// 16 lines; 11 cover the 165 lines of a 33-line tile.
//
// Precision: each flux F and each Dm entry is split into a TF32 head and a
// TF32 tail (F = F_h + F_l, both rounded to nearest), and three products are
// accumulated in FP32: F_h Dm_h + F_l Dm_h + F_h Dm_l (the dropped F_l Dm_l
// is ~2^-22 of the result's terms).  Shared memory holds the heads and tails
// of both directions (4 arrays of 26.4 KB): two CTAs fit an SM, against four
// of the CUDA-core plane kernel.
//
// After the products the node-centric assembly of the CUDA-core kernel is
// replayed from D: an element-interior node takes row a of its segment, a
// face node adds row N of the segment before (for the tile's first node
// that segment lies in the halo and its row N is computed on the CUDA
// cores), a wall node doubles its one-sided row.
#pragma once

#include <cuda_runtime.h>

#include "xg_plane_f32.cuh"
#include "xg_tc.cuh"

namespace xg {

// 8 warps: the epilogue splits the 11 products of a direction between warps
// 0-3 and 4-7 (one TMEM lane quarter each), and threads 0..164 take the
// 165 halo rows
constexpr int kPlaneTcThreads = 256;

struct PlaneTcLayout {
  static constexpr int N = 4, E = 8;
  static constexpr int LO = E * N + 1;               // owned extent across a line: 33
  static constexpr int PT = 40;                      // line pitch (floats): 37 loaded, then zeros
  static constexpr int LINES = 5 * LO;               // lines of one direction: 165
  static constexpr int BLOCKS = (LINES + 15) / 16;   // products of M = 128 rows: 11
  static constexpr int ARR = LINES * PT;             // floats of one array
  static constexpr int B16 = 16 * 8;                 // one B operand: 16 x 8 TF32 values
  static constexpr int OFF_B = 4 * ARR;              // XH, XL, YH, YL, then DXH, DXL, DYH, DYL
  static constexpr int TAIL = (BLOCKS * 16 - LINES) * PT;   // read by the last product's spare rows
  static constexpr int FLOATS = OFF_B + 4 * B16 + TAIL;
  static constexpr int RN = 28;                      // a line's row-N results start here (tail arrays)
  static constexpr int COLS = 256;                   // TMEM columns (11 x 16 used)
  static constexpr size_t bytes = sizeof(float) * FLOATS + 16;   // + mbarrier, TMEM address
};
static_assert(PlaneTcLayout::N * 4 == 16, "segments must start 16 bytes apart");
static_assert(PlaneTcLayout::LINES <= kPlaneTcThreads, "one thread per halo row");
static_assert(PlaneTcLayout::RN + PlaneTcLayout::E + 1 <= PlaneTcLayout::PT, "row-N slots fit a line");

// The products of one direction: D[16 b ...] for the 11 blocks, three split
// terms each, issued by one thread; the mbarrier at bar completes when done.
__device__ __forceinline__ void tc_plane_products(const float* H, const float* Lo, const float* BH,
                                                  const float* BL, uint32_t tm, uint32_t bar) {
  using L = PlaneTcLayout;
  constexpr uint32_t idesc = tc::idesc_tf32(128, 16);
  const uint64_t bh = tc::smem_desc(tc::smem_addr(BH), 16 * 16, 128);
  const uint64_t bl = tc::smem_desc(tc::smem_addr(BL), 16 * 16, 128);
  const uint32_t h0 = tc::smem_addr(H + L::N), l0 = tc::smem_addr(Lo + L::N);
#pragma unroll 1
  for (int b = 0; b < L::BLOCKS; ++b) {
    const uint32_t off = 16u * L::PT * 4u * (uint32_t)b;
    const uint64_t ah = tc::smem_desc(h0 + off, 16, L::PT * 4);
    const uint64_t al = tc::smem_desc(l0 + off, 16, L::PT * 4);
    const uint32_t d = tm + 16u * (uint32_t)b;
    tc::mma_tf32(d, ah, bh, idesc, false);
    tc::mma_tf32(d, al, bh, idesc, true);
    tc::mma_tf32(d, ah, bl, idesc, true);
  }
  tc::commit(bar);
}

// This thread's rows of D: rows 0..N-1 of a segment go in place into the head
// array (at the flux position of the node), row N into slot s + 1 of the
// line's row-N slots in the tail array.  nlines: valid lines of the
// direction's variable, nseg: valid segments.
__device__ __forceinline__ void tc_plane_epilogue(float* H, float* Lo, uint32_t tm, int nlines, int nseg) {
  using L = PlaneTcLayout;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, b0 = warp < 4 ? 0 : 6, b1 = warp < 4 ? 6 : L::BLOCKS;
  const int row = 32 * q + lane, s = row & 7;
#pragma unroll 1
  for (int b = b0; b < b1; ++b) {
    uint32_t r[8];
    tc::tmem_ld8(tm + ((uint32_t)(32 * q) << 16) + 16u * (uint32_t)b, r);
    tc::tmem_wait_ld();
    const int ln = 16 * b + (row >> 3);
    if (ln < L::LINES) {
      const int c = ln / L::LO, j = ln - c * L::LO;
      if (j < nlines && s < nseg) {
        float* h = H + ln * L::PT + L::N + s * L::N;
#pragma unroll
        for (int a = 0; a < L::N; ++a) h[a] = __uint_as_float(r[a]);
        Lo[ln * L::PT + L::RN + s + 1] = __uint_as_float(r[L::N]);
      }
    }
  }
}

// Row N of the halo segment before the first node of line tid (head + tail
// of the stored fluxes), or 0 when the thread has no such line.
__device__ __forceinline__ float tc_plane_halo(const FParams& P, int dir, const float* H, const float* Lo,
                                               int nlines, bool has) {
  using L = PlaneTcLayout;
  const int ln = threadIdx.x;
  if (!has || ln >= L::LINES) return 0.0f;
  const int c = ln / L::LO, j = ln - c * L::LO;
  if (j >= nlines) return 0.0f;
  float acc = 0.0f;
#pragma unroll
  for (int l = 0; l <= L::N; ++l) acc = fmaf(P.Dm[dir][L::N][l], H[ln * L::PT + l] + Lo[ln * L::PT + l], acc);
  return acc;
}

template <bool CG>
__device__ __forceinline__ void f_plane_tile_tc(const FParams& P, const FBufs& B, int bx, int by, int z,
                                                float* sm) {
  using L = PlaneTcLayout;
  constexpr int N = L::N, LO = L::LO, PT = L::PT;
  float* XH = sm;
  float* XL = sm + L::ARR;
  float* YH = sm + 2 * L::ARR;
  float* YL = sm + 3 * L::ARR;
  float* DB = sm + L::OFF_B;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::FLOATS);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5;
  const uint32_t bar_a = tc::smem_addr(bar);

  PlaneTile T;
  T.init<N, L::E>(P, bx, by);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), L::COLS);
  if (tid == 0) tc::mbar_init(bar_a, 1);
  // B operands: Dm^T of x and y, heads and tails
  for (int k = tid; k < 2 * L::B16; k += nthr) {
    const int d = k / L::B16, a = (k >> 3) & 15, l = k & 7;
    const float v = (a <= N && l <= N) ? P.Dm[d][a][l] : 0.0f;
    const float h = tc::to_tf32(v);
    DB[2 * d * L::B16 + tc::kmajor32(16, a, l)] = h;
    DB[(2 * d + 1) * L::B16 + tc::kmajor32(16, a, l)] = tc::to_tf32(v - h);
  }
  // zeros after the loaded extent of every owned line (the last segment's
  // second K-chunk reads them)
  const int wx = T.ekx * N + N + 1, wy = T.eky * N + N + 1;
  const int padx = PT - wx, pady = PT - wy;
  for (int k = tid; k < 5 * T.oy * padx; k += nthr) {
    const int line = k / padx, ii = wx + (k - line * padx);
    const int c = line / T.oy, ln = c * LO + (line - c * T.oy);
    XH[ln * PT + ii] = 0.0f;
    XL[ln * PT + ii] = 0.0f;
  }
  for (int k = tid; k < 5 * T.ox * pady; k += nthr) {
    const int line = k / pady, jj = wy + (k - line * pady);
    const int c = line / T.ox, ln = c * LO + (line - c * T.ox);
    YH[ln * PT + jj] = 0.0f;
    YL[ln * PT + jj] = 0.0f;
  }
  f_plane_pointwise<N, kPlaneBatch, CG, false>(
      P, B, T, z, tid, nthr,
      [&](int j, int ii, const float (&F)[5]) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const float h = tc::to_tf32(F[c]);
          XH[(c * LO + j) * PT + ii] = h;
          XL[(c * LO + j) * PT + ii] = tc::to_tf32(F[c] - h);
        }
      },
      [&](int jj, int i, const float (&F)[5]) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const float h = tc::to_tf32(F[c]);
          YH[(c * LO + i) * PT + jj] = h;
          YL[(c * LO + i) * PT + jj] = tc::to_tf32(F[c] - h);
        }
      });
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = *tslot;

  // ---- x: products, the halo rows meanwhile, then the epilogue
  if (tid == 0) tc_plane_products(XH, XL, DB, DB + L::B16, tm, bar_a);
  const float hx = tc_plane_halo(P, 0, XH, XL, T.oy, T.hxl);
  bool ok = tc::mbar_wait(bar_a, 0, tc::kWaitNs);
  int bad = __syncthreads_or(!ok);
  uint32_t bad_parity = 0;                             // the phase whose completion was not seen
  tc::fence_after_sync();
  if (!bad) {
    tc_plane_epilogue(XH, XL, tm, T.oy, T.ekx);
    if (tid < L::LINES) XL[tid * PT + L::RN] = hx;
    // ---- y: the TMEM columns are free once every thread's loads are done
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) tc_plane_products(YH, YL, DB + 2 * L::B16, DB + 3 * L::B16, tm, bar_a);
    const float hy = tc_plane_halo(P, 1, YH, YL, T.ox, T.hyl);
    ok = tc::mbar_wait(bar_a, 1, tc::kWaitNs);
    bad = __syncthreads_or(!ok);
    bad_parity = 1;
    tc::fence_after_sync();
    if (!bad) {
      tc_plane_epilogue(YH, YL, tm, T.ox, T.eky);
      if (tid < L::LINES) YL[tid * PT + L::RN] = hy;
    }
  }
  // products whose completion was not seen may still write tensor memory:
  // wait (bounded) once more for their commit before freeing it
  if (bad && tid == 0) tc::mbar_wait(bar_a, bad_parity, tc::kWaitNs);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tm, L::COLS);
  }
  if (bad) {
    if (tid == 0) atomicOr(B.flag, 2);
    return;
  }

  // ---- each owned node: x part + y part from the assembled rows
  const int nx = P.n[0], ny = P.n[1];
  const int ekx = T.ekx, eky = T.eky, ox = T.ox, oy = T.oy;
  const long long np = P.np;
  const long long zoff = (long long)nx * ny * z;
  const float rox = 1.0f / (float)ox;
  float* __restrict__ To = B.T;
  for (int idx = tid; idx < ox * oy; idx += nthr) {
    const int j = small_div(idx, ox, rox), i = idx - j * ox;
    const long long I = zoff + (T.x0 + i) + (long long)nx * (T.y0 + j);
    const int sx = min(i / N, ekx - 1), ax = i - sx * N;   // the wall node is row N of the last
    const int sy = min(j / N, eky - 1), ay = j - sy * N;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int lx = (c * LO + j) * PT, ly = (c * LO + i) * PT;
      float v = ax < N ? XH[lx + N + i] : XL[lx + L::RN + sx + 1];
      if (ax == 0) v += (sx > 0 || T.hxl) ? XL[lx + L::RN + sx] : v;
      else if (ax == N) v += v;                          // wall: the one-sided row counts twice
      float w = ay < N ? YH[ly + N + j] : YL[ly + L::RN + sy + 1];
      if (ay == 0) w += (sy > 0 || T.hyl) ? YL[ly + L::RN + sy] : w;
      else if (ay == N) w += w;
      To[c * np + I] = v + w;
    }
  }
}

__global__ void __launch_bounds__(kPlaneTcThreads, 2) k_f_plane_xy_tc(const FParams P, const FBufs B) {
  extern __shared__ __align__(128) float sm_plane_tc[];
  f_plane_tile_tc<false>(P, B, blockIdx.x, blockIdx.y, blockIdx.z, sm_plane_tc);
}

}  // namespace xg
