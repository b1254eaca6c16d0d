// xg_plane_h16.cuh -- the FP32 plane kernel (x and y passes of one level)
// with the derivative contractions on the tensor cores in IEEE half
// precision: tcgen05.mma of kind f16, each value split into three halves
// after a power-of-two scale per element segment, for order N = 4.
//
// As in the TF32 form, a direction's contraction is one GEMM per tile whose
// rows are the (variable, line, element segment) triples and whose columns
// are the segment's N + 1 output rows a:
//   D[(c, line, s)][a] = sum_{l >= 1} Dm[a][l] (F_c(line, s N + l) - F_c(line, s N)),
// the difference form of Eqs. 8-12 (each row of the derivative matrix sums to
// zero, so subtracting the segment's first value changes nothing but the
// rounding).  For rho' and Theta' the differences are formed from the rho'
// flux m = rho u_d and theta = Theta / rho exactly as the CUDA-core kernel
// does (f_drows): F_l - F_0 = theta_l (m_l - m_0) + (theta_l - theta_0) m_0.
//
// Range and precision.  Half precision has an 11-bit significand and a
// range of 2^-24 .. 65504, far too narrow for the fluxes of a box of
// kilometre-sized elements.  Every segment row is therefore scaled by its own
// power of two 2^k, chosen so that its largest difference lies in
// [2^14, 2^15), and split into three halves, v 2^k = h + t + u (each the
// rounded remainder of the one before: 11 + 11 + 11 bits hold the 24 of an
// FP32 value, so the split is exact up to half subnormals far below the
// row's largest value).  Dm is scaled (one power of two per direction) and
// split the same way.  In difference form the value at l = 0 is zero, so a
// row has N = 4 values per level and one K = 16 row of A holds
//   [h_1..4  t_1..4 | u_1..4  h_1..4]
// against the two B operands
//   B1 = [Dh  Dh | Dh  Dt]   and   B2 = [Du  Dt | 0  0]   (each over l = 1..4),
// so the two products accumulate, in FP32 in tensor memory,
//   (h + t + u) Dh + h Dt + h Du + t Dt,
// which misses v Dm only by u Dt + (t + u) Du, ~2^-33 of the row's largest
// term; what remains is the FP32 accumulation.  The epilogue multiplies each
// row by its inverse scales (exact powers of two).
//
// Operand layout (K-major, no swizzle).  A line's A operand is two core
// matrices of 8 rows x 16 bytes (K-chunk 0, then K-chunk 1 of its 8
// segments), so the leading byte offset is 128 and the stride byte offset
// (one line to the next, one 8-row group) 256.  One product covers 16 lines;
// 11 cover the 165 lines of a 33-line tile, and the 11 lines after them are
// zero rows.  The face node of two segments enters both rows.
//
// Shared memory (110 KB, two CTAs per SM).  A direction's operand region is
// used three times: first as FP32 staging of the fluxes (each segment row 8
// floats at the row's place, face values written twice), then -- after a
// barrier -- as the half-precision operands, and after the products as the
// FP32 results read by the node-centric assembly.  The halo segment before
// the tile's first node is staged apart and its row N is formed on the CUDA
// cores.  The x products run while the y operands are converted.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "xg_plane_f32.cuh"
#include "xg_tc.cuh"

namespace xg {

constexpr int kPlaneH16Threads = 256;

struct PlaneH16Layout {
  static constexpr int N = 4, E = 8;
  static constexpr int LO = E * N + 1;                 // owned extent across a line: 33
  static constexpr int LINES = 5 * LO;                 // lines of one direction: 165
  static constexpr int BLOCKS = (LINES + 15) / 16;     // products of M = 128 rows: 11
  static constexpr int LPAD = 16 * BLOCKS;             // lines with an operand: 176
  static constexpr int ITEMS = LPAD * E;               // segment rows of one direction: 1408
  static constexpr int LINE_BYTES = 256;               // the two K-chunk core matrices of one line
  static constexpr int ST = LINE_BYTES / 4;            // FP32 staging pitch of a line (floats): 64
  static constexpr int RP = 48;                        // result pitch (floats): rows 0..N-1 in place,
  static constexpr int RN = 36;                        //   row-N slots (halo, then segment s + 1) here
  static constexpr int OP_BYTES = LPAD * LINE_BYTES;   // one direction: 45,056
  static constexpr int HALO = 8;                       // staged halo values per line (N + 1 used)
  static constexpr int B_HALVES = 16 * 16;             // one B operand: 16 output rows x K = 16
  // byte offsets
  static constexpr int OFF_OPX = 0;
  static constexpr int OFF_OPY = OP_BYTES;
  static constexpr int OFF_B = 2 * OP_BYTES;                          // 4 B operands (x1, x2, y1, y2)
  static constexpr int OFF_SC = OFF_B + 4 * B_HALVES * 2;             // row scales [2][ITEMS]
  static constexpr int OFF_DSC = OFF_SC + 2 * ITEMS * 4;              // the two directions' Dm scales
  static constexpr int OFF_HALO = OFF_DSC + 16;                       // [2][LINES][HALO] floats
  static constexpr int OFF_BAR = OFF_HALO + 2 * LINES * HALO * 4;     // mbarrier, TMEM address
  static constexpr size_t bytes = OFF_BAR + 16;
  static constexpr int COLS = 256;                     // TMEM columns (11 x 16 used)
};
static_assert(PlaneH16Layout::LINES <= kPlaneH16Threads, "one thread per halo row");
static_assert(PlaneH16Layout::N == 4, "a K-chunk of 8 halves holds two levels of N = 4 values");
static_assert(PlaneH16Layout::RN >= PlaneH16Layout::N + PlaneH16Layout::E * PlaneH16Layout::N,
              "row-N slots after the in-place rows");
static_assert(PlaneH16Layout::RN + PlaneH16Layout::E + 1 <= PlaneH16Layout::RP, "row-N slots fit a line");
static_assert(PlaneH16Layout::LINES * PlaneH16Layout::RP * 4 <= PlaneH16Layout::OP_BYTES,
              "results fit the operand region");
static_assert(PlaneH16Layout::OFF_B % 128 == 0 && PlaneH16Layout::OFF_OPY % 128 == 0, "operand alignment");
static_assert(2 * (PlaneH16Layout::bytes + 1024) <= 233472, "two CTAs per SM");

// The power of two that brings mx (> 0) into [2^14, 2^15): its exponent k,
// clamped to the normal range of a float so that 2^k and 2^-k both exist.
__device__ __forceinline__ int h16_scale_exp(float mx) {
  const int e = max((int)((__float_as_uint(mx) >> 23) & 0xffu) - 127, -126);
  return min(14 - e, 126);
}
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(127 + k) << 23); }

// v = h + t + u, each the nearest half to the remainder of the one before
// (the remainders are exact in FP32)
__device__ __forceinline__ void h16_split3(float v, uint16_t& h, uint16_t& t, uint16_t& u) {
  const __half hh = __float2half_rn(v);
  const float r1 = v - __half2float(hh);
  const __half th = __float2half_rn(r1);
  const float r2 = r1 - __half2float(th);
  h = __half_as_ushort(hh);
  t = __half_as_ushort(th);
  u = __half_as_ushort(__float2half_rn(r2));
}

// The FP32 staging of the flux value v of line ln at local node i of the
// line (i in [-N, E N]): the segment rows holding it, or the halo.
__device__ __forceinline__ void h16_stage(float* st, float* halo, int ln, int i, float v) {
  using L = PlaneH16Layout;
  if (i <= 0) halo[ln * L::HALO + i + L::N] = v;
  if (i >= 0) {
    const int s = i / L::N, l = i - s * L::N;
    if (s < L::E) st[ln * L::ST + s * 8 + l] = v;
    if (l == 0 && s > 0) st[ln * L::ST + (s - 1) * 8 + L::N] = v;
  }
}

// One direction's B operands from Dm (columns l = 1..N; rows a > N zero):
// B1 = [Dh Dh | Dh Dt] and B2 = [Du Dt | 0 0] along K, in the K-major
// layout.  The direction's inverse scale goes to *dsc.
__device__ __forceinline__ void h16_b_operands(const FParams& P, int d, uint16_t* b1, uint16_t* b2, float* dsc,
                                               int tid, int nthr) {
  using L = PlaneH16Layout;
  constexpr int N = L::N;
  float mx = 0.0f;
#pragma unroll
  for (int a = 0; a <= N; ++a)
#pragma unroll
    for (int l = 1; l <= N; ++l) mx = fmaxf(mx, fabsf(P.Dm[d][a][l]));
  const int k = mx > 0.0f ? h16_scale_exp(mx) : 0;
  const float sc = pow2f(k);
  if (tid == 0) *dsc = pow2f(-k);
  for (int idx = tid; idx < L::B_HALVES; idx += nthr) {
    const int a = idx >> 4, kk = idx & 15, g = kk >> 2, l = (kk & 3) + 1;   // g: group of 4 along K
    uint16_t h = 0, t = 0, u = 0;
    if (a <= N) h16_split3(P.Dm[d][a][l] * sc, h, t, u);
    b1[tc::kmajor(16, a, kk)] = g < 3 ? h : t;
    b2[tc::kmajor(16, a, kk)] = g == 0 ? u : g == 1 ? t : (uint16_t)0;
  }
}

// Up to kH16Items segment rows of one direction per thread, read from the
// FP32 staging into registers as packed halves (the staging and the operands
// share the region: every thread reads before anyone writes).  R.h is a
// row's K-chunk 0, R.t its K-chunk 1.
constexpr int kH16Items = (PlaneH16Layout::ITEMS + kPlaneH16Threads - 1) / kPlaneH16Threads;

struct H16Rows {
  uint32_t h[kH16Items][4], t[kH16Items][4];
  float isc[kH16Items];
};

__device__ __forceinline__ void h16_convert_read(const float* st, int nlines, int nseg, int tid, int nthr,
                                                 H16Rows& R) {
  using L = PlaneH16Layout;
  constexpr int N = L::N;
#pragma unroll
  for (int u = 0; u < kH16Items; ++u) {
    const int item = tid + u * nthr;
#pragma unroll
    for (int w = 0; w < 4; ++w) R.h[u][w] = R.t[u][w] = 0u;
    R.isc[u] = 0.0f;
    const int ln = item >> 3, s = item & 7;
    if (item >= L::ITEMS || ln >= L::LINES) continue;
    const int c = ln / L::LO, j = ln - c * L::LO;
    if (j >= nlines || s >= nseg) continue;
    const float* f = st + ln * L::ST + s * 8;
    float d[N + 1];
    d[0] = 0.0f;
    if (c == 4) {                                   // slot 4 holds theta; m is the rho' flux line
      const float* m = st + j * L::ST + s * 8;
      const float m0 = m[0], t0 = f[0];
#pragma unroll
      for (int l = 1; l <= N; ++l) {
        const float dm = m[l] - m0;
        d[l] = fmaf(f[l], dm, (f[l] - t0) * m0);
      }
    } else {
      const float f0 = f[0];
#pragma unroll
      for (int l = 1; l <= N; ++l) d[l] = f[l] - f0;
    }
    float mx = 0.0f;
#pragma unroll
    for (int l = 1; l <= N; ++l) mx = fmaxf(mx, fabsf(d[l]));
    if (!(mx > 0.0f)) {                             // an all-zero row; a NaN reaches the results
      bool nan = false;
#pragma unroll
      for (int l = 1; l <= N; ++l) nan |= d[l] != d[l];
      if (nan) R.isc[u] = __uint_as_float(0x7fc00000u);
      continue;
    }
    const int k = h16_scale_exp(mx);
    const float sc = pow2f(k);
    R.isc[u] = pow2f(-k);
    uint16_t hh[N], tt[N], uu[N];
#pragma unroll
    for (int l = 0; l < N; ++l) h16_split3(d[l + 1] * sc, hh[l], tt[l], uu[l]);
    // chunk 0: h_1..4 t_1..4; chunk 1: u_1..4 h_1..4
    R.h[u][0] = (uint32_t)hh[0] | ((uint32_t)hh[1] << 16);
    R.h[u][1] = (uint32_t)hh[2] | ((uint32_t)hh[3] << 16);
    R.h[u][2] = (uint32_t)tt[0] | ((uint32_t)tt[1] << 16);
    R.h[u][3] = (uint32_t)tt[2] | ((uint32_t)tt[3] << 16);
    R.t[u][0] = (uint32_t)uu[0] | ((uint32_t)uu[1] << 16);
    R.t[u][1] = (uint32_t)uu[2] | ((uint32_t)uu[3] << 16);
    R.t[u][2] = R.h[u][0];
    R.t[u][3] = R.h[u][1];
  }
}

__device__ __forceinline__ void h16_convert_write(unsigned char* op, float* sc, int tid, int nthr,
                                                  const H16Rows& R) {
  using L = PlaneH16Layout;
#pragma unroll
  for (int u = 0; u < kH16Items; ++u) {
    const int item = tid + u * nthr;
    if (item >= L::ITEMS) continue;
    const int ln = item >> 3, s = item & 7;
    *reinterpret_cast<uint4*>(op + ln * L::LINE_BYTES + s * 16) =
        make_uint4(R.h[u][0], R.h[u][1], R.h[u][2], R.h[u][3]);
    *reinterpret_cast<uint4*>(op + ln * L::LINE_BYTES + 128 + s * 16) =
        make_uint4(R.t[u][0], R.t[u][1], R.t[u][2], R.t[u][3]);
    sc[item] = R.isc[u];
  }
}

// The two products of every block of one direction (issued by one thread);
// the mbarrier at bar completes when they are done.
__device__ __forceinline__ void h16_products(const unsigned char* op, const uint16_t* b1, const uint16_t* b2,
                                             uint32_t tm, uint32_t bar) {
  using L = PlaneH16Layout;
  constexpr uint32_t idesc = tc::idesc_f16(128, 16);
  const uint64_t d1 = tc::smem_desc(tc::smem_addr(b1), 16 * 16, 128);
  const uint64_t d2 = tc::smem_desc(tc::smem_addr(b2), 16 * 16, 128);
  const uint32_t a0 = tc::smem_addr(op);
#pragma unroll 1
  for (int b = 0; b < L::BLOCKS; ++b) {
    const uint64_t ad = tc::smem_desc(a0 + (uint32_t)(16 * L::LINE_BYTES * b), 128, L::LINE_BYTES);
    const uint32_t d = tm + 16u * (uint32_t)b;
    tc::mma_bf16(d, ad, d1, idesc, false);
    tc::mma_bf16(d, ad, d2, idesc, true);
  }
  tc::commit(bar);
}

// This thread's rows of D, unscaled, into the result layout over the
// (finished) operand region: rows 0..N-1 of segment s at N + s N + a, row N
// in slot RN + s + 1.
__device__ __forceinline__ void h16_epilogue(float* res, const float* sc, float dsc, uint32_t tm, int nlines,
                                             int nseg) {
  using L = PlaneH16Layout;
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
        const float f = sc[ln * L::E + s] * dsc;
        float* o = res + ln * L::RP;
#pragma unroll
        for (int a = 0; a < L::N; ++a) o[L::N + s * L::N + a] = __uint_as_float(r[a]) * f;
        o[L::RN + s + 1] = __uint_as_float(r[L::N]) * f;
      }
    }
  }
}

// Row N of the halo segment before the first node of line tid, in the
// difference form of the CUDA-core kernel, or 0 when there is none.
template <int D>
__device__ __forceinline__ float h16_halo(const FParams& P, const float* halo, int nlines, bool has) {
  using L = PlaneH16Layout;
  constexpr int N = L::N;
  const int ln = threadIdx.x;
  if (!has || ln >= L::LINES) return 0.0f;
  const int c = ln / L::LO, j = ln - c * L::LO;
  if (j >= nlines) return 0.0f;
  float f[N + 1];
  if (c == 0 || c == 4) {
    float m[N + 1], r0 = 0.0f, r4 = 0.0f;
#pragma unroll
    for (int l = 0; l <= N; ++l) {
      m[l] = halo[j * L::HALO + l];
      f[l] = halo[(4 * L::LO + j) * L::HALO + l];
    }
    f_drows<N, D>(P, N, m, f, r0, r4);
    return c == 0 ? r0 : r4;
  }
#pragma unroll
  for (int l = 0; l <= N; ++l) f[l] = halo[ln * L::HALO + l];
  return f_row_from<N, D>(P, N, f, 0.0f);
}

__device__ __forceinline__ void f_plane_tile_h16(const FParams& P, const FBufs& B, int bx, int by, int z,
                                                 unsigned char* sm) {
  using L = PlaneH16Layout;
  constexpr int N = L::N, LO = L::LO, RP = L::RP;
  unsigned char* OPX = sm + L::OFF_OPX;
  unsigned char* OPY = sm + L::OFF_OPY;
  float* STX = reinterpret_cast<float*>(OPX);      // staging, then results
  float* STY = reinterpret_cast<float*>(OPY);
  uint16_t* BO = reinterpret_cast<uint16_t*>(sm + L::OFF_B);
  float* SC = reinterpret_cast<float*>(sm + L::OFF_SC);
  float* DSC = reinterpret_cast<float*>(sm + L::OFF_DSC);
  float* HX = reinterpret_cast<float*>(sm + L::OFF_HALO);
  float* HY = HX + L::LINES * L::HALO;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::OFF_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5;
  const uint32_t bar_a = tc::smem_addr(bar);

  PlaneTile T;
  T.init<N, L::E>(P, bx, by);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), L::COLS);
  if (tid == 0) tc::mbar_init(bar_a, 1);
  h16_b_operands(P, 0, BO, BO + L::B_HALVES, DSC, tid, nthr);
  h16_b_operands(P, 1, BO + 2 * L::B_HALVES, BO + 3 * L::B_HALVES, DSC + 1, tid, nthr);
  f_plane_pointwise<N, kPlaneBatch, false, true>(
      P, B, T, z, tid, nthr,
      [&](int j, int ii, const float (&F)[5]) {
#pragma unroll
        for (int c = 0; c < 5; ++c) h16_stage(STX, HX, c * LO + j, ii - N, F[c]);
      },
      [&](int jj, int i, const float (&F)[5]) {
#pragma unroll
        for (int c = 0; c < 5; ++c) h16_stage(STY, HY, c * LO + i, jj - N, F[c]);
      });
  __syncthreads();

  // halo rows on the CUDA cores (their staging is not overwritten)
  const float hx = h16_halo<0>(P, HX, T.oy, T.hxl);
  const float hy = h16_halo<1>(P, HY, T.ox, T.hyl);
  // ---- x operands, then the x products while the y operands are converted
  {
    H16Rows R;
    h16_convert_read(STX, T.oy, T.ekx, tid, nthr, R);
    __syncthreads();
    h16_convert_write(OPX, SC, tid, nthr, R);
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = *tslot;
  if (tid == 0) h16_products(OPX, BO, BO + L::B_HALVES, tm, bar_a);
  {
    H16Rows R;
    h16_convert_read(STY, T.ox, T.eky, tid, nthr, R);
    __syncthreads();
    h16_convert_write(OPY, SC + L::ITEMS, tid, nthr, R);
  }
  tc::fence_proxy_async();
  bool ok = tc::mbar_wait(bar_a, 0, tc::kWaitNs);
  int bad = __syncthreads_or(!ok);
  uint32_t bad_parity = 0;                             // the phase whose completion was not seen
  tc::fence_after_sync();
  if (!bad) {
    h16_epilogue(STX, SC, DSC[0], tm, T.oy, T.ekx);
    if (tid < L::LINES) STX[tid * RP + L::RN] = hx;
    // ---- y: the TMEM columns are free once every thread's loads are done
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) h16_products(OPY, BO + 2 * L::B_HALVES, BO + 3 * L::B_HALVES, tm, bar_a);
    ok = tc::mbar_wait(bar_a, 1, tc::kWaitNs);
    bad = __syncthreads_or(!ok);
    bad_parity = 1;
    tc::fence_after_sync();
    if (!bad) {
      h16_epilogue(STY, SC + L::ITEMS, DSC[1], tm, T.ox, T.eky);
      if (tid < L::LINES) STY[tid * RP + L::RN] = hy;
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
      const float* rx = STX + (c * LO + j) * RP;
      const float* ry = STY + (c * LO + i) * RP;
      float v = ax < N ? rx[N + i] : rx[L::RN + sx + 1];
      if (ax == 0) v += (sx > 0 || T.hxl) ? rx[L::RN + sx] : v;
      else if (ax == N) v += v;                          // wall: the one-sided row counts twice
      float w = ay < N ? ry[N + j] : ry[L::RN + sy + 1];
      if (ay == 0) w += (sy > 0 || T.hyl) ? ry[L::RN + sy] : w;
      else if (ay == N) w += w;
      To[c * np + I] = v + w;
    }
  }
}

__global__ void __launch_bounds__(kPlaneH16Threads, 2) k_f_plane_xy_h16(const FParams P, const FBufs B) {
  extern __shared__ __align__(1024) unsigned char sm_plane_h16[];
  f_plane_tile_h16(P, B, blockIdx.x, blockIdx.y, blockIdx.z, sm_plane_h16);
}

}  // namespace xg
