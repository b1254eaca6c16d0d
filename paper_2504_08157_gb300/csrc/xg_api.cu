// xg_api.cu -- C ABI of the explicit CG Euler path (see include/xg.h).
//
// Host side: contexts and their device buffers, the reference-state table
// p_0 = p(Theta_0) (Eq. 3), and the launch sequence of one SSP-RK3 stage
// (three line kernels).  Mesh checks and the launch constants (LGL
// derivative matrix, equation-of-state series) are in xg_setup.h.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/xg.h"
#include "xg_kernels.cuh"
#include "xg_column_f32.cuh"
#include "xg_kernels_df.cuh"
#include "xg_plane_h16.cuh"
#include "xg_plane_tc.cuh"
#include "xg_setup.h"
#include "xg_ctx.h"

using xg::DfBufs;
using xg::DfParams;
using xg::LineParams;
using xg::StageBufs;
using xg::df;

namespace xg {
bool encode_tma_4d_f32(CUtensorMap* map, const float* base, const uint64_t dims[4], const uint32_t box[4]) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) return false;
  const cuuint64_t gdim[4] = {dims[0], dims[1], dims[2], dims[3]};
  const cuuint64_t gstride[3] = {dims[0] * 4, dims[0] * dims[1] * 4, dims[0] * dims[1] * dims[2] * 4};
  const cuuint32_t bdim[4] = {box[0], box[1], box[2], box[3]};
  const cuuint32_t estride[4] = {1, 1, 1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), gdim, gstride, bdim, estride,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(df v) { return df_to_double(v); }
}  // namespace xg


namespace {

// Reciprocal self-check: out[i] = rcp_newton(x[i]) (positive normal x).
__global__ void k_rcp_check(const double* __restrict__ x, double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = xg::rcp_newton(x[i]);
}

// Equation-of-state self-check: p' of Eq. 3 at every node from Theta' (FP64
// values, converted as the state is) and the node level's reference values,
// through the device function each precision's kernels call.
__global__ void k_eos_check_fp64(const xg::LineParams P, const double* __restrict__ base,
                                 const double* __restrict__ tp, double* __restrict__ out,
                                 long long np, long long nxy, int nz) {
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < np;
       I += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(I / nxy);
    out[I] = base[2 * nz + z] * xg::eos_phi(P, tp[I] * base[3 * nz + z]);
  }
}

__global__ void k_eos_check_df(const xg::DfParams P, const xg::df* __restrict__ base,
                               const double* __restrict__ tp, double* __restrict__ out,
                               long long np, long long nxy, int nz) {
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < np;
       I += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(I / nxy);
    const xg::df x = xg::df_mul(xg::df_of_double(tp[I]), base[3 * nz + z]);
    out[I] = xg::df_to_double(xg::df_mul(base[2 * nz + z], xg::df_eos_phi(P, x)));
  }
}

__global__ void k_eos_check_f32(const xg::FParams P, const xg::df* __restrict__ base,
                                const double* __restrict__ tp, double* __restrict__ out,
                                long long np, long long nxy, int nz) {
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < np;
       I += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(I / nxy);
    out[I] = (double)xg::f_pressure_pert(P, __double2float_rn(tp[I]), base[2 * nz + z], base[3 * nz + z]);
  }
}

// Partition faces (values of 8 bytes: FP64 or double-float pairs).  Face
// arrays are [5][n_z][n_x].  pack: the slab's first y plane of T (x part
// plus row 0 of the first y segment) into out.  combine: the first plane
// gets the left neighbour's row N (t0 + carry, the order of k_line_y at a
// shared face), the last plane the right neighbour's t0 plus this slab's own
// row N -- so both slabs hold bit for bit the value a single domain has.
template <typename V>
__global__ void k_face_pack(const V* __restrict__ T, V* __restrict__ out, int nx, int ny, int nz,
                            long long np) {
  const long long nf = (long long)nx * nz;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 5 * nf;
       k += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(k / nf);
    const long long r = k - c * nf;
    const int z = (int)(r / nx), x = (int)(r - (long long)z * nx);
    out[k] = T[c * np + x + (long long)nx * ny * z];
  }
}

// MIXED: slots 0 and 4 hold doubles and 1..3 double-float pairs (XG_DF64)
template <bool MIXED>
__global__ void k_face_combine(double* __restrict__ T, const double* __restrict__ recv_lo,
                               const double* __restrict__ recv_hi, const double* __restrict__ own_hi,
                               int nx, int ny, int nz, long long np) {
  const long long nf = (long long)nx * nz;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 5 * nf;
       k += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(k / nf);
    const long long r = k - c * nf;
    const int z = (int)(r / nx), x = (int)(r - (long long)z * nx);
    const long long I0 = c * np + x + (long long)nx * ny * z;
    const long long I1 = I0 + (long long)nx * (ny - 1);
    if (MIXED && c != 0 && c != 4) {
      xg::df* Tm = reinterpret_cast<xg::df*>(T);
      if (recv_lo) Tm[I0] = xg::df_add(Tm[I0], reinterpret_cast<const xg::df*>(recv_lo)[k]);
      if (recv_hi)
        Tm[I1] = xg::df_add(reinterpret_cast<const xg::df*>(recv_hi)[k], reinterpret_cast<const xg::df*>(own_hi)[k]);
    } else {
      if (recv_lo) T[I0] = T[I0] + recv_lo[k];
      if (recv_hi) T[I1] = recv_hi[k] + own_hi[k];
    }
  }
}

}  // namespace

namespace xg {
__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = __double2float_rn(in[i]);
}
__global__ void k_from_f32(const float* __restrict__ in, double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}
}  // namespace xg

namespace {

constexpr int kDiagBlocks = 512;
constexpr int kDiagThreads = 256;

// Per-block FP64 sums of M_I q_v,I (v = 0..4), M_I = Wx(gx) Wy(gy) Wz(gz)
// with the Jacobian folded into Wx; a fixed tree order in shared memory.
template <typename R>
__global__ void k_diag_partial(const R* __restrict__ q, const double* __restrict__ wasm, int nx,
                               int ny, int nz, long long np, double* __restrict__ partial) {
  __shared__ double red[5][kDiagThreads];
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < np;
       I += (long long)gridDim.x * blockDim.x) {
    const int gx = (int)(I % nx);
    const long long r = I / nx;
    const int gy = (int)(r % ny), gz = (int)(r / ny);
    const double m = wasm[gx] * wasm[nx + gy] * wasm[nx + ny + gz];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += m * xg::to_double(q[v * np + I]);
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) red[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int h = kDiagThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
#pragma unroll
      for (int v = 0; v < 5; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x < 5) partial[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_diag_final(const double* __restrict__ partial, double* __restrict__ out) {
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int b = 0; b < kDiagBlocks; ++b) s += partial[b * 5 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

unsigned conv_blocks(long long n) {
  const long long b = (n + 255) / 256;
  return (unsigned)(b < 16384 ? b : 16384);
}

xg_status fail_cuda(xg_ctx* c, cudaError_t e, const char* what) {
  if (c) c->failed = true;
  fprintf(stderr, "xg: %s: %s\n", what, cudaGetErrorString(e));
  return XG_ERR_CUDA;
}

#define XG_CUDA(ctx, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return fail_cuda((ctx), e_, #call); \
  } while (0)

// Records the start (end = false) or end event of kernel k's launch.
void prof_mark(xg_ctx* c, int k, bool end, cudaStream_t st) {
  if (!c->profiling) return;
  const size_t i = 2 * c->ev_used + (end ? 1 : 0);
  while (c->events.size() <= i) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { c->profiling = false; return; }
    c->events.push_back(e);
  }
  cudaEventRecord(c->events[i], st);
  if (end) {
    if (c->ev_kernel.size() <= c->ev_used) c->ev_kernel.resize(c->ev_used + 1);
    c->ev_kernel[c->ev_used] = k;
    ++c->ev_used;
  }
}

// Folds the recorded pairs into the per-kernel totals (the stream has been
// synchronised by the caller).
void prof_fold(xg_ctx* c) {
  for (size_t p = 0; p < c->ev_used; ++p) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c->events[2 * p], c->events[2 * p + 1]) == cudaSuccess) {
      c->k_ms[c->ev_kernel[p]] += ms;
      c->k_launches[c->ev_kernel[p]] += 1;
    }
  }
  c->ev_used = 0;
}

// parts: bit 0 the x and y passes, bit 1 the z pass (a partitioned stage
// exchanges the partition faces' rows in between)
template <int N>
void launch_stage_n(xg_ctx* c, const StageBufs& B, cudaStream_t st, int parts) {
  if (parts & 1) {
    dim3 gx(c->n[1], c->n[2]);
    prof_mark(c, 0, false, st);
    xg::k_line_x<N><<<gx, xg::kXThreads, c->xsmem, st>>>(c->P, B);
    prof_mark(c, 0, true, st);
    dim3 gy((c->n[0] + 127) / 128, c->nchunk_y, c->n[2]);
    prof_mark(c, 1, false, st);
    xg::k_line_y<N><<<gy, 128, 0, st>>>(c->P, B, c->chunk_y);
    prof_mark(c, 1, true, st);
  }
  if (parts & 2) {
    dim3 gz((c->n[0] + 127) / 128, c->nchunk_z, c->n[1]);
    prof_mark(c, 2, false, st);
    xg::k_line_z<N><<<gz, 128, 0, st>>>(c->P, B, c->chunk_z);
    prof_mark(c, 2, true, st);
  }
}

template <int N>
cudaError_t configure_n(xg_ctx* c) {
  cudaError_t e = xg::raise_dynamic_smem(xg::k_line_x<N>, c->xsmem);
  if (e == cudaSuccess) e = xg::raise_dynamic_smem(xg::k_df_line_x<N>, c->xsmem);
  if (e == cudaSuccess) e = xg::raise_dynamic_smem(xg::k_f_plane_xy<N>, xg::PlaneLayoutF<N>::bytes);
  if (N == xg::PlaneTcLayout::N && e == cudaSuccess)
    e = xg::raise_dynamic_smem(xg::k_f_plane_xy_tc, xg::PlaneTcLayout::bytes);
  if (N == xg::ColLayout::N && e == cudaSuccess) e = xg::raise_dynamic_smem(xg::k_f_column<true>, xg::ColLayout::bytes);
  if (N == xg::ColLayout::N && e == cudaSuccess) e = xg::raise_dynamic_smem(xg::k_f_column<false>, xg::ColLayout::bytes);
  if (N == xg::PlaneH16Layout::N && e == cudaSuccess) {
    e = xg::raise_dynamic_smem(xg::k_f_plane_xy_h16, xg::PlaneH16Layout::bytes);
    // two CTAs of 111 KB per SM need the whole shared-memory carveout
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)xg::k_f_plane_xy_h16, cudaFuncAttributePreferredSharedMemoryCarveout,
                               100);
  }
  return e;
}

template <int N>
void launch_df_stage_n(xg_ctx* c, const DfBufs& B, cudaStream_t st, int parts) {
  if (parts & 1) {
    dim3 gx(c->n[1], c->n[2]);
    prof_mark(c, 0, false, st);
    xg::k_df_line_x<N><<<gx, xg::kXThreads, c->xsmem, st>>>(c->Pdf, B);
    prof_mark(c, 0, true, st);
    constexpr int K = xg::df_tile_segments(N, 1);
    const dim3 blk(xg::kTileCols, K * N + 1);
    const unsigned xb = (c->n[0] + xg::kTileCols - 1) / xg::kTileCols;
    dim3 gy(xb, (c->d.nel[1] + K - 1) / K, c->n[2]);
    prof_mark(c, 1, false, st);
    xg::k_df_tline<N, 1><<<gy, blk, 0, st>>>(c->Pdf, B);
    prof_mark(c, 1, true, st);
  }
  if (parts & 2) {
    constexpr int K = xg::df_tile_segments(N, 2);
    const dim3 blk(xg::kTileCols, K * N + 1);
    const unsigned xb = (c->n[0] + xg::kTileCols - 1) / xg::kTileCols;
    dim3 gz(xb, (c->d.nel[2] + K - 1) / K, c->n[1]);
    prof_mark(c, 2, false, st);
    xg::k_df_tline<N, 2><<<gz, blk, 0, st>>>(c->Pdf, B);
    prof_mark(c, 2, true, st);
  }
}

// The fused column pass applies: FP32 form, order 4, the CUDA-core
// contraction, walls at the bottom and top.
bool column_on(const xg_ctx* c) {
  return c->f32 && c->fused && c->d.order == xg::ColLayout::N && c->contract == XG_CONTRACT_FMA &&
         !c->Pf.per[2];
}

// The TMA map of stage input q (the 4-D view [5][n_z][n_y][n_x] with the
// column kernel's box), or null where the pitch does not allow one.
const CUtensorMap* column_map(xg_ctx* c, const float* q) {
  if (c->n[0] % 4 != 0) return nullptr;
  for (int k = 0; k < 4; ++k)
    if (c->col_key[k] == q) return &c->col_map[k];
  const int k = c->col_next;
  const uint64_t dims[4] = {(uint64_t)c->n[0], (uint64_t)c->n[1], (uint64_t)c->n[2], 5};
  const uint32_t box[4] = {xg::ColLayout::QX, xg::ColLayout::LX, 1, 5};
  if (!xg::encode_tma_4d_f32(&c->col_map[k], q, dims, box)) return nullptr;
  c->col_key[k] = q;
  c->col_next = (k + 1) % 4;
  return &c->col_map[k];
}

template <int N>
void launch_f32_stage_n(xg_ctx* c, const xg::FBufs& B, cudaStream_t st) {
  if (N == xg::ColLayout::N && column_on(c)) {   // x, y, z and the stage in one pass
    constexpr int E = xg::ColLayout::E;
    const dim3 g((c->d.nel[0] + E - 1) / E, (c->d.nel[1] + E - 1) / E);
    const CUtensorMap* m = column_map(c, B.q);
    prof_mark(c, 0, false, st);
    if (m) {
      xg::k_f_column<true><<<g, xg::kColThreads, xg::ColLayout::bytes, st>>>(c->Pf, B, *m);
    } else {
      CUtensorMap unused;
      std::memset(&unused, 0, sizeof(unused));
      xg::k_f_column<false><<<g, xg::kColThreads, xg::ColLayout::bytes, st>>>(c->Pf, B, unused);
    }
    prof_mark(c, 0, true, st);
    return;
  }
  // x and y passes fused over element tiles of each level, then the z pass
  constexpr int E = xg::plane_elems_f32(N);
  dim3 gp((c->d.nel[0] + E - 1) / E, (c->d.nel[1] + E - 1) / E, c->n[2]);
  prof_mark(c, 0, false, st);
  if (N == xg::PlaneTcLayout::N && c->contract == XG_CONTRACT_TF32X3) {
    static_assert(xg::plane_elems_f32(4) == xg::PlaneTcLayout::E, "same tiles");
    xg::k_f_plane_xy_tc<<<gp, xg::kPlaneTcThreads, xg::PlaneTcLayout::bytes, st>>>(c->Pf, B);
  } else if (N == xg::PlaneH16Layout::N && c->contract == XG_CONTRACT_F16X3) {
    static_assert(xg::plane_elems_f32(4) == xg::PlaneH16Layout::E, "same tiles");
    xg::k_f_plane_xy_h16<<<gp, xg::kPlaneH16Threads, xg::PlaneH16Layout::bytes, st>>>(c->Pf, B);
  } else {
    xg::k_f_plane_xy<N><<<gp, xg::kPlaneThreads, xg::PlaneLayoutF<N>::bytes, st>>>(c->Pf, B);
  }
  prof_mark(c, 0, true, st);
  constexpr int K = xg::f32_tile_segments(N);
  const dim3 blk(xg::kTileCols, K * N + 1);
  const unsigned xb = (c->n[0] + xg::kTileCols - 1) / xg::kTileCols;
  dim3 gz(xb, (c->d.nel[2] + K - 1) / K, c->n[1]);
  prof_mark(c, 2, false, st);
  xg::k_f_tline<N, 2><<<gz, blk, 0, st>>>(c->Pf, B);
  prof_mark(c, 2, true, st);
}

cudaError_t launch_f32_stage(xg_ctx* c, const xg::FBufs& B, cudaStream_t st) {
  switch (c->d.order) {
    case 1: launch_f32_stage_n<1>(c, B, st); break;
    case 2: launch_f32_stage_n<2>(c, B, st); break;
    case 3: launch_f32_stage_n<3>(c, B, st); break;
    case 4: launch_f32_stage_n<4>(c, B, st); break;
    case 5: launch_f32_stage_n<5>(c, B, st); break;
    case 6: launch_f32_stage_n<6>(c, B, st); break;
    case 7: launch_f32_stage_n<7>(c, B, st); break;
    case 8: launch_f32_stage_n<8>(c, B, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_df_stage(xg_ctx* c, const DfBufs& B, cudaStream_t st, int parts) {
  switch (c->d.order) {
    case 1: launch_df_stage_n<1>(c, B, st, parts); break;
    case 2: launch_df_stage_n<2>(c, B, st, parts); break;
    case 3: launch_df_stage_n<3>(c, B, st, parts); break;
    case 4: launch_df_stage_n<4>(c, B, st, parts); break;
    case 5: launch_df_stage_n<5>(c, B, st, parts); break;
    case 6: launch_df_stage_n<6>(c, B, st, parts); break;
    case 7: launch_df_stage_n<7>(c, B, st, parts); break;
    case 8: launch_df_stage_n<8>(c, B, st, parts); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_stage(xg_ctx* c, const StageBufs& B, cudaStream_t st, int parts) {
  switch (c->d.order) {
    case 1: launch_stage_n<1>(c, B, st, parts); break;
    case 2: launch_stage_n<2>(c, B, st, parts); break;
    case 3: launch_stage_n<3>(c, B, st, parts); break;
    case 4: launch_stage_n<4>(c, B, st, parts); break;
    case 5: launch_stage_n<5>(c, B, st, parts); break;
    case 6: launch_stage_n<6>(c, B, st, parts); break;
    case 7: launch_stage_n<7>(c, B, st, parts); break;
    case 8: launch_stage_n<8>(c, B, st, parts); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t configure(xg_ctx* c) {
  switch (c->d.order) {
    case 1: return configure_n<1>(c);
    case 2: return configure_n<2>(c);
    case 3: return configure_n<3>(c);
    case 4: return configure_n<4>(c);
    case 5: return configure_n<5>(c);
    case 6: return configure_n<6>(c);
    case 7: return configure_n<7>(c);
    case 8: return configure_n<8>(c);
    default: return cudaErrorInvalidValue;
  }
}

StageBufs make_bufs(xg_ctx* c, const double* q, const double* qn, double* out, double dt,
                    double alpha, double beta, int rhs_only) {
  StageBufs B;
  B.q = q;
  B.qn = qn;
  B.out = out;
  B.W = c->W;
  B.T = c->T;
  B.S = c->has_forcing ? c->S : nullptr;
  B.base = c->base;
  B.flag = c->flag;
  B.dt = dt;
  B.alpha = alpha;
  B.beta = beta;
  B.rhs_only = rhs_only;
  B.face_hi = c->part_send[1];
  return B;
}

// One pass of the hot path: the tendency of q, stored as dq/dt (rhs_only)
// or combined as out = alpha qn + beta (q + dt L(q)).  Buffers are device
// arrays of the context's precision.
cudaError_t run_stage(xg_ctx* c, const void* q, const void* qn, void* out, double dt,
                      double alpha, double beta, int rhs_only, cudaStream_t st, int parts = 3) {
  if (c->f32) {
    xg::FBufs F;
    F.C = nullptr;
    if (c->closure) {
      if (!c->cl_fixed) {
        const cudaError_t e = closure_launch(c, (const float*)q, st);
        if (e != cudaSuccess) return e;
      }
      F.C = c->cl_C;
    }
    F.q = (const float*)q;
    F.qn = (const float*)qn;
    F.out = (float*)out;
    F.W = (float*)c->W;
    F.T = (float*)c->T;
    F.S = c->has_forcing ? (const float*)c->S : nullptr;
    F.base = (const df*)c->base;
    F.flag = c->flag;
    F.dt = (float)dt;
    F.alpha = (float)alpha;
    F.beta = (float)beta;
    F.rhs_only = rhs_only;
    return launch_f32_stage(c, F, st);
  }
  if (!c->dfm) {
    StageBufs B = make_bufs(c, (const double*)q, (const double*)qn, (double*)out, dt, alpha, beta,
                            rhs_only);
    if (c->dyn) {
      const cudaError_t e = dynamics_launch(c, (const double*)q, st);
      if (e != cudaSuccess) return e;
      B.E = c->dyn_E;
    }
    return launch_stage(c, B, st, parts);
  }
  DfBufs B;
  B.q = (const double*)q;
  B.qn = (const double*)qn;
  B.out = (double*)out;
  B.W = (df*)c->W;
  B.W64 = c->W + 3 * c->np;
  B.T = c->T;
  B.Tm = (df*)c->T;
  B.S = c->has_forcing ? c->S : nullptr;
  B.base = (const df*)c->base;
  B.base64 = c->base64;
  B.flag = c->flag;
  B.dt = xg::split_df(dt);
  B.alpha = xg::split_df(alpha);
  B.beta = xg::split_df(beta);
  B.bdt = xg::split_df((double)((long double)beta * (long double)dt));
  B.dt64 = dt;
  B.alpha64 = alpha;
  B.beta64 = beta;
  B.rhs_only = rhs_only;
  B.face_hi = c->part_send[1];
  B.Fy = c->Fy;
  return launch_df_stage(c, B, st, parts);
}

// Device FP64 array -> the context's device representation (n values; FP64
// and XG_DF64 contexts hold FP64 arrays).
cudaError_t import_values(xg_ctx* c, const double* src, void* dst, long long n, cudaStream_t st) {
  if (c->f32) {
    xg::k_to_f32<<<conv_blocks(n), 256, 0, st>>>(src, (float*)dst, n);
    return cudaGetLastError();
  }
  return cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st);
}

// The context's device representation -> device FP64 array.
cudaError_t export_values(xg_ctx* c, const void* src, double* dst, long long n, cudaStream_t st) {
  if (c->f32) {
    xg::k_from_f32<<<conv_blocks(n), 256, 0, st>>>((const float*)src, dst, n);
    return cudaGetLastError();
  }
  return cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st);
}

}  // namespace

cudaError_t rhs_f64_state(xg_ctx* c, const double* q, double* out, cudaStream_t st) {
  return run_stage(c, q, nullptr, out, 0.0, 0.0, 1.0, 1, st);
}

extern "C" {

const char* xg_status_str(xg_status s) {
  switch (s) {
    case XG_OK: return "XG_OK";
    case XG_ERR_ARG: return "XG_ERR_ARG";
    case XG_ERR_CUDA: return "XG_ERR_CUDA";
    case XG_ERR_OOM: return "XG_ERR_OOM";
    case XG_ERR_NONFINITE: return "XG_ERR_NONFINITE";
    case XG_ERR_TIMEOUT: return "XG_ERR_TIMEOUT";
    case XG_ERR_UNSUPPORTED: return "XG_ERR_UNSUPPORTED";
  }
  return "XG_UNKNOWN";
}

xg_status xg_mesh_create(const xg_mesh_desc* d, xg_ctx** out) {
  if (!out) return XG_ERR_ARG;
  *out = nullptr;
  if (!d) return XG_ERR_ARG;
  xg::MeshGeom geo;
  const xg_status st = xg::check_desc(d, &geo);
  if (st != XG_OK) return st;
  const int* n = geo.n;
  const long long np = geo.np;
  const size_t xsmem = geo.xsmem;

  xg_ctx* c = new (std::nothrow) xg_ctx();
  if (!c) return XG_ERR_OOM;
  c->d = *d;
  c->n[0] = n[0]; c->n[1] = n[1]; c->n[2] = n[2];
  c->np = np;
  c->xsmem = xsmem;
  cudaError_t e = cudaGetDevice(&c->dev);
  if (e != cudaSuccess) { fail_cuda(c, e, "cudaGetDevice"); delete c; return XG_ERR_CUDA; }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
  if (sms <= 0) sms = 1;

  xg::fill_line_params(d, geo, &c->P);
  c->dfm = d->precision == XG_DF64;
  c->f32 = d->precision == XG_FP32;
  if (c->dfm) xg::fill_df_params(c->P, &c->Pdf);
  if (c->f32) xg::fill_f32_params(c->P, &c->Pf);
  xg::plan_marches(d, geo, sms, &c->chunk_y, &c->nchunk_y, &c->chunk_z, &c->nchunk_z);

  const size_t vec = sizeof(double) * (size_t)np;
  struct { double** p; size_t bytes; } allocs[] = {
      {&c->A, 5 * vec}, {&c->Bq, 5 * vec}, {&c->Cq, 5 * vec}, {&c->Dq, 5 * vec}, {&c->W, 4 * vec},
      {&c->T, 5 * vec}, {&c->S, vec}, {&c->base, sizeof(double) * 4 * (size_t)n[2]},
      {&c->base64, sizeof(double) * 4 * (size_t)n[2]}};
  for (auto& a : allocs) {
    e = cudaMalloc((void**)a.p, a.bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      xg_destroy(c);
      return e == cudaErrorMemoryAllocation ? XG_ERR_OOM : XG_ERR_CUDA;
    }
  }
  e = cudaMalloc((void**)&c->flag, sizeof(int));
  if (e == cudaSuccess && c->dfm)
    e = cudaMalloc((void**)&c->Fy, sizeof(double) * 5 * (size_t)c->P.nseg[1] * (size_t)n[2] * (size_t)n[0]);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->hflag, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->wasm, sizeof(double) * (size_t)(n[0] + n[1] + n[2]));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->partial, sizeof(double) * 5 * kDiagBlocks);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->hdiag, sizeof(double) * 5);
  if (e == cudaSuccess) {
    // assembled 1-D LGL weights per direction (Eq. 8-9 on the uniform box):
    // w_a inside an element, 2 w_0 on a shared face, w_0 on a wall; the
    // Jacobian (h_x h_y h_z / 8) is folded into the x weights
    double wl[xg::kMaxOrder + 1];
    xg::lgl_weights(d->order, wl);
    std::vector<double> wa(n[0] + n[1] + n[2]);
    double J = 1.0;
    for (int k = 0; k < 3; ++k) J *= (d->hi[k] - d->lo[k]) / d->nel[k] / 2.0;
    int off = 0;
    for (int k = 0; k < 3; ++k) {
      for (int g = 0; g < n[k]; ++g) {
        const int a = g % d->order;
        double w = wl[a];
        if (a == 0) w = (d->periodic[k] || (g > 0 && g < n[k] - 1)) ? 2.0 * wl[0] : wl[0];
        wa[off + g] = k == 0 ? w * J : w;
      }
      off += n[k];
    }
    e = cudaMemcpy(c->wasm, wa.data(), sizeof(double) * wa.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = configure(c);
  if (e != cudaSuccess) {
    const bool oom = e == cudaErrorMemoryAllocation;
    fail_cuda(c, e, "xg_mesh_create");
    xg_destroy(c);
    return oom ? XG_ERR_OOM : XG_ERR_CUDA;
  }
  *out = c;
  return XG_OK;
}

xg_status xg_mesh_np(const xg_ctx* c, long long* np) {
  if (!c || !np) return XG_ERR_ARG;
  *np = c->np;
  return XG_OK;
}

xg_status xg_mesh_dims(const xg_ctx* c, int n[3]) {
  if (!c || !n) return XG_ERR_ARG;
  n[0] = c->n[0]; n[1] = c->n[1]; n[2] = c->n[2];
  return XG_OK;
}

xg_status xg_set_state(xg_ctx* c, const double* q, const double* rho0, const double* rhotheta0,
                       int where, void* stream) {
  if (!c || !q) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (where != XG_HOST && where != XG_DEVICE) return XG_ERR_ARG;
  if ((rho0 == nullptr) != (rhotheta0 == nullptr)) return XG_ERR_ARG;
  if (!rho0 && !c->has_base) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int nz = c->n[2];
  if (rho0) {
    double* hb = (double*)malloc(sizeof(double) * 6 * (size_t)nz);
    if (!hb) return XG_ERR_OOM;
    double* r0 = hb + 4 * nz;
    double* t0 = hb + 5 * nz;
    if (where == XG_DEVICE) {
      cudaError_t e = cudaMemcpyAsync(r0, rho0, sizeof(double) * nz, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(t0, rhotheta0, sizeof(double) * nz, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { free(hb); return fail_cuda(c, e, "xg_set_state reference copy"); }
    } else {
      memcpy(r0, rho0, sizeof(double) * nz);
      memcpy(t0, rhotheta0, sizeof(double) * nz);
    }
    const double gamma = c->d.cp / c->d.cv;
    for (int k = 0; k < nz; ++k) {
      if (!(xg::finite_pos(r0[k]) && xg::finite_pos(t0[k]))) { free(hb); return XG_ERR_ARG; }
      hb[k] = r0[k];
      hb[nz + k] = t0[k];
      hb[2 * nz + k] = c->d.p_a * pow(c->d.R * t0[k] / c->d.p_a, gamma);  // Eq. 3
      hb[3 * nz + k] = 1.0 / t0[k];
    }
    // the FP64 table (the rho' and Theta' path of XG_DF64), then for the
    // double-float and FP32 kernels the table as pairs (8 bytes each, in place)
    cudaError_t e = cudaMemcpyAsync(c->base64, hb, sizeof(double) * 4 * nz, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (c->dfm || c->f32) {
      for (int k = 0; k < 4 * nz; ++k) {
        const df v = xg::split_df(hb[k]);
        memcpy(hb + k, &v, sizeof(df));
      }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->base, hb, sizeof(double) * 4 * nz, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    free(hb);
    if (e != cudaSuccess) return fail_cuda(c, e, "xg_set_state reference upload");
    c->has_base = true;
  }
  const long long n5 = 5 * c->np;
  if (!c->f32) {
    XG_CUDA(c, cudaMemcpyAsync(c->A, q, sizeof(double) * (size_t)n5,
                               where == XG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  } else if (where == XG_DEVICE) {
    XG_CUDA(c, import_values(c, q, c->A, n5, st));
  } else {  // host data goes through the stage buffer B as FP64
    XG_CUDA(c, cudaMemcpyAsync(c->Bq, q, sizeof(double) * (size_t)n5, cudaMemcpyHostToDevice, st));
    XG_CUDA(c, import_values(c, c->Bq, c->A, n5, st));
  }
  c->has_state = true;
  return XG_OK;
}

xg_status xg_set_forcing(xg_ctx* c, const double* S, int where, void* stream) {
  if (!c) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (where != XG_HOST && where != XG_DEVICE) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!S) {
    c->has_forcing = false;
    return XG_OK;
  }
  if (!c->f32) {
    XG_CUDA(c, cudaMemcpyAsync(c->S, S, sizeof(double) * (size_t)c->np,
                               where == XG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  } else if (where == XG_DEVICE) {
    XG_CUDA(c, import_values(c, S, c->S, c->np, st));
  } else {
    XG_CUDA(c, cudaMemcpyAsync(c->Cq, S, sizeof(double) * (size_t)c->np, cudaMemcpyHostToDevice, st));
    XG_CUDA(c, import_values(c, c->Cq, c->S, c->np, st));
  }
  c->has_forcing = true;
  return XG_OK;
}

xg_status xg_rhs(xg_ctx* c, double* dqdt, int where, void* stream) {
  if (!c || !dqdt) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (c->part_open[0] || c->part_open[1]) return XG_ERR_UNSUPPORTED;   // xg_partition_stage
  if (where != XG_HOST && where != XG_DEVICE) return XG_ERR_ARG;
  if (!c->has_state) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  double* dst = where == XG_DEVICE ? dqdt : c->Bq;
  const bool tc_waits = c->closure || c->contract != XG_CONTRACT_FMA || column_on(c);   // bounded waits
  if (tc_waits) XG_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int), st));
  if (!c->f32) {
    XG_CUDA(c, run_stage(c, c->A, nullptr, dst, 0.0, 0.0, 1.0, 1, st));
  } else {
    XG_CUDA(c, run_stage(c, c->A, nullptr, c->Cq, 0.0, 0.0, 1.0, 1, st));
    XG_CUDA(c, export_values(c, c->Cq, dst, 5 * c->np, st));
  }
  if (where == XG_HOST) {
    XG_CUDA(c, cudaMemcpyAsync(dqdt, c->Bq, sizeof(double) * 5 * (size_t)c->np,
                               cudaMemcpyDeviceToHost, st));
  }
  if (tc_waits) {   // reports a tensor-core wait that ran out (bit 1 of the flag); waits
    XG_CUDA(c, cudaMemcpyAsync(c->hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    XG_CUDA(c, cudaStreamSynchronize(st));
    prof_fold(c);
    return (*c->hflag & 2) ? XG_ERR_TIMEOUT : XG_OK;
  }
  if (where == XG_HOST || c->profiling) {
    XG_CUDA(c, cudaStreamSynchronize(st));
    prof_fold(c);
  }
  return XG_OK;
}

// nsteps SSP-RK3 steps of the context's state on stream st (no wait)
cudaError_t rk3_steps(xg_ctx* c, double dt, int nsteps, cudaStream_t st) {
  for (int it = 0; it < nsteps; ++it) {
    cudaError_t e = run_stage(c, c->A, nullptr, c->Bq, dt, 0.0, 1.0, 0, st);
    if (e == cudaSuccess) e = run_stage(c, c->Bq, c->A, c->Cq, dt, 0.75, 0.25, 0, st);
    if (e == cudaSuccess) e = run_stage(c, c->Cq, c->A, c->Dq, dt, 1.0 / 3.0, 2.0 / 3.0, 0, st);
    if (e != cudaSuccess) return e;
    double* t = c->A;  // every kernel's arrays stay distinct (no in-place stage)
    c->A = c->Dq;
    c->Dq = t;
  }
  return cudaSuccess;
}

xg_status xg_step(xg_ctx* c, double dt, int nsteps, void* stream) {
  if (!c) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (c->part_open[0] || c->part_open[1]) return XG_ERR_UNSUPPORTED;   // xg_partition_stage
  if (!std::isfinite(dt) || nsteps < 0) return XG_ERR_ARG;
  if (!c->has_state) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  XG_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int), st));
  XG_CUDA(c, rk3_steps(c, dt, nsteps, st));
  XG_CUDA(c, cudaMemcpyAsync(c->hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  XG_CUDA(c, cudaStreamSynchronize(st));
  prof_fold(c);
  if (*c->hflag & 2) return XG_ERR_TIMEOUT;   // the closure kernel's bounded wait ran out
  return *c->hflag ? XG_ERR_NONFINITE : XG_OK;
}

// The staging arrays, copy streams and events of xg_step_stream.
cudaError_t stream_setup(xg_ctx* c) {
  if (c->ss_ready) return cudaSuccess;
  const size_t bytes = sizeof(double) * 5 * (size_t)c->np;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    if (!c->ss_in[b]) e = cudaMalloc((void**)&c->ss_in[b], bytes);
    if (e == cudaSuccess && !c->ss_out[b]) e = cudaMalloc((void**)&c->ss_out[b], bytes);
  }
  int made = 0;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->ss_h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->ss_d2h, cudaStreamNonBlocking);
  for (; made < 12 && e == cudaSuccess; ++made)
    e = cudaEventCreateWithFlags(&c->ss_ev[made], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    for (int b = 0; b < 2; ++b) {
      cudaFree(c->ss_in[b]);
      cudaFree(c->ss_out[b]);
      c->ss_in[b] = c->ss_out[b] = nullptr;
    }
    for (int k = 0; k < made; ++k) cudaEventDestroy(c->ss_ev[k]);
    if (c->ss_h2d) cudaStreamDestroy(c->ss_h2d);
    if (c->ss_d2h) cudaStreamDestroy(c->ss_d2h);
    c->ss_h2d = c->ss_d2h = nullptr;
    return e;
  }
  c->ss_ready = true;
  return cudaSuccess;
}

// xg_step_stream for FP64-state contexts (XG_FP64, XG_DF64): the inputs are
// stepped where they were uploaded.  The state pointer moves to each input's
// array and the output is downloaded from the array the steps leave it in,
// so no state is copied on the device.  Six state-sized arrays rotate: the
// one being stepped (A), the spare of the steps (Dq), and the others, which
// wait in a pool for uploads (oldest first) once their download, or the
// work already queued on st for the state array the call starts from, is
// done.  The context's fields never alias: after every change of A the four
// arrays that are neither A nor Dq are the ss_in / ss_out fields.
xg_status stream_in_place(xg_ctx* c, int count, const double* const* q_in, double* const* q_out, double dt,
                          int nsteps, cudaStream_t st) {
  const size_t bytes = sizeof(double) * 5 * (size_t)c->np;
  double* arr[6] = {c->ss_in[0], c->ss_in[1], c->ss_out[0], c->ss_out[1], c->A, c->Dq};
  cudaEvent_t* ready = c->ss_ev;       // the upload into arr[i] (h2d), later its output (st)
  cudaEvent_t* freed = c->ss_ev + 6;   // arr[i] may be overwritten
  bool pending[6] = {false, false, false, false, false, false};
  auto index_of = [&](const double* p) {
    for (int i = 0; i < 6; ++i)
      if (arr[i] == p) return i;
    return -1;
  };
  auto reassign = [&]() {   // the four arrays that are neither A nor Dq
    double** f[4] = {&c->ss_in[0], &c->ss_in[1], &c->ss_out[0], &c->ss_out[1]};
    int j = 0;
    for (int i = 0; i < 6; ++i)
      if (arr[i] != c->A && arr[i] != c->Dq) *f[j++] = arr[i];
  };
  std::deque<int> pool = {0, 1, 2, 3};
  XG_CUDA(c, cudaEventRecord(freed[4], st));   // the starting state array, after st's queued work
  pending[4] = true;
  pool.push_back(4);
  int next = -1;
  auto upload = [&](int k) -> cudaError_t {
    next = pool.front();
    pool.pop_front();
    cudaError_t e = pending[next] ? cudaStreamWaitEvent(c->ss_h2d, freed[next], 0) : cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(arr[next], q_in[k], bytes, cudaMemcpyHostToDevice, c->ss_h2d);
    if (e == cudaSuccess) e = cudaEventRecord(ready[next], c->ss_h2d);
    return e;
  };
  XG_CUDA(c, upload(0));
  for (int k = 0; k < count; ++k) {
    const int cur = next;
    if (k + 1 < count) XG_CUDA(c, upload(k + 1));
    XG_CUDA(c, cudaStreamWaitEvent(st, ready[cur], 0));
    c->A = arr[cur];
    reassign();
    c->has_state = true;
    XG_CUDA(c, rk3_steps(c, dt, nsteps, st));   // swaps A and Dq only
    const int out = index_of(c->A);
    if (out < 0) return fail_cuda(c, cudaErrorUnknown, "xg_step_stream state array");
    XG_CUDA(c, cudaEventRecord(ready[out], st));
    XG_CUDA(c, cudaStreamWaitEvent(c->ss_d2h, ready[out], 0));
    XG_CUDA(c, cudaMemcpyAsync(q_out[k], arr[out], bytes, cudaMemcpyDeviceToHost, c->ss_d2h));
    XG_CUDA(c, cudaEventRecord(freed[out], c->ss_d2h));
    pending[out] = true;
    pool.push_back(out);
  }
  return XG_OK;
}

xg_status xg_step_stream(xg_ctx* c, int count, const double* const* q_in, double* const* q_out, double dt,
                         int nsteps, void* stream) {
  if (!c || count < 0 || (count > 0 && (!q_in || !q_out))) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (c->part_open[0] || c->part_open[1]) return XG_ERR_UNSUPPORTED;   // xg_partition_stage
  if (!std::isfinite(dt) || nsteps < 0 || !c->has_base) return XG_ERR_ARG;
  for (int k = 0; k < count; ++k)
    if (!q_in[k] || !q_out[k]) return XG_ERR_ARG;
  if (count == 0) return XG_OK;
  {  // an output that overlaps any input would race with the uploads (other stream)
    const uintptr_t len = sizeof(double) * 5 * (uintptr_t)c->np;
    for (int k = 0; k < count; ++k)
      for (int i = 0; i < count; ++i) {
        const uintptr_t o = (uintptr_t)q_out[k], p = (uintptr_t)q_in[i];
        if (o < p + len && p < o + len) return XG_ERR_ARG;
      }
  }
  {
    const cudaError_t e = stream_setup(c);
    if (e == cudaErrorMemoryAllocation) return XG_ERR_OOM;
    if (e != cudaSuccess) return fail_cuda(c, e, "xg_step_stream setup");
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long long n5 = 5 * c->np;
  const size_t bytes = sizeof(double) * (size_t)n5;
  cudaEvent_t* in_ready = c->ss_ev;
  cudaEvent_t* in_used = c->ss_ev + 2;
  cudaEvent_t* out_ready = c->ss_ev + 4;
  cudaEvent_t* drained = c->ss_ev + 6;
  XG_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int), st));
  if (!c->f32) {
    const xg_status r = stream_in_place(c, count, q_in, q_out, dt, nsteps, st);
    if (r != XG_OK) return r;
    XG_CUDA(c, cudaMemcpyAsync(c->hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    XG_CUDA(c, cudaStreamSynchronize(c->ss_d2h));
    XG_CUDA(c, cudaStreamSynchronize(c->ss_h2d));
    XG_CUDA(c, cudaStreamSynchronize(st));
    prof_fold(c);
    if (*c->hflag & 2) return XG_ERR_TIMEOUT;
    return *c->hflag ? XG_ERR_NONFINITE : XG_OK;
  }
  // XG_FP32: FP64 staging arrays, converted on the device.  The first input;
  // later ones are uploaded while the one before runs
  XG_CUDA(c, cudaMemcpyAsync(c->ss_in[0], q_in[0], bytes, cudaMemcpyHostToDevice, c->ss_h2d));
  XG_CUDA(c, cudaEventRecord(in_ready[0], c->ss_h2d));
  for (int k = 0; k < count; ++k) {
    const int b = k & 1, nb = b ^ 1;
    if (k + 1 < count) {   // upload input k + 1 once input k - 1's staging array is read
      XG_CUDA(c, cudaStreamWaitEvent(c->ss_h2d, in_used[nb], 0));
      XG_CUDA(c, cudaMemcpyAsync(c->ss_in[nb], q_in[k + 1], bytes, cudaMemcpyHostToDevice, c->ss_h2d));
      XG_CUDA(c, cudaEventRecord(in_ready[nb], c->ss_h2d));
    }
    XG_CUDA(c, cudaStreamWaitEvent(st, in_ready[b], 0));
    XG_CUDA(c, import_values(c, c->ss_in[b], c->A, n5, st));
    XG_CUDA(c, cudaEventRecord(in_used[b], st));
    c->has_state = true;
    XG_CUDA(c, rk3_steps(c, dt, nsteps, st));
    // output k into staging once output k - 2 has left it, then download it
    XG_CUDA(c, cudaStreamWaitEvent(st, drained[b], 0));
    XG_CUDA(c, export_values(c, c->A, c->ss_out[b], n5, st));
    XG_CUDA(c, cudaEventRecord(out_ready[b], st));
    XG_CUDA(c, cudaStreamWaitEvent(c->ss_d2h, out_ready[b], 0));
    XG_CUDA(c, cudaMemcpyAsync(q_out[k], c->ss_out[b], bytes, cudaMemcpyDeviceToHost, c->ss_d2h));
    XG_CUDA(c, cudaEventRecord(drained[b], c->ss_d2h));
  }
  XG_CUDA(c, cudaMemcpyAsync(c->hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  XG_CUDA(c, cudaStreamSynchronize(c->ss_d2h));
  XG_CUDA(c, cudaStreamSynchronize(c->ss_h2d));
  XG_CUDA(c, cudaStreamSynchronize(st));
  prof_fold(c);
  if (*c->hflag & 2) return XG_ERR_TIMEOUT;
  return *c->hflag ? XG_ERR_NONFINITE : XG_OK;
}

xg_status xg_get_state(xg_ctx* c, double* q, int where, void* stream) {
  if (!c || !q) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (where != XG_HOST && where != XG_DEVICE) return XG_ERR_ARG;
  if (!c->has_state) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long long n5 = 5 * c->np;
  if (!c->f32) {
    XG_CUDA(c, cudaMemcpyAsync(q, c->A, sizeof(double) * (size_t)n5,
                               where == XG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  } else if (where == XG_DEVICE) {
    XG_CUDA(c, export_values(c, c->A, q, n5, st));
  } else {
    XG_CUDA(c, export_values(c, c->A, c->Bq, n5, st));
    XG_CUDA(c, cudaMemcpyAsync(q, c->Bq, sizeof(double) * (size_t)n5, cudaMemcpyDeviceToHost, st));
  }
  if (where == XG_HOST) XG_CUDA(c, cudaStreamSynchronize(st));
  return XG_OK;
}

xg_status xg_set_fused(xg_ctx* c, int fused) {
  if (!c || (fused != 0 && fused != 1)) return XG_ERR_ARG;
  c->fused = fused != 0;
  return XG_OK;
}

xg_status xg_set_contraction(xg_ctx* c, int mode) {
  if (!c) return XG_ERR_ARG;
  if (mode != XG_CONTRACT_FMA && mode != XG_CONTRACT_TF32X3 && mode != XG_CONTRACT_F16X3) return XG_ERR_ARG;
  static_assert(xg::PlaneTcLayout::N == xg::PlaneH16Layout::N, "both tensor-core forms are of one order");
  if (mode != XG_CONTRACT_FMA && (!c->f32 || c->d.order != xg::PlaneTcLayout::N))
    return XG_ERR_UNSUPPORTED;
  c->contract = mode;
  return XG_OK;
}

xg_status xg_profile(xg_ctx* c, int enable) {
  if (!c) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  c->profiling = enable != 0;
  return XG_OK;
}

xg_status xg_kernel_times(xg_ctx* c, double ms[3], long long launches[3], int reset) {
  if (!c) return XG_ERR_ARG;
  for (int k = 0; k < 3; ++k) {
    if (ms) ms[k] = c->k_ms[k];
    if (launches) launches[k] = c->k_launches[k];
    if (reset) { c->k_ms[k] = 0.0; c->k_launches[k] = 0; }
  }
  return XG_OK;
}

xg_status xg_reciprocal(const double* x, double* out, long long n, void* stream) {
  if (!x || !out || n < 0) return XG_ERR_ARG;
  if (n == 0) return XG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const long long blocks = (n + 255) / 256;
  k_rcp_check<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(x, out, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(nullptr, e, "xg_reciprocal");
  return XG_OK;
}

xg_status xg_partition_set(xg_ctx* c, int open_lo, int open_hi, double* send_lo, double* recv_lo,
                           double* send_hi, double* recv_hi) {
  if (!c) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if ((open_lo != 0 && open_lo != 1) || (open_hi != 0 && open_hi != 1)) return XG_ERR_ARG;
  if ((open_lo || open_hi) && c->d.periodic[1]) return XG_ERR_ARG;
  if (open_lo && (!send_lo || !recv_lo)) return XG_ERR_ARG;
  if (open_hi && (!send_hi || !recv_hi)) return XG_ERR_ARG;
  if ((open_lo || open_hi) && (c->f32 || c->dyn || c->closure)) return XG_ERR_UNSUPPORTED;
  c->part_open[0] = open_lo;
  c->part_open[1] = open_hi;
  c->part_send[0] = open_lo ? send_lo : nullptr;
  c->part_recv[0] = open_lo ? recv_lo : nullptr;
  c->part_send[1] = open_hi ? send_hi : nullptr;
  c->part_recv[1] = open_hi ? recv_hi : nullptr;
  c->P.open_y[0] = c->Pdf.open_y[0] = c->Pdf.P64.open_y[0] = open_lo;
  c->P.open_y[1] = c->Pdf.open_y[1] = c->Pdf.P64.open_y[1] = open_hi;
  return XG_OK;
}

xg_status xg_partition_stage(xg_ctx* c, int half, int stage, double dt, double* dqdt, int where,
                             void* stream) {
  if (!c) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (!c->part_open[0] && !c->part_open[1]) return XG_ERR_ARG;
  if ((half != 0 && half != 1) || stage < -1 || stage > 2 || !std::isfinite(dt)) return XG_ERR_ARG;
  if (stage < 0 && half == 1 && (!dqdt || (where != XG_HOST && where != XG_DEVICE))) return XG_ERR_ARG;
  if (!c->has_state) return XG_ERR_ARG;
  if (c->dyn) return XG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  // the stage's buffers, as in xg_step / xg_rhs
  const void* q = c->A;
  const void* qn = nullptr;
  void* out = c->Bq;
  double alpha = 0.0, beta = 1.0;
  if (stage == 1) { q = c->Bq; qn = c->A; out = c->Cq; alpha = 0.75; beta = 0.25; }
  if (stage == 2) { q = c->Cq; qn = c->A; out = c->Dq; alpha = 1.0 / 3.0; beta = 2.0 / 3.0; }
  if (stage < 0) out = where == XG_DEVICE ? (void*)dqdt : (void*)c->Bq;
  const int rhs = stage < 0 ? 1 : 0;
  const long long nf5 = 5ll * c->n[0] * c->n[2];
  const unsigned g = conv_blocks(nf5);
  if (half == 0) {
    if (stage <= 0) XG_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int), st));
    XG_CUDA(c, run_stage(c, q, qn, out, rhs ? 0.0 : dt, alpha, beta, rhs, st, 1));
    if (c->part_open[0]) {
      k_face_pack<double><<<g, 256, 0, st>>>(c->T, c->part_send[0], c->n[0], c->n[1], c->n[2], c->np);
      XG_CUDA(c, cudaGetLastError());
    }
    return XG_OK;
  }
  if (c->dfm)
    k_face_combine<true><<<g, 256, 0, st>>>(c->T, c->part_recv[0], c->part_recv[1], c->part_send[1],
                                            c->n[0], c->n[1], c->n[2], c->np);
  else
    k_face_combine<false><<<g, 256, 0, st>>>(c->T, c->part_recv[0], c->part_recv[1], c->part_send[1],
                                             c->n[0], c->n[1], c->n[2], c->np);
  XG_CUDA(c, cudaGetLastError());
  XG_CUDA(c, run_stage(c, q, qn, out, rhs ? 0.0 : dt, alpha, beta, rhs, st, 2));
  if (stage < 0) {
    if (where == XG_HOST) {
      XG_CUDA(c, cudaMemcpyAsync(dqdt, c->Bq, sizeof(double) * 5 * (size_t)c->np,
                                 cudaMemcpyDeviceToHost, st));
      XG_CUDA(c, cudaStreamSynchronize(st));
    }
    return XG_OK;
  }
  if (stage == 2) {
    double* t = c->A;
    c->A = c->Dq;
    c->Dq = t;
    XG_CUDA(c, cudaMemcpyAsync(c->hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    XG_CUDA(c, cudaStreamSynchronize(st));
    prof_fold(c);
    return *c->hflag ? XG_ERR_NONFINITE : XG_OK;
  }
  return XG_OK;
}

xg_status xg_pressure_perturbation(const xg_ctx* c, const double* theta_p, double* p,
                                   double* x_max, void* stream) {
  if (!c || !theta_p || !p) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (!c->has_base) return XG_ERR_ARG;
  if (x_max) *x_max = c->P.eos_xmax;
  cudaStream_t st = (cudaStream_t)stream;
  const long long nxy = (long long)c->n[0] * c->n[1];
  const unsigned g = conv_blocks(c->np);
  if (c->f32)
    k_eos_check_f32<<<g, 256, 0, st>>>(c->Pf, (const df*)c->base, theta_p, p, c->np, nxy, c->n[2]);
  else if (c->dfm)
    k_eos_check_df<<<g, 256, 0, st>>>(c->Pdf, (const df*)c->base, theta_p, p, c->np, nxy, c->n[2]);
  else
    k_eos_check_fp64<<<g, 256, 0, st>>>(c->P, c->base, theta_p, p, c->np, nxy, c->n[2]);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(const_cast<xg_ctx*>(c), e, "xg_pressure_perturbation");
  return XG_OK;
}

xg_status xg_diagnostics(xg_ctx* c, double out[5], void* stream) {
  if (!c || !out) return XG_ERR_ARG;
  if (c->failed) return XG_ERR_CUDA;
  if (!c->has_state) return XG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (c->f32)
    k_diag_partial<float><<<kDiagBlocks, kDiagThreads, 0, st>>>((const float*)c->A, c->wasm, c->n[0],
                                                                c->n[1], c->n[2], c->np, c->partial);
  else
    k_diag_partial<double><<<kDiagBlocks, kDiagThreads, 0, st>>>(c->A, c->wasm, c->n[0], c->n[1],
                                                                 c->n[2], c->np, c->partial);
  XG_CUDA(c, cudaGetLastError());
  k_diag_final<<<1, 32, 0, st>>>(c->partial, c->T);   // T is free between stages
  XG_CUDA(c, cudaGetLastError());
  XG_CUDA(c, cudaMemcpyAsync(c->hdiag, c->T, sizeof(double) * 5, cudaMemcpyDeviceToHost, st));
  XG_CUDA(c, cudaStreamSynchronize(st));
  for (int v = 0; v < 5; ++v) out[v] = c->hdiag[v];
  return XG_OK;
}

void xg_destroy(xg_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  cudaFree(c->wasm);
  cudaFree(c->partial);
  if (c->hdiag) cudaFreeHost(c->hdiag);
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  cudaFree(c->A);
  cudaFree(c->Bq);
  cudaFree(c->Cq);
  cudaFree(c->Dq);
  cudaFree(c->W);
  cudaFree(c->T);
  cudaFree(c->Fy);
  cudaFree(c->S);
  cudaFree(c->base);
  cudaFree(c->base64);
  cudaFree(c->flag);
  if (c->hflag) cudaFreeHost(c->hflag);
  for (int b = 0; b < 2; ++b) {
    cudaFree(c->ss_in[b]);
    cudaFree(c->ss_out[b]);
  }
  if (c->ss_ready) {
    for (cudaEvent_t e : c->ss_ev) cudaEventDestroy(e);
    cudaStreamDestroy(c->ss_h2d);
    cudaStreamDestroy(c->ss_d2h);
  }
  closure_free(c);
  dynamics_free(c);
  imex_free(c);
  delete c;
}

}  // extern "C"
