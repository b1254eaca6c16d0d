// xg_noalloc.cu -- the right-hand side for callers that must not allocate
// device memory (see xg_rhs_noalloc in include/xg.h).
//
// The line kernels need scratch beyond their inputs and outputs: W (v, w, p',
// theta per node), T (x + y parts of the tendency), the per-level reference table
// and the non-finite flag.  A context allocates those with cudaMalloc.  Here
// they live in one file-scope __device__ array of fixed size instead, so a
// call allocates nothing: no cudaMalloc, no cudaFree, no allocating library
// routine.  The array exists once per device that loads this library and
// stays until the process exits.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/xg.h"
#include "xg_kernels.cuh"
#include "xg_setup.h"

namespace {

constexpr size_t kScratchDoubles = (size_t)XG_NOALLOC_SCRATCH_BYTES / sizeof(double);
constexpr int kFlagSlots = 32;   // doubles reserved at the end for the int flag

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  In host code the name
// g_scratch is only a host-side stand-in, so the address is looked up once
// per device with cudaGetSymbolAddress (with that device current) and kept.
// The kept address belongs to the device's primary context, the one the CUDA
// runtime uses; it stays valid for the life of the process as long as that
// context is not destroyed (no cudaDeviceReset of the device between calls).
xg_status scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    fprintf(stderr, "xg_rhs_noalloc: cudaGetDevice: %s\n", cudaGetErrorString(e));
    return XG_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return XG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "xg_rhs_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
      return XG_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return XG_OK;
}

// Per-level reference table rho0, Theta0, p0 = p(Theta0) (Eq. 3), 1/Theta0.
__global__ void k_base_table(const double* __restrict__ rho0, const double* __restrict__ rt0,
                             int nz, double p_a, double R, double gamma, double* __restrict__ base) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nz; k += gridDim.x * blockDim.x) {
    const double r = rho0[k], t = rt0[k];
    base[k] = r;
    base[nz + k] = t;
    base[2 * nz + k] = p_a * pow(R * t / p_a, gamma);
    base[3 * nz + k] = 1.0 / t;
  }
}

template <int N>
cudaError_t launch_rhs(const xg::LineParams& P, const xg::StageBufs& B, size_t xsmem,
                       int chunk_y, int nchunk_y, int chunk_z, int nchunk_z, cudaStream_t st) {
  cudaError_t e = xg::raise_dynamic_smem(xg::k_line_x<N>, xsmem);
  if (e != cudaSuccess) return e;
  dim3 gx(P.n[1], P.n[2]);
  xg::k_line_x<N><<<gx, xg::kXThreads, xsmem, st>>>(P, B);
  dim3 gy((P.n[0] + 127) / 128, nchunk_y, P.n[2]);
  xg::k_line_y<N><<<gy, 128, 0, st>>>(P, B, chunk_y);
  dim3 gz((P.n[0] + 127) / 128, nchunk_z, P.n[1]);
  xg::k_line_z<N><<<gz, 128, 0, st>>>(P, B, chunk_z);
  return cudaGetLastError();
}

}  // namespace

extern "C" xg_status xg_rhs_noalloc(const xg_mesh_desc* d, const double* q, const double* rho0,
                                    const double* rhotheta0, const double* S_theta, double* dqdt,
                                    void* stream) {
  if (!d || !q || !rho0 || !rhotheta0 || !dqdt) return XG_ERR_ARG;
  xg::MeshGeom geo;
  const xg_status st = xg::check_desc(d, &geo);
  if (st != XG_OK) return st;
  if (d->precision != XG_FP64) return XG_ERR_UNSUPPORTED;
  const long long np = geo.np;
  // the kernels read q (and S_theta) in other CTAs while dqdt is written:
  // the output must not overlap them (a host-side address comparison)
  auto overlaps = [](const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
  };
  const size_t bytes5 = sizeof(double) * 5 * (size_t)np;
  if (overlaps(q, bytes5, dqdt, bytes5)) return XG_ERR_ARG;
  if (S_theta && overlaps(S_theta, sizeof(double) * (size_t)np, dqdt, bytes5)) return XG_ERR_ARG;
  const int nz = geo.n[2];
  const unsigned long long need = 9ull * (unsigned long long)np + 4ull * (unsigned long long)nz +
                                  kFlagSlots;
  if (need > kScratchDoubles) {
    fprintf(stderr,
            "xg_rhs_noalloc: a mesh of %lld nodes needs %llu bytes of scratch; the static "
            "scratch holds %llu bytes (at most about %llu nodes)\n",
            np, need * 8ull, (unsigned long long)XG_NOALLOC_SCRATCH_BYTES,
            (unsigned long long)((kScratchDoubles - kFlagSlots) / 9));
    return XG_ERR_UNSUPPORTED;
  }
  double* scratch = nullptr;
  xg_status s = scratch_address(&scratch);
  if (s != XG_OK) return s;

  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  xg::LineParams P;
  xg::fill_line_params(d, geo, &P);
  int chunk_y, nchunk_y, chunk_z, nchunk_z;
  xg::plan_marches(d, geo, sms, &chunk_y, &nchunk_y, &chunk_z, &nchunk_z);

  xg::StageBufs B;
  B.q = q;
  B.qn = nullptr;
  B.out = dqdt;
  B.W = scratch;                       // [4][np]
  B.T = scratch + 4 * np;              // [5][np]
  double* base = scratch + 9 * np;     // [4][nz]
  B.base = base;
  B.flag = reinterpret_cast<int*>(base + 4 * nz);
  B.S = S_theta;
  B.dt = 0.0;
  B.alpha = 0.0;
  B.beta = 1.0;
  B.rhs_only = 1;

  cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(B.flag, 0, sizeof(int), cs);
  if (e == cudaSuccess) {
    const double gamma = d->cp / d->cv;
    k_base_table<<<(nz + 127) / 128, 128, 0, cs>>>(rho0, rhotheta0, nz, d->p_a, d->R, gamma, base);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    switch (d->order) {
      case 1: e = launch_rhs<1>(P, B, geo.xsmem, chunk_y, nchunk_y, chunk_z, nchunk_z, cs); break;
      case 2: e = launch_rhs<2>(P, B, geo.xsmem, chunk_y, nchunk_y, chunk_z, nchunk_z, cs); break;
      case 3: e = launch_rhs<3>(P, B, geo.xsmem, chunk_y, nchunk_y, chunk_z, nchunk_z, cs); break;
      case 4: e = launch_rhs<4>(P, B, geo.xsmem, chunk_y, nchunk_y, chunk_z, nchunk_z, cs); break;
      case 5: e = launch_rhs<5>(P, B, geo.xsmem, chunk_y, nchunk_y, chunk_z, nchunk_z, cs); break;
      case 6: e = launch_rhs<6>(P, B, geo.xsmem, chunk_y, nchunk_y, chunk_z, nchunk_z, cs); break;
      case 7: e = launch_rhs<7>(P, B, geo.xsmem, chunk_y, nchunk_y, chunk_z, nchunk_z, cs); break;
      case 8: e = launch_rhs<8>(P, B, geo.xsmem, chunk_y, nchunk_y, chunk_z, nchunk_z, cs); break;
      default: e = cudaErrorInvalidValue;
    }
  }
  if (e != cudaSuccess) {
    fprintf(stderr, "xg_rhs_noalloc: %s\n", cudaGetErrorString(e));
    return XG_ERR_CUDA;
  }
  return XG_OK;
}
