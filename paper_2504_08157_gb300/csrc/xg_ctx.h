// xg_ctx.h -- the context behind the opaque xg_ctx handle of include/xg.h:
// one mesh, its launch constants and its device buffers.  Shared by the
// single-instance entry points (xg_api.cu) and the batched persistent form
// (xg_batch.cu), which advances many contexts in one launch.
#pragma once

#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/xg.h"
#include "xg_kernels.cuh"
#include "xg_kernels_df.cuh"
#include "xg_kernels_f32.cuh"

struct xg_ctx {
  xg_mesh_desc d;
  int n[3];
  long long np;
  int dev;
  xg::LineParams P;
  xg::DfParams Pdf;      // launch constants of the double-float kernels
  xg::FParams Pf;        // launch constants of the FP32 kernels
  bool dfm = false;      // precision XG_DF64: FP64 arrays, mixed FP64 / double-float kernels
  bool f32 = false;      // precision XG_FP32: device arrays hold floats
  int contract = 0;      // XG_FP32: arithmetic of the x and y contractions (XG_CONTRACT_*)
  // XG_FP32: the fused column pass where the mesh allows it (xg_set_fused,
  // opt-in), and the TMA maps of its stage inputs (one per distinct q
  // buffer, encoded on first use)
  bool fused = false;
  // xg_step_stream: four FP64 state-sized arrays for the streamed inputs and
  // outputs, the two copy streams and their events (allocated on first use).
  // XG_FP32 stages through them (in_ready[2], in_used[2], out_ready[2],
  // out_drained[2] in ss_ev[0..7]); FP64-state contexts rotate them with A
  // and Dq (ready[6], freed[6]), never aliasing A or Dq between calls
  double* ss_in[2] = {nullptr, nullptr};
  double* ss_out[2] = {nullptr, nullptr};
  cudaStream_t ss_h2d = nullptr, ss_d2h = nullptr;
  cudaEvent_t ss_ev[12] = {};
  bool ss_ready = false;
  CUtensorMap col_map[4];
  const void* col_key[4] = {nullptr, nullptr, nullptr, nullptr};
  int col_next = 0;
  double* A = nullptr;   // q^n (the state)
  double* Bq = nullptr;  // stage buffer
  double* Cq = nullptr;  // stage buffer
  double* Dq = nullptr;  // q^{n+1}; swapped with A after every step
  double* W = nullptr;   // [4][np] primitives v, w, p', theta (FP32: [3][np])
  double* T = nullptr;   // [5][np] partial tendency
  double* Fy = nullptr;  // XG_DF64: [5][nseg_y][nz][nx] y-face rows between the y and z passes
  double* S = nullptr;   // [np] heating
  double* base = nullptr;  // [4][nz] (double-float pairs for XG_DF64 and XG_FP32)
  double* base64 = nullptr;  // [4][nz] the same table in FP64
  double* wasm = nullptr;  // assembled 1-D mass weights: [n_x + n_y + n_z], J folded into x
  double* partial = nullptr;  // [kDiagBlocks][5] per-block conservation sums
  double* hdiag = nullptr;    // pinned [5]
  int* flag = nullptr;
  int* hflag = nullptr;  // pinned
  bool has_state = false;
  bool has_base = false;
  bool has_forcing = false;
  bool failed = false;
  int chunk_y = 1, nchunk_y = 1, chunk_z = 1, nchunk_z = 1;
  size_t xsmem = 0;
  // profiling: event pairs recorded around launches since the last fold
  bool profiling = false;
  std::vector<cudaEvent_t> events;
  std::vector<int> ev_kernel;   // kernel id of each recorded pair
  size_t ev_used = 0;           // pairs recorded
  double k_ms[3] = {0, 0, 0};
  long long k_launches[3] = {0, 0, 0};
  // learned closure (XG_FP32 only): packed bfloat16 network and the
  // correction of the current stage's input state
  bool closure = false;
  bool cl_fixed = false;  // C is a prescribed correction (xg_correction_set), not the network's
  void* cl_pack = nullptr;
  float* cl_C = nullptr;
  int cl_grid = 0;       // persistent grid of the closure kernel
  // hyper-diffusion and sponge (XG_FP64 only): line-operator constants,
  // work arrays and the extra tendency E of the current stage
  bool dyn = false, dyn_hyper = false;
  void* dyn_params = nullptr;
  double* dyn_L1 = nullptr;
  double* dyn_E = nullptr;
  double* dyn_gamma = nullptr;   // [n_z] sponge rate per level
  // IMEX work arrays (xg_imex.cu), allocated on first use
  void* imex = nullptr;
  // element partition along y (xg_partition_set): which y ends are
  // partition faces, and the caller's face buffers [5][n_z][n_x] (8-byte
  // values) sent to / received from the neighbours on those sides
  int part_open[2] = {0, 0};
  double* part_send[2] = {nullptr, nullptr};
  double* part_recv[2] = {nullptr, nullptr};
};

void imex_free(xg_ctx* c);
// the right-hand side S(q) of an FP64-state context (XG_FP64, or XG_DF64 by
// the mixed stage) into out, both [5][Np] doubles (xg_api.cu)
cudaError_t rhs_f64_state(xg_ctx* c, const double* q, double* out, cudaStream_t st);

// E = H(q) + sponge(q) of the FP64 stage input q into c->dyn_E
// (xg_dynamics.cu); and freeing its buffers.
cudaError_t dynamics_launch(xg_ctx* c, const double* q, cudaStream_t st);
void dynamics_free(xg_ctx* c);

// The closure's correction C = MLP(features(q)) of the stage input q into
// c->cl_C (xg_closure.cu); and freeing its buffers.
cudaError_t closure_launch(xg_ctx* c, const float* q, cudaStream_t st);
void closure_free(xg_ctx* c);
