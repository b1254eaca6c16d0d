// xg_batch.cu -- the batched persistent form (include/xg_batch.h).
//
// Many independent XG_FP32 instances (own mesh, order, reference state and
// forcing) advance in one cooperative launch of a persistent kernel.  Every
// stage is two passes over all instances -- x-y plane tiles (f_plane_tile:
// primitives, x and y parts) and z tiles (f_tline_tile: z part, sources,
// walls, inverse mass, SSP-RK3 combination) -- separated by a grid barrier
// with a bounded wait.  The per-node arithmetic is the single-context FP32
// path's (the same device functions), so results are bitwise those of an
// XG_FP32 context; what is batched is only the scheduling.
//
// Data written inside the launch (stage buffers, W, T) is read with
// L2-only loads (the CG variants of the tile functions): L1 is not coherent
// across SMs within a launch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <queue>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/xg_batch.h"
#include "xg_ctx.h"
#include "xg_plane_f32.cuh"
#include "xg_setup.h"

namespace xg {

constexpr int kBatchMinOrder = 3;
constexpr int kBatchMaxOrder = 6;
// 16 warps: z tiles of K segments with K N + 1 <= 16 planes of 32 columns
// (K = 5, 3, 3, 2 for N = 3, 4, 5, 6).  With 2 CTAs an SM sub-partition
// holds 8 warps, which leaves 64 registers per thread.
constexpr int kBatchThreads = kTileCols * 16;
__host__ __device__ constexpr int batch_z_segments(int N) { return (16 - 1) / N; }
constexpr int kBatchPlaneBatch = 1;   // measured: 4.59 vs 4.75 ms per step on the 96-instance batch

__host__ __device__ constexpr int batch_plane_elems(int N, int half) {
  return half ? (N >= 16 ? 1 : 16 / N) : plane_elems_f32(N);
}

// One instance as the persistent kernel reads it (copied to shared memory).
struct alignas(16) BInst {
  FParams P;
  float* buf[4];      // q^n, stage 1, stage 2, q^{n+1} at launch start
  float* W;
  float* T;
  const float* S;     // null: no heating
  const df* base;
  float dt;
  int order;
  int pad[2];
};

constexpr int kGroups = kBatchMaxOrder - kBatchMinOrder + 1;   // tiles grouped by order

// Launch arguments.  Each pass's tile list is grouped by order (group g:
// N = 3 + g) and, within a group, in instance order; goff/gcnt locate the
// groups.  XG_SCHED_LPT permutes the list so that CTA c's tiles of group g
// are lpt[pass][c (kGroups + 1) + g] .. lpt[pass][c (kGroups + 1) + g + 1] - 1.
struct BRun {
  const BInst* inst;
  const int4* items[2];   // pass 0 {inst, bx, by, z}; pass 1 {inst, bx, z-block, y}
  const int* lpt[2];
  int goff[2][kGroups], gcnt[2][kGroups];
  int schedule;
  int plane_half;
  unsigned long long* ctr;  // [2][kGroups] claim counters (XG_SCHED_DYNAMIC)
  unsigned int* bar;        // barrier arrivals since launch start
  int* err;                 // XG_ERR_TIMEOUT once a wait ran out
  int* flag;                // non-finite flag
  int nstages;              // stages in this launch (3 per step, or 1 for a RHS)
  int rhs_only;
  float alpha[3], beta[3];
  long long spin_limit;
  int selftest;             // 1: one barrier that waits for G + 1 arrivals, nothing else
};

static_assert(sizeof(BInst) % 16 == 0, "BInst is copied as int4");
constexpr size_t kInstBytes = (sizeof(BInst) + 127) / 128 * 128;

// Grid barrier with a bounded wait (one thread per CTA polls).  Returns
// false when the launch must end: this CTA's wait ran out (it records
// XG_ERR_TIMEOUT) or another CTA's did.
__device__ __forceinline__ bool grid_barrier(const BRun& R, unsigned target, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(R.bar, 1u);
    int ok = 1;
    long long spins = 0;
    while (true) {
      const unsigned v = *(volatile unsigned*)R.bar;
      if ((int)(v - target) >= 0) break;
      if (*(volatile int*)R.err != 0) { ok = 0; break; }
      if (++spins > R.spin_limit) {
        atomicCAS(R.err, 0, (int)XG_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// The stage's buffers of the instance in shared memory: stage st of step
// parity par (q^n and q^{n+1} trade places every step).
__device__ __forceinline__ FBufs stage_bufs(const BRun& R, const BInst& I, int st, int par) {
  FBufs B;
  float* A = I.buf[par ? 3 : 0];
  float* D = I.buf[par ? 0 : 3];
  B.q = st == 0 ? A : I.buf[st];
  B.qn = st == 0 ? nullptr : A;
  B.out = R.rhs_only ? I.buf[1] : (st == 2 ? D : I.buf[st + 1]);
  B.W = I.W;
  B.T = I.T;
  B.S = I.S;
  B.base = I.base;
  B.C = nullptr;
  B.flag = R.flag;
  B.dt = I.dt;
  B.alpha = R.alpha[st];
  B.beta = R.beta[st];
  B.rhs_only = R.rhs_only;
  return B;
}

// This CTA's tiles of order N in pass PASS of stage s (plane tiles of
// E = batch_plane_elems(N, HALF) elements per side, or z tiles).
template <int N, int HALF, int PASS>
__device__ __noinline__ void run_group(const BRun& R, int s, int st, int par, int& cur,
                                          unsigned char* smb, int* s_item) {
  constexpr int g = N - kBatchMinOrder;
  const int n = R.gcnt[PASS][g];
  if (n == 0) return;
  const int off = R.goff[PASS][g];
  const unsigned G = gridDim.x;
  const int4* items = R.items[PASS];
  BInst& I = *reinterpret_cast<BInst*>(smb);
  float* work = reinterpret_cast<float*>(smb + kInstBytes);
  int k, kend, kstep;
  if (R.schedule == XG_SCHED_LPT) {
    const int* t = R.lpt[PASS] + blockIdx.x * (kGroups + 1) + g;
    k = t[0];
    kend = t[1];
    kstep = 1;
  } else {   // round robin over the whole pass list: position p goes to CTA p mod G
    k = off + (int)((blockIdx.x + G - (unsigned)off % G) % G);
    kend = off + n;
    kstep = G;
  }
  const unsigned long long cbase = (unsigned long long)s * (unsigned long long)(n + G);
  while (true) {
    if (R.schedule == XG_SCHED_DYNAMIC) {
      if (threadIdx.x == 0) *s_item = (int)(atomicAdd(R.ctr + PASS * kGroups + g, 1ull) - cbase);
      __syncthreads();
      k = *s_item;
      __syncthreads();
      if (k >= n) break;
      k += off;
    } else if (k >= kend) {
      break;
    }
    const int4 it = __ldg(items + k);
    if (it.x != cur) {
      const int4* src = reinterpret_cast<const int4*>(R.inst + it.x);
      int4* dst = reinterpret_cast<int4*>(smb);
      for (int t = threadIdx.x; t < (int)(sizeof(BInst) / 16); t += blockDim.x) dst[t] = __ldg(src + t);
      cur = it.x;
      __syncthreads();
    }
    const FBufs B = stage_bufs(R, I, st, par);
    if (PASS == 0)
      f_plane_tile<N, batch_plane_elems(N, HALF), kBatchPlaneBatch, true>(I.P, B, it.y, it.z, it.w, work,
                                                                         threadIdx.x, blockDim.x);
    else   // warps beyond the tile's K N + 1 planes own nothing
      f_tline_tile<N, 2, true, batch_z_segments(N)>(I.P, B, it.y, it.z, it.w, threadIdx.x & 31,
                                                     threadIdx.x >> 5, work);
    __syncthreads();   // the tile's shared arrays are free again
    k += kstep;
  }
}

__global__ void __launch_bounds__(kBatchThreads, 2) k_batch(const __grid_constant__ BRun R) {
  extern __shared__ __align__(128) unsigned char smb[];
  __shared__ int s_ok, s_item;
  const unsigned G = gridDim.x;
  if (R.selftest) {
    grid_barrier(R, G + 1, &s_ok);
    return;
  }
  unsigned nbar = 0;
  int cur = -1;
  for (int s = 0; s < R.nstages; ++s) {
    const int st = R.rhs_only ? 0 : s % 3;
    const int par = R.rhs_only ? 0 : (s / 3) & 1;
    if (R.plane_half) {
      run_group<3, 1, 0>(R, s, st, par, cur, smb, &s_item);
      run_group<4, 1, 0>(R, s, st, par, cur, smb, &s_item);
      run_group<5, 1, 0>(R, s, st, par, cur, smb, &s_item);
      run_group<6, 1, 0>(R, s, st, par, cur, smb, &s_item);
    } else {
      run_group<3, 0, 0>(R, s, st, par, cur, smb, &s_item);
      run_group<4, 0, 0>(R, s, st, par, cur, smb, &s_item);
      run_group<5, 0, 0>(R, s, st, par, cur, smb, &s_item);
      run_group<6, 0, 0>(R, s, st, par, cur, smb, &s_item);
    }
    ++nbar;
    if (!grid_barrier(R, nbar * G, &s_ok)) return;
    run_group<3, 0, 1>(R, s, st, par, cur, smb, &s_item);
    run_group<4, 0, 1>(R, s, st, par, cur, smb, &s_item);
    run_group<5, 0, 1>(R, s, st, par, cur, smb, &s_item);
    run_group<6, 0, 1>(R, s, st, par, cur, smb, &s_item);
    if (s == R.nstages - 1) break;
    ++nbar;
    if (!grid_barrier(R, nbar * G, &s_ok)) return;
  }
}

// Shared memory of one CTA for the orders lo..hi and a plane tile choice.
size_t batch_smem(int lo, int hi, int half) {
  size_t m = 0;
  for (int N = lo; N <= hi; ++N) {
    const int E = batch_plane_elems(N, half);
    const size_t TS = (size_t)E * N;
    const size_t plane = sizeof(float) * 2 * 5 * (TS + 1) * (TS + N + 1);
    const size_t z = sizeof(float) * (size_t)tline_smem_floats(N, batch_z_segments(N));
    m = std::max(m, std::max(plane, z));
  }
  return kInstBytes + m;
}

}  // namespace xg

using xg::BInst;
using xg::BRun;

struct xg_batch {
  std::vector<xg_ctx*> inst;
  int count = 0;
  int lo_order = 8, hi_order = 1;
  int dev = 0;
  int sms = 1;
  xg_batch_tuning tune = {XG_SCHED_LPT, 0, 2, 0.0};
  int grid = 0;                  // CTAs of the current configuration
  size_t smem = 0;
  bool graph_ok = true;          // false once capturing the launch failed
  bool failed = false;
  BInst* dinst = nullptr;        // [count]
  BInst* hinst = nullptr;        // pinned [count]
  // tile lists per plane-tile choice and pass, grouped by order, with the
  // LPT permutation and per-CTA ranges for the grid they were built for
  int4* ditems[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int goff[2][2][xg::kGroups] = {}, gcnt[2][2][xg::kGroups] = {};
  std::vector<int4> hitems[2][2];
  std::vector<double> cost[2][2];
  int4* dlpt[2] = {nullptr, nullptr};   // current configuration's LPT order, per pass
  int* dtbl[2] = {nullptr, nullptr};    // [grid][kGroups + 1] range starts
  int lpt_grid = 0, lpt_half = -1;
  // launch bookkeeping: bar, err, flag, ctr[2][kGroups] (zeroed at every launch)
  unsigned char* dsync = nullptr;
  int* hsync = nullptr;          // pinned copy of err, flag
  cudaStream_t cap = nullptr;
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (stages, rhs_only)
  cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace {

constexpr size_t kSyncBytes = 128;   // bar @0, err @4, flag @8, ctr @16 (2 x 4 x 8 bytes)
constexpr long long kSpinLimit = 20000000;   // ~2 s of 100 ns polls

xg_status batch_fail(xg_batch* b, cudaError_t e, const char* where) {
  fprintf(stderr, "xg_batch: %s: %s\n", where, cudaGetErrorString(e));
  cudaGetLastError();
  b->failed = true;
  return XG_ERR_CUDA;
}

#define XB_CUDA(b, call)                                  \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return batch_fail(b, e_, #call); \
  } while (0)

void drop_graphs(xg_batch* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  b->graphs.clear();
}

// Tile lists of every instance for one plane-tile choice, grouped by
// order, with a cost per tile for the LPT schedule: loaded and owned nodes
// plus a fixed per-tile overhead (in node units).
void build_items(xg_batch* b, int half) {
  for (int pass = 0; pass < 2; ++pass) {
    b->hitems[half][pass].clear();
    b->cost[half][pass].clear();
  }
  const double overhead = 256.0;
  for (int g = 0; g < xg::kGroups; ++g) {
    for (int pass = 0; pass < 2; ++pass) b->goff[half][pass][g] = (int)b->hitems[half][pass].size();
    for (int i = 0; i < b->count; ++i) {
      const xg_ctx* c = b->inst[i];
      const int N = c->d.order;
      if (N != xg::kBatchMinOrder + g) continue;
      const int* nel = c->d.nel;
      const int E = xg::batch_plane_elems(N, half);
      for (int z = 0; z < c->n[2]; ++z)
        for (int by = 0; by < (nel[1] + E - 1) / E; ++by)
          for (int bx = 0; bx < (nel[0] + E - 1) / E; ++bx) {
            b->hitems[half][0].push_back(make_int4(i, bx, by, z));
            const int ex = std::min(E, nel[0] - bx * E), ey = std::min(E, nel[1] - by * E);
            const double own = (double)(ex * N + 1) * (ey * N + 1);
            const double halo = (double)N * ((ex + ey) * N + 2);
            b->cost[half][0].push_back(2.0 * own + halo + overhead);
          }
      const int K = xg::batch_z_segments(N);
      const int xb = (c->n[0] + xg::kTileCols - 1) / xg::kTileCols;
      for (int y = 0; y < c->n[1]; ++y)
        for (int zb = 0; zb < (nel[2] + K - 1) / K; ++zb)
          for (int bx = 0; bx < xb; ++bx) {
            b->hitems[half][1].push_back(make_int4(i, bx, zb, y));
            const int cols = std::min(xg::kTileCols, c->n[0] - bx * xg::kTileCols);
            const int kc = std::min(K, nel[2] - zb * K);
            b->cost[half][1].push_back((double)cols * (kc * N + 1) * 2.5 + (double)cols * N + overhead);
          }
    }
    for (int pass = 0; pass < 2; ++pass)
      b->gcnt[half][pass][g] = (int)b->hitems[half][pass].size() - b->goff[half][pass][g];
  }
}

cudaError_t upload_items(xg_batch* b, int half) {
  for (int pass = 0; pass < 2; ++pass) {
    const auto& h = b->hitems[half][pass];
    cudaError_t e = cudaMalloc((void**)&b->ditems[half][pass], sizeof(int4) * std::max<size_t>(h.size(), 1));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(b->ditems[half][pass], h.data(), sizeof(int4) * h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Longest-processing-time-first assignment of each pass's tiles to the
// grid's CTAs; every CTA's tiles are then ordered by group and instance.
cudaError_t build_lpt(xg_batch* b, int half, int grid) {
  if (b->lpt_grid == grid && b->lpt_half == half) return cudaSuccess;
  constexpr int NG = xg::kGroups;
  for (int pass = 0; pass < 2; ++pass) {
    const auto& items = b->hitems[half][pass];
    const auto& cost = b->cost[half][pass];
    const size_t n = items.size();
    std::vector<int> order(n), group(n);
    for (int g = 0; g < NG; ++g)
      for (int k = 0; k < b->gcnt[half][pass][g]; ++k) group[b->goff[half][pass][g] + k] = g;
    for (size_t k = 0; k < n; ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int g = 0; g < grid; ++g) heap.push({0.0, g});
    std::vector<int> owner(n);
    for (int k : order) {
      Load l = heap.top();
      heap.pop();
      owner[k] = l.second;
      l.first += cost[k];
      heap.push(l);
    }
    std::vector<int> tbl((size_t)grid * (NG + 1), 0), fill((size_t)grid * NG, 0);
    for (size_t k = 0; k < n; ++k) ++fill[(size_t)owner[k] * NG + group[k]];
    int pos = 0;
    for (int c = 0; c < grid; ++c) {
      for (int g = 0; g < NG; ++g) {
        tbl[(size_t)c * (NG + 1) + g] = pos;
        const int cnt = fill[(size_t)c * NG + g];
        fill[(size_t)c * NG + g] = pos;
        pos += cnt;
      }
      tbl[(size_t)c * (NG + 1) + NG] = pos;
    }
    std::vector<int4> perm(std::max<size_t>(n, 1));
    for (size_t k = 0; k < n; ++k) perm[fill[(size_t)owner[k] * NG + group[k]]++] = items[k];
    cudaFree(b->dlpt[pass]);
    cudaFree(b->dtbl[pass]);
    b->dlpt[pass] = nullptr;
    b->dtbl[pass] = nullptr;
    cudaError_t e = cudaMalloc((void**)&b->dlpt[pass], sizeof(int4) * perm.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->dtbl[pass], sizeof(int) * tbl.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->dlpt[pass], perm.data(), sizeof(int4) * perm.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->dtbl[pass], tbl.data(), sizeof(int) * tbl.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  b->lpt_grid = grid;
  b->lpt_half = half;
  return cudaSuccess;
}

// Bring the launch state in line with b->tune: tile lists, grid size, LPT
// ranges.  Drops cached graphs when anything changed.
cudaError_t apply_tuning(xg_batch* b) {
  const int half = b->tune.plane_tile;
  cudaError_t e = cudaSuccess;
  if (!b->ditems[half][0]) {
    build_items(b, half);
    e = upload_items(b, half);
    if (e != cudaSuccess) return e;
  }
  const size_t smem = xg::batch_smem(b->lo_order, b->hi_order, half);
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, xg::k_batch, xg::kBatchThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min(b->tune.ctas_per_sm, occ) * b->sms;
  if (b->tune.schedule == XG_SCHED_LPT) {
    e = build_lpt(b, half, grid);
    if (e != cudaSuccess) return e;
  }
  drop_graphs(b);   // a captured launch holds the old configuration's arguments
  b->grid = grid;
  b->smem = smem;
  return cudaSuccess;
}

BRun make_run(xg_batch* b, int nstages, int rhs_only, int selftest, long long spin_limit) {
  BRun R;
  memset(&R, 0, sizeof(R));
  const int half = b->tune.plane_tile;
  R.inst = b->dinst;
  for (int pass = 0; pass < 2; ++pass) {
    for (int g = 0; g < xg::kGroups; ++g) {
      R.goff[pass][g] = b->goff[half][pass][g];
      R.gcnt[pass][g] = b->gcnt[half][pass][g];
    }
    if (b->tune.schedule == XG_SCHED_LPT) {
      R.items[pass] = b->dlpt[pass];
      R.lpt[pass] = b->dtbl[pass];
    } else {
      R.items[pass] = b->ditems[half][pass];
      R.lpt[pass] = nullptr;
    }
  }
  R.schedule = b->tune.schedule;
  R.plane_half = half;
  R.bar = (unsigned int*)b->dsync;
  R.err = (int*)(b->dsync + 4);
  R.flag = (int*)(b->dsync + 8);
  R.ctr = (unsigned long long*)(b->dsync + 16);
  R.nstages = nstages;
  R.rhs_only = rhs_only;
  // the stage weights exactly as the single-context path rounds them
  const double al[3] = {0.0, 0.75, 1.0 / 3.0}, be[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int k = 0; k < 3; ++k) {
    R.alpha[k] = (float)al[k];
    R.beta[k] = (float)be[k];
  }
  R.spin_limit = spin_limit;
  R.selftest = selftest;
  return R;
}

cudaError_t launch(xg_batch* b, const BRun& R, cudaStream_t st) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(xg::kBatchThreads);
  cfg.dynamicSmemBytes = b->smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaMemsetAsync(b->dsync, 0, kSyncBytes, st);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, xg::k_batch, R);
}

// Refresh the instance records (buffer roles, dt) on `st`.
xg_status upload_instances(xg_batch* b, const double* dt, cudaStream_t st) {
  for (int i = 0; i < b->count; ++i) {
    xg_ctx* c = b->inst[i];
    BInst& h = b->hinst[i];
    h.P = c->Pf;
    h.buf[0] = (float*)c->A;
    h.buf[1] = (float*)c->Bq;
    h.buf[2] = (float*)c->Cq;
    h.buf[3] = (float*)c->Dq;
    h.W = (float*)c->W;
    h.T = (float*)c->T;
    h.S = c->has_forcing ? (const float*)c->S : nullptr;
    h.base = (const xg::df*)c->base;
    h.dt = dt ? (float)dt[i] : 0.0f;
    h.order = c->d.order;
  }
  XB_CUDA(b, cudaMemcpyAsync(b->dinst, b->hinst, sizeof(BInst) * b->count, cudaMemcpyHostToDevice, st));
  return XG_OK;
}

// One persistent launch (through a cached graph when possible); waits for
// it and returns the status it recorded.
xg_status run(xg_batch* b, int nstages, int rhs_only, cudaStream_t st, bool timed, float* ms) {
  const BRun R = make_run(b, nstages, rhs_only, 0, kSpinLimit);
  cudaGraphExec_t exec = nullptr;
  if (b->graph_ok) {
    auto key = std::make_pair(nstages, rhs_only);
    auto it = b->graphs.find(key);
    if (it != b->graphs.end()) {
      exec = it->second;
    } else {
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
      cudaError_t e2 = cudaSuccess;
      if (e == cudaSuccess) {
        e2 = launch(b, R, b->cap);
        e = cudaStreamEndCapture(b->cap, &g);
      }
      if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        exec = nullptr;
        b->graph_ok = false;   // launch directly from now on
      } else {
        b->graphs[key] = exec;
      }
    }
  }
  if (timed) XB_CUDA(b, cudaEventRecord(b->ev[0], st));
  if (exec) XB_CUDA(b, cudaGraphLaunch(exec, st));
  else XB_CUDA(b, launch(b, R, st));
  if (timed) XB_CUDA(b, cudaEventRecord(b->ev[1], st));
  XB_CUDA(b, cudaMemcpyAsync(b->hsync, b->dsync + 4, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  XB_CUDA(b, cudaStreamSynchronize(st));
  if (timed && ms) XB_CUDA(b, cudaEventElapsedTime(ms, b->ev[0], b->ev[1]));
  if (b->hsync[0]) return (xg_status)b->hsync[0];
  return b->hsync[1] ? XG_ERR_NONFINITE : XG_OK;
}

bool valid_tuning(const xg_batch_tuning* t) {
  return t && t->schedule >= XG_SCHED_ROUND_ROBIN && t->schedule <= XG_SCHED_DYNAMIC &&
         (t->plane_tile == 0 || t->plane_tile == 1) && (t->ctas_per_sm == 1 || t->ctas_per_sm == 2);
}

xg_status check_ready(xg_batch* b, const double* dt) {
  for (int i = 0; i < b->count; ++i) {
    if (b->inst[i]->closure) return XG_ERR_UNSUPPORTED;   // the batched kernel has no closure
    if (!b->inst[i]->has_state || b->inst[i]->failed) return XG_ERR_ARG;
    if (dt && !std::isfinite(dt[i])) return XG_ERR_ARG;
  }
  return XG_OK;
}

// Steps advance the roles of q^n and q^{n+1} once per step.
void swap_roles(xg_batch* b, int nsteps) {
  if (nsteps % 2 == 0) return;
  for (xg_ctx* c : b->inst) std::swap(c->A, c->Dq);
}

}  // namespace

extern "C" {

xg_status xg_batch_create(const xg_mesh_desc* d, int count, xg_batch** out) {
  if (!out) return XG_ERR_ARG;
  *out = nullptr;
  if (!d || count < 1 || count > 4096) return XG_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    if (d[i].precision != XG_FP32) return XG_ERR_UNSUPPORTED;
    if (d[i].order < xg::kBatchMinOrder || d[i].order > xg::kBatchMaxOrder) {
      return d[i].order >= 1 && d[i].order <= xg::kMaxOrder ? XG_ERR_UNSUPPORTED : XG_ERR_ARG;
    }
  }
  xg_batch* b = new (std::nothrow) xg_batch();
  if (!b) return XG_ERR_OOM;
  b->count = count;
  for (int i = 0; i < count; ++i) {
    xg_ctx* c = nullptr;
    const xg_status s = xg_mesh_create(&d[i], &c);
    if (s != XG_OK) {
      xg_batch_destroy(b);
      return s;
    }
    b->inst.push_back(c);
    b->lo_order = std::min(b->lo_order, d[i].order);
    b->hi_order = std::max(b->hi_order, d[i].order);
  }
  cudaError_t e = cudaGetDevice(&b->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev);
  if (e == cudaSuccess) {
    const size_t most = std::max(xg::batch_smem(xg::kBatchMinOrder, xg::kBatchMaxOrder, 0),
                                 xg::batch_smem(xg::kBatchMinOrder, xg::kBatchMaxOrder, 1));
    e = xg::raise_dynamic_smem(xg::k_batch, most);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->dinst, sizeof(BInst) * count);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->hinst, sizeof(BInst) * count);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->dsync, kSyncBytes);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->hsync, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev[1]);
  if (e == cudaSuccess) e = apply_tuning(b);
  if (e != cudaSuccess) {
    const bool oom = e == cudaErrorMemoryAllocation;
    batch_fail(b, e, "xg_batch_create");
    xg_batch_destroy(b);
    return oom ? XG_ERR_OOM : XG_ERR_CUDA;
  }
  *out = b;
  return XG_OK;
}

xg_status xg_batch_count(const xg_batch* b, int* count) {
  if (!b || !count) return XG_ERR_ARG;
  *count = b->count;
  return XG_OK;
}

xg_ctx* xg_batch_instance(xg_batch* b, int i) {
  if (!b || i < 0 || i >= b->count) return nullptr;
  return b->inst[i];
}

xg_status xg_batch_step(xg_batch* b, const double* dt, int nsteps, void* stream) {
  if (!b || !dt || nsteps < 0) return XG_ERR_ARG;
  if (b->failed) return XG_ERR_CUDA;
  xg_status s = check_ready(b, dt);
  if (s != XG_OK) return s;
  if (nsteps == 0) return XG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  s = upload_instances(b, dt, st);
  if (s != XG_OK) return s;
  s = run(b, 3 * nsteps, 0, st, false, nullptr);
  if (s == XG_OK || s == XG_ERR_NONFINITE) swap_roles(b, nsteps);
  return s;
}

xg_status xg_batch_rhs(xg_batch* b, double* const* dqdt, int where, void* stream) {
  if (!b || !dqdt) return XG_ERR_ARG;
  if (b->failed) return XG_ERR_CUDA;
  if (where != XG_HOST && where != XG_DEVICE) return XG_ERR_ARG;
  for (int i = 0; i < b->count; ++i)
    if (!dqdt[i]) return XG_ERR_ARG;
  xg_status s = check_ready(b, nullptr);
  if (s != XG_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  s = upload_instances(b, nullptr, st);
  if (s != XG_OK) return s;
  s = run(b, 1, 1, st, false, nullptr);
  if (s != XG_OK && s != XG_ERR_NONFINITE) return s;
  for (int i = 0; i < b->count; ++i) {
    xg_ctx* c = b->inst[i];
    const long long n5 = 5 * c->np;
    double* dst = where == XG_DEVICE ? dqdt[i] : c->Cq;
    const int blocks = (int)std::min<long long>((n5 + 255) / 256, 4096);
    xg::k_from_f32<<<blocks, 256, 0, st>>>((const float*)c->Bq, dst, n5);
    XB_CUDA(b, cudaGetLastError());
    if (where == XG_HOST)
      XB_CUDA(b, cudaMemcpyAsync(dqdt[i], c->Cq, sizeof(double) * (size_t)n5, cudaMemcpyDeviceToHost, st));
  }
  XB_CUDA(b, cudaStreamSynchronize(st));
  return XG_OK;
}

xg_status xg_batch_set_tuning(xg_batch* b, const xg_batch_tuning* t) {
  if (!b || !valid_tuning(t)) return XG_ERR_ARG;
  if (b->failed) return XG_ERR_CUDA;
  const xg_batch_tuning old = b->tune;
  b->tune = *t;
  b->tune.ms_per_step = 0.0;
  const cudaError_t e = apply_tuning(b);
  if (e != cudaSuccess) {
    b->tune = old;
    return batch_fail(b, e, "xg_batch_set_tuning");
  }
  return XG_OK;
}

xg_status xg_batch_get_tuning(const xg_batch* b, xg_batch_tuning* t) {
  if (!b || !t) return XG_ERR_ARG;
  *t = b->tune;
  return XG_OK;
}

xg_status xg_batch_autotune(xg_batch* b, const double* dt, int trial_steps, xg_batch_tuning* chosen,
                            void* stream) {
  if (!b || !dt || trial_steps < 1) return XG_ERR_ARG;
  if (b->failed) return XG_ERR_CUDA;
  xg_status s = check_ready(b, dt);
  if (s != XG_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // save every state (the trials advance it)
  std::vector<float*> saved(b->count, nullptr);
  auto release = [&]() {
    for (float* p : saved) cudaFree(p);
  };
  for (int i = 0; i < b->count; ++i) {
    const size_t bytes = sizeof(float) * 5 * (size_t)b->inst[i]->np;
    cudaError_t e = cudaMalloc((void**)&saved[i], bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(saved[i], b->inst[i]->A, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
      release();
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? XG_ERR_OOM : batch_fail(b, e, "xg_batch_autotune save");
    }
  }
  auto restore = [&]() -> cudaError_t {
    for (int i = 0; i < b->count; ++i) {
      cudaError_t e = cudaMemcpyAsync(b->inst[i]->A, saved[i], sizeof(float) * 5 * (size_t)b->inst[i]->np,
                                      cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(st);
  };
  const xg_batch_tuning start = b->tune;
  xg_batch_tuning best = start;
  best.ms_per_step = 0.0;
  xg_status result = XG_OK;
  for (int sched = XG_SCHED_ROUND_ROBIN; sched <= XG_SCHED_DYNAMIC && result == XG_OK; ++sched)
    for (int half = 0; half < 2 && result == XG_OK; ++half)
      for (int cps = 1; cps <= 2 && result == XG_OK; ++cps) {
        b->tune = {sched, half, cps, 0.0};
        cudaError_t e = apply_tuning(b);
        if (e != cudaSuccess) { result = batch_fail(b, e, "xg_batch_autotune"); break; }
        xg_status r = upload_instances(b, dt, st);
        if (r == XG_OK) r = run(b, 3, 0, st, false, nullptr);   // warm-up step
        if (r == XG_OK) swap_roles(b, 1);
        float ms = 0.0f;
        if (r == XG_OK) r = upload_instances(b, dt, st);
        if (r == XG_OK) r = run(b, 3 * trial_steps, 0, st, true, &ms);
        if (r == XG_OK) swap_roles(b, trial_steps);
        if (r != XG_OK) { result = r; break; }
        e = restore();
        if (e != cudaSuccess) { result = batch_fail(b, e, "xg_batch_autotune restore"); break; }
        const double per = ms / trial_steps;
        if (best.ms_per_step == 0.0 || per < best.ms_per_step) best = {sched, half, cps, per};
      }
  if (result != XG_OK && !b->failed) {
    const cudaError_t e = restore();
    if (e != cudaSuccess) batch_fail(b, e, "xg_batch_autotune restore");
  }
  release();
  if (result != XG_OK) {
    b->tune = start;
    if (!b->failed) apply_tuning(b);
    return result;
  }
  b->tune = best;
  const cudaError_t e = apply_tuning(b);
  if (e != cudaSuccess) return batch_fail(b, e, "xg_batch_autotune");
  b->tune.ms_per_step = best.ms_per_step;
  if (chosen) *chosen = b->tune;
  return XG_OK;
}

xg_status xg_batch_barrier_selftest(xg_batch* b, long long spin_limit, void* stream) {
  if (!b || spin_limit < 1 || spin_limit > 10000000) return XG_ERR_ARG;
  if (b->failed) return XG_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const BRun R = make_run(b, 0, 0, 1, spin_limit);
  XB_CUDA(b, launch(b, R, st));
  XB_CUDA(b, cudaMemcpyAsync(b->hsync, b->dsync + 4, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  XB_CUDA(b, cudaStreamSynchronize(st));
  return b->hsync[0] ? (xg_status)b->hsync[0] : XG_OK;
}

void xg_batch_destroy(xg_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  drop_graphs(b);
  for (xg_ctx* c : b->inst) xg_destroy(c);
  for (int h = 0; h < 2; ++h)
    for (int p = 0; p < 2; ++p) cudaFree(b->ditems[h][p]);
  for (int p = 0; p < 2; ++p) {
    cudaFree(b->dlpt[p]);
    cudaFree(b->dtbl[p]);
  }
  cudaFree(b->dinst);
  cudaFreeHost(b->hinst);
  cudaFree(b->dsync);
  cudaFreeHost(b->hsync);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  delete b;
}

}  // extern "C"
