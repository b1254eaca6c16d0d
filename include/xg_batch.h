/*
 * xg_batch.h -- batched persistent form of the explicit CG Euler path of
 * xg.h: many independent limited-area instances, each its own mesh (own
 * element counts and polynomial order), own reference state, vortex and
 * heating, advanced together by ONE persistent kernel launch per call.
 *
 * The paper runs one simulator per GPU (Sec. 4, Sec. 5); it notes the model
 * can hold several independent simulation objects, which is what a batch
 * is.  Every instance computes exactly what a single XG_FP32 context of
 * xg.h computes (the same kernels' arithmetic, node by node), so an
 * instance's results equal those of xg_step / xg_rhs on an XG_FP32 context
 * of the same description bit for bit.
 *
 * Execution: one cooperative launch of G = ctas_per_sm x (SM count) CTAs
 * per call runs every pass of every stage of every step of every instance.
 * A pass is a list of tiles (x-y plane tiles of E x E elements per level,
 * then z tiles of 32 columns x K elements); CTAs take tiles according to a
 * schedule (below) and meet at a grid barrier between passes.  Each barrier
 * wait is bounded: a CTA that waits longer than the spin limit records
 * XG_ERR_TIMEOUT and every CTA leaves the launch at its next barrier.  The
 * launch is captured once per step count into a CUDA graph and replayed.
 *
 * Schedules (element-to-CTA assignment):
 *   XG_SCHED_ROUND_ROBIN  tile t of a pass goes to CTA t mod G (tiles in
 *                         instance order);
 *   XG_SCHED_LPT          tiles are assigned ahead of time by longest
 *                         processing time first from a per-tile cost model
 *                         (owned nodes, halo nodes, order), each CTA a
 *                         contiguous range;
 *   XG_SCHED_DYNAMIC      CTAs claim the next tile with an atomic counter.
 * plane_tile selects the x-y tile: 0 = 32/N elements per side (up to 32 x
 * 32 nodes), 1 = 16/N.  xg_batch_autotune times the candidate (schedule,
 * plane_tile, ctas_per_sm) combinations on the batch itself and keeps the
 * fastest.
 *
 * Threads and streams as in xg.h.  Errors as in xg.h; XG_ERR_TIMEOUT is
 * returned by the call whose launch recorded it and leaves the batch usable.
 */
#ifndef XG_BATCH_H
#define XG_BATCH_H

#include "xg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xg_batch xg_batch;

enum { XG_SCHED_ROUND_ROBIN = 0, XG_SCHED_LPT = 1, XG_SCHED_DYNAMIC = 2 };

/* A launch configuration of the persistent kernel.
 *   schedule      XG_SCHED_*
 *   plane_tile    0 or 1 (see above)
 *   ctas_per_sm   1 or 2 (clamped to what fits on an SM)
 *   ms_per_step   filled by xg_batch_autotune / xg_batch_get_tuning: the
 *                 measured milliseconds per SSP-RK3 step of the whole batch
 *                 with this configuration (0 when not measured) */
typedef struct {
  int schedule;
  int plane_tile;
  int ctas_per_sm;
  double ms_per_step;
} xg_batch_tuning;

/* Create a batch of `count` instances (1 <= count <= 4096) from d[0..count-1].
 * Every description must have precision XG_FP32 and order 3..6; anything
 * else is XG_ERR_UNSUPPORTED (a different precision or order runs through
 * the single-instance contexts of xg.h).  Each instance is an xg_ctx owned
 * by the batch (xg_batch_instance).  The initial configuration is
 * {XG_SCHED_LPT, 0, 2}.  Errors: XG_ERR_ARG (NULL, count out of range, an
 * invalid description), XG_ERR_UNSUPPORTED, XG_ERR_OOM, XG_ERR_CUDA. */
xg_status xg_batch_create(const xg_mesh_desc* d, int count, xg_batch** out);

/* Number of instances. */
xg_status xg_batch_count(const xg_batch* b, int* count);

/* The context of instance i (owned by the batch; do not destroy it).  Use
 * the xg.h calls on it to set and read that instance's state, reference
 * state and heating, its right-hand side (xg_rhs) and conservation sums
 * (xg_diagnostics).  xg_step on an instance advances that instance alone.
 * Returns NULL for a NULL batch or i out of range. */
xg_ctx* xg_batch_instance(xg_batch* b, int i);

/* nsteps SSP-RK3 steps of every instance i with its own step dt[i] (host
 * array of `count` values), all in one persistent launch on `stream`.
 * Every instance must have a state.  Waits for the GPU at the end.
 * Errors: XG_ERR_ARG (NULL, nsteps < 0, a dt not finite, an instance
 * without state), XG_ERR_UNSUPPORTED (an instance has a learned closure
 * set, see xg_closure.h: the batched kernel evaluates the plain right-hand
 * side only), XG_ERR_NONFINITE (some instance produced a NaN or Inf),
 * XG_ERR_TIMEOUT, XG_ERR_CUDA. */
xg_status xg_batch_step(xg_batch* b, const double* dt, int nsteps, void* stream);

/* Right-hand sides of every instance for its current state, in one
 * persistent launch: dqdt[i] [5][Np_i] (an array of `count` pointers, each
 * host or device memory as `where` says).  Does not modify any state.
 * Errors: XG_ERR_ARG, XG_ERR_TIMEOUT, XG_ERR_CUDA. */
xg_status xg_batch_rhs(xg_batch* b, double* const* dqdt, int where, void* stream);

/* Time every candidate configuration (3 schedules x 2 plane tiles x
 * ctas_per_sm 1 and 2) over `trial_steps` steps (after one warm-up step)
 * with the steps dt[0..count-1], keep the fastest and return it in *chosen
 * (may be NULL).  The instances' states are saved before and restored
 * after, so the call does not advance the batch.  Waits for the GPU.
 * Errors: XG_ERR_ARG (NULL b or dt, trial_steps < 1, an instance without
 * state), XG_ERR_NONFINITE, XG_ERR_TIMEOUT, XG_ERR_OOM, XG_ERR_CUDA. */
xg_status xg_batch_autotune(xg_batch* b, const double* dt, int trial_steps,
                            xg_batch_tuning* chosen, void* stream);

/* Set or read the configuration.  Errors: XG_ERR_ARG (NULL, a field out of
 * range). */
xg_status xg_batch_set_tuning(xg_batch* b, const xg_batch_tuning* t);
xg_status xg_batch_get_tuning(const xg_batch* b, xg_batch_tuning* t);

/* Self-test of the bounded grid barrier: one persistent launch whose single
 * barrier waits for one arrival more than the grid has, so every CTA's
 * wait runs out after `spin_limit` polls (1 <= spin_limit <= 1e7, each poll
 * sleeps ~0.1 us) and the launch ends.  Returns XG_ERR_TIMEOUT when the
 * timeout was detected as designed and the batch stays usable; XG_OK would
 * mean the wait did not run out.  Errors: XG_ERR_ARG, XG_ERR_CUDA. */
xg_status xg_batch_barrier_selftest(xg_batch* b, long long spin_limit, void* stream);

/* Free the batch and its instances (synchronises the device first).  NULL
 * is a no-op. */
void xg_batch_destroy(xg_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* XG_BATCH_H */
