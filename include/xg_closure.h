/*
 * xg_closure.h -- learned subgrid closure of the explicit right-hand side
 * (an extension: the paper's model has no closure).
 *
 * A coarse XG_FP32 context can add a pointwise correction to its
 * right-hand side:  dq/dt = L(q) + s_out * MLP(clamp((x - mu) * s_in)),
 * (the normalised inputs clamped to [-8, 8]), where x
 * are 21 features of the node -- the five state variables q_v, their
 * assembled gradients d q_v / d x_d (the derivative operator of Eqs. 8-12
 * applied to q_v itself: M^-1 DSS(w J d q_v / d x_d)) and the heating
 * S_theta -- in the order q_0..q_4, dq_0/dx, dq_0/dy, dq_0/dz, dq_1/dx, ...,
 * dq_4/dz, S_theta.  The network is 21 -> 64 -> 64 -> 5 with SiLU
 * (z / (1 + e^-z)) after both hidden layers.  Parameters are one flat FP32
 * array of XG_CLOSURE_PARAMS values: W1 [64][21] (row = output), b1 [64],
 * W2 [64][64], b2 [64], W3 [5][64], b3 [5].
 *
 * Training runs on the GPU with these calls (FP32 arithmetic): features of
 * a state (xg_features), restriction of a fine run's fields to coarse nodes
 * (xg_restrict), per-column statistics (xg_column_stats), the mean-squared
 * error and its gradient over a set of samples (xg_mlp_loss_grad, computed
 * by back-propagation, deterministic), and the Adam update (xg_mlp_adam).
 * Inference (xg_mlp_forward with XG_MLP_BF16, and the closure inside
 * xg_rhs / xg_step) rounds the weights, the normalised features and the
 * hidden activations to bfloat16 and multiplies them on the tensor cores
 * (tcgen05.mma, FP32 accumulation in tensor memory); biases, SiLU and the
 * output scaling are FP32.
 *
 * Arrays: feature and target sets are structure of arrays with a leading
 * dimension: X [21][ld] holds sample s of feature f at X[f * ld + s];
 * T [5][ld] likewise.  All arrays are device memory of the current device
 * unless stated.  Errors as in xg.h.
 */
#ifndef XG_CLOSURE_H
#define XG_CLOSURE_H

#include "xg.h"

#ifdef __cplusplus
extern "C" {
#endif

#define XG_CLOSURE_IN 21
#define XG_CLOSURE_HIDDEN 64
#define XG_CLOSURE_OUT 5
#define XG_CLOSURE_PARAMS 5893

enum { XG_MLP_FP32 = 0, XG_MLP_BF16 = 1 };

/* Features of the current state of an XG_FP32 context into X [21][Np]
 * (float, ld = Np), on `stream`.  Errors: XG_ERR_ARG (NULL, no state),
 * XG_ERR_UNSUPPORTED (the context is not XG_FP32), XG_ERR_CUDA. */
xg_status xg_features(xg_ctx* ctx, float* X, void* stream);

/* Evaluate nvar FP64 fields src [nvar][Np_fine] of the mesh of `fine` at
 * the nodes of `coarse`: dst [nvar][Np_coarse].  Inside each fine element
 * the field is its tensor-product Lagrange interpolant on the element's LGL
 * nodes (Eq. 4); the value at a coarse node is that interpolant evaluated
 * there.  Both meshes must cover the same box with the same periodicity
 * (any element counts and orders).  Allocates and frees its own scratch;
 * waits for the GPU.  Errors: XG_ERR_ARG (NULL, nvar < 1, different boxes
 * or periodicity), XG_ERR_OOM, XG_ERR_CUDA. */
xg_status xg_restrict(const xg_ctx* fine, const xg_ctx* coarse, const double* src, int nvar,
                      double* dst, void* stream);

/* Mean and standard deviation (population, two passes, FP64 sums in a
 * fixed order) of each of the ncol columns of X [ncol][ld] over its first n
 * samples, into HOST arrays mean[ncol], stdev[ncol].  Waits for the GPU.
 * Errors: XG_ERR_ARG, XG_ERR_CUDA. */
xg_status xg_column_stats(const float* X, int ncol, long long ld, long long n, double* mean,
                          double* stdev, void* stream);

/* Mean-squared error over the n samples and 5 outputs of the network on
 * normalised inputs clamp((X - in_mean) * in_scale) against normalised targets
 * T / out_scale, and its gradient with respect to the parameters:
 * grad [XG_CLOSURE_PARAMS] (device), *loss (host).  FP32 arithmetic,
 * deterministic (per-block partial sums added in a fixed order).  Waits
 * for the GPU.  Errors: XG_ERR_ARG (NULL, n < 1, ld < n), XG_ERR_OOM,
 * XG_ERR_CUDA. */
xg_status xg_mlp_loss_grad(const float* params, const float* X, const float* T, long long ld,
                           long long n, const float* in_mean, const float* in_scale,
                           const float* out_scale, float* grad, double* loss, void* stream);

/* One Adam step (Kingma & Ba 2015) of t >= 1 on nparams values: m, v are
 * the moment arrays (zero before the first step).  Errors: XG_ERR_ARG,
 * XG_ERR_CUDA. */
xg_status xg_mlp_adam(float* params, float* m, float* v, const float* grad, int nparams, int t,
                      double lr, double beta1, double beta2, double eps, void* stream);

/* The correction out_scale * MLP(clamp((X - in_mean) * in_scale)) for n samples
 * into Y [5][ldy]: XG_MLP_FP32 (the training arithmetic) or XG_MLP_BF16
 * (the inference arithmetic, tensor cores).  Waits for the GPU.  Errors:
 * XG_ERR_ARG, XG_ERR_TIMEOUT (a bounded wait for the tensor cores ran out),
 * XG_ERR_OOM, XG_ERR_CUDA. */
xg_status xg_mlp_forward(const float* params, const float* X, long long ld, long long n,
                         const float* in_mean, const float* in_scale, const float* out_scale,
                         float* Y, long long ldy, int precision, void* stream);

/* Enable the closure on an XG_FP32 context: from now on xg_rhs and
 * xg_step evaluate L(q) + correction (before the wall condition, which
 * therefore still holds).  params, in_mean [21], in_scale [21] and
 * out_scale [5] are copied (bfloat16 weights for inference).  params NULL
 * disables it (the plain right-hand side).  Errors: XG_ERR_ARG,
 * XG_ERR_UNSUPPORTED (not XG_FP32), XG_ERR_OOM, XG_ERR_CUDA. */
xg_status xg_closure_set(xg_ctx* ctx, const float* params, const float* in_mean,
                         const float* in_scale, const float* out_scale, void* stream);

/* A prescribed correction instead of the network's, on an XG_FP32
 * context: from now on xg_rhs and xg_step evaluate L(q) + C in every stage
 * (before the wall condition), with C [5][Np] (device, FP64) rounded to FP32
 * and copied.  It replaces an enabled network (xg_closure_set replaces it in
 * turn); C NULL removes a prescribed correction.  This is how a correction
 * computed elsewhere -- e.g. the exact refined-minus-coarse tendency of the
 * training target, held over a step -- is tested in a coarse run.  Errors:
 * XG_ERR_ARG, XG_ERR_UNSUPPORTED (not XG_FP32), XG_ERR_OOM, XG_ERR_CUDA. */
xg_status xg_correction_set(xg_ctx* ctx, const double* C, void* stream);

/* The closure's training targets as one elementwise operation over n FP64
 * device values: out = s (a - b), e.g. R L_fine(q_fine) - L_coarse(R q_fine)
 * (s = 1) or (R q_fine(t + dt) - S_coarse(R q_fine(t))) / dt (s = 1 / dt).
 * out may alias a or b.  Errors: XG_ERR_ARG (NULL, n < 0), XG_ERR_CUDA. */
xg_status xg_closure_target(const double* a, const double* b, double s, long long n, double* out,
                            void* stream);

/* The failure path of the tensor-core kernels' bounded waits, exercised on
 * purpose: one CTA allocates tensor memory, waits at most limit_ns
 * nanoseconds (1 .. 1e9) on an mbarrier that nothing completes, then frees
 * the tensor memory and returns.  Returns XG_ERR_TIMEOUT when the wait ran
 * out (the expected result) and leaves the device usable.  Waits for the GPU.
 * Errors: XG_ERR_ARG, XG_ERR_CUDA. */
xg_status xg_tc_wait_selftest(long long limit_ns, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* XG_CLOSURE_H */
