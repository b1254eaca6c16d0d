/*
 * xg_imex.h -- IMEX time integration of the xg.h path (Sec. 2.3).
 *
 * The right-hand side S(q) is split into a slow part, S - L, taken
 * explicitly, and a linear part L, taken implicitly. L carries the fast
 * acoustic and gravity waves: S linearised about the resting hydrostatic
 * reference state, without Coriolis and heating.
 *   L_rho'   = -div(rho u)
 *   L_rho u  = -grad p'_lin - rho' g k,   p'_lin = gamma p_0 / Theta_0 * Theta'
 *   L_Theta' = -div(theta_0 rho u),       theta_0 = Theta_0 / rho_0
 * L uses the same CG discretisation and no-flux walls as S.
 *
 * Each step is the second-order additive Runge-Kutta scheme ARK2 of
 * Giraldo, Kelly & Constantinescu (2013).
 *   c = (0, 2g, 1), g = 1 - 1/sqrt(2), d = 1/(2 sqrt 2), a = (3 + 2 sqrt 2)/6
 *   explicit tableau:  a21 = 2g;  a31 = 1 - a, a32 = a
 *   implicit tableau:  a21 = a22 = g;  a31 = a32 = d, a33 = g
 *   weights b = (d, d, g) for both tableaux
 * Each implicit stage solves (I - dt g L) Q = b matrix-free with restarted
 * GMRES. Every product applies L on the fly; only the Krylov vectors are
 * stored. The inner product weights variable v by 1 / rms(b_v)^2, which is
 * GMRES on the system scaled per variable, so that rho', the momentum and
 * Theta' each reach the relative tolerance.
 *
 * XG_FP64 and XG_DF64 contexts. L, GMRES and every combination of
 * vectors are FP64 in both; the explicit part S is the context's own stage
 * in right-hand-side mode (in XG_DF64 the mixed stage of xg.h, the
 * rho' and Theta' tendencies in FP64 and the momentum in double-float).
 * Hyper-diffusion and the sponge of xg_dynamics.h (XG_FP64 only), when
 * set, belong to the explicit part.
 */
#ifndef XG_IMEX_H
#define XG_IMEX_H

#include "xg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Solver options.
 *   tol           relative residual of each stage solve, in the weighted
 *                 norm (default 1e-10; 0 < tol < 1)
 *   krylov        Krylov vectors per restart (default 20; 1..64)
 *   max_restarts  restarts before giving up (default 50; >= 1) */
typedef struct {
  double tol;
  int krylov;
  int max_restarts;
} xg_imex_opts;

/* Solver statistics of one xg_step_imex call.
 *   iterations      GMRES iterations (products with the operator) over all
 *                   stage solves
 *   max_iterations  the largest count of one solve
 *   solves          stage solves (2 per step)
 *   max_residual    the largest final relative residual
 *   reorthogonalised  Arnoldi steps whose first Gram-Schmidt pass cancelled
 *                   severely (removed more than 1 - 1e-4 of |w|^2) and that
 *                   took a second */
typedef struct {
  long long iterations;
  int max_iterations;
  int solves;
  double max_residual;
  long long reorthogonalised;
} xg_imex_stats;

/* nsteps ARK2 steps of size dt; opts and stats may be NULL. The first call
 * allocates the krylov + 9 work arrays of [5][Np] doubles. Waits for the GPU.
 * Errors:
 *   XG_ERR_ARG          NULL ctx, dt not finite or <= 0, nsteps < 0, an
 *                       option out of range, no state
 *   XG_ERR_UNSUPPORTED  an XG_FP32 context, or a partitioned one
 *   XG_ERR_TIMEOUT      a stage solve did not reach tol within its restarts;
 *                       the state is left at the start of that step
 *   XG_ERR_NONFINITE, XG_ERR_OOM, XG_ERR_CUDA */
xg_status xg_step_imex(xg_ctx* ctx, double dt, int nsteps, const xg_imex_opts* opts,
                       xg_imex_stats* stats, void* stream);

/* out [5][Np] = L(v) for device arrays v, out (the test hook of the linear
 * operator). Errors: XG_ERR_ARG, XG_ERR_UNSUPPORTED (XG_FP32), no
 * reference state yet, XG_ERR_CUDA. */
xg_status xg_linear_operator(xg_ctx* ctx, const double* v, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* XG_IMEX_H */
