/*
 * xg_dynamics.h -- the paper's remaining terms of the dynamics on an xg.h
 * context, and its RI-velocity diagnostic.
 *
 * Hyper-diffusion (Sec. 2.4, Eq. 14, alpha = 2): H = -(div tau grad)^2 q for
 * all five state variables, tau applied at each of the two Laplacians.  Each
 * Laplacian is the weak CG form M^-1 DSS(-sum w J grad psi . tau grad q)
 * with no boundary term (walls are natural zero-flux boundaries for it).  On
 * the library's axis-aligned box the tensor of Eq. 15 reduces to
 * tau = diag(nu_x, nu_y, nu_z), with nu = c^(1/2) (h/N)^2 / dt^(1/2) (Eq. 16)
 * and h the element size.  c[0] goes with the largest element size, c[2] with
 * the smallest (ascending eigenvalues of G = J^-1 J^-T); equal sizes keep the
 * x, y, z order.
 *
 * Sponge (Sec. 4.1): Rayleigh damping of the vertical momentum in the top
 * layer, -gamma(z) rho w with gamma = gamma_max sin^2(pi/2 (z - z_s) /
 * depth) above z_s = z_top - depth.
 *
 * With either term set, xg_rhs and xg_step evaluate S(q) + H(q) + sponge,
 * all before the wall condition.  Native FP64 contexts only.
 */
#ifndef XG_DYNAMICS_H
#define XG_DYNAMICS_H

#include "xg.h"

#ifdef __cplusplus
extern "C" {
#endif

/*   hyper_c[3]     c_i of Eq. 16 (>= 0; all zero: no hyper-diffusion)
 *   hyper_dt       the time step of Eq. 16 in seconds (> 0 when hyper_c is set)
 *   sponge_depth   layer thickness in metres (0: no sponge; <= box height)
 *   sponge_gamma   gamma_max in 1/s (>= 0) */
typedef struct {
  double hyper_c[3];
  double hyper_dt;
  double sponge_depth;
  double sponge_gamma;
} xg_dynamics;

/* Set the terms (copied); NULL switches both off.  Allocates two [5][Np]
 * FP64 work arrays on first use.  Errors: XG_ERR_ARG (NULL ctx, a value out
 * of range), XG_ERR_UNSUPPORTED (the context is not XG_FP64), XG_ERR_OOM,
 * XG_ERR_CUDA. */
xg_status xg_set_dynamics(xg_ctx* ctx, const xg_dynamics* dyn);

/* The terms' tendency H(q) + sponge(q) of the current state (no wall
 * condition) into out [5][Np] (host or device per `where`; XG_HOST waits).
 * Zero when no term is set.  Errors: XG_ERR_ARG (NULL, no state),
 * XG_ERR_UNSUPPORTED (not XG_FP64), XG_ERR_CUDA. */
xg_status xg_dynamics_tendency(xg_ctx* ctx, double* out, int where, void* stream);

/* RI velocity of the current state (Sec. 5): per level the centroid
 * x_c(z) = sum |u| x / sum |u| (sums over the level's nodes; the box centre
 * when |u| vanishes), the tangential speed u_theta = |(I - e_r e_r - e_z e_z) u|
 * about it (u = (rho u) / (rho_0 + rho'); the horizontal speed where r = 0),
 * its mean over the nodes of each of nstrips circular strips of width
 * R / nstrips, R = half the smaller horizontal box side (empty strips count
 * 0, nodes beyond R none), and *u_ri = the largest strip mean over all
 * levels.  centroid [n_z][2] and means [n_z][nstrips] are optional host
 * outputs (NULL to skip).  Any precision (FP64 arithmetic on the state read
 * back as FP64); deterministic; waits for the GPU.  Errors: XG_ERR_ARG
 * (NULL ctx or u_ri, nstrips outside [1, 1024], no state), XG_ERR_OOM,
 * XG_ERR_CUDA. */
xg_status xg_ri_velocity(xg_ctx* ctx, int nstrips, double* u_ri, double* centroid, double* means,
                         void* stream);

#ifdef __cplusplus
}
#endif

#endif /* XG_DYNAMICS_H */
