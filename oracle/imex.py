"""IMEX additive Runge-Kutta time integration (Sec. 2.3) with a matrix-free
Krylov solve.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper splits dq/dt = S(q) into [S(q) - L(q)] + L(q): the bracket (slow,
advective) explicitly, the linear operator L (fast acoustic and gravity
waves) implicitly, with the second-order ARK2 scheme of Giraldo, Kelly &
Constantinescu (2013) -- ARK(2,3,2)b in the paper's later naming -- and
solves each implicit stage with GMRES (Saad & Schultz 1986), matrix-free.

* ``TABLEAU``: c = (0, 2 gamma, 1); explicit a21 = 2 gamma,
  a31 = 1 - alpha, a32 = alpha; implicit a21 = a22 = gamma,
  a31 = a32 = delta, a33 = gamma; weights b = (delta, delta, gamma) for
  both; gamma = 1 - 1/sqrt(2), delta = 1/(2 sqrt(2)),
  alpha = (3 + 2 sqrt(2))/6.
* ``linear_operator``: L is S linearised about the reference state at rest
  (q = 0), without the Coriolis and heating terms (they stay explicit):
  L_rho' = -div(rho u), L_(rho u) = -grad p'_lin - rho' g k with
  p'_lin = gamma p_0/Theta_0 Theta', L_Theta' = -div(theta_0 rho u) with
  theta_0 = Theta_0/rho_0; the same CG discretisation (gather, derivatives,
  DSS, M^-1) and wall condition as S.
* ``ark2_step``: one step with stage solves (I - dt gamma L) Q_i = b_i, each
  solved on the per-variable scaled system (variable v divided by the
  root-mean-square of b_v) so every variable converges to the same relative
  tolerance.
"""

import numpy as np

from . import euler as E

GAMMA = 1.0 - 1.0 / np.sqrt(2.0)
DELTA = 1.0 / (2.0 * np.sqrt(2.0))
ALPHA = (3.0 + 2.0 * np.sqrt(2.0)) / 6.0

C = np.array([0.0, 2.0 * GAMMA, 1.0])
A_EXP = np.array([[0.0, 0.0, 0.0], [2.0 * GAMMA, 0.0, 0.0], [1.0 - ALPHA, ALPHA, 0.0]])
A_IMP = np.array([[0.0, 0.0, 0.0], [GAMMA, GAMMA, 0.0], [DELTA, DELTA, GAMMA]])
B = np.array([DELTA, DELTA, GAMMA])


def linear_operator(mesh, v, base, phys):
    """L(v) [5, Np] (see the module docstring)."""
    gz = mesh.gidx[2]
    rho0 = base.rho0[gz]
    Th0 = base.Theta0[gz]
    p0 = E.pressure(Th0, phys)
    cp_lin = phys.gamma * p0 / Th0
    th0 = Th0 / rho0
    zero = np.zeros(mesh.Np)
    out = np.zeros((5, mesh.Np))
    out[0] = -E.divergence(mesh, [v[1], v[2], v[3]])
    pl = cp_lin * v[4]
    for d in range(3):
        F = [pl if k == d else zero for k in range(3)]
        out[1 + d] = -E.divergence(mesh, F)
    out[3] -= phys.g * v[0]
    out[4] = -E.divergence(mesh, [th0 * v[1], th0 * v[2], th0 * v[3]])
    return E.apply_walls(mesh, out)


def _scaled_solve(Lfun, b, dt_gamma, x0, solve_tol):
    """Solve (I - dt_gamma L) x = b on the per-variable scaled system with
    scipy's GMRES (a library Krylov routine) to a tight tolerance."""
    from scipy.sparse.linalg import LinearOperator, gmres
    shape = b.shape
    s = np.sqrt(np.mean(b * b, axis=1))
    s = np.where(s > 0, s, 1.0)
    S = s[:, None]

    def mv(xs):
        x = xs.reshape(shape) * S
        return ((x - dt_gamma * Lfun(x)) / S).ravel()

    n = b.size
    A = LinearOperator((n, n), matvec=mv, dtype=np.float64)
    try:
        xs, info = gmres(A, (b / S).ravel(), x0=(x0 / S).ravel(), rtol=solve_tol, atol=0.0,
                         restart=60, maxiter=2000)
    except TypeError:   # SciPy before 1.12 names the relative tolerance ``tol``
        xs, info = gmres(A, (b / S).ravel(), x0=(x0 / S).ravel(), tol=solve_tol, atol=0.0,
                         restart=60, maxiter=2000)
    if info != 0:
        raise RuntimeError("GMRES did not converge (info %d)" % info)
    return xs.reshape(shape) * S


def ark2_step(S, L, q, dt, solve_tol=1e-13):
    """One ARK2 step of dq/dt = S(q) split as [S - L] + L."""
    Q = [q]
    Sv = [S(q)]
    Lv = [L(q)]
    for i in (1, 2):
        b = q.copy()
        for j in range(i):
            Nj = Sv[j] - Lv[j]
            b = b + dt * (A_EXP[i, j] * Nj + A_IMP[i, j] * Lv[j])
        Qi = _scaled_solve(L, b, dt * A_IMP[i, i], Q[-1], solve_tol)
        Q.append(Qi)
        Sv.append(S(Qi))
        Lv.append(L(Qi))
    out = q.copy()
    for i in range(3):
        out = out + dt * B[i] * Sv[i]
    return out


def ark2_step_dense(N, Lmat, y, dt):
    """The same scheme for a small system y' = N(y) + Lmat y with a dense
    direct solve (used by the pins)."""
    I = np.eye(len(y))
    Ys = [y]
    for i in (1, 2):
        b = y.copy()
        for j in range(i):
            b = b + dt * (A_EXP[i, j] * N(Ys[j]) + A_IMP[i, j] * (Lmat @ Ys[j]))
        Ys.append(np.linalg.solve(I - dt * A_IMP[i, i] * Lmat, b))
    return y + dt * sum(B[i] * (N(Ys[i]) + Lmat @ Ys[i]) for i in range(3))
