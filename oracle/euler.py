"""Explicit right-hand side of the compressible Euler equations for
perturbations about a hydrostatic reference state, on the CG mesh.

Sec. 2.1, Eq. 1 states the equations for (rho', u, theta') with the reference
fields rho_0(z), theta_0(z) in hydrostatic balance (dp_0/dz = -rho_0 g) and
the pressure from the equation of state, Eq. 3.  Written for the conservative
variables q = (rho', rho u, rho v, rho w, Theta') with rho = rho_0 + rho',
Theta = rho theta = Theta_0 + Theta', Theta_0 = rho_0 theta_0 (the product
rule applied to Eq. 1a-1c; this restatement is checked against Eq. 1 itself by
a manufactured-solution pin):

    d rho'/dt   = -div(rho u)
    d (rho u)/dt = -div(rho u (x) u + p' I) - rho' g k - f k x (rho u)
    d Theta'/dt = -div(Theta u) + rho S_theta

where p' = p(Theta_0 + Theta') - p(Theta_0) with p(Theta) = p_a (R Theta /
p_a)^gamma (Eq. 3), f k x is the f-plane Coriolis term and S_theta the
prescribed heating (a potential-temperature tendency, K/s).  The
hyper-diffusion H of Eq. 1 (Sec. 2.4) is not part of this path (H = 0).

The discrete operator follows Secs. 2.2 and 3.3-3.4:

1. gather the element-local state, q_e(i,j,k,e,m) = q(m, intma(i,j,k,e))
   (Alg. 1, global-to-local);
2. evaluate the fluxes at every element-local node and differentiate them in
   the reference coordinates with the LGL derivative matrix (Alg. 2);
3. form the physical divergence with the metric terms (chain rule, Eq. 5)
   and the pointwise S(q) at each node (Alg. 1, local-to-global: "evaluate
   f(grad q)"), i.e. collocated strong form;
4. multiply by the quadrature weight times Jacobian, w_ijk J_ijk (Eq. 8);
5. direct stiffness summation R_I = sum over (i,e) -> I (Eqs. 10-11, Alg. 3
   gathering, done serially here instead of with atomics), and likewise the
   diagonal mass M_I = sum w J (Eq. 9 with collocated quadrature, Eq. 12);
6. dq_I/dt = R_I / M_I (Eq. 12);
7. no-flux walls (Sec. 4.1): the wall-normal momentum tendency is zero at
   wall nodes.
"""

from dataclasses import dataclass

import numpy as np

from .mesh import apply_D


@dataclass(frozen=True)
class Physics:
    """Physical constants (Eq. 1, Eq. 3) and the f-plane Coriolis parameter."""
    g: float = 9.81
    R: float = 287.0
    cp: float = 1004.5
    cv: float = 717.5
    p_a: float = 1.0e5
    f: float = 0.0

    @property
    def gamma(self):
        return self.cp / self.cv


def pressure(Theta, phys):
    """Eq. 3: p = p_a (rho R theta / p_a)^gamma with Theta = rho theta."""
    return phys.p_a * np.power(phys.R * Theta / phys.p_a, phys.gamma)


def pressure_perturbation(Theta0, Theta_p, phys):
    """p' = p(Theta_0 + Theta') - p(Theta_0) (Eq. 3 minus its reference value).

    Evaluated as p(Theta_0) * expm1(gamma * log1p(Theta'/Theta_0)), which is
    the same quantity without the cancellation of the plain difference (for
    small Theta'/Theta_0 the difference loses digits in proportion to
    Theta_0/Theta')."""
    p0 = pressure(Theta0, phys)
    return p0 * np.expm1(phys.gamma * np.log1p(Theta_p / Theta0))


@dataclass
class Base:
    """Reference state on the global node levels gz = 0 .. n_z - 1 (Sec. 2.1:
    the reference fields depend on z only)."""
    rho0: np.ndarray    # [n_z] reference density
    Theta0: np.ndarray  # [n_z] reference rho_0 theta_0


def fluxes(rho0, Theta0, qv, phys):
    """Flux tensor F[m][d] of the conservative restatement of Eq. 1 at nodes,
    for q = (rho', rho u, rho v, rho w, Theta')."""
    rho = rho0 + qv[0]
    u = [qv[1 + d] / rho for d in range(3)]
    Theta = Theta0 + qv[4]
    pp = pressure_perturbation(Theta0, qv[4], phys)
    F = [[None] * 3 for _ in range(5)]
    for d in range(3):
        F[0][d] = qv[1 + d]                                   # rho u_d
        for i in range(3):
            F[1 + i][d] = qv[1 + i] * u[d] + (pp if i == d else 0.0)  # rho u_i u_d + p' delta
        F[4][d] = Theta * u[d]                                # Theta u_d
    return F


def local_tendency(mesh, q, base, S_theta, phys, elements=None):
    """Pointwise S(q) at every element-local node (steps 1-3 above).

    Returns S[m, e, c, b, a] for the selected elements (all by default)."""
    intma = mesh.intma if elements is None else mesh.intma[elements]
    # Alg. 1, global to local
    qe = q[:, intma]
    gz = mesh.gidx[2][intma]
    rho0 = base.rho0[gz]
    Theta0 = base.Theta0[gz]
    F = fluxes(rho0, Theta0, qe, phys)
    dxi_dx = mesh.dxi_dx if elements is None else mesh.dxi_dx[:, :, elements]
    # Alg. 2 reference derivatives, then div F = sum_d sum_j dxi_j/dx_d dF^d/dxi_j
    dt = np.result_type(qe, mesh.D)      # float64, or np.longdouble when extended
    div = []
    for m in range(5):
        acc = np.zeros(intma.shape, dtype=dt)
        for d in range(3):
            for j in range(3):
                acc += dxi_dx[j, d] * apply_D(mesh.D, F[m][d], j)
        div.append(acc)
    rho = rho0 + qe[0]
    Sth = S_theta[intma] if S_theta is not None else 0.0
    S = np.empty((5,) + intma.shape, dtype=dt)
    S[0] = -div[0]
    S[1] = -div[1] + phys.f * qe[2]          # -f k x (rho u), x component
    S[2] = -div[2] - phys.f * qe[1]          # y component
    S[3] = -div[3] - qe[0] * phys.g          # -rho' g k
    S[4] = -div[4] + rho * Sth               # rho S_theta
    return S


def assemble(mesh, S_local, elements=None):
    """DSS of w J S and of w J (Eqs. 9-11, Alg. 3): returns (R [5, Np], M [Np]).

    With ``elements`` the sums run over that subset only; they are complete
    at every node all of whose elements are in the subset."""
    intma = mesh.intma if elements is None else mesh.intma[elements]
    detJ = mesh.detJ if elements is None else mesh.detJ[elements]
    wJ = mesh.w3[None] * detJ
    dt = np.result_type(S_local, wJ)
    R = np.zeros((S_local.shape[0], mesh.Np), dtype=dt)
    for m in range(S_local.shape[0]):
        np.add.at(R[m], intma.ravel(), (wJ * S_local[m]).ravel())
    M = np.zeros(mesh.Np, dtype=wJ.dtype)
    np.add.at(M, intma.ravel(), wJ.ravel())
    return R, M


def apply_walls(mesh, dqdt):
    """No-flux walls (Sec. 4.1): zero the wall-normal momentum tendency at
    nodes on a non-periodic face (edges and corners: every normal involved)."""
    for d in range(3):
        mask = mesh.wall_nodes(d)
        dqdt[1 + d][mask] = 0.0
    return dqdt


def rhs(mesh, q, base, S_theta, phys):
    """dq/dt = M^{-1} DSS(w J S(q)) with the wall condition (Eq. 12)."""
    S = local_tendency(mesh, q, base, S_theta, phys)
    R, M = assemble(mesh, S)
    return apply_walls(mesh, R / M[None, :])


def rhs_at_nodes(mesh, q, base, S_theta, phys, nodes):
    """Eq. 12 at the given global nodes only: the same steps restricted to the
    stored elements that contain them (used to check large meshes by
    sampling; ``mesh`` may hold just the elements around the nodes, see
    ``mesh.elements_around``)."""
    nodes = np.asarray(nodes)
    el = mesh.elements_containing(nodes)
    S = local_tendency(mesh, q, base, S_theta, phys, elements=el)
    R, M = assemble(mesh, S, elements=el)
    out = R[:, nodes] / M[None, nodes]
    for d in range(3):
        out[1 + d][mesh.wall_nodes(d)[nodes]] = 0.0
    return out


def divergence(mesh, F):
    """Assembled divergence M^{-1} DSS(w J div F) of a nodal vector field
    F [3, Np] (the operator of steps 2-6 alone, for the metric pins)."""
    intma = mesh.intma
    Fe = [F[d][intma] for d in range(3)]
    acc = np.zeros(intma.shape, dtype=np.result_type(Fe[0], mesh.D))
    for d in range(3):
        for j in range(3):
            acc += mesh.dxi_dx[j, d] * apply_D(mesh.D, Fe[d], j)
    R, M = assemble(mesh, acc[None])
    return R[0] / M


def mass(mesh):
    """Diagonal mass M_I = DSS(w J) (Eq. 9 with collocated quadrature)."""
    _, M = assemble(mesh, np.zeros((1,) + mesh.intma.shape, dtype=mesh.D.dtype))
    return M
