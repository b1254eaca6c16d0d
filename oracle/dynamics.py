"""The paper's remaining terms of the dynamics and its RI-velocity diagnostic.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``laplacian`` -- the weak CG Laplacian with a viscosity tensor,
  M^-1 DSS(-sum_k w_k J_k grad(psi_I) . tau grad(q)), written with the
  per-node metric terms of the mesh (Sec. 2.2, Eqs. 8-12 applied to the
  weak form of div(tau grad q); no boundary term, so walls are natural
  zero-flux boundaries).
* ``viscosity_tensor`` -- tau = J E diag(nu_i lambda_i^-1) (J E)^T of
  Sec. 2.4 / Eq. 15: J = dx/dxi, G = J^-1 J^-T, E its orthonormal
  eigenvectors, lambda_i^-1 its eigenvalues in ascending order, with
  nu_i = c_i^(1/alpha) dx_i^2 / dt^(1/alpha) (Eq. 16) for element sizes
  dx_i along the same principal axes.
* ``hyperdiffusion`` -- H = (-1)^(alpha+1) (div tau grad)^alpha q (Eq. 14),
  tau applied at every Laplacian, for all five state variables.
* ``sponge`` -- Rayleigh damping of the vertical momentum in the top layer
  (the paper's implicit sponge after Klemp et al. 2008, Sec. 4.1):
  -gamma(z) rho w with gamma = gamma_max sin^2(pi/2 (z - z_s)/(z_top - z_s))
  above z_s = z_top - depth.
* ``ri_velocity`` -- Sec. 5 (Eq. 18-21): per level the centroid of |u|,
  the tangential speed |(I - e_r e_r - e_z e_z) u| about it, its average
  over equal-width circular strips, and the maximum over strips and levels.
"""

import numpy as np

from . import euler as E
from .mesh import apply_D


def _global(mesh, local):
    """Position of the global nodes from an element-local coordinate field:
    the smallest of a node's copies (a periodic direction's last element
    carries the wrapped image of the first node, one period further on)."""
    out = np.full(mesh.Np, np.inf)
    np.minimum.at(out, mesh.intma.ravel(), np.asarray(local).ravel())
    return out


def element_sizes(mesh):
    """Edge lengths of the (affine) elements along the reference axes."""
    h = (mesh.hi - mesh.lo) / np.asarray(mesh.nel, dtype=np.float64)
    return np.abs(mesh.A @ np.diag(h))          # columns: images of the element edges


def viscosity_tensor(mesh, c, dt, alpha=2):
    """tau [3, 3, Ne, c, b, a] per element-local node (Eq. 15-16)."""
    jac = np.empty((3, 3) + mesh.detJ.shape)
    for i in range(3):
        for j in range(3):
            jac[i, j] = apply_D(mesh.D, mesh.xyz[i], j)
    Jm = np.moveaxis(jac, (0, 1), (-2, -1))              # [..., i, j] = dx_i / dxi_j
    Jinv = np.linalg.inv(Jm)
    G = Jinv @ np.swapaxes(Jinv, -1, -2)
    lam_inv, Evec = np.linalg.eigh(G)                   # ascending eigenvalues lambda^-1
    # element size along each principal axis: the length of J applied to the
    # reference edge (2 units of xi) in the eigenvector direction, scaled by
    # the order to a node spacing
    edge = np.linalg.norm(Jm @ Evec, axis=-2) * 2.0 / mesh.N
    nu = np.asarray(c, dtype=np.float64) ** (1.0 / alpha) * edge ** 2 / dt ** (1.0 / alpha)
    JE = Jm @ Evec
    D = nu * lam_inv
    tau = JE @ (D[..., :, None] * np.swapaxes(JE, -1, -2))
    return np.moveaxis(tau, (-2, -1), (0, 1))


def laplacian(mesh, q, tau):
    """Weak Laplacian M^-1 DSS(-sum w J grad psi . tau grad q) of fields
    q [nv, Np] (collocated LGL quadrature, Eqs. 8-12)."""
    q = np.atleast_2d(q)
    intma = mesh.intma
    wJ = mesh.w3 * mesh.detJ
    out = np.zeros_like(q)
    for v in range(q.shape[0]):
        qe = q[v][intma]
        # physical gradient at element nodes: sum_j dxi_j/dx_d d q/dxi_j
        dq = [apply_D(mesh.D, qe, j) for j in range(3)]
        grad = [sum(mesh.dxi_dx[j, d] * dq[j] for j in range(3)) for d in range(3)]
        flux = [sum(tau[d, e] * grad[e] for e in range(3)) for d in range(3)]
        acc = np.zeros(intma.shape)
        for j in range(3):
            # contravariant component, weighted: w J (dxi_j/dx . tau grad q)
            Fj = wJ * sum(mesh.dxi_dx[j, d] * flux[d] for d in range(3))
            # sum_k D[k, a] F(k): the reference derivative's transpose along j
            acc -= apply_D(mesh.D.T, Fj, j)
        # DSS of the weak contributions (already weighted by w J), Eqs. 10-11
        R = np.zeros(mesh.Np)
        np.add.at(R, intma.ravel(), acc.ravel())
        out[v] = R / E.mass(mesh)
    return out


def hyperdiffusion(mesh, q, tau, alpha=2):
    """H = (-1)^(alpha+1) (div tau grad)^alpha q (Eq. 14)."""
    h = np.asarray(q, dtype=np.float64)
    for _ in range(alpha):
        h = laplacian(mesh, h, tau)
    return (-1.0) ** (alpha + 1) * h


def sponge_rate(z, z_top, depth, gamma_max):
    zs = z_top - depth
    s = np.clip((np.asarray(z) - zs) / depth, 0.0, 1.0)
    return np.where(np.asarray(z) > zs, gamma_max * np.sin(0.5 * np.pi * s) ** 2, 0.0)


def sponge(mesh, q, depth, gamma_max):
    """Tendency [5, Np]: -gamma(z) rho w in the vertical momentum."""
    z = _global(mesh, mesh.xyz[2])
    out = np.zeros_like(np.asarray(q, dtype=np.float64))
    out[3] = -sponge_rate(z, mesh.hi[2], depth, gamma_max) * q[3]
    return out


def ri_velocity(mesh, q, rho0_lev, nstrips=50):
    """(u_RI, centroids [nz, 2], strip means [nz, nstrips]).  Strips of width
    R/nstrips cover r in [0, R), R = half the smaller horizontal box side."""
    x = _global(mesh, mesh.xyz[0])
    y = _global(mesh, mesh.xyz[1])
    gz = mesh.gidx[2]
    rho = rho0_lev[gz] + q[0]
    u, v, w = q[1] / rho, q[2] / rho, q[3] / rho
    speed = np.sqrt(u * u + v * v + w * w)
    L = mesh.hi - mesh.lo
    R = 0.5 * min(L[0], L[1])
    eps = R / nstrips
    nz = mesh.n[2]
    cent = np.zeros((nz, 2))
    means = np.zeros((nz, nstrips))
    for k in range(nz):
        m = gz == k
        s = speed[m]
        tot = s.sum()
        cx = (s * x[m]).sum() / tot if tot > 0 else 0.5 * (mesh.lo[0] + mesh.hi[0])
        cy = (s * y[m]).sum() / tot if tot > 0 else 0.5 * (mesh.lo[1] + mesh.hi[1])
        cent[k] = cx, cy
        rx, ry = x[m] - cx, y[m] - cy
        r = np.sqrt(rx * rx + ry * ry)
        with np.errstate(invalid="ignore", divide="ignore"):
            erx = np.where(r > 0, rx / r, 0.0)
            ery = np.where(r > 0, ry / r, 0.0)
        ur = u[m] * erx + v[m] * ery
        # (I - e_r e_r - e_z e_z) u = horizontal u minus its radial part
        tx, ty = u[m] - ur * erx, v[m] - ur * ery
        ut = np.sqrt(tx * tx + ty * ty)
        idx = np.floor(r / eps).astype(np.int64)
        for j in range(nstrips):
            sel = idx == j
            means[k, j] = ut[sel].mean() if sel.any() else 0.0
    return float(means.max()), cent, means
