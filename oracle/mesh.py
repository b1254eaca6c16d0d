"""Hexahedral CG mesh of a box: elements, the local-to-global map and metrics.

Sec. 2.2: the domain is split into N_e disjoint hexahedra; inside each element
the state is expanded in (N+1)^3 tensor-product LGL nodes (Eqs. 4-5), the
reference coordinates (xi, eta, zeta) in E = [-1, 1]^3 map to physical x via
metric terms, and neighbouring elements share the nodes of their common faces,
edges and corners (the CG space of Eq. 6).  ``intma`` is the paper's
local-to-global node map (Alg. 1, Alg. 3).

Conventions (they are the library's data layout, so both sides use them):

* element e = ex + nel_x (ey + nel_y ez);
* local node (a, b, c) in [0, N]^3 is stored at [e, c, b, a] (xi fastest);
* global nodes per direction: n_d = N nel_d, or N nel_d + 1 when direction d
  is not periodic; global node I = gx + n_x (gy + n_y gz) with
  g_d = (N e_d + a_d) mod n_d;
* the physical point of a node is the affine image A @ (box point) of the
  box point lo + (e_d + (xi_a + 1) / 2) (hi - lo) / nel_d; A = identity is
  the axis-aligned box.

Metric terms are computed per node from the node coordinates with the
derivative matrix, the general isoparametric recipe (Eq. 5, Eq. 8), even
though every mesh here is affine.
"""

from dataclasses import dataclass, field

import numpy as np

from . import lgl


def apply_D(D, f, axis):
    """Reference derivative along one local direction of element arrays laid
    out [..., c, b, a] (Alg. 2: q_xi(i,j,k) = sum_l dphi/dxi(l,i) q(l,j,k)).
    axis 0 -> xi (last array axis), 1 -> eta, 2 -> zeta."""
    ax = f.ndim - 1 - axis
    g = np.moveaxis(f, ax, -1)
    g = g @ D.T  # out[..., i] = sum_l D[i, l] g[..., l]
    return np.moveaxis(g, -1, ax)


@dataclass
class Mesh:
    N: int
    nel: tuple
    periodic: tuple
    lo: np.ndarray
    hi: np.ndarray
    A: np.ndarray
    n: tuple                      # global nodes per direction (nx, ny, nz)
    Np: int
    xi: np.ndarray                # LGL points
    w: np.ndarray                 # LGL weights
    D: np.ndarray                 # derivative matrix
    intma: np.ndarray             # [Ne, N+1, N+1, N+1] -> global node
    xyz: np.ndarray               # [3, Ne, c, b, a] physical node coordinates
    gidx: tuple                   # (gx, gy, gz) integer indices of global nodes
    dxi_dx: np.ndarray = field(repr=False, default=None)  # [3 (xi_j), 3 (x_i), Ne, c, b, a]
    detJ: np.ndarray = field(repr=False, default=None)    # [Ne, c, b, a]
    w3: np.ndarray = field(repr=False, default=None)      # [c, b, a] tensor weights

    elem_ids: np.ndarray = field(repr=False, default=None)  # global ids of the stored elements

    @property
    def Ne(self):
        return int(self.intma.shape[0])

    def wall_nodes(self, d):
        """Boolean mask over global nodes lying on a wall normal to direction
        d (empty when d is periodic)."""
        if self.periodic[d]:
            return np.zeros(self.Np, dtype=bool)
        g = self.gidx[d]
        return (g == 0) | (g == self.n[d] - 1)

    def elements_containing(self, nodes):
        """Sorted positions (rows of intma) of the stored elements whose
        local nodes include any of the global node ids in ``nodes``."""
        hit = np.isin(self.intma.reshape(self.Ne, -1), np.asarray(nodes)).any(axis=1)
        return np.nonzero(hit)[0]


def elements_around(nel, N, periodic, nodes):
    """Global ids of every element that contains one of the global nodes:
    along each direction a node g belongs to element g // N, and also to
    element g // N - 1 when it sits on a face (g % N == 0); indices wrap in
    periodic directions and stop at walls."""
    n = [N * nel[d] + (0 if periodic[d] else 1) for d in range(3)]
    nodes = np.asarray(nodes, dtype=np.int64)
    g = [nodes % n[0], (nodes // n[0]) % n[1], nodes // (n[0] * n[1])]
    out = set()
    for k in range(nodes.size):
        choices = []
        for d in range(3):
            gd = int(g[d][k])
            c = []
            for e in (gd // N, gd // N - 1 if gd % N == 0 else None):
                if e is None:
                    continue
                if periodic[d]:
                    c.append(e % nel[d])
                elif 0 <= e < nel[d]:
                    c.append(e)
            choices.append(sorted(set(c)))
        for ex in choices[0]:
            for ey in choices[1]:
                for ez in choices[2]:
                    out.add(ex + nel[0] * (ey + nel[1] * ez))
    return np.array(sorted(out), dtype=np.int64)


def build_mesh(nel, N, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
               periodic=(False, False, False), A=None, elements=None, dtype=np.float64):
    """Build the CG mesh of a box of nel = (nel_x, nel_y, nel_z) order-N
    hexahedra (Sec. 2.2) and its per-node metric terms.  With ``elements``
    (global element ids) only those elements are stored; the global node
    numbering is that of the whole box.

    dtype=np.longdouble builds the same mesh in extended precision (LGL
    points from lgl_points_extended; box corners, A and every derived array
    in np.longdouble), for evaluating the same definitions with rounding far
    below FP64's where a result is a small residual of large terms; the
    euler functions then compute in extended precision when given
    np.longdouble state arrays."""
    nel = tuple(int(v) for v in nel)
    periodic = tuple(bool(p) for p in periodic)
    if min(nel) < 1 or N < 1:
        raise ValueError("need nel >= 1 and N >= 1")
    if dtype not in (np.float64, np.longdouble):
        raise ValueError("dtype must be np.float64 or np.longdouble")
    lo = np.asarray(lo, dtype=dtype)
    hi = np.asarray(hi, dtype=dtype)
    A = np.eye(3, dtype=dtype) if A is None else np.asarray(A, dtype=dtype)
    n = tuple(N * nel[d] + (0 if periodic[d] else 1) for d in range(3))
    Np = n[0] * n[1] * n[2]

    xi = lgl.lgl_points(N) if dtype == np.float64 else lgl.lgl_points_extended(N)
    w = lgl.lgl_weights(N, xi)
    D = lgl.derivative_matrix(xi)

    # element order e = ex + nel_x (ey + nel_y ez)
    if elements is None:
        elements = np.arange(nel[0] * nel[1] * nel[2], dtype=np.int64)
    elements = np.asarray(elements, dtype=np.int64)
    ex = elements % nel[0]
    ey = (elements // nel[0]) % nel[1]
    ez = elements // (nel[0] * nel[1])
    a = np.arange(N + 1)
    # broadcast to [Ne, c, b, a]
    gx = (N * ex[:, None, None, None] + a[None, None, None, :]) % n[0]
    gy = (N * ey[:, None, None, None] + a[None, None, :, None]) % n[1]
    gz = (N * ez[:, None, None, None] + a[None, :, None, None]) % n[2]
    intma = gx + n[0] * (gy + n[1] * gz)

    h = (hi - lo) / np.asarray(nel, dtype=dtype)
    bx = lo[0] + (ex[:, None, None, None] + (xi[None, None, None, :] + 1.0) / 2.0) * h[0]
    by = lo[1] + (ey[:, None, None, None] + (xi[None, None, :, None] + 1.0) / 2.0) * h[1]
    bz = lo[2] + (ez[:, None, None, None] + (xi[None, :, None, None] + 1.0) / 2.0) * h[2]
    shape = (len(ex), N + 1, N + 1, N + 1)
    box = np.stack([np.broadcast_to(bx, shape), np.broadcast_to(by, shape),
                    np.broadcast_to(bz, shape)])
    xyz = np.einsum("ij,j...->i...", A, box)

    I = np.arange(Np)
    gidx = (I % n[0], (I // n[0]) % n[1], I // (n[0] * n[1]))

    m = Mesh(N=N, nel=nel, periodic=periodic, lo=lo, hi=hi, A=A, n=n, Np=Np,
             xi=xi, w=w, D=D, intma=intma, xyz=xyz, gidx=gidx, elem_ids=elements)
    _metrics(m)
    return m


def _det_inv3(jac):
    """Determinant and inverse of 3 x 3 matrices jac[i, j, ...] by cofactors
    (any float dtype; numpy's linalg has no extended-precision routines):
    det = sum_j jac[0, j] C[0, j], inv[j, i] = C[i, j] / det with the
    cofactors C[i, j] = (-1)^(i+j) minor(i, j)."""
    C = np.empty_like(jac)
    for i in range(3):
        for j in range(3):
            r = [k for k in range(3) if k != i]
            c = [k for k in range(3) if k != j]
            minor = jac[r[0], c[0]] * jac[r[1], c[1]] - jac[r[0], c[1]] * jac[r[1], c[0]]
            C[i, j] = minor if (i + j) % 2 == 0 else -minor
    det = jac[0, 0] * C[0, 0] + jac[0, 1] * C[0, 1] + jac[0, 2] * C[0, 2]
    inv = np.empty_like(jac)
    for i in range(3):
        for j in range(3):
            inv[j, i] = C[i, j] / det
    return det, inv


def _metrics(m):
    """Per-node Jacobian matrix dx_i/dxi_j from the node coordinates with D,
    its determinant J (Eq. 8) and inverse dxi_j/dx_i (Eq. 5)."""
    jac = np.empty((3, 3) + m.xyz.shape[1:], dtype=m.xyz.dtype)  # [x_i, xi_j, ...]
    for i in range(3):
        for j in range(3):
            jac[i, j] = apply_D(m.D, m.xyz[i], j)
    if jac.dtype == np.float64:
        jm = np.moveaxis(jac, (0, 1), (-2, -1))    # [..., i, j]
        m.detJ = np.linalg.det(jm)
        inv = np.linalg.inv(jm)                    # [..., j, i] = dxi_j/dx_i
        m.dxi_dx = np.moveaxis(inv, (-2, -1), (0, 1))
    else:
        m.detJ, m.dxi_dx = _det_inv3(jac)
    w = m.w
    m.w3 = w[:, None, None] * w[None, :, None] * w[None, None, :]
