"""Node positions of the structured box meshes, for sampling analytic fields.

Global node g_d along direction d of a box with nel_d order-N elements sits at
lo_d + (e + (xi_a + 1)/2) h_d with g_d = N e + a and h_d = (hi_d - lo_d)/nel_d;
xi are the LGL points (-1, +1 and the roots of P_N'), taken here from numpy's
Legendre-series root finder.  Periodic directions have N nel_d nodes, walled
ones N nel_d + 1."""

import numpy as np
from numpy.polynomial import legendre as npleg


def lgl_points(N):
    if N == 1:
        return np.array([-1.0, 1.0])
    c = np.zeros(N + 1)
    c[N] = 1.0
    r = np.sort(np.real(npleg.legroots(npleg.legder(c))))
    return np.concatenate(([-1.0], r, [1.0]))


def axis_nodes(nel, N, lo, hi, periodic):
    """Positions of the global nodes along one axis."""
    xi = lgl_points(N)
    h = (hi - lo) / nel
    n = N * nel + (0 if periodic else 1)
    g = np.arange(n)
    e = np.minimum(g // N, nel - 1)
    a = g - N * e
    return lo + (e + (xi[a] + 1.0) / 2.0) * h


def node_coords(nel, N, lo, hi, periodic):
    """(x, y, z) arrays over global nodes, I = gx + n_x (gy + n_y gz)."""
    ax = [axis_nodes(nel[d], N, lo[d], hi[d], periodic[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X.reshape(-1), Y.reshape(-1), Z.reshape(-1), ax
