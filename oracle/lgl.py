"""Legendre-Gauss-Lobatto (LGL) points, weights and the nodal derivative matrix.

Sec. 2.2, Eq. 5: the basis is a tensor product of order-N Lagrange polynomials
h_alpha on the N+1 LGL points of [-1, 1]; Eq. 8 integrates with the LGL
weights at the same points (collocated, "inexact" integration, which makes the
mass matrix diagonal, Eq. 12).

The paper only names these objects; their textbook definitions are:

* LGL points: -1, +1 and the N-1 roots of P_N'(x).  P_N' is (up to a factor)
  the Jacobi polynomial P^{(1,1)}_{N-1}, so the interior points are the
  eigenvalues of the symmetric tridiagonal Jacobi matrix of the weight
  (1 - x^2) (Golub-Welsch).
* LGL weights: w_j = 2 / (N (N+1) P_N(x_j)^2).
* Derivative matrix: D[i, l] = h_l'(x_i), the derivative of the l-th Lagrange
  cardinal polynomial at point i, from the barycentric formula
  D[i, l] = (lam_l / lam_i) / (x_i - x_l) for i != l with
  lam_l = 1 / prod_{k != l} (x_l - x_k), and D[i, i] = -sum_{l != i} D[i, l]
  (the derivative of a constant is zero).

Alg. 2 stores the same matrix transposed (dphi/dxi(l, i)); ``D`` here is
indexed [output point i, input point l], so (D f)_i = sum_l D[i, l] f_l.
"""

import numpy as np


def _real(x):
    """x as a floating array: float64 unless it already is a wider float
    (the extended-precision evaluation keeps np.longdouble throughout)."""
    x = np.asarray(x)
    return x if x.dtype == np.longdouble else np.asarray(x, dtype=np.float64)


def legendre(n, x):
    """P_n(x) by the three-term (Bonnet) recurrence."""
    x = _real(x)
    p0 = np.ones_like(x)
    if n == 0:
        return p0
    p1 = x.copy()
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    return p1


def lgl_points(N):
    """The N+1 LGL points on [-1, 1], ascending (Sec. 2.2, Eq. 5)."""
    if N < 1:
        raise ValueError("order N must be >= 1")
    if N == 1:
        return np.array([-1.0, 1.0])
    m = N - 1  # number of interior points = degree of P^{(1,1)}_{N-1}
    k = np.arange(1, m, dtype=np.float64)
    # monic recurrence coefficients for the weight (1 - x^2):
    # beta_k = k (k + 2) / ((2k + 1)(2k + 3))
    beta = k * (k + 2.0) / ((2.0 * k + 1.0) * (2.0 * k + 3.0))
    J = np.diag(np.sqrt(beta), 1) + np.diag(np.sqrt(beta), -1)
    interior = np.linalg.eigvalsh(J) if m > 1 else np.zeros(1)
    x = np.concatenate(([-1.0], np.sort(interior), [1.0]))
    # symmetrise: the point set is symmetric about 0
    x = 0.5 * (x - x[::-1])
    return x


def lgl_points_extended(N):
    """The LGL points in extended precision (np.longdouble): the FP64 points
    of lgl_points polished by Newton's method on P_N'(x) in np.longdouble,
    with P_N' = N (x P_N - P_{N-1}) / (x^2 - 1) and, from Legendre's equation
    (1 - x^2) P'' - 2 x P' + N (N+1) P = 0, P_N'' = (2 x P_N' - N (N+1) P_N)
    / (1 - x^2).  Quadratic convergence: four steps from FP64 accuracy reach
    the working precision."""
    x = np.asarray(lgl_points(N), dtype=np.longdouble)
    if N < 2:
        return x
    inner = x[1:-1]
    for _ in range(4):
        p, pm = legendre(N, inner), legendre(N - 1, inner)
        dp = N * (inner * p - pm) / (inner * inner - 1)
        d2p = (2 * inner * dp - N * (N + 1) * p) / (1 - inner * inner)
        inner = inner - dp / d2p
    x[1:-1] = inner
    return x


def lgl_weights(N, x=None):
    """LGL quadrature weights w_j = 2 / (N (N+1) P_N(x_j)^2) (Eq. 8)."""
    if x is None:
        x = lgl_points(N)
    return 2.0 / (N * (N + 1) * legendre(N, x) ** 2)


def derivative_matrix(x):
    """D[i, l] = h_l'(x_i) for the Lagrange cardinal basis on points x
    (Alg. 2's dphi/dxi, transposed), barycentric form."""
    x = _real(x)
    n = x.size
    diff = x[:, None] - x[None, :]
    np.fill_diagonal(diff, 1.0)
    lam = 1.0 / np.prod(diff, axis=1)  # barycentric weights lam_l
    D = (lam[None, :] / lam[:, None]) / diff
    np.fill_diagonal(D, 0.0)
    D[np.arange(n), np.arange(n)] = -D.sum(axis=1)
    return D


def lagrange_eval(x, xe):
    """Matrix L[k, l] = h_l(xe_k): values of the cardinal polynomials on x at
    the evaluation points xe (used by the pins to interpolate)."""
    x = np.asarray(x, dtype=np.float64)
    xe = np.atleast_1d(np.asarray(xe, dtype=np.float64))
    L = np.ones((xe.size, x.size))
    for l in range(x.size):
        for k in range(x.size):
            if k != l:
                L[:, l] *= (xe - x[k]) / (x[l] - x[k])
    return L
