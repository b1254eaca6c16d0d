"""Pins for the oracle's LGL points, weights and derivative matrix (Sec. 2.2,
Eq. 5, Eq. 8): closed forms, polynomial exactness, invariants."""

import math

import numpy as np
import pytest

from oracle import lgl


# Closed forms: LGL points are -1, +1 and the roots of P_N'.
#   N = 2: P_2' ~ x                  -> 0;          w = 1/3, 4/3, 1/3
#   N = 3: P_3' ~ 5x^2 - 1           -> +-1/sqrt5;  w = 1/6, 5/6
#   N = 4: P_4' ~ x (7x^2 - 3)       -> 0, +-sqrt(3/7); w = 1/10, 49/90, 32/45
CLOSED = {
    2: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0],
        [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
    # N = 5: roots of P_5' ~ 21x^4 - 14x^2 + 1: x^2 = (7 -+ 2 sqrt7)/21,
    #        w = 1/15, (14 +- sqrt7)/30
    5: ([-1.0, -math.sqrt((7 + 2 * math.sqrt(7)) / 21), -math.sqrt((7 - 2 * math.sqrt(7)) / 21),
         math.sqrt((7 - 2 * math.sqrt(7)) / 21), math.sqrt((7 + 2 * math.sqrt(7)) / 21), 1.0],
        [1 / 15, (14 - math.sqrt(7)) / 30, (14 + math.sqrt(7)) / 30,
         (14 + math.sqrt(7)) / 30, (14 - math.sqrt(7)) / 30, 1 / 15]),
}


@pytest.mark.parametrize("N", sorted(CLOSED))
def test_closed_forms(N):
    x = lgl.lgl_points(N)
    w = lgl.lgl_weights(N, x)
    xc, wc = CLOSED[N]
    assert np.allclose(x, xc, rtol=0, atol=2e-16)
    assert np.allclose(w, wc, rtol=0, atol=4e-16)


@pytest.mark.parametrize("N", range(1, 9))
def test_quadrature_exactness(N):
    """LGL quadrature integrates x^k exactly for k <= 2N - 1 and not for
    k = 2N (which tells it apart from Gauss-Legendre)."""
    x = lgl.lgl_points(N)
    w = lgl.lgl_weights(N, x)
    for k in range(2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    k = 2 * N
    assert abs(np.dot(w, x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("N", range(1, 9))
def test_derivative_exact_for_degree_le_N(N):
    x = lgl.lgl_points(N)
    D = lgl.derivative_matrix(x)
    assert np.max(np.abs(D.sum(axis=1))) < 1e-13          # D 1 = 0
    for k in range(1, N + 1):
        err = np.max(np.abs(D @ x ** k - k * x ** (k - 1)))
        assert err < 1e-13 * max(1, k * k)
    # one degree higher is not differentiated exactly
    k = N + 1
    assert np.max(np.abs(D @ x ** k - k * x ** (k - 1))) > 1e-6


@pytest.mark.parametrize("N", range(1, 9))
def test_derivative_structure(N):
    """Endpoint diagonal entries -/+ N(N+1)/4, centro-antisymmetry
    D[N-i, N-l] = -D[i, l], and D agrees with differentiating the Lagrange
    interpolant by finite differences at an off-node point."""
    x = lgl.lgl_points(N)
    D = lgl.derivative_matrix(x)
    assert abs(D[0, 0] + N * (N + 1) / 4) < 1e-13 * N * N
    assert abs(D[N, N] - N * (N + 1) / 4) < 1e-13 * N * N
    assert np.max(np.abs(D[::-1, ::-1] + D)) < 1e-13 * N * N
    f = np.cos(1.3 * x + 0.2)
    dfn = D @ f
    h = 1e-6
    for i in range(N + 1):
        fd = (lgl.lagrange_eval(x, x[i] + h) - lgl.lagrange_eval(x, x[i] - h)) @ f / (2 * h)
        assert abs(fd[0] - dfn[i]) < 1e-7 * max(1.0, abs(dfn[i]))


def test_weights_sum_and_symmetry():
    for N in range(1, 9):
        x = lgl.lgl_points(N)
        w = lgl.lgl_weights(N, x)
        assert abs(w.sum() - 2.0) < 1e-14
        assert np.allclose(x, -x[::-1], atol=1e-16)
        assert np.allclose(w, w[::-1], atol=1e-15)
        assert abs(w[0] - 2.0 / (N * (N + 1))) < 1e-15
