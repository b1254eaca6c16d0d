"""Pins for oracle/imex.py: the ARK2 tableau's order conditions, the implicit
and explicit stability functions, second-order convergence on a stiff
nonlinear split system (a planted wrong gamma must lose it), the mesh step
against the dense-solve step, and the linear operator as the derivative of
S at the resting reference state."""

import numpy as np
import pytest

from inputs import rng, workloads as W
from oracle import euler as E, imex as X, mesh as M


def test_tableau_order_conditions():
    for A in (X.A_EXP, X.A_IMP):
        assert np.allclose(A.sum(axis=1), X.C, atol=1e-15)
        assert np.isclose(X.B.sum(), 1.0, atol=1e-15)
        assert np.isclose(X.B @ X.C, 0.5, atol=1e-15)
    assert np.isclose(X.GAMMA, 1 - 1 / np.sqrt(2)) and np.isclose(X.A_IMP[2, 2], X.GAMMA)


@pytest.mark.parametrize("z", [-0.3, -2.0, -40.0, 0.5j, -1.0 + 3.0j])
def test_stability_functions(z):
    one = np.ones(3)
    for A, N, Lm in ((X.A_IMP, lambda y: 0 * y, np.array([[z]])),
                     (X.A_EXP, lambda y: z * y, np.array([[0.0]]))):
        R = 1 + z * X.B @ np.linalg.solve(np.eye(3) - z * A, one)
        y1 = X.ark2_step_dense(N, Lm.astype(complex), np.array([1.0 + 0j]), 1.0)
        assert np.isclose(y1[0], R, rtol=1e-13)


def _convergence(A_imp=None):
    if A_imp is not None:
        saved = X.A_IMP.copy()
        X.A_IMP[:] = A_imp
    try:
        Lm = np.array([[-5.0, 1.0], [0.5, -40.0]])
        N = lambda y: np.array([-y[0] * y[1], 0.5 * y[0] ** 2])
        from scipy.integrate import solve_ivp
        y0 = np.array([1.0, 0.5])
        T = 1.0
        ref = solve_ivp(lambda t, y: N(y) + Lm @ y, (0, T), y0, method="Radau", rtol=1e-12,
                        atol=1e-14).y[:, -1]
        errs = []
        for n in (40, 80, 160):
            y = y0.copy()
            for _ in range(n):
                y = X.ark2_step_dense(N, Lm, y, T / n)
            errs.append(np.abs(y - ref).max())
        return np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    finally:
        if A_imp is not None:
            X.A_IMP[:] = saved


def test_second_order_convergence():
    p1, p2 = _convergence()
    assert 1.8 < p1 < 2.3 and 1.8 < p2 < 2.3, (p1, p2)


def test_planted_wrong_gamma_loses_second_order():
    g = 0.3
    A = np.array([[0.0, 0.0, 0.0], [g, g, 0.0], [X.DELTA, X.DELTA, g]])
    p1, p2 = _convergence(A)
    assert p2 < 1.5, (p1, p2)


def _small_case():
    wl = W.box((1, 1, 2), 2, (0.0, 0.0, 0.0), (1000.0, 1000.0, 2000.0), (True, False, False), f=1e-4,
               seed=21)
    m = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"])
    return wl, m, E.Physics(**wl["phys"]), E.Base(wl["rho0"], wl["Theta0"])


def test_mesh_step_matches_dense_solve():
    wl, m, phys, base = _small_case()
    S = lambda s: E.rhs(m, s, base, wl["S_theta"], phys)
    L = lambda s: X.linear_operator(m, s, base, phys)
    n = 5 * m.Np
    Lmat = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        Lmat[:, k] = L(e.reshape(5, m.Np)).ravel()
    N = lambda y: (S(y.reshape(5, m.Np)) - L(y.reshape(5, m.Np))).ravel()
    dt = 2.0
    got = X.ark2_step(S, L, wl["q"], dt)
    ref = X.ark2_step_dense(N, Lmat, wl["q"].ravel(), dt).reshape(5, m.Np)
    for v in range(5):
        assert np.linalg.norm(got[v] - ref[v]) <= 1e-10 * np.linalg.norm(ref[v]), v


def test_linear_operator_is_the_derivative_at_rest():
    """L(v) = d/de S(e v) at e = 0 (f = 0, no heating): central differences."""
    wl, m, phys, base = _small_case()
    phys0 = E.Physics(**dict(wl["phys"], f=0.0))
    v = wl["q"]
    L = X.linear_operator(m, v, base, phys0)
    eps = 1e-6
    fd = (E.rhs(m, eps * v, base, None, phys0) - E.rhs(m, -eps * v, base, None, phys0)) / (2 * eps)
    for k in range(5):
        assert np.linalg.norm(L[k] - fd[k]) <= 1e-6 * np.linalg.norm(fd[k]) + 1e-14, k
    # and it is linear
    u = rng.uniform(5, 5 * m.Np, -1.0, 1.0).reshape(5, m.Np)
    assert np.allclose(X.linear_operator(m, 2 * u + v, base, phys0),
                       2 * X.linear_operator(m, u, base, phys0) + L, rtol=1e-12, atol=1e-14)
