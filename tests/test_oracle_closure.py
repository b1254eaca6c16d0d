"""Pins for the oracle's closure pieces (oracle/closure.py): the MLP
gradient against central finite differences (with planted mistakes that the
check must catch), closed forms of SiLU, the network and the first Adam
step, bfloat16 rounding on known ties, features that are exact for
polynomial fields, and fine-to-coarse restriction that reproduces
polynomials and inverts prolongation."""

import numpy as np
import pytest

from inputs import rng
from oracle import closure as C, mesh as M

SMALL = (4, 6, 5, 3)


def _problem(sizes=SMALL, n=7, seed=5):
    u = rng.uniform(seed, C.param_count(sizes) + n * (sizes[0] + sizes[-1]), -1.0, 1.0)
    P = C.param_count(sizes)
    p = u[:P] * 0.8
    X = u[P:P + n * sizes[0]].reshape(n, sizes[0]) * 2.0
    T = u[P + n * sizes[0]:].reshape(n, sizes[-1])
    return p, X, T


def _fd_grad(f, p, h=1e-6):
    g = np.zeros_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        g[k] = (f(p + e) - f(p - e)) / (2 * h)
    return g


def test_param_count_of_the_closure_net():
    assert C.param_count() == 21 * 64 + 64 + 64 * 64 + 64 + 64 * 5 + 5 == 5893


def test_gradient_matches_finite_differences():
    p, X, T = _problem()
    loss, g = C.loss_and_grad(p, X, T, SMALL)
    assert np.isclose(loss, np.mean((C.forward(p, X, SMALL) - T) ** 2))
    fd = _fd_grad(lambda q: C.loss_and_grad(q, X, T, SMALL)[0], p)
    assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(fd)


def test_planted_gradient_mistakes_are_caught(monkeypatch):
    """The finite-difference check fails if the SiLU derivative is dropped
    or the output residual's factor 2 is lost."""
    p, X, T = _problem()
    fd = _fd_grad(lambda q: C.loss_and_grad(q, X, T, SMALL)[0], p)
    monkeypatch.setattr(C, "silu_prime", lambda z: np.ones_like(z))
    _, g = C.loss_and_grad(p, X, T, SMALL)
    assert np.linalg.norm(g - fd) > 1e-3 * np.linalg.norm(fd)
    monkeypatch.undo()
    _, g = C.loss_and_grad(p, X, T, SMALL)
    assert np.linalg.norm(0.5 * g - fd) > 1e-3 * np.linalg.norm(fd)


def test_silu_closed_forms():
    z = np.array([-40.0, -1.0, 0.0, 1.0, 40.0])
    s = C.silu(z)
    assert s[2] == 0.0 and abs(s[4] - 40.0) < 1e-12 and abs(s[0]) < 1e-15
    assert np.isclose(s[3], 1.0 / (1.0 + np.exp(-1.0)))
    fd = (C.silu(z + 1e-6) - C.silu(z - 1e-6)) / 2e-6
    assert np.allclose(C.silu_prime(z), fd, atol=1e-8)
    assert C.silu_prime(np.array([0.0]))[0] == 0.5


def test_forward_closed_form():
    """Zero hidden weights: the output is W3 silu(b2) + b3 whatever the input."""
    p = np.zeros(C.param_count())
    (W1, b1), (W2, b2), (W3, b3) = C.unpack(p)
    b1[:] = 0.3
    b2[:] = np.linspace(-1, 1, 64)
    W3[:] = np.arange(5 * 64).reshape(5, 64) / 100.0
    b3[:] = [1, 2, 3, 4, 5]
    X = np.random.default_rng(0).normal(size=(3, 21))
    want = W3 @ C.silu(b2) + b3
    assert np.allclose(C.forward(p, X), want[None, :], rtol=1e-14)


def test_first_adam_step_moves_each_parameter_by_lr():
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    p = np.zeros(4)
    p1, m, v = C.adam_step(p, np.zeros(4), np.zeros(4), g, 1, lr=0.01, eps=0.0)
    assert np.allclose(p1, -0.01 * np.sign(g), rtol=1e-14)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_minimises_a_quadratic():
    target = np.array([1.0, -2.0, 0.5])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 3001):
        p, m, v = C.adam_step(p, m, v, 2 * (p - target), t, lr=0.01)
    assert np.allclose(p, target, atol=1e-3)


def test_bf16_rounding_ties_to_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, -2.5, 3.0e38])
    r = C.bf16(x)
    assert list(r[:4]) == [1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7]
    assert r[4] == -2.5
    assert np.isfinite(r[5]) or r[5] == np.inf


# ---------------------------------------------------------------- features

def _global_coord(m, d):
    c = np.zeros(m.Np)
    c[m.intma.ravel()] = m.xyz[d].ravel()
    return c


def test_features_are_exact_for_polynomials():
    """Assembled gradients of a field of degree <= N per direction are its
    exact derivatives at every node (walls: the polynomial need not be
    periodic)."""
    N = 3
    m = M.build_mesh((2, 3, 2), N, (0.0, 0.0, 0.0), (2.0, 3.0, 1.5), (False, False, False))
    x, y, z = (_global_coord(m, d) for d in range(3))
    q = np.stack([x ** 3 * y, y ** 2 * z ** 3, x * y * z, 1.0 + 0 * x, z ** 2 - x])
    S = 0.1 * x
    X = C.features(m, q, S)
    exact = [
        (3 * x ** 2 * y, x ** 3, 0 * x),
        (0 * x, 2 * y * z ** 3, 3 * y ** 2 * z ** 2),
        (y * z, x * z, x * y),
        (0 * x, 0 * x, 0 * x),
        (-1 + 0 * x, 0 * x, 2 * z),
    ]
    assert np.array_equal(X[:5], q) and np.array_equal(X[20], S)
    for v in range(5):
        for d in range(3):
            got = X[5 + 3 * v + d]
            assert np.allclose(got, exact[v][d], atol=1e-10 * (1 + np.abs(exact[v][d]).max())), (v, d)


# ---------------------------------------------------------------- restriction

@pytest.mark.parametrize("per", [False, True])
def test_restriction_inverts_prolongation(per):
    N = 4
    coarse = (3, N, 0.0, 3000.0, per)
    fine = (6, N, 0.0, 3000.0, per)
    Rfc = C.restriction_1d(fine, coarse)
    Rcf = C.restriction_1d(coarse, fine)
    assert np.allclose(Rfc @ Rcf, np.eye(Rfc.shape[0]), atol=1e-13)
    assert np.allclose(Rfc.sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(C.restriction_1d(coarse, coarse), np.eye(Rfc.shape[0]), atol=1e-13)


def test_restriction_reproduces_polynomials():
    N = 3
    fine_axes = [(4, N, 0.0, 2.0, False), (2, N, -1.0, 1.0, False), (6, N, 0.0, 3.0, False)]
    coarse_axes = [(3, N, 0.0, 2.0, False), (1, N, -1.0, 1.0, False), (2, N, 0.0, 3.0, False)]
    pf = [C.axis_positions(*a) for a in fine_axes]
    pc = [C.axis_positions(*a) for a in coarse_axes]
    Z, Y, X = np.meshgrid(pf[2], pf[1], pf[0], indexing="ij")
    Zc, Yc, Xc = np.meshgrid(pc[2], pc[1], pc[0], indexing="ij")
    f = lambda x, y, z: x ** 3 - 2 * x * y ** 2 * z + z ** 3 * y ** 3 + 0.5
    got = C.restrict(fine_axes, coarse_axes, f(X, Y, Z).reshape(1, -1))[0]
    assert np.allclose(got, f(Xc, Yc, Zc).reshape(-1), atol=1e-11)

