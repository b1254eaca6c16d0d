"""Pins for oracle/dynamics.py: the weak Laplacian (conservation, symmetry,
negative semi-definiteness, exact interior second derivatives of quadratics,
spectral convergence on a Fourier mode), the viscosity tensor's closed form
on an axis-aligned box, hyper-diffusion of a Fourier mode, the sponge profile
and the RI-velocity diagnostic on solid-body rotation and radial flow."""

import numpy as np
import pytest

from inputs import rng
from oracle import dynamics as Y, euler as E, mesh as M


def _coords(m):
    return [Y._global(m, m.xyz[d]) for d in range(3)]


def _tau_diag(m, nu):
    t = np.zeros((3, 3) + m.detJ.shape)
    for d in range(3):
        t[d, d] = nu[d]
    return t


@pytest.mark.parametrize("per", [(False, False, False), (True, True, False), (True, True, True)])
def test_laplacian_conserves_is_symmetric_and_dissipative(per):
    A = np.array([[1.0, 0.2, 0.0], [0.0, 1.0, 0.1], [0.0, 0.0, 1.0]])
    m = M.build_mesh((2, 3, 2), 3, (0, 0, 0), (2.0, 3.0, 1.5), per, A=A)
    tau = Y.viscosity_tensor(m, (1.0, 2.0, 3.0), 0.5)
    u = rng.uniform(3, 2 * m.Np, -1.0, 1.0).reshape(2, m.Np)
    Lu = Y.laplacian(m, u, tau)
    W = E.mass(m)
    for v in range(2):
        assert abs(np.dot(W, Lu[v])) <= 1e-12 * np.dot(W, np.abs(Lu[v]))
    a = np.dot(W * u[0], Lu[1])
    b = np.dot(W * Lu[0], u[1])
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))
    assert np.dot(W * u[0], Lu[0]) < 0.0


def test_laplacian_of_quadratics_is_exact_inside():
    N = 4
    m = M.build_mesh((3, 2, 2), N, (0, 0, 0), (3.0, 2.0, 2.0), (False, False, False))
    x, y, z = _coords(m)
    nu = (0.5, 2.0, 3.0)
    tau = _tau_diag(m, nu)
    inside = np.ones(m.Np, dtype=bool)
    for d in range(3):
        inside &= ~m.wall_nodes(d)
    L = Y.laplacian(m, np.stack([x * x, y * y, z * z, x * y, np.ones(m.Np)]), tau)
    assert np.allclose(L[0][inside], 2 * nu[0], atol=1e-11)
    assert np.allclose(L[1][inside], 2 * nu[1], atol=1e-11)
    assert np.allclose(L[2][inside], 2 * nu[2], atol=1e-11)
    assert np.allclose(L[3][inside], 0.0, atol=1e-11)
    assert np.allclose(L[4], 0.0, atol=1e-12)


def test_laplacian_converges_spectrally_on_a_fourier_mode():
    k = 2 * np.pi / 2.0
    errs = []
    for N in (3, 5, 7):
        m = M.build_mesh((4, 1, 1), N, (0, 0, 0), (2.0, 1.0, 1.0), (True, True, True))
        x, _, _ = _coords(m)
        L = Y.laplacian(m, np.sin(k * x), _tau_diag(m, (1.0, 1.0, 1.0)))[0]
        errs.append(np.abs(L + k * k * np.sin(k * x)).max() / (k * k))
    assert errs[0] > 10 * errs[1] > 100 * errs[2]
    assert errs[2] < 1e-5


def test_viscosity_tensor_closed_form_on_a_box():
    """Axis-aligned box: tau = diag(nu) with nu = c^(1/2) (h/N)^2 / dt^(1/2),
    c_1 on the largest element size (smallest eigenvalue of G)."""
    N = 4
    m = M.build_mesh((2, 2, 4), N, (0, 0, 0), (8.0, 8.0, 2.0), (True, True, False))
    c = (4.0, 4.0, 9.0)
    dt = 0.25
    tau = Y.viscosity_tensor(m, c, dt)
    hs = (4.0, 4.0, 0.5)                     # element sizes: x and y are the largest
    want = [np.sqrt(c[0]) * (hs[0] / N) ** 2 / np.sqrt(dt), np.sqrt(c[1]) * (hs[1] / N) ** 2 / np.sqrt(dt),
            np.sqrt(c[2]) * (hs[2] / N) ** 2 / np.sqrt(dt)]
    for d in range(3):
        for e in range(3):
            assert np.allclose(tau[d, e], want[d] if d == e else 0.0, atol=1e-12 * max(want))


def test_hyperdiffusion_damps_a_fourier_mode_at_nu_squared_k4():
    k = 2 * np.pi / 2.0
    m = M.build_mesh((4, 1, 1), 7, (0, 0, 0), (2.0, 1.0, 1.0), (True, True, True))
    x, _, _ = _coords(m)
    nu = 0.3
    q = np.stack([np.sin(k * x)] * 5)
    H = Y.hyperdiffusion(m, q, _tau_diag(m, (nu, nu, nu)))
    assert np.abs(H + (nu * k * k) ** 2 * q).max() <= 2e-3 * (nu * k * k) ** 2
    assert abs(np.dot(E.mass(m), H[0])) < 1e-10


def test_sponge_profile_and_variable():
    m = M.build_mesh((1, 1, 8), 4, (0, 0, 0), (1.0, 1.0, 8.0), (True, True, False))
    z = Y._global(m, m.xyz[2])
    g = Y.sponge_rate(z, 8.0, 4.0, 0.2)
    assert np.all(g[z <= 4.0] == 0.0)
    assert np.isclose(Y.sponge_rate(np.array([8.0]), 8.0, 4.0, 0.2)[0], 0.2)
    assert np.isclose(Y.sponge_rate(np.array([6.0]), 8.0, 4.0, 0.2)[0], 0.1)
    q = np.ones((5, m.Np))
    s = Y.sponge(m, q, 4.0, 0.2)
    assert np.all(s[[0, 1, 2, 4]] == 0.0) and np.allclose(s[3], -g)


def test_ri_velocity_of_solid_body_rotation():
    """u = Omega k x (x - c) about the box centre: the centroid is the centre,
    the tangential speed is Omega r, a strip averages it over its radii."""
    m = M.build_mesh((8, 8, 2), 4, (-4.0, -4.0, 0.0), (4.0, 4.0, 2.0), (False, False, False))
    x, y, _ = _coords(m)
    rho0 = np.full(m.n[2], 1.2)
    Om = 0.5
    q = np.zeros((5, m.Np))
    q[1], q[2] = -Om * y * 1.2, Om * x * 1.2
    q[3] = 0.7 * 1.2                      # vertical motion does not count
    uri, cent, means = Y.ri_velocity(m, q, rho0, nstrips=8)
    assert np.allclose(cent, 0.0, atol=1e-12)
    r = np.sqrt(x * x + y * y)
    ok = 0
    for j in range(8):
        sel = (np.floor(r / 0.5) == j) & (m.gidx[2] == 0)
        if sel.any():
            assert np.isclose(means[0, j], Om * r[sel].mean(), rtol=1e-12)
            ok += 1
    assert ok >= 7 and np.isclose(uri, means.max())
    # purely radial flow has no tangential speed
    q2 = np.zeros((5, m.Np))
    q2[1], q2[2] = x * 1.2, y * 1.2
    assert Y.ri_velocity(m, q2, rho0, nstrips=8)[0] < 1e-12
