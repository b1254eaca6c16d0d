"""Pins for the oracle's mesh, local-to-global map, metric terms, mass matrix
and DSS (Sec. 2.2, Eqs. 8-12, Alg. 1, Alg. 3)."""

import numpy as np
import pytest

from oracle import euler, mesh as M

SHEAR = np.array([[1.0, 0.3, 0.1], [0.0, 1.0, -0.2], [0.05, 0.0, 1.0]])


def _mesh(nel, N, periodic=(False, False, False), A=None, lo=(0, 0, 0), hi=(1.0, 2.0, 1.5)):
    return M.build_mesh(nel, N, lo, hi, periodic, A)


@pytest.mark.parametrize("periodic", [(False, False, False), (True, True, False), (True, True, True)])
@pytest.mark.parametrize("nel", [(1, 1, 1), (2, 2, 2), (3, 2, 5)])
def test_intma_geometry(nel, periodic):
    """Every local copy of a global node sits at the same physical point
    (modulo the period in periodic directions), and every global node is
    used."""
    N = 3
    m = _mesh(nel, N, periodic)
    L = m.hi - m.lo
    xyz = m.xyz.reshape(3, -1)
    I = m.intma.reshape(-1)
    assert set(np.unique(I)) == set(range(m.Np))
    order = np.argsort(I, kind="stable")
    Is, pts = I[order], xyz[:, order]
    first = np.searchsorted(Is, Is)
    d = pts - pts[:, first]
    for k in range(3):
        if periodic[k]:
            d[k] = d[k] - L[k] * np.round(d[k] / L[k])
    assert np.max(np.abs(d)) < 1e-12


def test_multiplicity_8_elements():
    """On 2x2x2 walled elements: the centre node is shared by 8 elements, the
    centres of the interior faces' edges by 4, interior face nodes by 2,
    nodes interior to an element by 1."""
    N = 4
    m = _mesh((2, 2, 2), N)
    cnt = np.bincount(m.intma.reshape(-1), minlength=m.Np)
    gx, gy, gz = m.gidx
    on = [(g % N == 0) & (g > 0) & (g < 2 * N) for g in (gx, gy, gz)]
    k = on[0].astype(int) + on[1].astype(int) + on[2].astype(int)
    assert np.array_equal(cnt, 2 ** k)
    centre = N + (2 * N + 1) * (N + (2 * N + 1) * N)
    assert cnt[centre] == 8


@pytest.mark.parametrize("A", [None, SHEAR])
@pytest.mark.parametrize("periodic", [(False, False, False), (True, False, True)])
def test_mass_sums_to_volume(A, periodic):
    m = _mesh((3, 2, 2), 4, periodic, A)
    vol = np.prod(m.hi - m.lo) * (1.0 if A is None else np.linalg.det(A))
    assert abs(euler.mass(m).sum() - vol) < 1e-13 * vol


def test_mass_is_tensor_product_of_assembled_weights():
    """On a uniform axis-aligned box M_I = J W_x(gx) W_y(gy) W_z(gz), with W
    the 1-D assembled weight: w_a inside an element, 2 w_0 on a shared face,
    w_0 on a wall."""
    N, nel = 4, (3, 2, 4)
    m = _mesh(nel, N, (False, True, False))
    Mm = euler.mass(m)
    h = (m.hi - m.lo) / np.array(nel)
    J = np.prod(h) / 8.0

    def W(n, periodic):
        out = np.empty(n)
        for g in range(n):
            a = g % N
            if a:
                out[g] = m.w[a]
            elif periodic or 0 < g < n - 1:
                out[g] = 2 * m.w[0]
            else:
                out[g] = m.w[0]
        return out

    Wx, Wy, Wz = W(m.n[0], False), W(m.n[1], True), W(m.n[2], False)
    gx, gy, gz = m.gidx
    assert np.allclose(Mm, J * Wx[gx] * Wy[gy] * Wz[gz], rtol=1e-14, atol=0)


@pytest.mark.parametrize("periodic", [(False, False, False), (True, True, True)])
@pytest.mark.parametrize("nel", [(1, 1, 1), (2, 2, 2)])
def test_dss_brute_force(nel, periodic):
    """Dense Boolean scatter matrix Q (local x global) built from intma:
    M = Q^T (w J) and R = Q^T (w J S) against the oracle's gather."""
    N = 3
    m = _mesh(nel, N, periodic, SHEAR)
    nloc = m.intma.size
    Q = np.zeros((nloc, m.Np))
    Q[np.arange(nloc), m.intma.reshape(-1)] = 1.0
    rng = np.random.default_rng(3)
    S = rng.standard_normal((5,) + m.intma.shape)
    R, Mm = euler.assemble(m, S)
    wJ = (m.w3[None] * m.detJ).reshape(-1)
    assert np.allclose(Mm, Q.T @ wJ, rtol=1e-15, atol=1e-15)
    for v in range(5):
        assert np.allclose(R[v], Q.T @ (wJ * S[v].reshape(-1)), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_divergence_exact_for_polynomials_on_sheared_mesh(N):
    """On an affine (sheared) mesh the assembled divergence of a vector field
    whose components are polynomials of total degree <= N in x is exact at
    every node: each element differentiates it exactly, so the DSS average of
    the element values is the exact value."""
    m = _mesh((2, 3, 2), N, (False, False, False), SHEAR)
    x = np.zeros((3, m.Np))
    for k in range(3):
        x[k][m.intma.reshape(-1)] = m.xyz[k].reshape(-1)
    X, Y, Z = x
    p = N
    F = np.stack([X ** p + 2 * Y * Z ** (p - 1),
                  X ** (p - 1) * Y - Z ** p,
                  3 * Y ** p + X * Z ** (p - 1)])
    div_exact = p * X ** (p - 1) + X ** (p - 1) + (p - 1) * X * Z ** (p - 2) if p >= 2 else None
    div = euler.divergence(m, F)
    scale = np.max(np.abs(div_exact)) + 1.0
    assert np.max(np.abs(div - div_exact)) < 1e-11 * scale


def test_metric_terms_of_affine_map():
    """Metric terms from node coordinates reproduce the analytic Jacobian of
    the affine map: dx/dxi = A diag(h/2), det J = det(A) prod(h)/8."""
    nel, N = (2, 3, 4), 4
    m = _mesh(nel, N, (False, False, False), SHEAR)
    h = (m.hi - m.lo) / np.array(nel)
    Jm = SHEAR @ np.diag(h / 2)
    assert np.allclose(m.detJ, np.linalg.det(Jm), rtol=1e-13, atol=0)
    inv = np.linalg.inv(Jm)
    for j in range(3):
        for i in range(3):
            assert np.allclose(m.dxi_dx[j, i], inv[j, i], rtol=0, atol=1e-12 * np.abs(inv).max())
