"""Pins of the oracle's extended-precision evaluation (build_mesh with
dtype=np.longdouble; the euler functions then run in np.longdouble).

At the cyclone box's pure-vortex state the rho' and Theta' tendencies are
residuals of horizontal flux derivatives that nearly cancel, and the FP64
oracle's own rounding there reaches ~1e-12 relative L2 at full size (about
2.5e-13 on the 16 x 16 x 16 sample): parity at that state is therefore taken
against the same definitions evaluated in extended precision.  These tests
tie that evaluation to closed forms and to the FP64 oracle where FP64 is
accurate."""

import numpy as np

from inputs import workloads as W
from oracle import euler as E, lgl, mesh as M

from helpers import oracle_of, rel_l2_per_var

LD = np.longdouble
EPS_LD = float(np.finfo(LD).eps)


def _ld_oracle_rhs(wl, q=None):
    m = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"], dtype=LD)
    S = None if wl["S_theta"] is None else wl["S_theta"].astype(LD)
    return E.rhs(m, (wl["q"] if q is None else q).astype(LD), E.Base(wl["rho0"], wl["Theta0"]), S,
                 E.Physics(**wl["phys"]))


def test_extended_is_wider_than_fp64():
    assert EPS_LD < 1e-18


def test_extended_lgl_points_closed_forms():
    x = lgl.lgl_points_extended(4)
    assert x.dtype == LD
    r = np.sqrt(LD(3) / LD(7))
    ref = np.array([-1, -r, 0, r, 1], dtype=LD)
    assert np.max(np.abs(x - ref)) <= 8 * EPS_LD
    x3 = lgl.lgl_points_extended(3)
    r5 = 1 / np.sqrt(LD(5))
    assert np.max(np.abs(x3 - np.array([-1, -r5, r5, 1], dtype=LD))) <= 8 * EPS_LD
    w = lgl.lgl_weights(4, x)
    refw = np.array([LD(1) / 10, LD(49) / 90, LD(32) / 45, LD(49) / 90, LD(1) / 10])
    assert np.max(np.abs(w - refw)) <= 16 * EPS_LD


def test_extended_derivative_exact_for_polynomials():
    for N in (3, 4, 5, 6):
        x = lgl.lgl_points_extended(N)
        D = lgl.derivative_matrix(x)
        assert D.dtype == LD
        for k in range(N + 1):
            exact = k * x ** (k - 1) if k > 0 else np.zeros_like(x)
            assert np.max(np.abs(D @ x ** k - exact)) <= 200 * N * N * EPS_LD, (N, k)


def test_cofactor_inverse_matches_linalg():
    rng = np.random.default_rng(5)
    a = rng.normal(size=(3, 3, 7)) + 3 * np.eye(3)[:, :, None]
    det, inv = M._det_inv3(a)
    jm = np.moveaxis(a, (0, 1), (-2, -1))
    assert np.allclose(det, np.linalg.det(jm), rtol=1e-13, atol=0)
    ref = np.moveaxis(np.linalg.inv(jm), (-2, -1), (0, 1))
    assert np.allclose(inv, ref, rtol=1e-12, atol=1e-14)


def test_extended_mesh_sheared_metrics():
    """The extended mesh of a sheared box has the affine map's metric terms
    and volume, to extended precision."""
    A = np.array([[1.0, 0.2, 0.0], [0.0, 1.0, 0.1], [0.05, 0.0, 1.0]])
    m = M.build_mesh((2, 3, 2), 4, (0, 0, 0), (2.0, 3.0, 2.0), (False, True, False), A=A, dtype=LD)
    assert m.dxi_dx.dtype == LD and m.detJ.dtype == LD
    mass = E.mass(m)
    vol = LD(12) * LD(np.linalg.det(A))
    assert abs(np.sum(mass) - vol) <= 1e-15 * vol
    Ainv = np.linalg.inv(A)
    for j in range(3):
        for i in range(3):
            h = (1.0, 1.0, 1.0)[j]
            assert np.max(np.abs(m.dxi_dx[j, i] - 2.0 / h * Ainv[j, i])) <= 1e-14


def test_extended_rhs_agrees_with_fp64_where_fp64_is_accurate():
    """A seeded smooth random state (no cancellation): the two evaluations of
    the same definitions agree to FP64 rounding."""
    wl = W.tc(nel=(6, 5, 4), state="random")
    m, phys, base = oracle_of(wl)
    ref64 = E.rhs(m, wl["q"], base, wl["S_theta"], phys)
    refx = _ld_oracle_rhs(wl)
    assert refx.dtype == LD
    assert np.all(rel_l2_per_var(ref64, refx.astype(np.float64)) <= 2e-14)


def test_fp64_oracle_rounding_at_the_vortex():
    """At the pure-vortex state the FP64 oracle's rho' and Theta' differ from
    the extended evaluation by far more than at a random state (the residual
    is ~1/100 of the cancelling parts), while the momentum tendencies agree
    to FP64 rounding.  This is why the vortex-state parity tests compare
    against the extended evaluation."""
    wl = W.tc(nel=(16, 16, 16))
    m, phys, base = oracle_of(wl)
    ref64 = E.rhs(m, wl["q"], base, wl["S_theta"], phys)
    refx = _ld_oracle_rhs(wl).astype(np.float64)
    e = rel_l2_per_var(ref64, refx)
    assert np.all(e[[0, 4]] > 5e-14), e
    assert np.all(e[[0, 4]] < 1e-12), e
    assert np.all(e[1:3] < 2e-14), e
