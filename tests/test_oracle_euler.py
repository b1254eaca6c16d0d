"""Pins for the oracle's right-hand side (Eq. 1 restated, Eq. 3, Eqs. 8-12)
and its SSP-RK3 update: a manufactured solution whose exact tendency is
derived symbolically from Eq. 1 in the paper's own (rho', u, theta') form,
rest and free-stream states, mass conservation, Coriolis rotation, mirror
symmetry, the equation of state and the wall condition."""

import math

import numpy as np
import pytest

from inputs import workloads as W
from oracle import euler as E, mesh as M, ssprk3

PHYS0 = dict(g=9.81, R=287.0, cp=1004.5, cv=717.5, p_a=1.0e5)


def _setup(wl):
    m = M.build_mesh(wl["nel"], wl["N"], wl["lo"], wl["hi"], wl["periodic"])
    return m, E.Physics(**wl["phys"]), E.Base(wl["rho0"], wl["Theta0"])


# ---------------------------------------------------------------- manufactured solution

def _mms_problem():
    """Exact conservative tendencies of a smooth periodic state, derived with
    sympy from Eq. 1 as printed: d rho'/dt = -div(rho u);
    du/dt = -u.grad u - grad p'/rho - (rho'/rho) g k - f k x u;
    d theta'/dt = -u.grad(theta_0 + theta') + S_theta; with
    p' = p_a (R rho theta/p_a)^gamma - p_a (R rho_0 theta_0/p_a)^gamma.
    Conservative tendencies follow by the product rule:
    d(rho u)/dt = rho du/dt + u d rho'/dt, d Theta'/dt = rho dtheta'/dt +
    theta d rho'/dt."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    Lx, Ly, Lz = 3000.0, 2000.0, 2500.0
    kx, ky, kz = 2 * sp.pi / Lx, 2 * sp.pi / Ly, 2 * sp.pi / Lz
    g, R, cp, cv, pa, f = (PHYS0["g"], PHYS0["R"], PHYS0["cp"], PHYS0["cv"], PHYS0["p_a"], 1.0e-3)
    gam = sp.Rational(int(cp * 10), int(cv * 10))
    rho0 = 1.1 + 0.05 * sp.cos(kz * z)
    th0 = 300.0 + 4.0 * sp.sin(kz * z)
    rp = 0.01 * sp.sin(kx * x + 0.3) * sp.cos(ky * y) * sp.cos(kz * z + 0.2)
    u = 6.0 * sp.cos(kx * x) * sp.sin(ky * y + 0.5) + 2.0
    v = -4.0 * sp.sin(kx * x + 0.1) * sp.cos(kz * z) + 1.0
    w = 2.0 * sp.sin(ky * y) * sp.sin(kz * z + 0.7)
    thp = 1.5 * sp.cos(kx * x - 0.4) * sp.sin(ky * y) * sp.sin(kz * z) + 0.3
    sth = 5.0 * sp.cos(kx * x) * sp.cos(ky * y + 1.0) * sp.sin(kz * z)
    rho = rho0 + rp
    th = th0 + thp
    p = pa * (R * rho * th / pa) ** gam
    p0 = pa * (R * rho0 * th0 / pa) ** gam
    pp = p - p0
    U = [u, v, w]
    X = [x, y, z]

    def adv(s):
        return sum(U[i] * sp.diff(s, X[i]) for i in range(3))

    drho = -sum(sp.diff(rho * U[i], X[i]) for i in range(3))
    du = [-adv(U[i]) - sp.diff(pp, X[i]) / rho for i in range(3)]
    du[2] += -(rp / rho) * g
    du[0] += f * v     # -f k x u = (f v, -f u, 0)
    du[1] += -f * u
    dth = -adv(th) + sth
    T = [drho] + [rho * du[i] + U[i] * drho for i in range(3)] + [rho * dth + th * drho]
    state = [rp, rho * u, rho * v, rho * w, rho * th - rho0 * th0]
    lam = lambda e: sp.lambdify((x, y, z), e, "numpy")
    return dict(state=[lam(s) for s in state], T=[lam(t) for t in T], sth=lam(sth),
                rho0=lam(rho0), th0=lam(th0), L=(Lx, Ly, Lz), f=f)


@pytest.fixture(scope="module")
def mms():
    return _mms_problem()


def _mms_error(mms, nel, N):
    L = mms["L"]
    m = M.build_mesh((nel, nel, nel), N, (0, 0, 0), L, (True, True, True))
    X = np.zeros((3, m.Np))
    for k in range(3):
        X[k][m.intma.reshape(-1)] = m.xyz[k].reshape(-1)
    ev = lambda fn: np.broadcast_to(fn(X[0], X[1], X[2]), (m.Np,)).astype(np.float64)
    q = np.stack([ev(fn) for fn in mms["state"]])
    zl = np.zeros(m.n[2])
    zl[m.gidx[2]] = X[2]
    rho0 = np.broadcast_to(mms["rho0"](0, 0, zl), zl.shape).astype(np.float64)
    th0 = np.broadcast_to(mms["th0"](0, 0, zl), zl.shape).astype(np.float64)
    base = E.Base(rho0, rho0 * th0)
    phys = E.Physics(**PHYS0, f=mms["f"])
    r = E.rhs(m, q, base, ev(mms["sth"]), phys)
    T = np.stack([ev(fn) for fn in mms["T"]])
    return np.array([np.max(np.abs(r[v] - T[v])) / np.max(np.abs(T[v])) for v in range(5)])


@pytest.mark.parametrize("N", [3, 4])
def test_mms_design_order(mms, N):
    """The CG right-hand side converges to the exact Eq. 1 tendency at every
    node, for every variable, at (close to) the design order N."""
    e1 = _mms_error(mms, 8, N)
    e2 = _mms_error(mms, 12, N)
    rate = np.log(e1 / e2) / np.log(12 / 8)
    assert np.all(rate > N - 0.5), (e1, e2, rate)
    assert np.all(e2 < (1e-3 if N == 3 else 1e-4)), e2


# ---------------------------------------------------------------- invariants

def test_hydrostatic_rest_gives_zero_tendency():
    """Resting perturbation-free atmosphere: every tendency vanishes."""
    wl = W.tc(nel=(4, 4, 4))
    m, phys, base = _setup(wl)
    q = np.zeros_like(wl["q"])
    r = E.rhs(m, q, base, None, phys)
    scale = np.max(base.rho0) * phys.g
    assert np.max(np.abs(r)) <= 1e-12 * scale


@pytest.mark.parametrize("N", [3, 4])
def test_free_stream_on_sheared_mesh(N):
    """Constant density, velocity and Theta on a sheared periodic affine mesh
    with g = f = 0 and no heating: the tendency vanishes."""
    A = np.array([[1.0, 0.4, 0.0], [0.0, 1.0, 0.25], [0.1, 0.0, 1.0]])
    m = M.build_mesh((3, 2, 2), N, (0, 0, 0), (3000.0, 2000.0, 1000.0), (True, True, True), A)
    phys = E.Physics(**dict(PHYS0, g=0.0), f=0.0)
    rho0 = np.full(m.n[2], 1.15)
    base = E.Base(rho0, rho0 * 305.0)
    u = np.array([12.0, -7.0, 3.0])
    q = np.zeros((5, m.Np))
    q[0] = 0.02
    q[1:4] = (1.17 * u)[:, None]
    q[4] = 0.8
    r = E.rhs(m, q, base, None, phys)
    scale = 1.17 * 12.0 ** 2 / 1000.0
    assert np.max(np.abs(r)) <= 1e-12 * scale


def test_mass_conserved_under_walls():
    """Bubble in a closed box: sum_I M_I rho'_I is unchanged to 1e-13 of the
    total mass after 20 SSP-RK3 steps (Eq. 1a in conservation form, exact
    LGL integration of the divergence, zero normal flux at walls)."""
    wl = W.bubble()
    m, phys, base = _setup(wl)
    Mm = E.mass(m)
    L = lambda q: E.rhs(m, q, base, None, phys)
    q0 = wl["q"]
    q = ssprk3.run(L, q0, wl["dt"], 20)
    rho_total = np.dot(Mm, base.rho0[m.gidx[2]] + q0[0])
    assert abs(np.dot(Mm, q[0] - q0[0])) <= 1e-13 * rho_total
    assert np.max(np.abs(q[3])) > 0  # it did move


def test_mass_conserved_random_state_walls():
    wl = W.box((3, 2, 3), 4, (0, 0, 0), (3000.0, 2000.0, 3000.0), (False, True, False), seed=11)
    m, phys, base = _setup(wl)
    Mm = E.mass(m)
    L = lambda q: E.rhs(m, q, base, wl["S_theta"], phys)
    q0 = wl["q"]
    q = ssprk3.run(L, q0, 0.02, 5)
    rho_total = np.dot(Mm, base.rho0[m.gidx[2]] + q0[0])
    assert abs(np.dot(Mm, q[0] - q0[0])) <= 1e-13 * rho_total


def test_inertial_rotation_sign_and_rate():
    """Uniform horizontal momentum in a periodic box with g = 0 turns at the
    inertial frequency: (rho u, rho v) = U (cos ft, -sin ft) for f > 0."""
    f = 0.05
    m = M.build_mesh((2, 2, 2), 3, (0, 0, 0), (1000.0, 1000.0, 1000.0), (True, True, True))
    phys = E.Physics(**dict(PHYS0, g=0.0), f=f)
    rho0 = np.full(m.n[2], 1.0)
    base = E.Base(rho0, rho0 * 300.0)
    q = np.zeros((5, m.Np))
    q[1] = 10.0
    dt, n = 0.05, 200   # acoustic Courant number ~0.25; f dt = 2.5e-3
    q = ssprk3.run(lambda s: E.rhs(m, s, base, None, phys), q, dt, n)
    t = dt * n
    # c = rho u + i rho v obeys dc/dt = -i f c; SSP-RK3 multiplies c by
    # R(z) = 1 + z + z^2/2 + z^3/6, z = -i f dt, per step
    z = -1j * f * dt
    cn = 10.0 * (1 + z + z * z / 2 + z ** 3 / 6) ** n
    assert np.allclose(q[1], cn.real, rtol=0, atol=1e-11)
    assert np.allclose(q[2], cn.imag, rtol=0, atol=1e-11)
    assert np.allclose(q[1], 10.0 * math.cos(f * t), rtol=0, atol=1e-8)
    assert np.allclose(q[2], -10.0 * math.sin(f * t), rtol=0, atol=1e-8)
    assert np.max(np.abs(q[[0, 3, 4]])) < 1e-12


def test_bubble_mirror_symmetry():
    """The centred bubble in the walled cube stays mirror-symmetric in x and
    y and symmetric under the x <-> y swap."""
    wl = W.bubble(nel=(4, 4, 4))
    m, phys, base = _setup(wl)
    q = ssprk3.run(lambda s: E.rhs(m, s, base, None, phys), wl["q"], wl["dt"], 5)
    nx, ny, nz = m.n
    g = q.reshape(5, nz, ny, nx)
    sx = [1, -1, 1, 1, 1]
    sy = [1, 1, -1, 1, 1]
    scale = np.max(np.abs(g), axis=(1, 2, 3)) + 1e-300
    for v in range(5):
        assert np.max(np.abs(g[v] - sx[v] * g[v][:, :, ::-1])) <= 1e-12 * scale[v]
        assert np.max(np.abs(g[v] - sy[v] * g[v][:, ::-1, :])) <= 1e-12 * scale[v]
    swap = [0, 2, 1, 3, 4]
    for v in range(5):
        assert np.max(np.abs(g[v] - np.swapaxes(g[swap[v]], 1, 2))) <= 1e-12 * scale[v]


def test_wall_normal_momentum_tendency_zero():
    wl = W.box((2, 2, 2), 4, (0, 0, 0), (2000.0, 2000.0, 2000.0), (False, False, False), seed=5)
    m, phys, base = _setup(wl)
    r = E.rhs(m, wl["q"], base, wl["S_theta"], phys)
    for d in range(3):
        mask = m.wall_nodes(d)
        assert mask.any()
        assert np.all(r[1 + d][mask] == 0.0)
        assert np.any(r[1 + d][~mask] != 0.0)


def test_rhs_at_nodes_matches_full():
    wl = W.tc(nel=(4, 4, 3), state="random")
    m, phys, base = _setup(wl)
    r = E.rhs(m, wl["q"], base, wl["S_theta"], phys)
    nodes = np.array([0, 1, 4, 17, m.Np // 2, m.Np - 1, m.n[0] * m.n[1] * 4 + 3])
    rs = E.rhs_at_nodes(m, wl["q"], base, wl["S_theta"], phys, nodes)
    assert np.allclose(rs, r[:, nodes], rtol=1e-14, atol=0)


# ---------------------------------------------------------------- equation of state

def test_pressure_perturbation_against_extended_precision():
    """p' = p(Theta_0 + Theta') - p(Theta_0) (Eq. 3) against 50-digit
    arithmetic, across |Theta'/Theta_0| from 1e-9 to 0.3."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    phys = E.Physics(**PHYS0)
    gam = mp.mpf(phys.cp) / mp.mpf(phys.cv)
    Th0 = 350.0
    for rel in (1e-9, -3e-7, 1e-4, -2e-3, 0.05, -0.3):
        Tp = rel * Th0
        exact = (mp.mpf(phys.p_a) * (mp.mpf(phys.R) * (mp.mpf(Th0) + mp.mpf(Tp)) / mp.mpf(phys.p_a)) ** gam
                 - mp.mpf(phys.p_a) * (mp.mpf(phys.R) * mp.mpf(Th0) / mp.mpf(phys.p_a)) ** gam)
        got = E.pressure_perturbation(np.array(Th0), np.array(Tp), phys)
        assert abs(float((mp.mpf(float(got)) - exact) / exact)) < 5e-15


def test_pressure_special_value():
    """Eq. 3 at rho R theta = p_a gives p = p_a for any gamma."""
    phys = E.Physics(**PHYS0)
    assert abs(E.pressure(phys.p_a / phys.R, phys) - phys.p_a) < 1e-10


# ---------------------------------------------------------------- SSP-RK3

def test_ssprk3_amplification_polynomial():
    """On y' = lambda y one SSP-RK3 step multiplies by 1 + z + z^2/2 + z^3/6."""
    for z in (0.3, -1.2, 0.5j, -0.4 + 1.1j):
        got = ssprk3.ssprk3_step(lambda y: z * y, np.array(1.0 + 0j), 1.0)
        assert abs(got - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-15


def test_ssprk3_third_order():
    """Global error on y' = -y at t = 1 falls like dt^3."""
    errs = []
    for n in (10, 20, 40):
        y = ssprk3.run(lambda s: -s, np.array(1.0), 1.0 / n, n)
        errs.append(abs(float(y) - math.exp(-1.0)))
    assert 2.8 < math.log2(errs[0] / errs[1]) < 3.2
    assert 2.8 < math.log2(errs[1] / errs[2]) < 3.2


def test_dof_convention_matches_paper():
    """The paper's DOF counts for its grids (tests/golden/paper_dof_counts.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_dof_counts.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for nx, ny, nz, N, dof in rows:
        _, local = W.dof_counts((int(nx), int(ny), int(nz)), int(N), (True, True, False))
        assert local == int(dof)


# ---------------------------------------------------------------- planted mistakes
# Each plausible mistake, planted in the oracle on the CPU, must be caught by
# the manufactured-solution pin (error no longer near discretisation level).

def _mms_error_with(mms, monkeypatch, patch):
    with monkeypatch.context() as mp:
        patch(mp)
        return _mms_error(mms, 8, 4)


@pytest.mark.parametrize("mistake", ["transposed_D", "wrong_gamma", "coriolis_sign",
                                     "no_gravity", "heating_rho0"])
def test_planted_mistakes_are_caught(mms, monkeypatch, mistake):
    good = _mms_error(mms, 8, 4)
    if mistake == "transposed_D":
        orig = E.apply_D
        patch = lambda mp: mp.setattr(E, "apply_D", lambda D, f, ax: orig(D.T, f, ax))
    elif mistake == "wrong_gamma":
        patch = lambda mp: mp.setattr(E.Physics, "gamma", property(lambda s: s.cp / s.R))
    elif mistake == "coriolis_sign":
        orig_f = mms["f"]
        patch = lambda mp: mp.setitem(mms, "f", -orig_f)
    elif mistake == "no_gravity":
        patch = lambda mp: mp.setitem(PHYS0, "g", 0.0)
    else:  # heating multiplied by rho_0 instead of rho = rho_0 + rho'
        orig_lt = E.local_tendency

        def lt(mesh, q, base, S_theta, phys, elements=None):
            S = orig_lt(mesh, q, base, S_theta, phys, elements)
            intma = mesh.intma if elements is None else mesh.intma[elements]
            S[4] -= q[0][intma] * S_theta[intma]
            return S
        patch = lambda mp: mp.setattr(E, "local_tendency", lt)
    bad = _mms_error_with(mms, monkeypatch, patch)
    assert np.max(bad / good) > 3.0, (mistake, good, bad)


# ---------------------------------------------------------------- linear acoustics

def _acoustic_error(nel, N, eps=1e-5):
    """A right-going sound wave in a uniform resting atmosphere without
    gravity: rho' = e rho0 s, rho u = e rho0 c s, Theta' = e Theta0 s with
    s = sin(k x) and c^2 = gamma p0 / rho0 obeys dq/dt = -c dq/dx to first
    order in e.  The oracle's tendency (its odd part in e, by a central
    difference, so the O(e^2) terms cancel) against -c dq/dx, max relative
    error over the three wave variables."""
    L = 4000.0
    m = M.build_mesh((nel, 1, 1), N, (0.0, 0.0, 0.0), (L, 500.0, 500.0), (True, True, True))
    X = np.zeros(m.Np)
    X[m.intma.reshape(-1)] = m.xyz[0].reshape(-1)
    phys = E.Physics(**dict(PHYS0, g=0.0), f=0.0)
    rho0, Th0 = 1.2, 1.2 * 300.0
    # the sound speed from the constants, not from the oracle's own gamma or pressure
    gam = PHYS0["cp"] / PHYS0["cv"]
    p0 = PHYS0["p_a"] * (PHYS0["R"] * Th0 / PHYS0["p_a"]) ** gam
    c = math.sqrt(gam * p0 / rho0)
    base = E.Base(np.full(m.n[2], rho0), np.full(m.n[2], Th0))
    k = 2 * math.pi / L
    s, ds = np.sin(k * X), k * np.cos(k * X)
    amp = np.array([rho0, rho0 * c, 0.0, 0.0, Th0])
    q = amp[:, None] * s[None, :]
    r = (E.rhs(m, eps * q, base, None, phys) - E.rhs(m, -eps * q, base, None, phys)) / (2 * eps)
    exact = -c * amp[:, None] * ds[None, :]
    return max(np.max(np.abs(r[v] - exact[v])) / np.max(np.abs(exact[v])) for v in (0, 1, 4))


def test_linear_acoustics_speed_and_order():
    """The sound speed c = sqrt(gamma p0 / rho0) and the sign of propagation
    (a wrong gamma, a missing pressure term or a flipped flux fails the
    coarse check), and design-order convergence of the dispersion error."""
    e8, e16 = _acoustic_error(8, 4), _acoustic_error(16, 4)
    assert e8 < 4e-4, e8            # a 1 % error in c alone would give 1e-2
    assert math.log2(e8 / e16) > 3.5, (e8, e16)


@pytest.mark.parametrize("mistake", ["gamma", "pressure"])
def test_acoustics_catches_planted_mistakes(monkeypatch, mistake):
    """A 1 % error in the oracle's gamma, or 2 % in its equation of state,
    moves the sound speed and fails the acoustic pin."""
    if mistake == "gamma":
        monkeypatch.setattr(E.Physics, "gamma", property(lambda self: 1.01 * self.cp / self.cv))
    else:
        orig = E.pressure
        monkeypatch.setattr(E, "pressure", lambda Th, phys: 1.02 * orig(Th, phys))
    assert _acoustic_error(8, 4) > 4e-3
