"""Named synthetic workloads.

``bubble``  -- dry rising thermal: 10 x 10 x 10 km box, 8^3 elements, N = 4
               (33^3 nodes), isentropic theta_0 = 300 K, +2 K cosine bubble of
               radius 2 km centred at (5, 5, 2) km, no-flux walls on all six
               faces, no Coriolis, no heating, dt = 0.02 s.
``batch``   -- the batched form: ``count`` independent limited-area boxes of
               512 x 512 x 20 km (doubly periodic laterally, no-flux bottom
               and top, stable sounding, f = 5e-5 1/s), each with seeded
               element counts (uniform in 4..24 horizontally, 4..12
               vertically), order N uniform in {3, 4, 5, 6}, its own
               modified-Rankine vortex (Vmax U(10, 30) m/s at radius
               U(30, 80) km) and heating ring, and a step dt at the acoustic
               Courant number of ``tc`` (0.1 s for 216 m vertical spacing).
``closure_case`` -- a run of the learned-closure form: config 1's 10 km cube
               (no-flux walls, isentropic theta_0 = 300 K), a seeded warm
               bubble (+1..3 K, radius 1.5..2.5 km) and a seeded vortex scaled
               to the box (Vmax 5..15 m/s at 1..2 km, cut off beyond 3.5 km
               so the wall-normal momentum vanishes), and a heating ring
               scaled down from ``tc``'s (peak 5..15 K/h at 2 km, width
               0.5 km, below 8 km); dt at the acoustic Courant number of
               ``tc``.
``tc``      -- tropical-cyclone-shaped box: 1024 x 1024 x 20 km, 128 x 128 x 16
               elements, N = 4, doubly periodic laterally with no-flux bottom
               and top (512 x 512 x 65 nodes), stable sounding N_BV = 0.01 1/s,
               f = 5e-5 1/s, modified-Rankine vortex (15 m/s at 50 km) and the
               ring-plus-32-cells heating (seed 2504), dt = 0.1 s.
               ``scale`` shrinks the element counts (and the box with them, so
               the spacing stays that of the full case).

Each workload is a dict: mesh parameters (nel, N, lo, hi, periodic),
physics (g, R, cp, cv, p_a, f), dt, the state q [5, Np] (rho', rho u, rho v,
rho w, Theta'), the reference state on node levels (rho0 [n_z],
Theta0 [n_z]) and the heating S_theta [Np] in K/s (or None).
"""

import numpy as np

from . import atmosphere as atm
from . import grid
from . import rng

PHYS = dict(g=9.81, R=287.0, cp=1004.5, cv=717.5, p_a=1.0e5)


def _levels(ax_z):
    return np.asarray(ax_z)


def bubble(nel=(8, 8, 8), N=4, state="initial", seed=1):
    lo, hi = (0.0, 0.0, 0.0), (10.0e3, 10.0e3, 10.0e3)
    periodic = (False, False, False)
    X, Y, Z, ax = grid.node_coords(nel, N, lo, hi, periodic)
    rho0, Th0 = atm.isentropic_sounding(ax[2])
    n_xy = ax[0].size * ax[1].size
    if state == "initial":
        q = atm.bubble_state(X, Y, Z, ax[2], rho0, Th0, n_xy)
    elif state == "random":
        q = atm.smooth_random_state(X, Y, Z, lo, hi, periodic, seed)
    else:
        raise ValueError(state)
    return dict(name="bubble", nel=tuple(nel), N=N, lo=lo, hi=hi, periodic=periodic,
                phys=dict(PHYS, f=0.0), dt=0.02, q=q, rho0=rho0, Theta0=Th0, S_theta=None)


def tc(nel=(128, 128, 16), N=4, state="initial", seed=1, heating_seed=2504):
    hx = 1024.0e3 / 128 * nel[0]
    hy = 1024.0e3 / 128 * nel[1]
    hz = 20.0e3 / 16 * nel[2]
    lo, hi = (-hx / 2, -hy / 2, 0.0), (hx / 2, hy / 2, hz)
    periodic = (True, True, False)
    X, Y, Z, ax = grid.node_coords(nel, N, lo, hi, periodic)
    rho0, Th0 = atm.stable_sounding(ax[2], nbv=0.01)
    n_xy = ax[0].size * ax[1].size
    centre = (0.0, 0.0)
    if state == "initial":
        q = atm.vortex_state(X, Y, Z, rho0, n_xy, centre)
    elif state == "random":
        q = atm.smooth_random_state(X, Y, Z, lo, hi, periodic, seed)
        q += atm.vortex_state(X, Y, Z, rho0, n_xy, centre)
    else:
        raise ValueError(state)
    S = atm.heating(X, Y, Z, centre, seed=heating_seed)
    return dict(name="tc", nel=tuple(nel), N=N, lo=lo, hi=hi, periodic=periodic,
                phys=dict(PHYS, f=5.0e-5), dt=0.1, q=q, rho0=rho0, Theta0=Th0, S_theta=S)


def tc_paper(nel=(80, 80, 24), N=5, heating_seed=2504):
    """The cyclone box on the grid of the paper's timing runs (Sec. 4.1 and
    Table 1): 800 x 800 x 20 km, doubly periodic, 80 x 80 x 24 elements of
    order 5 (2 km horizontal and 167 m vertical node spacing); the same
    stable sounding, vortex and heating recipe as ``tc``."""
    lo, hi = (-400.0e3, -400.0e3, 0.0), (400.0e3, 400.0e3, 20.0e3)
    periodic = (True, True, False)
    X, Y, Z, ax = grid.node_coords(nel, N, lo, hi, periodic)
    rho0, Th0 = atm.stable_sounding(ax[2], nbv=0.01)
    n_xy = ax[0].size * ax[1].size
    q = atm.vortex_state(X, Y, Z, rho0, n_xy, (0.0, 0.0))
    S = atm.heating(X, Y, Z, (0.0, 0.0), seed=heating_seed)
    return dict(name="tc_paper", nel=tuple(nel), N=N, lo=lo, hi=hi, periodic=periodic,
                phys=dict(PHYS, f=5.0e-5), dt=0.5, q=q, rho0=rho0, Theta0=Th0, S_theta=S)


def box(nel, N, lo, hi, periodic, f=1.0e-4, seed=7, heating_amp=1.0e-3, sounding="stable"):
    """Generic box with a seeded smooth random state (for parity sweeps over
    orders, sizes and boundary types)."""
    X, Y, Z, ax = grid.node_coords(nel, N, lo, hi, periodic)
    if sounding == "stable":
        rho0, Th0 = atm.stable_sounding(ax[2] - lo[2], nbv=0.01)
    else:
        rho0, Th0 = atm.isentropic_sounding(ax[2] - lo[2])
    q = atm.smooth_random_state(X, Y, Z, lo, hi, periodic, seed)
    S = heating_amp * atm.smooth_random_state(X, Y, Z, lo, hi, (True, True, True), seed + 1000,
                                              amps=(1.0, 0, 0, 0, 0))[0]
    return dict(name="box", nel=tuple(nel), N=N, lo=tuple(lo), hi=tuple(hi),
                periodic=tuple(periodic), phys=dict(PHYS, f=f), dt=0.02, q=q, rho0=rho0,
                Theta0=Th0, S_theta=S)


def eos_span(nel=(4, 3, 8), N=4, seed=11, lo_ratio=1.0e-4, hi_ratio=0.3):
    """A box whose Theta' reaches |Theta'/Theta_0| = ``lo_ratio`` at the
    bottom level and ``hi_ratio`` at the top (an amplitude geometric in
    height, times a seeded smooth pattern in [-1, 1] kept at least 1e-3 in
    magnitude), so that the equation of state is evaluated on both sides of
    any switch point in between; the other variables are a seeded smooth
    random state.  Walls on all sides, stable sounding."""
    lo, hi = (0.0, 0.0, 0.0), (4000.0, 3000.0, 8000.0)
    periodic = (False, False, False)
    X, Y, Z, ax = grid.node_coords(nel, N, lo, hi, periodic)
    rho0, Th0 = atm.stable_sounding(ax[2], nbv=0.01)
    q = atm.smooth_random_state(X, Y, Z, lo, hi, periodic, seed)
    s = atm.smooth_random_state(X, Y, Z, lo, hi, (True, True, True), seed + 1,
                                amps=(1.0, 0, 0, 0, 0))[0]
    s = s / np.max(np.abs(s))
    s = np.sign(s) * np.maximum(np.abs(s), 1.0e-3)
    nxy = ax[0].size * ax[1].size
    gz = np.arange(X.size) // nxy
    t = Z / hi[2]
    ratio = lo_ratio * (hi_ratio / lo_ratio) ** t
    q[4] = Th0[gz] * ratio * s
    return dict(name="eos_span", nel=tuple(nel), N=N, lo=lo, hi=hi, periodic=periodic,
                phys=dict(PHYS, f=1.0e-4), dt=0.02, q=q, rho0=rho0, Theta0=Th0, S_theta=None)


def dof_counts(nel, N, periodic):
    """(unique-node DOF, element-local DOF): 5 variables times the unique
    global nodes, and the paper's convention N_e (N+1)^3 x 5 (Sec. 5.2)."""
    n = [N * nel[d] + (0 if periodic[d] else 1) for d in range(3)]
    return 5 * n[0] * n[1] * n[2], 5 * nel[0] * nel[1] * nel[2] * (N + 1) ** 3


BATCH_BOX = (512.0e3, 512.0e3, 20.0e3)


def batch_specs(count=96, seed=4096):
    """Seeded per-instance parameters of the batched form: a list of dicts
    with nel, N, vmax, rmax, ring radius and peak, centre offset."""
    u = rng.uniform(seed, 8 * count).reshape(count, 8)
    specs = []
    for i in range(count):
        nel = (4 + int(21 * u[i, 0]), 4 + int(21 * u[i, 1]), 4 + int(9 * u[i, 2]))
        specs.append(dict(nel=nel, N=3 + int(4 * u[i, 3]), vmax=10.0 + 20.0 * u[i, 4],
                          rmax=30.0e3 + 50.0e3 * u[i, 5], ring_peak=5.0 + 10.0 * u[i, 6],
                          centre=(40.0e3 * (u[i, 7] - 0.5), -40.0e3 * (u[i, 7] - 0.5))))
    return specs


def _min_vertical_spacing(nel_z, N):
    xi = grid.lgl_points(N)
    return (BATCH_BOX[2] / nel_z) * (xi[1] - xi[0]) / 2.0


def batch_instance(spec, state="initial", seed=1):
    """Workload dict of one instance of the batched form (as ``tc``)."""
    nel, N = spec["nel"], spec["N"]
    lo = (-BATCH_BOX[0] / 2, -BATCH_BOX[1] / 2, 0.0)
    hi = (BATCH_BOX[0] / 2, BATCH_BOX[1] / 2, BATCH_BOX[2])
    periodic = (True, True, False)
    X, Y, Z, ax = grid.node_coords(nel, N, lo, hi, periodic)
    rho0, Th0 = atm.stable_sounding(ax[2], nbv=0.01)
    n_xy = ax[0].size * ax[1].size
    c = spec["centre"]
    q = atm.vortex_state(X, Y, Z, rho0, n_xy, c, vmax=spec["vmax"], rmax=spec["rmax"])
    if state == "random":
        q += atm.smooth_random_state(X, Y, Z, lo, hi, periodic, seed)
    elif state != "initial":
        raise ValueError(state)
    S = atm.heating(X, Y, Z, c, seed=seed, ncells=0, ring_peak=spec["ring_peak"],
                    ring_r=0.8 * spec["rmax"])
    dt = 0.1 * _min_vertical_spacing(nel[2], N) / _min_vertical_spacing(16, 4)
    return dict(name="batch", nel=tuple(nel), N=N, lo=lo, hi=hi, periodic=periodic,
                phys=dict(PHYS, f=5.0e-5), dt=dt, q=q, rho0=rho0, Theta0=Th0, S_theta=S)


CLOSURE_BOX = 10.0e3


def closure_case(seed, nel=(64, 64, 16), N=4):
    """One seeded run of the learned-closure form on the 10 km cube (see the
    module docstring).  The same seed gives the same analytic fields on any
    mesh (the fine and coarse runs of a pair share it)."""
    u = rng.uniform(seed, 8)
    lo, hi = (0.0, 0.0, 0.0), (CLOSURE_BOX,) * 3
    periodic = (False, False, False)
    X, Y, Z, ax = grid.node_coords(nel, N, lo, hi, periodic)
    rho0, Th0 = atm.isentropic_sounding(ax[2])
    n_xy = ax[0].size * ax[1].size
    c = (5.0e3 + 1.0e3 * (u[0] - 0.5), 5.0e3 + 1.0e3 * (u[1] - 0.5))
    q = atm.bubble_state(X, Y, Z, ax[2], rho0, Th0, n_xy, dtheta=1.0 + 2.0 * u[2],
                         radius=1.5e3 + 1.0e3 * u[3], centre=(c[0], c[1], 2.0e3 + 1.0e3 * u[4]))
    q += atm.vortex_state(X, Y, Z, rho0, n_xy, c, vmax=5.0 + 10.0 * u[5], rmax=1.0e3 + 1.0e3 * u[6],
                          D1=4.0e3, D2=3.5e3)
    s = [(X - lo[0]) / CLOSURE_BOX, (Y - lo[1]) / CLOSURE_BOX]
    for d in range(2):   # no flux through the lateral walls
        q[1 + d][(s[d] < 1e-9) | (s[d] > 1.0 - 1e-9)] = 0.0
    S = atm.heating(X, Y, Z, c, seed=seed, ncells=0, ring_peak=5.0 + 10.0 * u[7], ring_r=2.0e3,
                    ring_w=0.5e3, ztop=8.0e3)
    xi = grid.lgl_points(N)
    dmin = min(CLOSURE_BOX / nel[d] * (xi[1] - xi[0]) / 2.0 for d in range(3))
    dt = 0.1 * dmin / _min_vertical_spacing(16, 4)
    return dict(name="closure", nel=tuple(nel), N=N, lo=lo, hi=hi, periodic=periodic,
                phys=dict(PHYS, f=0.0), dt=dt, q=q, rho0=rho0, Theta0=Th0, S_theta=S)
