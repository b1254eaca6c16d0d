"""Synthetic atmospheric inputs: reference soundings, initial states and the
heating source, sampled at node positions.

The paper's tropical-cyclone case reads its reference sounding from a table
(Sec. 4.1, Fig. 3) and its heating from airborne radar data (Fig. 4); neither
is available, so analytic stand-ins of the same shape are used:

* isentropic reference state theta_0 = 300 K (the rising-bubble box) and a
  stable sounding with constant Brunt-Vaisala frequency N_BV (the cyclone
  box), both in hydrostatic balance through the Exner function
  pi = (p/p_a)^(R/c_p);
* a cosine potential-temperature bubble with unperturbed Exner pressure;
* a warm-core vortex with a modified-Rankine surface wind, the height decay
  and lateral cut-off factors of Sec. 4.1's vortex (Eq. 17, read as
  exp(-z^sigma/(sigma D1^sigma)) exp(-(r/D2)^6));
* a heating field: an azimuthal ring plus seeded Gaussian convective cells
  with a sine vertical profile over 0-15 km, in K/h, returned in K/s.
"""

import numpy as np

from . import rng

G, R_D, CP, P_A = 9.81, 287.0, 1004.5, 1.0e5


def isentropic_sounding(z, theta0=300.0, g=G, R=R_D, cp=CP, p_a=P_A):
    """Reference (rho_0, Theta_0 = rho_0 theta_0) of a constant-theta
    atmosphere: pi_0 = 1 - g z / (c_p theta_0)."""
    z = np.asarray(z, dtype=np.float64)
    pi0 = 1.0 - g * z / (cp * theta0)
    p0 = p_a * pi0 ** (cp / R)
    th = np.full_like(z, theta0)
    rho0 = p0 / (R * pi0 * th)
    return rho0, rho0 * th


def stable_sounding(z, nbv=0.01, theta_s=300.0, g=G, R=R_D, cp=CP, p_a=P_A):
    """Reference state with constant Brunt-Vaisala frequency nbv:
    theta_0 = theta_s exp(nbv^2 z / g) and the hydrostatic Exner function
    pi_0 = 1 + g^2 / (c_p theta_s nbv^2) (exp(-nbv^2 z / g) - 1)."""
    z = np.asarray(z, dtype=np.float64)
    s = nbv * nbv / g
    th = theta_s * np.exp(s * z)
    pi0 = 1.0 + g * g / (cp * theta_s * nbv * nbv) * (np.exp(-s * z) - 1.0)
    p0 = p_a * pi0 ** (cp / R)
    rho0 = p0 / (R * pi0 * th)
    return rho0, rho0 * th


def bubble_state(X, Y, Z, z_levels, rho0_lev, Theta0_lev, n_xy, dtheta=2.0, radius=2000.0,
                 centre=(5000.0, 5000.0, 2000.0)):
    """Cosine warm bubble: theta' = dtheta (1 + cos(pi r / radius)) / 2 for
    r <= radius, Exner pressure unperturbed, so Theta' = 0 and
    rho' = rho_0 theta_0 / (theta_0 + theta') - rho_0; momentum zero."""
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    thp = np.where(r <= radius, 0.5 * dtheta * (1.0 + np.cos(np.pi * r / radius)), 0.0)
    gz = np.arange(X.size) // n_xy
    rho0 = rho0_lev[gz]
    th0 = Theta0_lev[gz] / rho0
    q = np.zeros((5, X.size))
    q[0] = rho0 * th0 / (th0 + thp) - rho0
    return q


def vortex_state(X, Y, Z, rho0_lev, n_xy, centre, vmax=15.0, rmax=50.0e3, decay=0.5,
                 sigma=2.0, D1=5823.0, D2=200.0e3):
    """Warm-core vortex momentum: tangential wind
    u_t = V(r) exp(-z^sigma / (sigma D1^sigma)) exp(-(r/D2)^6) with the
    modified-Rankine V(r) = vmax r / rmax inside rmax and vmax (rmax/r)^decay
    outside, counter-clockwise; rho' = Theta' = 0, w = 0."""
    dx, dy = X - centre[0], Y - centre[1]
    r = np.sqrt(dx * dx + dy * dy)
    V = np.where(r <= rmax, vmax * r / rmax, vmax * (rmax / np.maximum(r, 1e-30)) ** decay)
    ut = V * np.exp(-Z ** sigma / (sigma * D1 ** sigma)) * np.exp(-(r / D2) ** 6)
    rs = np.maximum(r, 1e-30)
    gz = np.arange(X.size) // n_xy
    rho0 = rho0_lev[gz]
    q = np.zeros((5, X.size))
    q[1] = rho0 * (-ut * dy / rs)
    q[2] = rho0 * (ut * dx / rs)
    return q


def heating(X, Y, Z, centre, seed=2504, ncells=32, ring_peak=10.0, ring_r=40.0e3,
            ring_w=10.0e3, cell_r=5.0e3, cell_amp=(5.0, 20.0), annulus=(20.0e3, 120.0e3),
            ztop=15.0e3):
    """Heating S_theta [K/s]: ring ring_peak exp(-((r - ring_r)/ring_w)^2) plus
    ``ncells`` Gaussian cells amp exp(-(d/cell_r)^2) with seeded centres uniform
    in the annulus and amplitudes U(cell_amp) K/h, all times sin(pi z/ztop) for
    z <= ztop (zero above)."""
    dx, dy = X - centre[0], Y - centre[1]
    r = np.sqrt(dx * dx + dy * dy)
    horiz = ring_peak * np.exp(-((r - ring_r) / ring_w) ** 2)
    u = rng.uniform(seed, 3 * ncells).reshape(ncells, 3)
    rc = np.sqrt(annulus[0] ** 2 + u[:, 0] * (annulus[1] ** 2 - annulus[0] ** 2))
    phi = 2.0 * np.pi * u[:, 1]
    amp = cell_amp[0] + (cell_amp[1] - cell_amp[0]) * u[:, 2]
    for k in range(ncells):
        cx = centre[0] + rc[k] * np.cos(phi[k])
        cy = centre[1] + rc[k] * np.sin(phi[k])
        horiz = horiz + amp[k] * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / cell_r ** 2)
    vert = np.where(Z <= ztop, np.sin(np.pi * np.clip(Z, 0.0, ztop) / ztop), 0.0)
    return horiz * vert / 3600.0


def smooth_random_state(X, Y, Z, lo, hi, periodic, seed, amps=(2e-3, 1.0, 1.0, 0.5, 0.3),
                        modes=4):
    """Sum of ``modes`` seeded sine modes per variable, with wavelengths that
    fit the box (integer wave numbers 1..3 in each direction); the momentum
    component normal to a walled direction is multiplied by sin(pi s) of the
    normalised coordinate so that it vanishes on those walls."""
    L = [hi[d] - lo[d] for d in range(3)]
    s = [(X - lo[0]) / L[0], (Y - lo[1]) / L[1], (Z - lo[2]) / L[2]]
    q = np.zeros((5, X.size))
    u = rng.uniform(seed, 5 * modes * 7).reshape(5, modes, 7)
    for v in range(5):
        for m in range(modes):
            k = 1.0 + np.floor(3.0 * u[v, m, :3])
            ph = 2.0 * np.pi * u[v, m, 3:6]
            a = amps[v] * (0.5 + u[v, m, 6]) / modes
            q[v] += a * (np.sin(2 * np.pi * k[0] * s[0] + ph[0])
                         * np.sin(2 * np.pi * k[1] * s[1] + ph[1])
                         * np.sin(2 * np.pi * k[2] * s[2] + ph[2]))
    for d in range(3):
        if not periodic[d]:
            q[1 + d] *= np.sin(np.pi * s[d])
            q[1 + d][(s[d] < 1e-9) | (s[d] > 1.0 - 1e-9)] = 0.0
    return q
