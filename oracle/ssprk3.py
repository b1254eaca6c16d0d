"""Three-stage SSP Runge-Kutta (Shu-Osher form) applied to Eq. 12.

The paper advances Eq. 12 with IMEX ARK2 (Sec. 2.3); the explicit path built
here advances the same semi-discrete system with the classical third-order
strong-stability-preserving scheme:

    q1      = q^n + dt L(q^n)
    q2      = 3/4 q^n + 1/4 (q1 + dt L(q1))
    q^{n+1} = 1/3 q^n + 2/3 (q2 + dt L(q2))
"""


def ssprk3_step(L, q, dt):
    """One SSP-RK3 step of dq/dt = L(q)."""
    q1 = q + dt * L(q)
    q2 = 0.75 * q + 0.25 * (q1 + dt * L(q1))
    return q / 3.0 + (2.0 / 3.0) * (q2 + dt * L(q2))


def run(L, q, dt, nsteps):
    """nsteps SSP-RK3 steps."""
    for _ in range(nsteps):
        q = ssprk3_step(L, q, dt)
    return q
