"""Explicit time integration of the spatially homogeneous equations of
Sec. 4.2, df/dt = Q(f,f) and df/dt = L[f], by the classical fourth-order
Runge-Kutta scheme (the paper's choice, step 0.1).  Oracle: test
infrastructure only."""


def rk4(op, f, dt, nsteps):
    """nsteps steps of k1 = op(f), k2 = op(f + dt/2 k1), k3 = op(f + dt/2 k2),
    k4 = op(f + dt k3), f <- f + dt/6 (k1 + 2 k2 + 2 k3 + k4); returns f."""
    for _ in range(nsteps):
        k1 = op(f)
        k2 = op(f + 0.5 * dt * k1)
        k3 = op(f + 0.5 * dt * k2)
        k4 = op(f + dt * k3)
        f = f + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return f
