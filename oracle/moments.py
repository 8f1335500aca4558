"""Moments of Sec. 2.1 on the collocation grid, and the FP64 conservation
projection.  Oracle: test infrastructure only.

Integrals are the trapezoid (spectral) rule  int phi dv ~= h^3 sum_l phi(v_l).
"""
import numpy as np

from . import grid


def moments(f, n, L):
    """rho, u (3,), theta, p_ij (3,3), q (3,) of Sec. 2.1 for f on the cyclic
    grid."""
    h = grid.spacing(n, L)
    v = grid.velocity_grid(n, L)
    w = h ** 3
    rho = w * f.sum()
    u = np.array([w * (vd * f).sum() for vd in v]) / rho
    c = [v[d] - u[d] for d in range(3)]
    c2 = c[0] ** 2 + c[1] ** 2 + c[2] ** 2
    theta = w * (c2 * f).sum() / (3.0 * rho)
    p = np.array([[w * (c[i] * c[j] * f).sum() for j in range(3)] for i in range(3)])
    q = np.array([0.5 * w * (c2 * c[i] * f).sum() for i in range(3)])
    return rho, u, theta, p, q


def invariant_moments(x, n, L):
    """(int x, int v1 x, int v2 x, int v3 x, int |v|^2 x) by the grid rule."""
    h = grid.spacing(n, L)
    v1, v2, v3 = grid.velocity_grid(n, L)
    w = h ** 3
    return np.array([w * x.sum(), w * (v1 * x).sum(), w * (v2 * x).sum(),
                     w * (v3 * x).sum(), w * ((v1 ** 2 + v2 ** 2 + v3 ** 2) * x).sum()])


def conservation_projection(x, n, L):
    """Least-squares (Euclidean on the grid) projection of x onto
    {y : int phi y = 0 for phi in 1, v1, v2, v3, |v|^2}:
        x <- x - C^T (C C^T)^{-1} C x,  C the 5 x n^3 matrix of phi(v_l).
    The paper only cites such a post-processing (Sec. 1); this is the reading
    used for the library's moment-correction option."""
    v1, v2, v3 = grid.velocity_grid(n, L)
    one = np.ones((n, n, n))
    rows = [one, v1 * one, v2 * one, v3 * one, (v1 ** 2 + v2 ** 2 + v3 ** 2) * one]
    Cm = np.stack([r.ravel() for r in rows])
    y = x.ravel()
    lam = np.linalg.solve(Cm @ Cm.T, Cm @ y)
    return (y - Cm.T @ lam).reshape(x.shape)
