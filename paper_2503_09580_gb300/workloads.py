"""Seeded synthetic inputs shaped like the paper's tests (Sec. 4) and the
library's benchmark workloads.  This module holds no step of the collision
operator itself: it only draws random numbers and evaluates the input fields
(a Gaussian times a polynomial, plus grid noise) on the collocation grid.

Layout: centred order, g[b, i1, i2, i3] at v = (i - n/2) * (2L/n);
params[b] = (rho, u1, u2, u3, theta).
"""
import itertools

import numpy as np


def velocity_axis(n, L):
    """1-D collocation points v_i = (i - n/2) * 2L/n, centred order."""
    return (np.arange(n) - n // 2) * (2.0 * L / n)


def monomial_exponents(degree):
    """All alpha in N^3 with |alpha| <= degree (20 for 3, 35 for 4)."""
    return [a for a in itertools.product(range(degree + 1), repeat=3) if sum(a) <= degree]


def gaussian_times_polynomial(n, L, rho, u, theta, coeffs, degree):
    """g(v) = rho (2 pi theta)^{-3/2} exp(-|v-u|^2/(2 theta)) p(xi),
    xi = (v - u)/sqrt(theta), p(xi) = sum_alpha c_alpha xi^alpha."""
    a = velocity_axis(n, L)
    x = [(a - u[d]) / np.sqrt(theta) for d in range(3)]
    X = (x[0][:, None, None], x[1][None, :, None], x[2][None, None, :])
    p = np.zeros((n, n, n))
    for c, al in zip(coeffs, monomial_exponents(degree)):
        p += c * X[0] ** al[0] * X[1] ** al[1] * X[2] ** al[2]
    r2 = X[0] ** 2 + X[1] ** 2 + X[2] ** 2
    return rho * (2.0 * np.pi * theta) ** -1.5 * np.exp(-0.5 * r2) * p


def maxwellian_polynomial_batch(n, L, batch, seed, degree=4, noise=1e-3,
                                rho_range=(0.5, 2.0), u_range=(-0.5, 0.5),
                                theta_range=(0.5, 2.0), fixed_params=None):
    """(params (B,5), g (B,n,n,n)) with per-instance background Maxwellian
    parameters drawn uniformly (or ``fixed_params``), polynomial coefficients
    ~ N(0,1) and iid N(0, noise^2) grid noise, all from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nc = len(monomial_exponents(degree))
    params = np.empty((batch, 5))
    g = np.empty((batch, n, n, n))
    for b in range(batch):
        if fixed_params is None:
            rho = rng.uniform(*rho_range)
            u = rng.uniform(*u_range, size=3)
            theta = rng.uniform(*theta_range)
        else:
            rho, u, theta = fixed_params[0], np.asarray(fixed_params[1:4]), fixed_params[4]
        coeffs = rng.standard_normal(nc)
        g[b] = gaussian_times_polynomial(n, L, rho, u, theta, coeffs, degree)
        if noise:
            g[b] += noise * rng.standard_normal((n, n, n))
        params[b] = (rho, u[0], u[1], u[2], theta)
    return params, g


def single_instance(n=16, L=8.0, seed=0):
    """Homogeneous single instance: rho=1, u=0, theta=1, cubic polynomial
    with N(0,1) coefficients, no noise."""
    return maxwellian_polynomial_batch(n, L, 1, seed, degree=3, noise=0.0,
                                       fixed_params=(1.0, 0.0, 0.0, 0.0, 1.0))


def batched_instances(n=32, L=8.0, batch=256, seed=0, noise=1e-3):
    """Per-instance Maxwellians rho~U[0.5,2], u_i~U[-0.5,0.5],
    theta~U[0.5,2]; quartic polynomial; 1e-3 grid noise (0 for the
    noise-free twin)."""
    return maxwellian_polynomial_batch(n, L, batch, seed, degree=4, noise=noise)


def paper_f1(n, L):
    """Smooth test function f^(1) of Sec. 4 (four Gaussians of temperature
    1/3 shifted by sqrt(2) along +-v1 and +-v2), normalised to unit density
    (the printed prefactor 1/(4 pi^{3/2}) gives density 0.544; Tables 1 and 3
    are reproduced with unit density).  Centred order."""
    a = velocity_axis(n, L)
    v1, v2, v3 = a[:, None, None], a[None, :, None], a[None, None, :]
    th, s = 1.0 / 3.0, np.sqrt(2.0)

    def e(x, y, z):
        return np.exp(-(x * x + y * y + z * z) / (2.0 * th))
    return (e(v1 + s, v2, v3) + e(v1 - s, v2, v3) + e(v1, v2 + s, v3)
            + e(v1, v2 - s, v3)) / (4.0 * (2.0 * np.pi * th) ** 1.5)


def paper_f2(n, L):
    """Discontinuous test function f^(2) of Sec. 4 (unit density, zero
    velocity, unit temperature).  On the plane v1 = 0, where the paper leaves
    it undefined, it takes the mean of its two branches.  Centred order."""
    a = velocity_axis(n, L)
    v1, v2, v3 = a[:, None, None], a[None, :, None], a[None, None, :]
    r2 = v1 ** 2 + v2 ** 2 + v3 ** 2
    c = 2.0 ** 0.25 * (2.0 - np.sqrt(2.0)) / np.pi ** 1.5
    pos = c * np.exp(-r2 / np.sqrt(2.0))
    neg = 0.25 * c * np.exp(-r2 / (2.0 * np.sqrt(2.0)))
    return np.where(v1 > 0, pos, np.where(v1 < 0, neg, 0.5 * (pos + neg)))
