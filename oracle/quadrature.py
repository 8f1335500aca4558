"""Quadrature rules of Eq. (2.13) (Sec. 2.3).  Oracle: test infrastructure only.

Radial rule:   int_0^R g^2 psi(g) dg  ~=  sum_j w_j psi(g_j)
Hemisphere:    int_{S^2_+} phi(sigma) dsigma ~= 2*pi * sum_m w_m phi(sigma_m)

The paper uses Jacobi-Gauss-Radau radially and Lebedev rules on the sphere
(Sec. 4.1).  The reading used here: Gauss-Legendre on [0, R] with the g^2
factor folded into the weights, and a product rule on the hemisphere
(Gauss-Legendre in cos(theta) on (0, 1) times a uniform azimuth), with the
weights normalised so that sum_m w_m = 1 (the 2*pi in Eq. (2.13) is the
hemisphere's area).
"""
import numpy as np
from scipy.special import eval_legendre, roots_jacobi


def gauss_legendre(J):
    """Nodes/weights of the J-point Gauss-Legendre rule on [-1, 1]
    (a library routine used as a step)."""
    x, w = np.polynomial.legendre.leggauss(int(J))
    return x, w


def radial_rule(J, R):
    """(g_j, w_j) with  sum_j w_j psi(g_j) ~= int_0^R g^2 psi(g) dg  (Eq. 2.13).

    Gauss-Legendre on [0, R]: g_j = R (x_j + 1)/2, w_j = (R/2) w_j^GL g_j^2.
    Exact for psi a polynomial of degree <= 2J - 3."""
    x, w = gauss_legendre(J)
    g = 0.5 * R * (x + 1.0)
    return g, 0.5 * R * w * g * g


def radial_rule_jgr(J, R, fixed_end=+1):
    """Jacobi-Gauss-Radau rule for int_0^R g^2 psi(g) dg (the paper's radial
    rule, Sec. 4.1): weight (1+x)^2 on [-1, 1] with one node fixed at
    x = fixed_end (g = R for +1, g = 0 for -1), the other J-1 nodes the zeros
    of the Jacobi polynomial P_{J-1}^{(1,2)} (resp. P_{J-1}^{(0,3)}).
    Exact for psi of degree <= 2J - 2.  Weights solve the exactness
    conditions on Legendre polynomials P_0..P_{J-1}."""
    if fixed_end == +1:
        xi, _ = roots_jacobi(J - 1, 1.0, 2.0)
    else:
        xi, _ = roots_jacobi(J - 1, 0.0, 3.0)
    x = np.sort(np.concatenate([xi, [float(fixed_end)]]))
    xg, wg = gauss_legendre(J + 4)
    A = np.array([eval_legendre(k, x) for k in range(J)])
    b = np.array([(wg * (1.0 + xg) ** 2 * eval_legendre(k, xg)).sum() for k in range(J)])
    w = np.linalg.solve(A, b)
    return 0.5 * R * (1.0 + x), (0.5 * R) ** 3 * w


def radial_rule_kind(J, R, kind="gl"):
    """Dispatch: 'gl' (default reading), 'jgr' (Radau node at g = R) or
    'jgr0' (Radau node at g = 0)."""
    if kind == "gl":
        return radial_rule(J, R)
    if kind == "jgr":
        return radial_rule_jgr(J, R, +1)
    if kind == "jgr0":
        return radial_rule_jgr(J, R, -1)
    raise ValueError(kind)


def hemisphere_rule(p):
    """Product rule with M = p * 2p points on the upper hemisphere.

    Returns sigma (M, 3) and weights w (M,) with sum w = 1, so that
    int_{S^2_+} phi dsigma ~= 2*pi * sum_m w_m phi(sigma_m)   (Eq. 2.13).
    cos(theta) uses p-point Gauss-Legendre mapped to (0, 1); the azimuth uses
    2p equispaced angles (exact for trigonometric degree < 2p)."""
    x, w = gauss_legendre(p)
    mu = 0.5 * (x + 1.0)            # cos(theta) in (0, 1)
    wmu = 0.5 * w                   # sums to 1 over (0, 1)
    na = 2 * p
    phi = (np.arange(na) + 0.5) * (2.0 * np.pi / na)
    st = np.sqrt(1.0 - mu * mu)
    sig = np.stack([
        (st[:, None] * np.cos(phi)[None, :]).ravel(),
        (st[:, None] * np.sin(phi)[None, :]).ravel(),
        np.repeat(mu, na),
    ], axis=1)
    wm = np.repeat(wmu, na) / na
    return sig, wm


def hemisphere_rule_M(M):
    """Product hemisphere rule for M = 2 p^2 points (M = 32 -> p = 4)."""
    p = int(round(np.sqrt(M / 2.0)))
    if 2 * p * p != M:
        raise ValueError("product hemisphere rule needs M = 2 p^2")
    return hemisphere_rule(p)


def vhs_kernel(g, omega, C=1.0 / (4.0 * np.pi)):
    """Variable hard-sphere kernel B(g) = C g^{2(1 - omega)}, Eq. (2.4),
    with C = 1/(4 pi) as in Eq. (4.1)."""
    return C * np.power(g, 2.0 * (1.0 - omega))
