"""Pins of two oracle functions against their definitions (no GPU), each with
a planted mistake that the check must reject.

* ``cutoff_mask`` (Eq. (3.9), Sec. 3.4) is a rewritten form of "M/rho < eps";
  the check forms M from its definition (Sec. 2.1) and compares the masks at
  grid points away from the tie M/rho = eps.
* ``conservation_projection`` is the least-squares projection onto zero mass,
  momentum and energy: its output has vanishing invariant moments, it is
  idempotent, and what it removes lies in span{1, v, |v|^2} (orthogonality of
  the least-squares residual).  An oblique projection passes the first two
  checks but not the third.
"""
import numpy as np
import pytest

from oracle import grid
from oracle.linearized import cutoff_mask
from oracle.moments import conservation_projection, invariant_moments

CASES = [(1.0, (0.0, 0.0, 0.0), 1.0), (1.7, (0.3, -0.4, 0.2), 0.8), (0.6, (-0.5, 0.1, 0.45), 1.9),
         (2.0, (0.2, 0.2, -0.3), 0.5)]


def maxwellian_from_definition(n, L, rho, u, theta):
    """M(v) = rho (2 pi theta)^{-3/2} exp(-|v-u|^2/(2 theta)) (Sec. 2.1), point
    by point on the cyclic grid, with |v-u|^2 returned alongside."""
    ax = grid.velocity_axes(n, L)
    d2 = np.empty((n, n, n))
    M = np.empty((n, n, n))
    for a in range(n):
        for b in range(n):
            for c in range(n):
                s = (ax[a] - u[0]) ** 2 + (ax[b] - u[1]) ** 2 + (ax[c] - u[2]) ** 2
                d2[a, b, c] = s
                M[a, b, c] = rho * (2.0 * np.pi * theta) ** -1.5 * np.exp(-s / (2.0 * theta))
    return M, d2


def mask_mismatches(mask_fn, n, L, eps):
    """Number of grid points, over CASES and away from ties, where
    mask_fn(d2, theta, eps) differs from M/rho < eps; also the number of
    points compared and of points cut."""
    bad = compared = cut = 0
    for rho, u, th in CASES:
        M, d2 = maxwellian_from_definition(n, L, rho, u, th)
        ratio = M / rho
        away = np.abs(np.log(ratio) - np.log(eps)) > 1e-6
        want = ratio < eps
        got = mask_fn(d2, th, eps)
        bad += int(np.count_nonzero((got != want) & away))
        compared += int(np.count_nonzero(away))
        cut += int(np.count_nonzero(want & away))
    return bad, compared, cut


@pytest.mark.parametrize("eps", [1e-9, 1e-5])
def test_cutoff_mask_is_m_over_rho_below_eps(eps):
    n, L = 24, 8.0
    bad, compared, cut = mask_mismatches(cutoff_mask, n, L, eps)
    assert compared > 0.99 * len(CASES) * n ** 3
    assert 0 < cut < compared  # both sides of the threshold are exercised
    assert bad == 0


def _mask_sign_flipped(d2, theta, eps):
    return d2 / (2.0 * theta) > np.log(1.0 / eps) + 1.5 * np.log(2.0 * np.pi * theta)


def _mask_without_rho(d2, theta, eps, rho_of_theta={1.0: 1.0, 0.8: 1.7, 1.9: 0.6, 0.5: 2.0}):
    # "M < eps" in place of "M/rho < eps": the density enters the threshold
    rho = rho_of_theta[theta]
    return d2 / (2.0 * theta) > np.log(rho / eps) - 1.5 * np.log(2.0 * np.pi * theta)


def _mask_wrong_factor(d2, theta, eps):
    return d2 / theta > np.log(1.0 / eps) - 1.5 * np.log(2.0 * np.pi * theta)


@pytest.mark.parametrize("planted", [_mask_sign_flipped, _mask_without_rho, _mask_wrong_factor])
def test_cutoff_check_rejects_planted_mistakes(planted):
    bad, _, _ = mask_mismatches(planted, 24, 8.0, 1e-9)
    assert bad > 0


# ------------------------------------------------------------ projection
def invariant_basis(n, L):
    v1, v2, v3 = grid.velocity_grid(n, L)
    one = np.ones((n, n, n))
    return np.stack([(one * b).ravel() for b in (1.0, v1, v2, v3, v1 ** 2 + v2 ** 2 + v3 ** 2)], axis=1)


def projection_defects(proj, n, L, x):
    """(max |moments of P x|, |P P x - P x|, distance of x - P x from
    span{1, v, |v|^2}), each relative to |x|."""
    y = proj(x, n, L)
    scale = np.abs(x).max()
    mom = np.abs(invariant_moments(y, n, L)).max() / ((2 * L / n) ** 3 * np.abs(x).sum())
    idem = np.abs(proj(y, n, L) - y).max() / scale
    d = (x - y).ravel()
    Bm = invariant_basis(n, L)
    coef, *_ = np.linalg.lstsq(Bm, d, rcond=None)
    off = np.abs(d - Bm @ coef).max() / scale
    return mom, idem, off


def test_conservation_projection_is_least_squares():
    n, L = 16, 8.0
    rng = np.random.default_rng(21)
    x = rng.standard_normal((n, n, n))
    mom, idem, off = projection_defects(conservation_projection, n, L, x)
    assert mom < 1e-13 and idem < 1e-12 and off < 1e-12
    # least squares: the projection is the closest admissible point
    y = conservation_projection(x, n, L)
    z = conservation_projection(rng.standard_normal((n, n, n)), n, L)
    for t in (1e-3, -0.2, 1.0):
        assert np.linalg.norm(x - y) <= np.linalg.norm(x - (y + t * z)) + 1e-12


def _oblique_projection(x, n, L):
    """x - D C^T (C D C^T)^{-1} C x with a positive diagonal D: zero moments
    and idempotent, but not the least-squares projection."""
    v1, v2, v3 = grid.velocity_grid(n, L)
    D = np.exp(-0.05 * (v1 ** 2 + v2 ** 2 + v3 ** 2)).ravel()
    Cm = invariant_basis(n, L).T
    y = x.ravel()
    lam = np.linalg.solve(Cm @ (D[:, None] * Cm.T), Cm @ y)
    return (y - D * (Cm.T @ lam)).reshape(x.shape)


def test_projection_check_rejects_oblique_projection():
    n, L = 16, 8.0
    x = np.random.default_rng(22).standard_normal((n, n, n))
    mom, idem, off = projection_defects(_oblique_projection, n, L, x)
    assert mom < 1e-12 and idem < 1e-10  # passes the two weaker checks
    assert off > 1e-3                    # fails the span check


# ------------------------------------------------ Eq. (2.16) mass fix of Q
def _q_mass(Q, n, L):
    return (2 * L / n) ** 3 * Q.sum(), (2 * L / n) ** 3 * np.abs(Q).sum()


def _anisotropic_f(n, L):
    from oracle.linearized import maxwellians
    M, *_ = maxwellians(n, L, 1.0, np.array([0.3, -0.2, 0.1]), 0.9)
    v1, v2, v3 = grid.velocity_grid(n, L)
    return M * (1 + 0.4 * v1 * v2 - 0.3 * v3 ** 2 + 0.2 * v1 ** 3)


def test_sinc_quadrature_loss_conserves_mass():
    """Sec. 2.3: with the loss multiplier's sinc replaced by its hemisphere
    quadrature, Eq. (2.16), the bracket of Eq. (2.15) vanishes term by term,
    so Q^_0 = 0 up to rounding; with the exact sinc it does not."""
    from oracle.linearized import Tables
    from oracle.quadratic import quadratic_operator
    from oracle.quadrature import hemisphere_rule
    n, L = 16, 8.0
    tab = Tables(n, L, 0.5, n)
    f = _anisotropic_f(n, L)
    sig, w = hemisphere_rule(2)
    for p in (2, 4):
        sig, w = hemisphere_rule(p)
        m0, a0 = _q_mass(quadratic_operator(tab, f, sig, w), n, L)
        m1, a1 = _q_mass(quadratic_operator(tab, f, sig, w, mass_fix="sinc_quadrature"), n, L)
        assert abs(m0) > 1e-6 * a0     # the plain M-point form loses mass
        assert abs(m1) < 1e-13 * a1    # Eq. (2.16) keeps it to rounding


def test_sinc_quadrature_check_rejects_the_plain_nyquist_cosine():
    """A planted mistake at the Nyquist planes: cos(2 alpha_d N_p) (the loss
    argument's own cosine) in place of the gain's squared factor
    cos^2(alpha_d N_p) breaks the cancellation of Eq. (2.15)."""
    from oracle.linearized import FFT, InvFFT, Tables
    from oracle.quadratic import phase_multiplier, quadratic_operator
    from oracle.quadrature import hemisphere_rule
    n, L = 16, 8.0
    tab = Tables(n, L, 0.5, n)
    f = _anisotropic_f(n, L)
    sig, w = hemisphere_rule(2)
    _, Qp, _ = quadratic_operator(tab, f, sig, w, return_parts=True)
    om = np.zeros((n,) * 3)
    for j in range(tab.J):
        acc = sum(w[m] * np.real(phase_multiplier(n, np.pi * tab.g[j] * sig[m] / L)) for m in range(len(w)))
        om += tab.w[j] * tab.B[j] * acc
    m, a = _q_mass(Qp - f * np.real(InvFFT(FFT(f) * 16 * np.pi ** 2 * om)), n, L)
    assert abs(m) > 1e-3 * a


def test_sinc_quadrature_check_rejects_the_gain_argument():
    """A planted mistake: the loss quadrature taken at the gain's argument
    pi g_j sigma . k / (2L) (Eq. (2.14)) instead of pi g_j sigma . k / L
    (Eq. (2.16))."""
    from oracle.linearized import FFT, InvFFT, Tables
    from oracle.quadratic import phase_multiplier, quadratic_operator
    from oracle.quadrature import hemisphere_rule
    n, L = 16, 8.0
    tab = Tables(n, L, 0.5, n)
    f = _anisotropic_f(n, L)
    sig, w = hemisphere_rule(2)
    _, Qp, _ = quadratic_operator(tab, f, sig, w, return_parts=True)
    om = np.zeros((n,) * 3)
    for j in range(tab.J):
        acc = sum(w[m] * np.real(phase_multiplier(n, np.pi * tab.g[j] * sig[m] / (2 * L))) for m in range(len(w)))
        om += tab.w[j] * tab.B[j] * acc
    Qbad = Qp - f * np.real(InvFFT(FFT(f) * 16 * np.pi ** 2 * om))
    m, a = _q_mass(Qbad, n, L)
    assert abs(m) > 1e-3 * a
