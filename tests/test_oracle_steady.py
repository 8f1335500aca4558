"""Pins of the oracle's discrete slab problem (Sec. 5, the supplement's upwind
finite-volume scheme) against properties fixed by its definition: the sweep
solves its upwind system, diffuse walls conserve mass, a uniform inflow state
is transport-free, and the continuation step tends to the explicit pseudo-time
step as dtau -> 0."""
import numpy as np
import pytest

from oracle.quadrature import hemisphere_rule
from oracle.steady import Slab, initial_state

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _maxwell(a, st):
    rho, u1, u2, u3, th = st
    return rho * (2 * np.pi * th) ** -1.5 * np.exp(
        -((a[:, None, None] - u1) ** 2 + (a[None, :, None] - u2) ** 2 + (a[None, None, :] - u3) ** 2) / (2 * th))


def test_sweep_solves_upwind_system():
    """z = sweep(r) satisfies v1^+ D^- z + v1^- D^+ z + (nu_j/Kn + s) z = r
    with zero ghost values, checked cell by cell with explicit neighbours."""
    S = Slab(8, 5.0, 1.0, 4, nx=5, kn=0.3, hemisphere=hemisphere_rule(1))
    rng = np.random.default_rng(3)
    r = rng.standard_normal((5, 8, 8, 8))
    nu = rng.uniform(0.5, 2.0, 5)
    for shift in (0.0, 1.7):
        z = S.sweep(r, nu, shift)
        for j in range(5):
            left = z[j - 1] if j > 0 else 0.0 * z[0]
            right = z[j + 1] if j < 4 else 0.0 * z[0]
            lhs = (S.vp * (z[j] - left) + S.vm * (right - z[j])) / S.dx + (nu[j] / S.kn + shift) * z[j]
            assert np.abs(lhs - r[j]).max() <= 1e-12 * np.abs(r).max()


def test_discrete_diffuse_walls_conserve_mass():
    """With the grid-sum wall factor, each wall re-emits exactly the mass
    that reaches it, so the transport term has zero total mass."""
    S = Slab(8, 5.0, 1.0, 4, nx=4, kn=1.0, hemisphere=hemisphere_rule(1), wall_flux="discrete",
             wall_left=(1.0, 0.0, 0.3, 0.0), wall_right=(2.0, 0.0, 0.0, -0.2))
    rng = np.random.default_rng(4)
    f = rng.uniform(0.0, 1.0, (4, 8, 8, 8))
    assert abs(S.mass(S.transport(f))) <= 1e-13 * S.mass(np.abs(S.transport(f)))
    # a correction's ghost values follow the same linear wall map
    assert abs(S.mass(S.transport(f - 0.5, linear=True))) <= 1e-12 * S.mass(np.abs(f))


def test_uniform_inflow_state_is_transport_free():
    """Both inflow sides carrying the state that fills the slab: every upwind
    difference vanishes, and the residual reduces to -Q(M, M)/Kn per cell."""
    st = (1.3, 0.8, 0.0, 0.0, 1.1)
    S = Slab(8, 6.0, 0.5, 4, nx=3, kn=0.2, hemisphere=hemisphere_rule(1), inflow_left=st, inflow_right=st)
    a = (np.arange(8) - 4) * S.h
    f = np.stack([_maxwell(a, st)] * 3)
    assert np.abs(S.transport(f)).max() <= 1e-15 * np.abs(f).max() / S.dx
    # the linear (correction) ghosts are zero: only the boundary cells feel them
    g = np.stack([_maxwell(a, st)] * 3)
    tg = S.transport(g, linear=True)
    assert np.abs(tg[1]).max() <= 1e-15 * np.abs(g).max() / S.dx
    assert np.allclose(tg[0], S.vp * g[0] / S.dx, rtol=0, atol=1e-15 * np.abs(g).max() / S.dx)
    assert np.allclose(tg[2], -S.vm * g[2] / S.dx, rtol=0, atol=1e-15 * np.abs(g).max() / S.dx)


def test_large_shift_gives_explicit_pseudo_time_step():
    """(A + s I) g = R with s -> infinity: s g -> R (forward Euler in pseudo
    time); the deviation is O(|A| / s)."""
    up = (1.0, 1.2, 0.0, 0.0, 1.0)
    down = (1.5, 0.8, 0.0, 0.0, 1.3)
    S = Slab(8, 6.0, 0.5, 4, nx=3, kn=0.5, hemisphere=hemisphere_rule(1), inflow_left=up, inflow_right=down)
    a = (np.arange(8) - 4) * S.h
    f = np.stack([_maxwell(a, up), _maxwell(a, (1.2, 1.0, 0.0, 0.0, 1.15)), _maxwell(a, down)])
    R = S.residual(f)
    errs = []
    for s in (1e4, 1e6):
        _, g, rn = S.newton_step(f.copy(), 0.0, rtol=1e-12, shift=s)
        assert abs(rn - S.norm(R)) <= 1e-12 * rn
        errs.append(np.abs(s * g - R).max() / np.abs(R).max())
    assert errs[1] < 1e-3
    assert errs[1] < 0.05 * errs[0]  # shrinks like 1/s


def test_exact_jacobian_is_the_derivative_of_the_residual():
    """R is quadratic in f (transport is linear, Q(f,f) is the diagonal of a
    symmetric bilinear form), so its central difference is exact for any
    step: (R(f + e g) - R(f - e g)) / (2 e) equals the exact Jacobian applied
    to g, which the oracle forms from the bilinear form instead of Q(f,f).
    With walls the ghost map is linear too; the check holds for both sides."""
    for inflow in (False, True):
        kw = dict(inflow_left=(1.0, 0.6, 0.0, 0.0, 1.0), inflow_right=(1.3, 0.4, 0.0, 0.0, 1.2)) if inflow else {}
        S = Slab(8, 6.0, 0.5, 4, nx=3, kn=0.4, hemisphere=hemisphere_rule(1), wall_flux="discrete", **kw)
        a = (np.arange(8) - 4) * S.h
        f = np.stack([_maxwell(a, (1.0 + 0.1 * j, 0.2 * j, 0.0, 0.1, 1.0 + 0.2 * j)) for j in range(3)])
        rng = np.random.default_rng(5)
        g = rng.standard_normal(f.shape) * f
        Jg = S.exact_jacobian(f)(g)
        if not inflow:  # the residual's ghost cells are the linear wall map of f
            for e in (1e-3, 0.7):
                fd = (S.residual(f + e * g) - S.residual(f - e * g)) / (2 * e)
                assert np.abs(fd - Jg).max() <= 1e-9 * np.abs(Jg).max()
        else:  # inflow ghosts are constant data: they cancel in the difference
            fd = (S.residual(f + 0.5 * g) - S.residual(f - 0.5 * g)) / 1.0
            assert np.abs(fd - Jg).max() <= 1e-9 * np.abs(Jg).max()


def test_bordered_newton_step_lands_on_the_total_mass():
    """Walls with the grid-sum wall flux and a mass-conserving Q (zero mode
    removed): every residual has zero total mass, and with the exact
    Jacobian (whose Q carries the same fix) so does every operator image, so
    the bordered system of the Newton step gives m(f - g) = C exactly
    (Eq. (5.3)), from a state of another mass."""
    S = Slab(8, 5.0, 1.0, 8, nx=3, kn=1.0, hemisphere=hemisphere_rule(1), wall_flux="discrete",
             q_mass_fix="zero_mode")
    a = (np.arange(8) - 4) * S.h
    f = np.stack([_maxwell(a, (1.0 + 0.1 * j, 0.0, 0.0, 0.0, 1.0 + 0.3 * j)) for j in range(3)])
    R = S.residual(f)
    assert abs(S.mass(R)) <= 1e-13 * S.mass(np.abs(R))
    C = 1.1 * S.mass(f)
    f_new, g, _ = S.newton_step(f, C, rtol=1e-12, restart=80, maxiter=200, jacobian="exact")
    assert abs(S.mass(f_new) - C) <= 1e-11 * C


def test_exact_jacobian_at_a_maxwellian_approaches_the_linearized_operator():
    """At a global Maxwellian the exact Jacobian's collision part is the
    M-point bilinear form Q(M, g) + Q(g, M), the form Sec. 4.1 compares with
    the M-free L[g]: at N = 16 they differ by the truncation (the paper's
    Table 1 gives 3.2e-3 at this resolution), a difference that no longer
    changes with the hemisphere order."""
    a = (np.arange(16) - 8) * (2 * 6.0 / 16)
    M = _maxwell(a, (1.0, 0.0, 0.0, 0.0, 1.0))
    g = M * (1.0 + 0.3 * a[:, None, None] - 0.2 * a[None, :, None] ** 2 + 0.1 * a[None, None, :])
    errs = []
    for p in (4, 8):
        S = Slab(16, 6.0, 1.0, 16, nx=1, kn=1.0, hemisphere=hemisphere_rule(p), wall_flux="discrete")
        lin = S.linear_operator(np.array([[1.0, 0.0, 0.0, 0.0, 1.0]]))(g[None])
        ex = S.exact_jacobian(M[None])(g[None])
        errs.append(np.abs(ex - lin).max() / np.abs(lin).max())
    assert 1e-4 < errs[0] < 5e-3
    assert abs(errs[0] - errs[1]) < 0.05 * errs[0]


def _wall_slab(kn):
    S = Slab(8, 5.0, 1.0, 4, nx=4, kn=kn, hemisphere=hemisphere_rule(1), wall_flux="discrete",
             wall_left=(1.0, 0.0, 0.0, 0.0), wall_right=(1.6, 0.0, 0.0, 0.0))
    a = (np.arange(8) - 4) * S.h
    f = np.stack([_maxwell(a, (1.0, 0.05 * j, 0.0, 0.0, 1.0 + 0.15 * j)) for j in range(4)])
    return S, f


def test_source_iteration_is_the_printed_update():
    """The supplement's update S g^{l+1} = (nu_j g^l + L_j[g^l])/Kn + r, with
    the wall and border couplings of g^l added to the right-hand side, equals
    the oracle's S g^{l+1} = (S - A) g^l + rhs and the sweep-preconditioned
    Richardson step g^l + sweep(rhs - A g^l), iterate by iterate."""
    S, f = _wall_slab(0.5)
    params = S.local_params(f)
    nu = params[:, 0]
    A = S.bordered_operator(params, f)
    L = S.linear_operator(params)
    e = f / S.mass(f)
    rng = np.random.default_rng(11)
    rhs = rng.standard_normal(f.shape) * f
    g = np.zeros_like(f)
    for _ in range(4):
        # printed form: collision part from L_j itself, transport part from
        # the ghost cells that S (zero ghosts) leaves out
        # L_j[g]/Kn = transport(g) - L(g) for the oracle's L(g) = transport(g) - L_j[g]/Kn
        coll = nu[:, None, None, None] * g / S.kn + (S.transport(g, linear=True) - L(g))
        ghost = S.transport(g, linear=True) - (S.sweep_operator(g, nu) - (nu[:, None, None, None] / S.kn) * g)
        printed = S.sweep(coll - ghost - e * S.mass(g) + rhs, nu)
        oracle_form = S.sweep(S.sweep_operator(g, nu) - A(g) + rhs, nu)
        richardson = g + S.sweep(rhs - A(g), nu)
        scale = np.abs(printed).max()
        assert np.abs(oracle_form - printed).max() <= 1e-12 * scale
        assert np.abs(richardson - printed).max() <= 1e-12 * scale
        g = printed


def _newton_system(kn, omega):
    """The bordered Newton system of the first step on a 4-cell wall slab at
    N = 16 (walls theta 1 and 2, the oracle's initial state)."""
    S = Slab(16, 5.5, omega, 16, nx=4, kn=kn, hemisphere=hemisphere_rule(1))
    f = initial_state(S)
    params = S.local_params(f)
    A = S.bordered_operator(params, f)
    rhs = S.residual(f)  # the initial state has the target mass: no border source
    return S, A, rhs, params[:, 0]


def test_source_iteration_converges_faster_at_large_kn():
    """Maxwell molecules: the source iteration reaches the solution of the
    bordered system (|rhs - A g| <= 1e-8 |rhs| with the oracle's own A), and
    it needs more iterations at the smaller Knudsen number, as Sec. 5.3
    reports for the Couette flow."""
    its = {}
    for kn in (0.2, 2.0):
        S, A, rhs, rho = _newton_system(kn, 1.0)
        g, it, ok = S.source_iteration(A, rhs, rho, rtol=1e-8, maxiter=400)
        assert ok, (kn, it)
        assert S.norm(rhs - A(g)) <= 1e-8 * S.norm(rhs)
        its[kn] = it
    assert its[0.2] > 1.5 * its[2.0], its


def test_hard_sphere_source_iteration_needs_the_positivity_condition():
    """Sec. 5.2 asks nu_j + L_j to be positive.  For hard spheres the loss
    frequency grows with |v| beyond rho_j, so nu_j = rho_j (the paper's
    practical choice) lets the iteration grow, while nu_j = 2 rho_j
    converges."""
    S, A, rhs, rho = _newton_system(2.0, 0.5)
    r0 = S.norm(rhs)
    g = np.zeros_like(rhs)
    for _ in range(20):
        g = g + S.sweep(rhs - A(g), rho)
    assert S.norm(rhs - A(g)) > r0
    g2, it, ok = S.source_iteration(A, rhs, 2.0 * rho, rtol=1e-6, maxiter=200)
    assert ok, it
