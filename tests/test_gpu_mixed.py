"""Slab whose cells carry different velocity grids (lbo_solver_create_mixed)
against the oracle's MixedSlab: the residual (collisions per cell, upwind
neighbours spectrally resampled to the cell's grid), one Newton step, and the
Mach-2 shock with N in {24, 32, 48} per cell solved to 1e-10."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.quadrature import hemisphere_rule
from oracle.steady import MixedSlab
from paper_2503_09580_gb300 import lbo

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GAMMA = 5.0 / 3.0


def _rh(mach):
    u1 = mach * np.sqrt(GAMMA)
    r = (GAMMA + 1) * mach ** 2 / ((GAMMA - 1) * mach ** 2 + 2)
    p2 = 1 + 2 * GAMMA / (GAMMA + 1) * (mach ** 2 - 1)
    return (1.0, u1, 0.0, 0.0, 1.0), (r, u1 / r, 0.0, 0.0, p2 / r)


def _blend(ns, L, up, down, width=0.15, x_left=-1.0, x_right=1.0, wobble=0.0):
    nx = len(ns)
    x = x_left + (np.arange(nx) + 0.5) * (x_right - x_left) / nx
    cells = []
    for j, (n, wj) in enumerate(zip(ns, 0.5 * (1 + np.tanh(x / width)))):
        rho, u1, _, _, th = [(1 - wj) * p + wj * q for p, q in zip(up, down)]
        a = (np.arange(n) - n // 2) * (2 * L / n)
        m = rho * (2 * np.pi * th) ** -1.5 * np.exp(-((a[:, None, None] - u1) ** 2 + a[None, :, None] ** 2
                                                      + a[None, None, :] ** 2) / (2 * th))
        if wobble:
            m = m * (1 + wobble * np.cos(j + a[:, None, None] + 0.5 * a[None, None, :]))
        cells.append(m)
    return cells


def _flat(cells):
    return np.concatenate([c.ravel() for c in cells])


def _small_case(jacobian="local_maxwellian", pdt=0.0, precond="sweep"):
    up, down = _rh(1.4)
    ns, L = [16, 24, 24, 16], 8.0
    oracle = MixedSlab(ns, L, 0.5, x_left=-0.5, x_right=0.5, kn=0.5, hemisphere=hemisphere_rule(1),
                       inflow_left=up, inflow_right=down)
    plans = [lbo.Plan(16, L, 0.5, 16, hemisphere_p=1), lbo.Plan(24, L, 0.5, 24, hemisphere_p=1)]
    solver = lbo.mixed_solver(plans, [0, 1, 1, 0], kind="slab", x_left=-0.5, x_right=0.5, kn=0.5,
                              inflow_left=up, inflow_right=down, krylov_rtol=1e-11, krylov_atol=0.0,
                              krylov_restart=80, krylov_maxit=1200, precond=precond, pseudo_dt=pdt,
                              jacobian=jacobian)
    f = _blend(ns, L, up, down, width=0.3, x_left=-0.5, x_right=0.5, wobble=0.05)
    return oracle, plans, solver, f


def test_mixed_residual_matches_oracle():
    oracle, plans, solver, f = _small_case()
    assert solver.state_length() == 2 * 16 ** 3 + 2 * 24 ** 3
    tf = torch.from_numpy(_flat(f)).to(DEV)
    out = torch.empty_like(tf)
    nrm = solver.residual(tf, out)
    ref = _flat(oracle.residual(f))
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    assert abs(nrm - oracle.norm(oracle.residual(f))) <= 1e-12 * nrm


def test_mixed_solver_with_one_n_is_the_uniform_solver():
    up, down = _rh(1.4)
    L = 8.0
    plan = lbo.Plan(16, L, 0.5, 16, hemisphere_p=1)
    kw = dict(kind="slab", x_left=-0.5, x_right=0.5, kn=0.5, inflow_left=up, inflow_right=down,
              krylov_rtol=1e-8, krylov_atol=0.0, krylov_restart=40, krylov_maxit=400, precond="sweep",
              pseudo_dt=0.5)
    uni = plan.solver(nx=3, total_mass=1.0, **kw)
    mix = lbo.mixed_solver([plan], [0, 0, 0], **kw)
    f = _flat(_blend([16] * 3, L, up, down, width=0.3, x_left=-0.5, x_right=0.5, wobble=0.05))
    out_u, out_m = torch.empty(f.size, dtype=torch.float64, device=DEV), torch.empty(f.size, dtype=torch.float64,
                                                                                        device=DEV)
    a = uni.residual(torch.from_numpy(f).to(DEV), out_u)
    b = mix.residual(torch.from_numpy(f).to(DEV), out_m)
    assert abs(a - b) <= 1e-13 * a
    assert torch.allclose(out_u, out_m, rtol=0, atol=1e-13 * float(out_u.abs().max()))
    tu, tm = torch.from_numpy(f.copy()).to(DEV), torch.from_numpy(f.copy()).to(DEV)
    su, sm = uni.newton_step(tu), mix.newton_step(tm)
    assert su["converged_inner"] and sm["converged_inner"]
    assert float((tu - tm).abs().max()) <= 1e-9 * float(tu.abs().max())


@pytest.mark.parametrize("jacobian", ["local_maxwellian", "exact"])
def test_mixed_newton_step_matches_oracle(jacobian):
    """One continuation step (shift 2) on the mixed slab: the GPU's
    sweep-preconditioned FGMRES and the oracle's plain GMRES solve the same
    system; the corrections agree to the solver tolerance."""
    oracle, plans, solver, f = _small_case(jacobian=jacobian, pdt=0.5)
    f_ref, g_ref, rn_ref = oracle.newton_step(f, rtol=1e-11, shift=2.0, jacobian=jacobian)
    tf = torch.from_numpy(_flat(f)).to(DEV)
    st = solver.newton_step(tf)
    g = _flat(f) - tf.cpu().numpy()
    gr = _flat(g_ref)
    print(jacobian, st["krylov_iterations"], st["linear_residual"] / st["rhs_norm"])
    assert st["converged_inner"]
    assert abs(st["residual_norm"] - rn_ref) <= 1e-12 * rn_ref
    assert np.abs(g - gr).max() <= 1e-7 * np.abs(gr).max()


def test_mixed_mach2_shock_converges():
    """Mach-2 shock, Kn = 0.1, 32 cells with N drawn per cell from {24, 32,
    48} (seeded, probabilities 0.5 / 0.35 / 0.15): continuation with
    exact-Jacobian steps, FP32 operator, FP64 residual per N, sweep on the
    finest grid, converges to |R| < 1e-10."""
    up, down = _rh(2.0)
    L, nx = 8.0, 32
    rng = np.random.default_rng(5)
    choice = rng.choice(3, size=nx, p=[0.5, 0.35, 0.15])
    Ns = (24, 32, 48)
    plans = [lbo.Plan(n, L, 0.5, n, hemisphere_p=2, precision="fp32", mass_fix=1) for n in Ns]
    res_plans = [lbo.Plan(n, L, 0.5, n, hemisphere_p=2, mass_fix=1) for n in Ns]
    solver = lbo.mixed_solver(plans, list(choice), kind="slab", x_left=-1.0, x_right=1.0, kn=0.1,
                              inflow_left=up, inflow_right=down, krylov_rtol=1e-3, krylov_atol=1e-14,
                              krylov_restart=40, krylov_maxit=600, precond="sweep", pseudo_dt=0.3,
                              jacobian="exact")
    for p in res_plans:
        solver.set_residual_plan(p)
    f = _blend([Ns[c] for c in choice], L, up, down)
    tf = torch.from_numpy(_flat(f)).to(DEV)
    hist = []
    for _ in range(24):
        st = solver.newton_step(tf)
        hist.append((st["residual_norm"], st["krylov_iterations"]))
        if st["residual_norm"] < 1e-10:
            break
    print("mixed shock:", [("%.1e" % r, k) for r, k in hist])
    assert hist[-1][0] < 1e-10
    assert np.isfinite(tf.cpu().numpy()).all()
