"""Learned preconditioner: hand-written GPU backward pass against the CPU
oracle of the network, training on solver-generated pairs, and the safety
property (the exact operator measures convergence; a poor network costs
iterations only).  The measured gain over the plain sweep is printed; it is
negative: an error dc in a cell's predicted coefficients reaches the
residual through the transport of the lifted correction, amplified by about
|v1|max / dx, so even a well-fitted network leaves a larger residual than
the sweep alone; the fallback keeps the solve exact."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.network import loss_and_grad, param_count
from oracle.quadrature import hemisphere_rule
from oracle.steady import Slab, initial_state
from paper_2503_09580_gb300 import lbo

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_network_gradient_matches_oracle():
    rng = np.random.default_rng(0)
    for H, P, nx in ((8, 4, 12), (32, 3, 40)):
        theta = (0.3 * rng.standard_normal(param_count(H))).astype(np.float32)
        x = rng.standard_normal((P, nx, 26)).astype(np.float32)
        t = rng.standard_normal((P, nx, 5)).astype(np.float32)
        l_ref, g_ref = loss_and_grad(theta.astype(np.float64), H, x.astype(np.float64), t.astype(np.float64))
        l, g = lbo.network_loss_grad(H, torch.from_numpy(theta).to(DEV), torch.from_numpy(x).to(DEV),
                                     torch.from_numpy(t).to(DEV))
        g = g.cpu().numpy()
        assert abs(l - l_ref) <= 1e-5 * l_ref
        assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()


def test_learned_preconditioner_trains_and_keeps_the_solve_exact():
    n, L, nx, kn = 32, 8.0, 16, 0.1
    orc = Slab(n, L, 1.0, n, nx=nx, kn=kn, hemisphere=hemisphere_rule(2), wall_flux="discrete")
    f0 = initial_state(orc)
    C = orc.mass(f0)

    def make(prec):
        plan = lbo.Plan(n, L, 1.0, n, hemisphere_p=2, mass_fix=1)
        return plan, plan.solver(kind="slab", nx=nx, kn=kn, wall_left=(1.0, 0, 0, 0), wall_right=(2.0, 0, 0, 0),
                                 total_mass=C, wall_flux="discrete", krylov_rtol=1e-4, krylov_atol=1e-10,
                                 krylov_restart=40, krylov_maxit=400, precond=prec)

    def run(solver):
        f = torch.from_numpy(f0.copy()).to(DEV)
        its, ms = 0, 0.0
        for _ in range(12):
            st = solver.newton_step(f)
            its += st["krylov_iterations"]
            ms += st["ms_linear"]
            if st["residual_norm"] < 3e-7:
                break
        out = torch.empty_like(f)
        return f.cpu().numpy(), solver.residual(f, out), its, ms

    planA, A = make("sweep")
    A.collect(2000)
    fa, ra, its_a, ms_a = run(A)
    assert A.pair_count > 50
    l_first = A.train_network(hidden=32, epochs=1, lr=3e-3, seed=1)
    l_final = A.train_network(hidden=32, epochs=800, lr=3e-3, seed=1)
    assert l_final < 0.8 * l_first
    planB, B = make("learned")
    B.set_network(*A.get_network())
    fb, rb, its_b, ms_b = run(B)
    print("sweep: %d Krylov iterations, %.0f ms; learned: %d iterations, %.0f ms; train loss %.3f -> %.3f"
          % (its_a, ms_a, its_b, ms_b, l_first, l_final))
    assert ra < 1e-6 and rb < 1e-6
    # both converge to the same discrete steady state (to the accuracy a
    # residual of 1e-6 fixes at Kn = 0.1, where the linearised operator is stiff)
    assert np.abs(fa - fb).max() <= 1e-3 * np.abs(fa).max()
