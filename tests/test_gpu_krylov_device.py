"""FGMRES with the device-resident Arnoldi (problem.device_krylov = 1: the
Gram-Schmidt coefficients, norms, Givens rotations and the stopping test on
the GPU, each restart cycle a CUDA graph with a WHILE node) against the
host-side Arnoldi on the same Newton steps: equal Krylov counts, restarts
and statuses, states equal to rounding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_09580_gb300 import lbo

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _slab_state(n, L, nx):
    a = (np.arange(n) - n // 2) * (2 * L / n)
    v2 = a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2
    x = (np.arange(nx) + 0.5) / nx
    return np.stack([(2 * np.pi * (1 + xi)) ** -1.5 * np.exp(-v2 / (2 * (1 + xi))) for xi in x])


def _run(plan, f0, steps, f_prev=None, **kw):
    out = []
    for dk in (False, True):
        solver = plan.solver(device_krylov=dk, **kw)
        f = torch.from_numpy(f0.copy()).to(DEV)
        fp = None if f_prev is None else torch.from_numpy(f_prev.copy()).to(DEV)
        stats = [solver.newton_step(f, fp) for _ in range(steps)]
        torch.cuda.synchronize()
        out.append((f.cpu().numpy(), stats))
        solver.close()
    return out


def _same(host, dev, tol=1e-9):
    """Same iteration; the two differ only in the rounding of the Givens
    rotations (host and device hypot), which the Krylov process carries into
    the last digits of the solution."""
    (fh, sh), (fd, sd) = host, dev
    for a, b in zip(sh, sd):
        assert a["krylov_iterations"] == b["krylov_iterations"]
        assert a["restarts"] == b["restarts"]
        assert a["converged_inner"] == b["converged_inner"]
        assert abs(a["linear_residual"] - b["linear_residual"]) <= 1e-9 * a["rhs_norm"]
    assert np.abs(fh - fd).max() <= tol * np.abs(fh).max()


@pytest.mark.parametrize("precond,restart", [("sweep", 8), ("none", 30)])
def test_slab_device_arnoldi_equals_host(precond, restart):
    n, L, nx = 32, 6.0, 16
    plan = lbo.Plan(n, L, 1.0, 12, hemisphere_p=2)
    f0 = _slab_state(n, L, nx)
    h3 = (2 * L / n) ** 3
    C = h3 * f0.sum() / nx
    host, dev = _run(plan, f0, 2, kind="slab", nx=nx, x_left=0.0, x_right=1.0, kn=1.0,
                     wall_left=(1.0, 0, 0, 0), wall_right=(2.0, 0, 0, 0), total_mass=C, krylov_rtol=1e-6,
                     krylov_atol=1e-12, krylov_restart=restart, krylov_maxit=400, precond=precond)
    assert host[1][0]["restarts"] > 0 or precond == "none"
    _same(host, dev)
    plan.close()


def test_iteration_cap_and_fp32_operator():
    """The cap on the total iteration count ends a cycle in its middle (not
    converged, the step applied all the same), in FP32 as in FP64."""
    n, L, nx = 32, 6.0, 8
    for prec in ("fp64", "fp32"):
        plan = lbo.Plan(n, L, 1.0, 12, hemisphere_p=2, precision=prec)
        f0 = _slab_state(n, L, nx)
        C = (2 * L / n) ** 3 * f0.sum() / nx
        host, dev = _run(plan, f0, 1, kind="slab", nx=nx, x_left=0.0, x_right=1.0, kn=0.1,
                         wall_left=(1.0, 0, 0, 0), wall_right=(2.0, 0, 0, 0), total_mass=C, krylov_rtol=1e-12,
                         krylov_atol=0.0, krylov_restart=5, krylov_maxit=13, precond="sweep")
        assert not host[1][0]["converged_inner"] and host[1][0]["krylov_iterations"] == 13
        _same(host, dev)
        plan.close()


def test_homogeneous_backward_euler_device_arnoldi():
    n, L, dt = 32, 8.0, 0.05
    a = (np.arange(n) - n // 2) * (2 * L / n)
    v2 = a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2
    K = 0.6
    fn = ((2 * np.pi * K) ** -1.5 * np.exp(-v2 / (2 * K)) * ((5 * K - 3) / (2 * K) + (1 - K) / (2 * K * K) * v2))
    fn = np.stack([fn, 0.5 * fn])
    plan = lbo.Plan(n, L, 1.0, n, hemisphere_p=3)
    host, dev = _run(plan, fn, 3, f_prev=fn, kind="homogeneous", nx=2, dt=dt, krylov_rtol=1e-12,
                     krylov_atol=0.0, krylov_restart=30, krylov_maxit=200, precond="none")
    _same(host, dev)
    assert host[1][-1]["residual_norm"] < 1e-4 * host[1][0]["residual_norm"]
    plan.close()
