"""The slab-block primitives on the GPU (lbo_slab_block_*, lbo_vec_*)
against their definitions (the numpy restatements of slab_standin.py), and
the partitioned slab driver on one rank with the library's kernels against
the single-GPU solver (lbo_newton_step) on the same problem."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from slab_standin import NumpyBlock  # noqa: E402

pytestmark = pytest.mark.gpu


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2503_09580_gb300 import lbo
    return lbo


def _host(t):
    return t.cpu()


def test_block_primitives_match_their_definitions():
    lbo = _cuda()
    N, L, nx, dx, kn, shift = 16, 5.0, 5, 0.2, 0.7, 0.3
    plan = lbo.Plan(N, L, 1.0, 8)
    ref = NumpyBlock(N, L)
    n3 = N ** 3
    rng = np.random.default_rng(11)
    v = torch.from_numpy(rng.standard_normal(nx * n3))
    gl, gr = torch.from_numpy(rng.standard_normal(n3)), torch.from_numpy(rng.standard_normal(n3))
    nu = torch.from_numpy(rng.uniform(0.5, 1.5, nx))
    dv, dgl, dgr, dnu = v.cuda(), gl.cuda(), gr.cuda(), nu.cuda()
    # transport with both, one and no neighbour cells
    for a, b, ha, hb in ((dgl, dgr, gl, gr), (None, dgr, None, gr), (None, None, None, None)):
        out = torch.zeros_like(dv)
        plan.block_transport(dv, a, b, out, nx, dx)
        exp = torch.zeros_like(v)
        ref.transport(v, ha, hb, exp, nx, dx)
        assert np.abs(_host(out).numpy() - exp.numpy()).max() <= 1e-12 * np.abs(exp.numpy()).max()
    # sweep: both halves, then each half with incoming values
    for direction in (0, 1, -1):
        z = torch.zeros_like(dv)
        plan.block_sweep(dv, dnu, dgl, dgr, z, nx, dx, kn, shift, direction)
        exp = torch.zeros_like(v)
        ref.sweep(v, nu, gl, gr, exp, nx, dx, kn, shift, direction)
        assert np.abs(_host(z).numpy() - exp.numpy()).max() <= 1e-12 * np.abs(exp.numpy()).max()
    # moments, wall flux and Maxwellian cell
    th = np.array([0.8, 1.0, 1.3, 0.9, 1.1])
    f = np.concatenate([ref.maxwellian(1 + 0.1 * j, (0.1 * j, -0.2, 0.05), th[j]) for j in range(nx)])
    params = torch.zeros(5 * nx, dtype=torch.float64, device="cuda")
    dnu2 = torch.zeros(nx, dtype=torch.float64, device="cuda")
    plan.block_moments(torch.from_numpy(f).cuda(), nx, params, dnu2)
    P = _host(params).numpy().reshape(nx, 5)
    for j in range(nx):
        rho, u, t = ref.cell_moments(f[j * n3:(j + 1) * n3])
        assert np.allclose(P[j], [rho, *u, t], rtol=1e-12, atol=1e-13)
        assert np.isclose(_host(dnu2).numpy()[j], rho, rtol=1e-13)
    cell = torch.from_numpy(f[:n3]).cuda()
    for side in (0, 1):
        assert np.isclose(plan.cell_flux(cell, side), ref.cell_flux(torch.from_numpy(f[:n3]), side), rtol=1e-12)
    w = torch.zeros(n3, dtype=torch.float64, device="cuda")
    plan.maxwellian_cell(1.3, (0.0, 0.2, -0.1), 0.7, w)
    assert np.allclose(_host(w).numpy(), ref.maxwellian(0.7, (0.0, 0.2, -0.1), 1.3), rtol=1e-13, atol=1e-300)
    # dots, axpby, combination
    K, n = 7, nx * n3
    V = torch.from_numpy(rng.standard_normal((K, n)))
    y = torch.from_numpy(rng.standard_normal(n))
    dV, dy = V.cuda(), y.cuda()
    d = plan.vec_dots(dV, n, K, dy, n)
    assert np.allclose(d, V.numpy() @ y.numpy(), rtol=1e-12, atol=1e-10)
    c = rng.standard_normal(K)
    plan.vec_combination(dy, dV, n, K, c, n)
    assert np.allclose(_host(dy).numpy(), y.numpy() - c @ V.numpy(), rtol=1e-12, atol=1e-12)
    plan.vec_axpby(dy, dV[2], 0.5, -2.0, n)
    assert np.allclose(_host(dy).numpy(), 0.5 * V.numpy()[2] - 2.0 * (y.numpy() - c @ V.numpy()), rtol=1e-12,
                       atol=1e-12)
    plan.close()


def test_one_rank_driver_matches_the_single_gpu_solver():
    lbo = _cuda()
    from paper_2503_09580_gb300 import distributed as D
    N, nx, R = 16, 8, 3.5
    L = (3 + np.sqrt(2)) * R / 4
    pb = dict(nx=nx, x_left=-0.5, x_right=0.5, kn=1.0, wall_left=(1.0, 0.0, -0.1, 0.0),
              wall_right=(1.0, 0.0, 0.1, 0.0), total_mass=1.0, krylov_rtol=1e-8, krylov_atol=1e-12,
              krylov_restart=10, krylov_maxit=300, precond="sweep")
    plan = lbo.Plan(N, L, 1.0, 9, R=R, hemisphere_p=2)
    a = (np.arange(N) - N // 2) * (2 * L / N)
    v2 = a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2
    x = -0.5 + (np.arange(nx) + 0.5) / nx
    f0 = np.stack([(2 * np.pi * (1 + 0.1 * xi)) ** -1.5 * np.exp(-v2 / (2 * (1 + 0.1 * xi))) for xi in x])
    solver = plan.solver(kind="slab", **pb)
    fc = torch.from_numpy(f0.copy()).cuda()
    c_stats = [solver.newton_step(fc) for _ in range(2)]
    solver.close()
    slab = D.DistributedSlab(D.GpuBlock(plan), D.Comm(device="cuda"), **pb)
    fd = torch.from_numpy(f0.copy()).cuda().reshape(-1)
    d_stats = [slab.newton_step(fd) for _ in range(2)]
    torch.cuda.synchronize()
    for c, d in zip(c_stats, d_stats):
        assert d["krylov_iterations"] == c["krylov_iterations"]
        assert d["restarts"] == c["restarts"]
        assert np.isclose(d["residual_norm"], c["residual_norm"], rtol=1e-10)
    diff = (fd - fc.reshape(-1)).abs().max().item()
    assert diff <= 1e-10 * fc.abs().max().item()
    assert d_stats[1]["residual_norm"] < 0.2 * d_stats[0]["residual_norm"]
    plan.close()
