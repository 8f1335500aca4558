"""Host logic of the partitioned slab solver (distributed.py) on CPU: the
cell partition; a single rank's residual against the discrete equations of
the supplement written out; its FGMRES solve against a dense solve of the
same bordered system; and world sizes 2 and 3 on gloo (each rank one block
of cells, halo exchange, sums over ranks, sweep chained across the blocks)
reproducing the single-rank Newton steps.  The per-block operations come
from the numpy stand-in (slab_standin.py)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from paper_2503_09580_gb300 import distributed as D  # noqa: E402
from slab_standin import NumpyBlock  # noqa: E402

BOX = 4.0


def _problem(**kw):
    p = dict(nx=7, x_left=-0.5, x_right=0.5, kn=0.5, wall_left=(1.0, 0.0, -0.2, 0.0),
             wall_right=(1.3, 0.0, 0.2, 0.0), total_mass=1.0, wall_flux="discrete", krylov_rtol=1e-10,
             krylov_atol=1e-13, krylov_restart=6, krylov_maxit=400, precond="sweep")
    p.update(kw)
    return p


def _initial_state(N, nx, seed=3):
    """Cells of a temperature ramp between the walls, slightly perturbed."""
    b = NumpyBlock(N, BOX)
    rng = np.random.default_rng(seed)
    cells = []
    for j in range(nx):
        th = 1.0 + 0.3 * (j + 0.5) / nx
        m = b.maxwellian(1.0, (0.0, 0.05 * np.sin(j), 0.0), th)
        cells.append(m * (1 + 0.05 * rng.standard_normal(b.n3)))
    return np.concatenate(cells)


def test_partition_blocks():
    assert D.partition(7, 3) == [(0, 3), (3, 2), (5, 2)]
    assert D.partition(8, 2) == [(0, 4), (4, 4)]
    assert D.partition(5, 1) == [(0, 5)]
    for nx, w in ((200, 8), (513, 7), (9, 9)):
        parts = D.partition(nx, w)
        assert parts[0][0] == 0 and sum(n for _, n in parts) == nx
        assert all(a + n == b for (a, n), (b, _) in zip(parts, parts[1:]))
        assert max(n for _, n in parts) - min(n for _, n in parts) <= 1
    with pytest.raises(ValueError):
        D.partition(3, 4)


def _reference_residual(b, f, pb):
    """T f - Q(f)/Kn from the upwind scheme of the supplement, ghost cells
    sigma W with sigma from the outgoing flux of the boundary cells."""
    nx, n3, h3 = pb["nx"], b.n3, b.h ** 3
    dx = (pb["x_right"] - pb["x_left"]) / nx
    F = f.reshape(nx, n3)
    WL = b.maxwellian(1.0, pb["wall_left"][1:], pb["wall_left"][0])
    WR = b.maxwellian(1.0, pb["wall_right"][1:], pb["wall_right"][0])
    kL = 1.0 / (h3 * (np.maximum(b.v1, 0) @ WL))
    kR = 1.0 / (h3 * (-np.minimum(b.v1, 0) @ WR))
    g0 = -kL * h3 * (np.minimum(b.v1, 0) @ F[0]) * WL
    g1 = kR * h3 * (np.maximum(b.v1, 0) @ F[-1]) * WR
    ext = np.vstack([g0, F, g1])
    out = np.empty_like(F)
    for j in range(nx):
        rho, u, th = b.cell_moments(F[j])
        q = rho * (b.project(b.maxwellian(rho, u, th), F[j]) - F[j])
        tv = np.where(b.v1 > 0, b.v1 * (ext[j + 1] - ext[j]), b.v1 * (ext[j + 2] - ext[j + 1])) / dx
        out[j] = tv - q / pb["kn"]
    return out.ravel()


def test_single_rank_residual_matches_the_discrete_equations():
    N, pb = 6, _problem()
    b = NumpyBlock(N, BOX)
    f0 = _initial_state(N, pb["nx"])
    slab = D.DistributedSlab(b, D.Comm(), **pb)
    out = torch.zeros(len(f0), dtype=torch.float64)
    rn = slab.residual(torch.from_numpy(f0.copy()), out)
    ref = _reference_residual(b, f0, pb)
    assert np.allclose(out.numpy(), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert np.isclose(rn, np.sqrt(slab.wnorm * (ref @ ref)), rtol=1e-13)
    # the stand-in collision conserves the five discrete moments
    q = torch.zeros_like(out)
    b.quadratic(torch.from_numpy(f0.copy()), pb["nx"], q)
    assert np.abs(b.phi @ q.numpy().reshape(pb["nx"], -1).T).max() < 1e-12


@pytest.mark.parametrize("precond,restart", [("sweep", 6), ("none", 200)])
def test_single_rank_fgmres_matches_dense_solve(precond, restart):
    N, pb = 6, _problem(nx=5, precond=precond, krylov_restart=restart, krylov_maxit=800, pseudo_dt=0.0)
    b = NumpyBlock(N, BOX)
    f0 = _initial_state(N, pb["nx"])
    slab = D.DistributedSlab(b, D.Comm(), **pb)
    ns = {"krylov_iterations": 0, "restarts": 0, "status": "ok"}
    slab.prepare(torch.from_numpy(f0.copy()), ns)
    n = slab.len
    A = np.empty((n, n))
    e = torch.zeros(n, dtype=torch.float64)
    col = torch.zeros(n, dtype=torch.float64)
    for i in range(n):
        e.zero_()
        e[i] = 1.0
        slab.apply_op(e, col)
        A[:, i] = col.numpy()
    x = np.linalg.solve(A, slab.rhs.numpy())
    slab.fgmres(ns)
    assert ns["status"] == "ok"
    if precond == "sweep":
        assert ns["restarts"] > 0   # the restart path ran
    assert np.abs(slab.x.numpy() - x).max() <= 1e-8 * np.abs(x).max()
    # the bordered operator is nonsingular: the mass mode is fixed
    assert np.linalg.cond(A) < 1e12


def _run_steps(block, comm, f_block, pb, steps):
    slab = D.DistributedSlab(block, comm, **pb)
    f = torch.from_numpy(f_block.copy())
    stats = [slab.newton_step(f) for _ in range(steps)]
    return f.numpy(), stats


def _worker(rank, world, port, N, pb, steps, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = D.Comm()
        c0, n = D.partition(pb["nx"], world)[rank]
        b = NumpyBlock(N, BOX)
        f0 = _initial_state(N, pb["nx"])
        f, stats = _run_steps(b, comm, f0[c0 * b.n3:(c0 + n) * b.n3], pb, steps)
        out.put((rank, f, stats))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_reproduce_the_single_rank_newton_steps(world):
    N, steps = 6, 3
    pb = _problem(nx=7, krylov_rtol=1e-6, krylov_atol=1e-12, pseudo_dt=0.0)
    b = NumpyBlock(N, BOX)
    f0 = _initial_state(N, pb["nx"])
    f1, stats1 = _run_steps(b, D.Comm(), f0, pb, steps)
    # the Newton iteration converges on the stand-in (consistent discrete mass balance)
    assert stats1[-1]["residual_norm"] < 2e-3 * stats1[0]["residual_norm"]
    assert stats1[0]["restarts"] > 0
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, N, pb, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    fw = np.concatenate([r[1] for r in res])
    assert np.abs(fw - f1).max() <= 1e-11 * np.abs(f1).max()
    for rank_stats in (r[2] for r in res):
        for a, s in zip(rank_stats, stats1):
            assert a["krylov_iterations"] == s["krylov_iterations"]
            assert a["restarts"] == s["restarts"]
            assert np.isclose(a["residual_norm"], s["residual_norm"], rtol=1e-10)
