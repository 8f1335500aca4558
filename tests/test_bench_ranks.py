"""Host-side logic of bench.py's multi-rank run (one process per GPU under
torchrun), exercised with world_size 2 on the gloo backend on CPU: the
max-over-ranks timing, the barrier, per-rank instance sharding (each rank
applies L to its own batch; no data-path collective) and the reference arm
running on rank 0 only."""
import importlib.util
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    bench = _load_bench()
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(backend="gloo")
    bench.barrier(w)
    ms = bench.max_over_ranks(1.0 + 2.0 * r, w)  # this rank's step time
    from paper_2503_09580_gb300 import workloads
    params, g = workloads.batched_instances(16, 8.0, batch=2, seed=7 + r, noise=1e-3)
    # the reference arm prints on rank 0 only; other ranks return at once
    class Args:
        seed, omega, warmup, steps, ref_per_core, gpus = 0, 0.5, 0, 0, 1, w
    skipped = r != 0 and bench.run_reference(Args, w, r) is None
    out.put((r, w, ms, float(params[0, 0]), float(g.sum()), skipped))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, ms0, p0, g0, _), (r1, w1, ms1, p1, g1, skipped1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert ms0 == ms1 == 3.0          # max over ranks, seen by both
    assert p0 != p1 and g0 != g1      # each rank its own instances
    assert skipped1                   # reference arm: rank 1 does no work
    # value = all ranks' applications / max time (weak scaling)
    assert np.isclose(2 * 256 / (ms0 * 1e-3), 170666.66, rtol=1e-6)
