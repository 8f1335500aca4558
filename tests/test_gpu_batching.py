"""Mixed-N batches through plan groups (own streams, CUDA-graph replay) and
the launch-shape autotuner."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.linearized import Tables, apply_linearized
from paper_2503_09580_gb300 import lbo, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _inputs(sizes, batches, seed, L=8.0):
    ps, gs = [], []
    for i, (n, b) in enumerate(zip(sizes, batches)):
        p, g = workloads.batched_instances(n, L, batch=b, seed=seed + i, noise=1e-4)
        ps.append(torch.from_numpy(p).to(DEV))
        gs.append(torch.from_numpy(g).to(DEV))
    return ps, gs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_group_matches_members_and_graph_replays(precision):
    sizes, batches, L = (24, 32, 48), (5, 4, 2), 8.0
    # FP64 at N = 32 with the 8-plane tile of the register plane kernel (the
    # shape with more than 48 KB of shared memory) inside the captured graph
    plans = [lbo.Plan(n, L, 0.5, n, precision=precision, **({"planes": 8} if precision == "fp64" and n == 32 else {}))
             for n in sizes]
    ps, gs = _inputs(sizes, batches, seed=50)
    ref = []
    for p, tp, tg in zip(plans, ps, gs):
        o = torch.empty_like(tg)
        p.apply_linearized(tp, tg, o)
        ref.append(o)
    torch.cuda.synchronize()
    for graph in (False, True):
        grp = lbo.Group(plans, graph=graph)
        outs = [torch.full_like(g, float("nan")) for g in gs]
        for _ in range(3):  # eager, capture + launch, replay
            grp.apply_linearized(ps, gs, outs)
            torch.cuda.synchronize()
            for o, r in zip(outs, ref):
                assert torch.equal(o, r)
        # replay reads the arrays' current contents
        for g in gs:
            g.mul_(0.5)
        grp.apply_linearized(ps, gs, outs)
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert torch.allclose(o, 0.5 * r, rtol=1e-6 if precision == "fp32" else 1e-12, atol=0)
        for g in gs:
            g.mul_(2.0)
        grp.close()


def test_autotune_picks_a_shape_and_keeps_results():
    n, L = 32, 8.0
    params, g = workloads.batched_instances(n, L, batch=64, seed=60, noise=0.0)
    plan = lbo.Plan(n, L, 0.5, n, precision="fp32")
    tp, tg = torch.from_numpy(params).to(DEV), torch.from_numpy(g).to(DEV)
    out = torch.empty_like(tg)
    choice = plan.autotune(tp, tg, out)
    assert choice in (1, 2, 3, 4, 6, 8)
    plan.apply_linearized(tp, tg, out)
    torch.cuda.synchronize()
    ref = apply_linearized(Tables(n, L, 0.5, n), params[:2], g[:2])
    got = out.cpu().numpy()[:2]
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    # FP64 at N = 32: planes per CTA of the register plane kernel; results
    # do not depend on the shape
    plan64 = lbo.Plan(n, L, 0.5, n)
    plan64.apply_linearized(tp, tg, out)
    torch.cuda.synchronize()
    ref64 = out.cpu().numpy()
    assert plan64.autotune(tp, tg, out) in (2, 4, 8)
    plan64.apply_linearized(tp, tg, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref64)
    # nothing to tune on the generic kernels at another N
    p16, g16 = workloads.batched_instances(16, L, batch=4, seed=61, noise=0.0)
    t16, s16 = torch.from_numpy(p16).to(DEV), torch.from_numpy(g16).to(DEV)
    assert lbo.Plan(16, L, 0.5, 16).autotune(t16, s16, torch.empty_like(s16)) == 0
