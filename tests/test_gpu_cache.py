"""lbo_plan_cache_maxwellians: the Maxwellian-dependent factors of
Algorithm 1 (u^_j of every radial node, the loss factor InvFFT(FFT(M) omega))
computed once and reused by later applications with the same Maxwellians.
The cached path evaluates the same arithmetic in the same order, so its
result equals the uncached one; the cache is keyed by the params pointer,
the batch, the precision and the kernel set, and can be dropped."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_09580_gb300 import lbo, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def apply(plan, tp, tg):
    out = torch.empty_like(tg)
    plan.apply_linearized(tp, tg, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("n,precision", [(16, "fp64"), (32, "fp64"), (32, "fp32"), (24, "fp32"), (16, "fp32x2")])
def test_cached_application_equals_uncached(n, precision):
    L = 8.0
    params, g = workloads.batched_instances(n, L, batch=5, seed=51, noise=1e-3)
    _, g2 = workloads.batched_instances(n, L, batch=5, seed=52, noise=1e-3)
    tp = torch.from_numpy(params).to(DEV)
    tg, tg2 = torch.from_numpy(g).to(DEV), torch.from_numpy(g2).to(DEV)
    plan = lbo.Plan(n, L, 0.5, n, precision=precision)
    ref, ref2 = apply(plan, tp, tg), apply(plan, tp, tg2)
    launches_plain = plan.last_launches
    plan.cache_maxwellians(tp)
    got, got2 = apply(plan, tp, tg), apply(plan, tp, tg2)  # two products with the same Maxwellians
    assert plan.last_launches < launches_plain
    scale = np.abs(ref).max()
    print("%s n=%d: cached vs uncached max diff %.3e (bitwise: %s)"
          % (precision, n, np.abs(got - ref).max() / scale, np.array_equal(got, ref)))
    assert np.abs(got - ref).max() <= 1e-14 * scale
    assert np.abs(got2 - ref2).max() <= 1e-14 * np.abs(ref2).max()
    plan.close()


def test_cache_is_keyed_by_params_and_can_be_dropped():
    n, L = 16, 8.0
    pa, g = workloads.batched_instances(n, L, batch=3, seed=53, noise=0.0)
    pb, _ = workloads.batched_instances(n, L, batch=3, seed=54, noise=0.0)
    tpa, tpb, tg = (torch.from_numpy(x).to(DEV) for x in (pa, pb, g))
    plan = lbo.Plan(n, L, 1.0, n)
    ref_b = apply(plan, tpb, tg)
    plan.cache_maxwellians(tpa)
    # other Maxwellians: the cache is not used
    assert np.array_equal(apply(plan, tpb, tg), ref_b)
    # the same pointer with other contents is the caller's error; after a drop
    # the plan computes everything again
    tpa.copy_(tpb)
    plan.cache_maxwellians(None)
    assert np.array_equal(apply(plan, tpa, tg), ref_b)
    # a smaller batch of the same pointer does not use the cache either
    plan.cache_maxwellians(tpa)
    assert np.array_equal(apply(plan, tpa[:2], tg[:2]), ref_b[:2])
    plan.close()
