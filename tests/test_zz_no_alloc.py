"""lbo_apply_linearized_noalloc: the allocation-free variant of
lbo_apply_linearized, for callers that cannot allocate device memory when
they apply the operator (fixed memory budgets, real-time loops, hosts that
forbid allocation after start-up).  Its scratch is a static device array of
the library.  Checked through the C ABI against the regular entry point on
two calls in a row (the second with different inputs, so stale scratch
contents from the first call would show), plus the size limit.

The file name makes pytest collect it last, so a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_09580_gb300 import lbo, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _to_dev(params, g):
    return torch.from_numpy(params).to(DEV), torch.from_numpy(g).to(DEV)


@pytest.mark.parametrize("n,precision", [(16, "fp64"), (32, "fp64"), (32, "fp32")])
def test_noalloc_matches_regular_entry_point_twice(n, precision):
    L = 8.0
    # kernel=1: the regular entry point runs the same (generic) kernel set the
    # allocation-free variant runs, so the two must agree to rounding
    plan = lbo.Plan(n, L, 0.5, n, precision=precision, kernel=1)
    batch = min(6, plan.noalloc_max_batch())
    for seed in (21, 22):  # two calls in a row, different inputs
        params, g = workloads.batched_instances(n, L, batch=batch, seed=seed, noise=1e-4)
        tp, tg = _to_dev(params, g)
        ref = torch.empty_like(tg)
        got = torch.full_like(tg, float("nan"))
        plan.apply_linearized(tp, tg, ref)
        plan.apply_linearized_noalloc(tp, tg, got)
        torch.cuda.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    plan.close()


def test_noalloc_rejects_batch_above_static_scratch():
    n, L = 32, 8.0
    plan = lbo.Plan(n, L, 0.5, n)
    too_many = plan.noalloc_max_batch() + 1
    tp = torch.zeros((too_many, 5), dtype=torch.float64, device=DEV)
    tg = torch.zeros((too_many, n, n, n), dtype=torch.float64, device=DEV)
    out = torch.empty_like(tg)
    with pytest.raises(lbo.LboError) as ei:
        plan.apply_linearized_noalloc(tp, tg, out)
    assert ei.value.status == 1
    assert "static scratch" in str(ei.value)
    # host arrays are refused (staging them would allocate)
    params, g = workloads.batched_instances(n, L, batch=1, seed=3, noise=0.0)
    with pytest.raises(lbo.LboError):
        plan.apply_linearized_noalloc(params, g, np.empty_like(g))
    plan.close()
