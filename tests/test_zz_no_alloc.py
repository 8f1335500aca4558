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


@pytest.mark.parametrize("n,precision", [(16, "fp64"), (24, "fp64"), (32, "fp64"), (32, "fp32"), (64, "fp64")])
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
        launches = plan.last_launches
        plan.apply_linearized_noalloc(tp, tg, got)
        torch.cuda.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
        assert plan.last_launches == launches  # the same launch sequence
    plan.close()


def test_noalloc_allocates_nothing_on_a_fresh_plan():
    """On a plan that has never run the regular entry point (so it owns no
    workspace), the call leaves the device's free memory unchanged.  A
    first call on another plan of the same N loads the library's kernels and
    its static array beforehand, so that their one-time loading is not
    counted."""
    n, L = 16, 8.0
    params, g = workloads.batched_instances(n, L, batch=4, seed=23, noise=1e-4)
    tp, tg = _to_dev(params, g)
    out = torch.empty_like(tg)
    warm = lbo.Plan(n, L, 0.5, n)
    warm.apply_linearized_noalloc(tp, tg, out)
    torch.cuda.synchronize()
    fresh = lbo.Plan(n, L, 0.5, n)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    fresh.apply_linearized_noalloc(tp, tg, out)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before
    ref = torch.empty_like(tg)
    warm.set("kernel", 1)
    warm.apply_linearized(tp, tg, ref)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref.cpu().numpy()).max() <= 1e-12 * np.abs(ref.cpu().numpy()).max()
    warm.close()
    fresh.close()


def test_noalloc_rejects_fix_options_and_stale_tables():
    n, L = 16, 8.0
    params, g = workloads.batched_instances(n, L, batch=1, seed=24, noise=0.0)
    tp, tg = _to_dev(params, g)
    out = torch.empty_like(tg)
    plan = lbo.Plan(n, L, 0.5, n, mass_fix=1)
    with pytest.raises(lbo.LboError) as ei:
        plan.apply_linearized_noalloc(tp, tg, out)
    assert ei.value.status == 7  # LBO_EUNSUPPORTED
    plan.close()
    plan = lbo.Plan(n, L, 0.5, n)
    plan.set("R", 5.0)  # the tables are rebuilt at the next regular call only
    with pytest.raises(lbo.LboError) as ei:
        plan.apply_linearized_noalloc(tp, tg, out)
    assert ei.value.status == 1  # LBO_EINVAL
    assert "out of date" in str(ei.value)
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
