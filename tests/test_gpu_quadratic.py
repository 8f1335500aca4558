"""Parity of the CUDA quadratic operator Q(f,f) (M-point form, Eq. (2.14))
with the CPU oracle, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grid
from oracle.linearized import Tables
from oracle.quadratic import apply_quadratic
from oracle.quadrature import hemisphere_rule
from paper_2503_09580_gb300 import lbo, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def run_q(plan, f):
    tf = torch.from_numpy(f).to(DEV)
    out = torch.empty_like(tf)
    plan.apply_quadratic(tf, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def maxwell_batch(n, L, params):
    a = workloads.velocity_axis(n, L)
    out = []
    for rho, u1, u2, u3, th in params:
        d2 = (a[:, None, None] - u1) ** 2 + (a[None, :, None] - u2) ** 2 + (a[None, None, :] - u3) ** 2
        out.append(rho * (2 * np.pi * th) ** -1.5 * np.exp(-d2 / (2 * th)))
    return np.stack(out)


@pytest.mark.parametrize("n,p,omega", [(16, 4, 0.5), (16, 2, 1.0), (32, 1, 0.74)])
def test_quadratic_fp64_matches_oracle(n, p, omega):
    L = 8.0
    params, g = workloads.batched_instances(n, L, batch=2, seed=31, noise=0.0)
    f = maxwell_batch(n, L, params) + 0.3 * g
    plan = lbo.Plan(n, L, omega, n, hemisphere_p=p)
    got = run_q(plan, f)
    sig, w = hemisphere_rule(p)
    ref = apply_quadratic(Tables(n, L, omega, n), f, sig, w)
    assert relerr(got, ref) <= 1e-12


def test_quadratic_mass_fix_and_host_path():
    n, L = 16, 8.0
    params, g = workloads.batched_instances(n, L, batch=2, seed=32, noise=0.0)
    f = maxwell_batch(n, L, params) + 0.2 * g
    plan = lbo.Plan(n, L, 0.5, n, hemisphere_p=2, mass_fix=1)
    got = run_q(plan, f)
    sig, w = hemisphere_rule(2)
    ref = apply_quadratic(Tables(n, L, 0.5, n), f, sig, w, mass_fix="zero_mode")
    assert relerr(got, ref) <= 1e-12
    host = np.empty_like(f)
    plan.apply_quadratic(f, host)
    assert np.array_equal(host, got)


def test_quadratic_maxwellian_equilibrium_and_fp32():
    n, L = 32, 8.0
    params = np.array([[1.0, 0.2, 0.0, -0.1, 1.0], [1.5, -0.3, 0.1, 0.2, 0.8]])
    M = maxwell_batch(n, L, params)
    plan = lbo.Plan(n, L, 0.74, n, hemisphere_p=2)
    q = run_q(plan, M)
    for b in range(2):
        loss = params[b, 0] * M[b]  # scale of Q^- for this instance
        assert np.abs(q[b]).max() < 1e-5 * np.abs(loss).max()  # grid resolution at theta = 0.8
    plan32 = lbo.Plan(n, L, 0.74, n, hemisphere_p=2, precision="fp32")
    q32 = run_q(plan32, M)
    f = M + 0.1 * workloads.batched_instances(n, L, batch=2, seed=3, noise=0.0)[1]
    a, b = run_q(plan32, f), run_q(plan, f)
    assert relerr(a, b) <= 2.0 ** -24 * 64
    assert np.abs(q32).max() < 1e-5 * np.abs(M).max()


def test_quadratic_bkw_rate_on_gpu():
    """d f_BKW/dt = Q(f_BKW, f_BKW), Maxwell molecules, K = 1 - exp(-t/6)."""
    n, L, K = 32, 8.0, 0.8
    a = workloads.velocity_axis(n, L)
    v2 = a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2

    def bkw(K):
        return ((2 * np.pi * K) ** -1.5 * np.exp(-v2 / (2 * K))
                * ((5 * K - 3) / (2 * K) + (1 - K) / (2 * K * K) * v2))
    dK = 1e-5
    dfdt = (bkw(K + dK) - bkw(K - dK)) / (2 * dK) * (1 - K) / 6
    plan = lbo.Plan(n, L, 1.0, n, hemisphere_p=3)
    q = run_q(plan, bkw(K)[None])[0]
    assert np.abs(q - dfdt).max() < 2e-4 * np.abs(dfdt).max()


def test_quadratic_radix3_size():
    n, L = 24, 8.0
    params, g = workloads.batched_instances(n, L, batch=1, seed=33, noise=0.0)
    f = maxwell_batch(n, L, params) + 0.3 * g
    plan = lbo.Plan(n, L, 0.74, n, hemisphere_p=1)
    got = run_q(plan, f)
    sig, w = hemisphere_rule(1)
    ref = apply_quadratic(Tables(n, L, 0.74, n), f, sig, w)
    assert relerr(got, ref) <= 1e-12


@pytest.mark.parametrize("jgroups", [1, 3])
def test_fused_fp32_quadratic_n32(jgroups):
    """Fused FP32 Q at N = 32 (one block per instance and group of radial
    nodes) against the FP64 oracle and the generic FP32 kernels."""
    n, L, p = 32, 8.0, 2
    params, g = workloads.batched_instances(n, L, batch=3, seed=34, noise=0.0)
    f = maxwell_batch(n, L, params) + 0.3 * g
    fused = lbo.Plan(n, L, 0.5, n, hemisphere_p=p, precision="fp32", jgroups=jgroups)
    generic = lbo.Plan(n, L, 0.5, n, hemisphere_p=p, precision="fp32", kernel=1)
    a = run_q(fused, f)
    assert fused.last_launches == 3
    b = run_q(generic, f)
    sig, w = hemisphere_rule(p)
    ref = apply_quadratic(Tables(n, L, 0.5, n), f[:1], sig, w)
    print("fused Q fp32 vs oracle %.2e, vs generic fp32 %.2e" % (relerr(a[:1], ref), relerr(a, b)))
    assert relerr(a[:1], ref) <= 2.0 ** -24 * 64
    assert relerr(a, b) <= 2.0 ** -24 * 64


def test_quadratic_fp64_n32_p4_matches_oracle():
    """The hemisphere order the Newton and BKW workloads use (p = 4, M = 32
    points) at N = 32, generic FP64 kernels, one radial node per grid point."""
    n, L, p = 32, 8.0, 4
    params, g = workloads.batched_instances(n, L, batch=2, seed=33, noise=0.0)
    f = maxwell_batch(n, L, params) + 0.3 * g
    plan = lbo.Plan(n, L, 0.5, n, hemisphere_p=p)
    got = run_q(plan, f)
    sig, w = hemisphere_rule(p)
    ref = apply_quadratic(Tables(n, L, 0.5, n), f, sig, w)
    assert relerr(got, ref) <= 1e-12


def test_quadratic_fused_fp32_n32_p4_matches_oracle():
    """Fused FP32 Q (the default kernels for FP32 at N = 32) at p = 4 against
    the FP64 oracle.  Bound: 64 u32 normwise (transform rounding of the
    2 J M + J transforms, observed ~1e-6)."""
    n, L, p = 32, 8.0, 4
    params, g = workloads.batched_instances(n, L, batch=2, seed=34, noise=0.0)
    f = maxwell_batch(n, L, params) + 0.3 * g
    plan = lbo.Plan(n, L, 0.74, n, hemisphere_p=p, precision="fp32")
    got = run_q(plan, f)
    sig, w = hemisphere_rule(p)
    ref = apply_quadratic(Tables(n, L, 0.74, n), f, sig, w)
    assert relerr(got, ref) <= 64 * 2.0 ** -24


def test_quadratic_fp64_n64_bkw_configuration_matches_oracle():
    """The BKW workload's operator: N = 64, J = 64, Maxwell molecules,
    M = 32 hemisphere points, generic FP64 kernels, one instance (the numpy
    oracle takes about a minute here)."""
    n, L, p = 64, 8.0, 4
    params, g = workloads.batched_instances(n, L, batch=1, seed=35, noise=0.0)
    f = maxwell_batch(n, L, params) + 0.3 * g
    plan = lbo.Plan(n, L, 1.0, n, hemisphere_p=p)
    got = run_q(plan, f)
    sig, w = hemisphere_rule(p)
    ref = apply_quadratic(Tables(n, L, 1.0, n), f, sig, w)
    assert relerr(got, ref) <= 1e-12


@pytest.mark.parametrize("n,p,precision,tol", [(16, 2, "fp64", 1e-12), (32, 4, "fp64", 1e-12),
                                               (32, 2, "fp32", 64 * 2.0 ** -24), (16, 2, "fp32x2", 1e-12)])
def test_quadratic_sinc_quadrature_fix(n, p, precision, tol):
    """Eq. (2.16): Q with the hemisphere quadrature of the loss multiplier
    against the oracle, and its mass zero to rounding (Sec. 2.3)."""
    L = 8.0
    params, g = workloads.batched_instances(n, L, batch=2, seed=36, noise=0.0)
    f = maxwell_batch(n, L, params) + 0.3 * g
    plan = lbo.Plan(n, L, 0.5, n, hemisphere_p=p, precision=precision, q_sinc_quadrature=1)
    got = run_q(plan, f)
    sig, w = hemisphere_rule(p)
    ref = apply_quadratic(Tables(n, L, 0.5, n), f, sig, w, mass_fix="sinc_quadrature")
    assert relerr(got, ref) <= tol
    for b in range(2):
        assert abs(got[b].sum()) <= 64 * (2.0 ** -24 if precision == "fp32" else 2.0 ** -48) * np.abs(got[b]).sum()
    plain = run_q(lbo.Plan(n, L, 0.5, n, hemisphere_p=p, precision=precision), f)
    assert abs(plain[0].sum()) > 1e-7 * np.abs(plain[0]).sum()
