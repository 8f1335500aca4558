"""The accuracy reading for noisy inputs (Sec. 3.3: FFT evaluations of the
gain term lose accuracy in proportion to max|r|, r = g/M) checked against an
extended-precision reference: the oracle's direct sums compiled with long
double (oracle/direct_ld.c).  The direct sums do not amplify the rounding
of r the way the FFT form does, so they and the extended sums agree to
~1e-14, while the FFT form sits within u max|r| of them."""
import os

import numpy as np

from oracle import grid
from oracle.direct import direct_linearized
from oracle.linearized import Tables, collision_operator
from paper_2503_09580_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "noisy_n16_extended.txt")


def load_extended_golden():
    """(max |L[g]|, max |g/M| kept by the cut-off, [(centred flat index, value)])"""
    vals, meta = [], {}
    for line in open(GOLDEN):
        if line.startswith("#"):
            continue
        a, b = line.split()
        if a in ("max_abs", "max_ratio"):
            meta[a] = float(b)
        else:
            vals.append((int(a), float(b)))
    return meta["max_abs"], meta["max_ratio"], vals


def test_extended_and_double_direct_sums_agree_without_noise():
    params, g = workloads.batched_instances(8, 8.0, batch=2, seed=3, noise=0.0)
    tab = Tables(8, 8.0, 0.5, 8)
    for p, x in zip(params, g):
        xc = grid.to_cyclic(x)
        ext = direct_linearized(tab, p[0], p[1:4], p[4], xc, extended=True)
        dbl = direct_linearized(tab, p[0], p[1:4], p[4], xc)
        fft = collision_operator(tab, p[0], p[1:4], p[4], xc)
        scale = np.abs(ext).max()
        assert np.abs(dbl - ext).max() <= 1e-14 * scale
        assert np.abs(fft - ext).max() <= 1e-12 * scale  # r = p, a random quartic: max|r| ~ 1e3


def test_fft_oracle_within_u_max_r_of_the_extended_reference():
    """Noisy N = 16 instance (benchmark recipe): the numpy FFT form of
    Algorithm 1 is within u64 max|r| of the extended-precision values, the
    FP64 direct sums within 1e-13."""
    max_abs, max_ratio, vals = load_extended_golden()
    params, g = workloads.batched_instances(16, 8.0, batch=1, seed=31, noise=1e-3)
    p = params[0]
    tab = Tables(16, 8.0, 0.5, 16)
    fft = grid.to_centred(collision_operator(tab, p[0], p[1:4], p[4], grid.to_cyclic(g[0]))).ravel()
    idx = np.array([i for i, _ in vals])
    ref = np.array([v for _, v in vals])
    assert np.abs(fft).max() == np.abs(fft[idx[0]]) or abs(np.abs(fft).max() - max_abs) <= 1e-10 * max_abs
    err = np.abs(fft[idx] - ref).max() / max_abs
    assert err <= 2.0 ** -53 * max_ratio
    assert err > 1e-14  # the amplification is visible: the FFT form is not at FP64 rounding here


def test_rk4_is_fourth_order_on_a_linear_system():
    """The oracle's RK4 (Sec. 4.2's scheme) on dy/dt = A y against exp(A t):
    the error falls by ~2^4 when dt halves."""
    import scipy.linalg
    from oracle.evolve import rk4
    rng = np.random.default_rng(3)
    A = rng.standard_normal((6, 6))
    A = A - A.T - 0.5 * np.eye(6)  # stable
    y0 = rng.standard_normal(6)
    exact = scipy.linalg.expm(A) @ y0
    e = [np.abs(rk4(lambda y: A @ y, y0, 1.0 / k, k) - exact).max() for k in (20, 40)]
    assert 14.0 < e[0] / e[1] < 18.0
