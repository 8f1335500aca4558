"""Pins of the oracle's spectral resampling between velocity grids of
different n (the mixed-n slab) and of its mixed-n slab residual."""
import numpy as np

from oracle import grid
from oracle.quadrature import hemisphere_rule
from oracle.resample import resample, resample_centred
from oracle.steady import MixedSlab, Slab


def test_padding_then_truncation_is_the_identity():
    rng = np.random.default_rng(0)
    for na, nb in ((16, 24), (24, 48), (16, 32)):
        f = rng.standard_normal((na, na, na))
        back = resample(resample(f, nb), na)
        assert np.abs(back - f).max() <= 1e-13 * np.abs(f).max()


def test_band_limited_polynomial_is_resampled_exactly():
    """A real trigonometric polynomial with modes |k| < 8 sampled on any grid
    n >= 16 is moved to any other such grid exactly (closed form)."""
    L = 5.0
    rng = np.random.default_rng(1)
    terms = [(rng.integers(-7, 8, 3), rng.standard_normal(), rng.uniform(0, 2 * np.pi)) for _ in range(12)]

    def sample(n):
        v = grid.velocity_grid(n, L)
        out = np.zeros((n, n, n))
        for k, amp, ph in terms:
            out += amp * np.cos(np.pi * (k[0] * v[0] + k[1] * v[1] + k[2] * v[2]) / L + ph)
        return out
    for na, nb in ((16, 24), (24, 16), (32, 48), (48, 16)):
        got = resample(sample(na), nb)
        assert np.abs(got - sample(nb)).max() <= 1e-12 * np.abs(sample(nb)).max()


def test_maxwellian_moves_between_grids_to_spectral_accuracy():
    L = 8.0

    def maxwell(n):
        a = (np.arange(n) - n // 2) * grid.spacing(n, L)
        return (2 * np.pi * 1.3) ** -1.5 * np.exp(
            -((a[:, None, None] - 0.7) ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2) / 2.6)
    for na, nb in ((24, 48), (48, 24), (32, 24)):
        err = np.abs(resample_centred(maxwell(na), nb) - maxwell(nb)).max() / maxwell(nb).max()
        assert err < 1e-6


def test_mixed_slab_with_one_n_is_the_uniform_slab():
    """With every cell on the same grid the mixed slab's residual is the
    uniform slab's (no resampling happens)."""
    up, down = (1.0, 1.2, 0.0, 0.0, 1.0), (1.4, 0.85, 0.0, 0.0, 1.25)
    hemi = hemisphere_rule(1)
    a = (np.arange(8) - 4) * grid.spacing(8, 6.0)
    f = np.stack([(1.0 + 0.1 * j) * (2 * np.pi) ** -1.5 * np.exp(
        -((a[:, None, None] - 0.9 + 0.1 * j) ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2) / 2)
        for j in range(3)])
    uni = Slab(8, 6.0, 0.5, 8, nx=3, kn=0.4, hemisphere=hemi, inflow_left=up, inflow_right=down)
    mix = MixedSlab([8, 8, 8], 6.0, 0.5, kn=0.4, hemisphere=hemi, inflow_left=up, inflow_right=down)
    r_uni, r_mix = uni.residual(f), mix.residual(list(f))
    assert max(np.abs(x - y).max() for x, y in zip(r_uni, r_mix)) <= 1e-14 * np.abs(r_uni).max()
    assert abs(uni.norm(r_uni) - mix.norm(r_mix)) <= 1e-14 * uni.norm(r_uni)
