"""Spectral resampling of a velocity field between grids of different n on
the same box [-L, L)^3, as the upwind flux between neighbouring cells of
different n needs it (the mixed-n slab; a library extension -- the paper
uses one n everywhere).  Oracle only: test infrastructure.

Reading.  A field given on the n_a grid stands for its trigonometric
interpolant (the Fourier representation of Sec. 2.3), with the Nyquist term
taken as a cosine: its coefficient is split equally between the wavenumbers
+-n_a/2.
  * n_b > n_a (zero padding): the interpolant is sampled on the n_b grid.
  * n_b < n_a (truncation): the modes |k| > n_b/2 are dropped and the
    interpolant restricted to |k| <= n_b/2 is sampled on the n_b grid, where
    the wavenumbers +-n_b/2 coincide (their coefficients add).
Both grids contain v = 0 and share the period 2L, so the sampling is an
inverse DFT on the target grid.  Separable: applied axis by axis, numpy FFTs
as the library routine.  Arrays in cyclic order (see grid.py).
"""
import numpy as np

from . import grid


def resample_axis(x, n_b, axis):
    """Resample one axis of x (cyclic order) to n_b points."""
    n_a = x.shape[axis]
    if n_a == n_b:
        return np.array(x, dtype=np.float64, copy=True)
    X = np.moveaxis(np.fft.fft(np.asarray(x, dtype=np.float64), axis=axis), axis, 0) / n_a
    Y = np.zeros((n_b,) + X.shape[1:], dtype=np.complex128)
    if n_b > n_a:
        for k in range(-n_a // 2 + 1, n_a // 2):
            Y[k % n_b] = X[k % n_a]
        half = 0.5 * X[n_a // 2]  # the Nyquist cosine of the n_a grid
        Y[n_a // 2] += half
        Y[(-n_a // 2) % n_b] += half
    else:
        for k in range(-n_b // 2 + 1, n_b // 2):
            Y[k % n_b] = X[k % n_a]
        Y[n_b // 2] = X[(n_b // 2) % n_a] + X[(-n_b // 2) % n_a]
    y = np.fft.ifft(Y, axis=0) * n_b
    return np.moveaxis(y.real, 0, axis)


def resample(f, n_b):
    """Resample a 3-D field (cyclic order) to the n_b grid."""
    out = np.asarray(f, dtype=np.float64)
    for axis in range(3):
        out = resample_axis(out, n_b, axis)
    return out


def resample_centred(f, n_b):
    """Same for a field in the library's centred order."""
    return grid.to_centred(resample(grid.to_cyclic(f), n_b))
