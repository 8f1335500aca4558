"""Collocation grid and cyclic multi-indices (Sec. 2.3).  Oracle only.

The paper's grid is v_l = l L / N_p with l = -N_p .. N_p-1 in each direction
(n = 2 N_p points), multi-indices cyclic modulo n.  The oracle stores every
array in *cyclic* order (index c = l mod n), which makes the paper's FFT and
InvFFT (Algorithm 1, with the c_k reading below) exactly numpy's fftn/ifftn.
The library's layout is *centred* order (index i = l + N_p); ``to_cyclic`` /
``to_centred`` convert between the two.
"""
import numpy as np


def centred_index(n):
    """Representative l in {-N_p, .., N_p-1} of each cyclic index 0..n-1."""
    c = np.arange(n)
    return np.where(c < n // 2, c, c - n)


def spacing(n, L):
    """Grid spacing h = L / N_p = 2L/n."""
    return 2.0 * L / n


def velocity_axes(n, L):
    """1-D velocity values in cyclic order."""
    return centred_index(n) * spacing(n, L)


def velocity_grid(n, L):
    """(v1, v2, v3) broadcastable arrays of shape (n,1,1), (1,n,1), (1,1,n),
    cyclic order."""
    a = velocity_axes(n, L)
    return a[:, None, None], a[None, :, None], a[None, None, :]


def wavenumber_norm(n):
    """|k| for the cyclic frequency grid.  The Nyquist index n/2 maps to
    k = -N_p; multipliers used here depend on |k| only, so the sign does
    not matter."""
    k = centred_index(n).astype(np.float64)
    return np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)


def to_cyclic(x):
    """Centred -> cyclic order on the last three axes."""
    return np.fft.ifftshift(x, axes=(-3, -2, -1))


def to_centred(x):
    """Cyclic -> centred order on the last three axes."""
    return np.fft.fftshift(x, axes=(-3, -2, -1))
