"""The M-point Fourier spectral quadratic collision operator, Eq. (2.14)
(Sec. 2.3), and its symmetric bilinear form Q(f,g) + Q(g,f).
Oracle: test infrastructure only.

With F = DFT(f) (standard n-point DFT, cyclic order), h = 2L/n and the
hemisphere rule normalised to sum_m w_m = 1, Eq. (2.14) in point values is

  Q+ = 16 pi^2 IDFT[ sum_{j,m} w_j w_m B(g_j) s_{j,k} DFT(A_c^2 - B_s^2) ]
  Q- = f * IDFT(F omega)

where A_c = IDFT(F cos(alpha.k)), A_s = IDFT(F sin(alpha.k)) = i B_s and
alpha = pi g_j sigma_m / (2L).  (The constant: 2 pi^2/L^3 of Eq. (2.14) times
h^6 n^3 from f^ = h^3 F, times (2L)^{-3} n^3 of the point-value synthesis.)
The sum cos.cos + sin.sin of I_{j,k,m} becomes A_c^2 + A_s^2 = A_c^2 - B_s^2
because a product in real space is a cyclic convolution in k.

Reading at the Nyquist planes: with the c_k weights of Sec. 2.3, a
non-even multiplier exp(i alpha_d k_d) at k_d = -N_p is the average over its
two images +-N_p, i.e. cos(alpha_d N_p).  This keeps cos(alpha.k) even and
sin(alpha.k) odd, so A_c and B_s are real.
"""
import numpy as np

from . import grid
from .linearized import FFT, InvFFT, sinc


def phase_multiplier(n, alpha):
    """E(k) = prod_d m_d(k_d) with m_d(k) = exp(i alpha_d k) for k != -N_p and
    cos(alpha_d N_p) at the Nyquist index (cyclic order)."""
    k = grid.centred_index(n).astype(np.float64)
    nyq = k == -(n // 2)
    facs = []
    for d in range(3):
        m = np.exp(1j * alpha[d] * k)
        m[nyq] = np.cos(alpha[d] * (n // 2))
        facs.append(m)
    return facs[0][:, None, None] * facs[1][None, :, None] * facs[2][None, None, :]


def _gain_pair_product(Ff, Fg, E):
    """A^f_c A^g_c - B^f_s B^g_s for one (j, m)."""
    c, s = np.real(E), np.imag(E)
    Acf = np.real(InvFFT(Ff * c))
    Bsf = np.imag(InvFFT(Ff * s))
    if Fg is Ff:
        return Acf * Acf - Bsf * Bsf
    Acg = np.real(InvFFT(Fg * c))
    Bsg = np.imag(InvFFT(Fg * s))
    return Acf * Acg - Bsf * Bsg


def loss_multiplier(tab, sig=None, wm=None, sinc_quadrature=False):
    """omega_k of Algorithm 1, or -- for the second mass fix of Sec. 2.3,
    Eq. (2.16) -- the same with sinc(pi g_j |k| / L) replaced by its M-point
    hemisphere quadrature sum_m w_m cos(pi g_j sigma_m . k / L).

    Reading at the Nyquist planes: Eq. (2.16) is there to make the bracket of
    Eq. (2.15) vanish, i.e. to give the loss term at k = 0 the gain's own
    kernel.  With the gain's per-axis factor E_d(k) = exp(i alpha_d k) and
    cos(alpha_d N_p) at the Nyquist index (alpha = pi g_j sigma_m / (2L)),
    that kernel is Re prod_d E_d(k_d)^2: cos(pi g_j sigma_m . k / L) away
    from the Nyquist planes and cos^2(alpha_d N_p) on them."""
    if not sinc_quadrature:
        return tab.omega
    om = np.zeros((tab.n,) * 3)
    for j in range(tab.J):
        acc = np.zeros((tab.n,) * 3)
        for m in range(len(wm)):
            acc += wm[m] * np.real(phase_multiplier(tab.n, np.pi * tab.g[j] * sig[m] / (2.0 * tab.L)) ** 2)
        om += tab.w[j] * tab.B[j] * acc
    return 16.0 * np.pi ** 2 * om


def quadratic_operator(tab, f, sig, wm, g=None, mass_fix=None, return_parts=False):
    """Q(f, f) by Eq. (2.14) on the cyclic grid; with ``g`` given, the
    symmetric bilinear form Q(f, g) + Q(g, f) (so that Q(M, g) + Q(g, M) is
    the M-point form of L[g], Sec. 4.1).

    mass_fix: None, 'zero_mode' (set Q^_0 = 0) or 'sinc_quadrature'
    (Eq. 2.16), the two fixes listed at the end of Sec. 2.3."""
    n, L = tab.n, tab.L
    f = np.asarray(f, dtype=np.float64)
    Ff = FFT(f)
    bil = g is not None
    if bil:
        g = np.asarray(g, dtype=np.float64)
        Fg = FFT(g)
    Qhat = np.zeros((n, n, n), dtype=np.complex128)
    for j in range(tab.J):
        for m in range(len(wm)):
            alpha = np.pi * tab.g[j] * sig[m] / (2.0 * L)
            E = phase_multiplier(n, alpha)
            if bil:
                P = 2.0 * _gain_pair_product(Ff, Fg, E)
            else:
                P = _gain_pair_product(Ff, Ff, E)
            Qhat += (tab.w[j] * wm[m] * tab.B[j]) * tab.s[j] * FFT(P)
    Qplus = 16.0 * np.pi ** 2 * np.real(InvFFT(Qhat))
    om = loss_multiplier(tab, sig, wm, sinc_quadrature=(mass_fix == "sinc_quadrature"))
    if bil:
        Qminus = f * np.real(InvFFT(Fg * om)) + g * np.real(InvFFT(Ff * om))
    else:
        Qminus = f * np.real(InvFFT(Ff * om))
    out = Qplus - Qminus
    if mass_fix == "zero_mode":
        out = out - out.mean()
    if return_parts:
        return out, Qplus, Qminus
    return out


def apply_quadratic(tab, f, sig, wm, mass_fix=None):
    """Batched Q(f,f) in the library's layout: f (B, n, n, n) centred."""
    f = np.asarray(f, dtype=np.float64).reshape(-1, tab.n, tab.n, tab.n)
    out = np.empty_like(f)
    for b in range(f.shape[0]):
        out[b] = grid.to_centred(quadratic_operator(tab, grid.to_cyclic(f[b]), sig, wm,
                                                    mass_fix=mass_fix))
    return out
