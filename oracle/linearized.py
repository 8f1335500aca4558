"""Algorithm 1 of the paper: the M-free Fourier spectral linearized collision
operator  L[g] = Q(M, g) + Q(g, M)  (Sec. 3, Eqs. (3.4)-(3.9)).
Oracle: test infrastructure only.

Readings of the paper taken here (each is pinned by a test):

* Gain constant.  Algorithm 1 prints phi_{j,k} = 32 pi^2 w_j B(g_j) s_{j,k}.
  Carrying Eqs. (3.5), (3.7), (3.8) through the FFT/InvFFT normalisations of
  Algorithm 1 gives 4 pi^2: InvFFT(FFT(u) FFT(r)) is the cyclic convolution
  u * r, which is psi / (8 pi^3), and the remaining factor h^3/(2 pi) cancels
  against the h^{-3} of the point-value synthesis.  With 4 pi^2, L[M] = 0 up
  to truncation; with 32 pi^2 the gain of L[M] is 8x its loss.
* FFT / InvFFT.  With cyclic multi-indices and the c_k weights, InvFFT(FFT(x))
  is the identity and both are the standard n-point DFT pair; the oracle
  stores arrays in cyclic order so they are numpy's fftn / ifftn.
* phi~_j = InvFFT(s_j) where s_j is given on k = -N..N.  ``nyquist='standard'``
  reads the k = +-N_p planes with the trapezoid weight 1/2 each (the c_k
  convention: phi~_j = IDFT of s_j on the n-point grid); ``'doubled'`` sums
  both planes with weight 1 as printed in Eq. (3.8).
* Cut-off, Eq. (3.9): r_l = 0 iff M_l / rho < eps, evaluated as
  |v_l - u|^2 / (2 theta) > ln(1/eps) - 1.5 ln(2 pi theta); the loss term uses
  the uncut g (Algorithm 1).
* M^ in the loss term is the numeric FFT of the sampled Maxwellian.
"""
import numpy as np

from . import grid
from .quadrature import radial_rule_kind, vhs_kernel


def sinc(x):
    """Unnormalised sinc, sin(x)/x with sinc(0) = 1 (Sec. 2.2)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x != 0.0
    out[nz] = np.sin(x[nz]) / x[nz]
    return out


def default_R(L):
    """Largest kernel cut-off allowed by the dealiasing rule L >= (3+sqrt2)R/4
    (Sec. 2.3)."""
    return 4.0 * L / (3.0 + np.sqrt(2.0))


class Tables:
    """Precomputation of Algorithm 1 (its first step): s_{j,k}, phi_{j,k},
    phi~_{j,k} = InvFFT(s_j) and omega_k, all in cyclic order."""

    def __init__(self, n, L, omega_vhs, J, R=None, C=1.0 / (4.0 * np.pi),
                 gain_const=4.0 * np.pi ** 2, nyquist="standard", radial="gl"):
        self.n, self.L, self.J = int(n), float(L), int(J)
        self.R = default_R(L) if R is None else float(R)
        self.omega_vhs, self.C = float(omega_vhs), float(C)
        self.g, self.w = radial_rule_kind(self.J, self.R, radial)
        self.B = vhs_kernel(self.g, self.omega_vhs, self.C)
        knorm = grid.wavenumber_norm(self.n)
        # s_{j,k} = sinc(pi g_j |k| / (2L))
        self.s = np.stack([sinc(np.pi * gj * knorm / (2.0 * self.L)) for gj in self.g])
        # phi_{j,k} = (gain constant) w_j B(g_j) s_{j,k}
        self.phi = (gain_const * self.w * self.B)[:, None, None, None] * self.s
        # phi~_j = InvFFT(s_j)
        if nyquist == "standard":
            sw = self.s
        elif nyquist == "doubled":
            nyq = (np.arange(self.n) == self.n // 2).astype(np.float64)
            mult = ((1.0 + nyq)[:, None, None] * (1.0 + nyq)[None, :, None]
                    * (1.0 + nyq)[None, None, :])
            sw = self.s * mult
        else:
            raise ValueError(nyquist)
        self.phit = np.real(np.fft.ifftn(sw, axes=(-3, -2, -1)))
        # omega_k = 16 pi^2 sum_j w_j B(g_j) sinc(pi g_j |k| / L)
        self.omega = 16.0 * np.pi ** 2 * sum(
            self.w[j] * self.B[j] * sinc(np.pi * self.g[j] * knorm / self.L)
            for j in range(self.J))


def maxwellians(n, L, rho, u, theta):
    """M, M^g, M^h of Algorithm 1 on the cyclic grid:
    M   = rho (2 pi theta)^{-3/2} exp(-|v-u|^2 / (2 theta))
    M^g = rho (pi theta)^{-3/2}   exp(-|v|^2 / theta)
    M^h = rho (pi theta)^{-3/2}   exp(-|v-u|^2 / theta)."""
    v1, v2, v3 = grid.velocity_grid(n, L)
    d2 = (v1 - u[0]) ** 2 + (v2 - u[1]) ** 2 + (v3 - u[2]) ** 2
    z2 = v1 ** 2 + v2 ** 2 + v3 ** 2
    M = rho * (2.0 * np.pi * theta) ** -1.5 * np.exp(-d2 / (2.0 * theta))
    Mg = rho * (np.pi * theta) ** -1.5 * np.exp(-z2 / theta)
    Mh = rho * (np.pi * theta) ** -1.5 * np.exp(-d2 / theta)
    return M, Mg, Mh, d2


def cutoff_mask(d2, theta, eps):
    """True where the cut-off of Eq. (3.9) zeroes r (M/rho < eps)."""
    thresh = np.log(1.0 / eps) - 1.5 * np.log(2.0 * np.pi * theta)
    return d2 / (2.0 * theta) > thresh


def FFT(x):
    return np.fft.fftn(x, axes=(-3, -2, -1))


def InvFFT(x):
    return np.fft.ifftn(x, axes=(-3, -2, -1))


def collision_operator(tab, rho, u, theta, f, cutoff=True, eps=1e-9,
                       mass_fix=False, return_parts=False):
    """CollisionOperator(rho, u, theta, f, cutoff) of Algorithm 1 for one
    instance.  ``f`` is given on the cyclic grid (n, n, n); returns L[f] on
    the cyclic grid.  Steps follow Algorithm 1 in order."""
    n, L = tab.n, tab.L
    f = np.asarray(f, dtype=np.float64)
    M, Mg, Mh, d2 = maxwellians(n, L, rho, np.asarray(u, dtype=np.float64), theta)
    # r = f / M, or 0 under the cut-off (Eq. 3.9)
    if cutoff:
        cut = cutoff_mask(d2, theta, eps)
        r = np.where(cut, 0.0, f / np.where(cut, 1.0, M))
    else:
        r = f / M
    # gain term
    rhat = FFT(r)
    Lhat = np.zeros((n, n, n), dtype=np.complex128)
    for j in range(tab.J):
        uj = Mg * tab.phit[j]
        uhat = FFT(uj)
        psi = np.real(InvFFT(uhat * rhat))
        psi = Mh * psi
        psihat = FFT(psi)
        Lhat += tab.phi[j] * psihat
    Lplus = np.real(InvFFT(Lhat))
    # loss term
    fhat = FFT(f)
    Mhat = FFT(M)
    uu = np.real(InvFFT(fhat * tab.omega))
    ww = np.real(InvFFT(Mhat * tab.omega))
    Lminus = uu * M + ww * f
    out = Lplus - Lminus
    if mass_fix:
        # L^_0 = 0 (Sec. 4.2, conservation study)
        out = out - out.mean()
    if return_parts:
        return out, Lplus, Lminus
    return out


def apply_linearized(tab, params, g, cutoff=True, eps=1e-9, mass_fix=False):
    """Batched L[g] in the library's layout: params (B, 5) = (rho, u1, u2, u3,
    theta), g (B, n, n, n) in centred order; returns (B, n, n, n) centred."""
    params = np.atleast_2d(np.asarray(params, dtype=np.float64))
    g = np.asarray(g, dtype=np.float64).reshape(params.shape[0], tab.n, tab.n, tab.n)
    out = np.empty_like(g)
    for b in range(params.shape[0]):
        rho, u1, u2, u3, th = params[b]
        out[b] = grid.to_centred(collision_operator(
            tab, rho, (u1, u2, u3), th, grid.to_cyclic(g[b]), cutoff, eps, mass_fix))
    return out
