"""Steady 1-D Boltzmann problem and its modified Newton step (Sec. 5 and the
supplement's fully discrete scheme).  Oracle: test infrastructure only.

State f[j, i1, i2, i3]: cell j = 1..nx (array index j-1), velocity on the
collocation grid in *centred* order (the library's layout).  Cell centres
x_j = x_L + (j - 1/2) dx.

Discrete residual (supplement, upwind finite volume):
  R_j = v1^+ (f_j - f_{j-1})/dx + v1^- (f_{j+1} - f_j)/dx - Q(f_j, f_j)/Kn
with ghost cells from Maxwell's diffuse walls, Eq. (5.2):
  f_0     = W_L(v) * ( -sqrt(2 pi/theta_L) h^3 sum_v v1^- f_1 ),
  f_{nx+1} = W_R(v) * (  sqrt(2 pi/theta_R) h^3 sum_v v1^+ f_nx ),
  W(v) = (2 pi theta)^{-3/2} exp(-|v - u_w|^2 / (2 theta)).
(Reading: the paper's rho_R formula uses f(x_L); the right wall uses f(x_R).)
Modified Newton, Eqs. (5.4), (5.6): solve
  v1^+ (g_j - g_{j-1})/dx + v1^- (g_{j+1} - g_j)/dx - L_j[g_j]/Kn = R_j
with the same linear wall map for g's ghost cells, L_j linearised about
the local Maxwellian of f_j; then f <- f - g.  The linear system
is singular along the mass mode (every residual has ~zero total mass:
diffuse walls carry no net flux and Q conserves mass), so the total-mass
condition dx h^3 sum f = C, Eq. (5.3), is imposed inside the solve
(reading): the bordered operator
  A'(g) = A g + e m(g),  e = f / m(f),  m(g) = dx h^3 sum g,
is solved with right-hand side R + e (m(f) - C), which gives A g = R and
m(f - g) = C whenever R has zero mass.
The inner solve uses scipy's GMRES (a library routine) on the exact
operator, or the paper's own inner solver, the source iteration (Eq. (5.7)
and the supplement's fully discrete form): with S the operator the upwind
sweep inverts (transport with zero incoming ghost values plus nu_j/Kn),
  S g^{l+1} = (S - A) g^l + rhs,  g^0 = 0,
which for A = transport - L/Kn is the printed update
S g^{l+1} = (nu_j g^l + L_j[g^l])/Kn + r.  (Reading: the wall's and the
border's couplings of g, which S leaves out, enter through (S - A) g^l,
one iteration behind; the fixed point is the solution of A g = rhs.)
"""
import numpy as np

from . import grid
from .linearized import Tables, collision_operator
from .moments import moments
from .quadratic import quadratic_operator


class Slab:
    def __init__(self, n, L, omega, J, nx, x_left=-0.5, x_right=0.5, kn=1.0,
                 wall_left=(1.0, 0.0, 0.0, 0.0), wall_right=(2.0, 0.0, 0.0, 0.0),
                 hemisphere=None, wall_flux="analytic", q_mass_fix=None, inflow_left=None, inflow_right=None):
        self.n, self.L, self.nx, self.kn = n, L, nx, kn
        self.tab = Tables(n, L, omega, J)
        self.dx = (x_right - x_left) / nx
        self.xc = x_left + (np.arange(nx) + 0.5) * self.dx
        self.h = grid.spacing(n, L)
        a = (np.arange(n) - n // 2) * self.h
        self.v1 = np.broadcast_to(a[:, None, None], (n, n, n))
        self.vp = np.maximum(self.v1, 0.0)
        self.vm = np.minimum(self.v1, 0.0)
        self.sig, self.wm = hemisphere
        v2 = a[None, :, None]
        v3 = a[None, None, :]

        def wall_shape(w):
            th, u1, u2, u3 = w
            return (2 * np.pi * th) ** -1.5 * np.exp(
                -((a[:, None, None] - u1) ** 2 + (v2 - u2) ** 2 + (v3 - u3) ** 2) / (2 * th))
        self.WL, self.WR = wall_shape(wall_left), wall_shape(wall_right)
        self.thL, self.thR = wall_left[0], wall_right[0]
        # wall-density factor per unit outgoing flux: sqrt(2 pi / theta) is the
        # inverse half-range flux of the unit Maxwellian (the paper's formula);
        # 'discrete' uses the grid sum instead, so the discrete net wall flux
        # vanishes exactly
        if wall_flux == "analytic":
            self.kL, self.kR = np.sqrt(2 * np.pi / self.thL), np.sqrt(2 * np.pi / self.thR)
        else:
            h3 = self.h ** 3
            self.kL = 1.0 / (h3 * (self.vp * self.WL).sum())
            self.kR = 1.0 / (h3 * (-self.vm * self.WR).sum())
        self.q_mass_fix = q_mass_fix
        # inflow sides (library extension for the shock workload): ghost cell =
        # the given Maxwellian (rho, u1, u2, u3, theta) for the residual, zero
        # for a Newton correction

        def maxwell(st):
            rho, u1, u2, u3, th = st
            return rho * (2 * np.pi * th) ** -1.5 * np.exp(
                -((a[:, None, None] - u1) ** 2 + (v2 - u2) ** 2 + (v3 - u3) ** 2) / (2 * th))
        self.inL = None if inflow_left is None else maxwell(inflow_left)
        self.inR = None if inflow_right is None else maxwell(inflow_right)

    def ghosts(self, f, linear=False):
        h3 = self.h ** 3
        if self.inL is not None:
            gl = 0.0 * self.WL if linear else self.inL
        else:
            gl = -self.kL * h3 * (self.vm * f[0]).sum() * self.WL
        if self.inR is not None:
            gr = 0.0 * self.WR if linear else self.inR
        else:
            gr = self.kR * h3 * (self.vp * f[-1]).sum() * self.WR
        return gl, gr

    def transport(self, f, linear=False):
        """v1^+ (f_j - f_{j-1})/dx + v1^- (f_{j+1} - f_j)/dx with ghost cells."""
        g0, g1 = self.ghosts(f, linear)
        ext = np.concatenate([g0[None], f, g1[None]], axis=0)
        return (self.vp * (ext[1:-1] - ext[:-2]) + self.vm * (ext[2:] - ext[1:-1])) / self.dx

    def collision_q(self, f):
        return np.stack([grid.to_centred(quadratic_operator(self.tab, grid.to_cyclic(f[j]), self.sig, self.wm,
                                                            mass_fix=self.q_mass_fix))
                         for j in range(self.nx)])

    def residual(self, f):
        return self.transport(f) - self.collision_q(f) / self.kn

    def local_params(self, f):
        out = np.empty((self.nx, 5))
        for j in range(self.nx):
            rho, u, th, _, _ = moments(grid.to_cyclic(f[j]), self.n, self.L)
            out[j] = (rho, u[0], u[1], u[2], th)
        return out

    def linear_operator(self, params):
        """g -> transport(g) - L_j[g_j]/Kn with L_j about params[j]."""
        def apply(g):
            Lg = np.stack([grid.to_centred(collision_operator(
                self.tab, p[0], p[1:4], p[4], grid.to_cyclic(g[j]))) for j, p in enumerate(params)])
            return self.transport(g, linear=True) - Lg / self.kn
        return apply

    def exact_jacobian(self, f):
        """g -> transport(g) - (Q(f_j, g_j) + Q(g_j, f_j))/Kn: the derivative
        of the discrete residual itself (Q(f,f) is the diagonal of the
        symmetric bilinear form of Eq. (2.14)), in place of the
        local-Maxwellian L_j of the modified step.  Library extension."""
        def apply(g):
            J = np.stack([grid.to_centred(quadratic_operator(
                self.tab, grid.to_cyclic(f[j]), self.sig, self.wm, g=grid.to_cyclic(g[j]),
                mass_fix=self.q_mass_fix)) for j in range(self.nx)])
            return self.transport(g, linear=True) - J / self.kn
        return apply

    def norm(self, r):
        """Discrete L2 norm sqrt(dx h^3 sum r^2), Sec. 5.3."""
        return np.sqrt(self.dx * self.h ** 3 * (r * r).sum())

    def mass(self, f):
        return self.dx * self.h ** 3 * f.sum()

    def sweep(self, r, nu, shift=0.0):
        """Upwind sweep of the source iteration, Eq. (5.7):
        (v1^+ D^- + v1^- D^+ + nu_j/Kn + shift) z = r, ghost values of z taken as 0."""
        z = np.zeros_like(r)
        c = np.abs(self.v1) / self.dx
        pos, neg = self.v1 > 0, self.v1 < 0
        zero = ~(pos | neg)
        prev = np.zeros(r.shape[1:])
        for j in range(self.nx):
            d = c + nu[j] / self.kn + shift
            zj = np.where(pos, (r[j] + c * prev) / d, 0.0)
            z[j][pos] = zj[pos]
            prev = np.where(pos, zj, 0.0)
        prev = np.zeros(r.shape[1:])
        for j in range(self.nx - 1, -1, -1):
            d = c + nu[j] / self.kn + shift
            zj = np.where(neg, (r[j] + c * prev) / d, 0.0)
            z[j][neg] = zj[neg]
            prev = np.where(neg, zj, 0.0)
        for j in range(self.nx):
            z[j][zero] = r[j][zero] / (nu[j] / self.kn + shift)
        return z

    def sweep_operator(self, z, nu, shift=0.0):
        """The operator ``sweep`` inverts: (v1^+ D^- + v1^- D^+ + nu_j/Kn + shift) z
        with zero ghost values."""
        zero = np.zeros((1,) + z.shape[1:])
        ext = np.concatenate([zero, z, zero], axis=0)
        tr = (self.vp * (ext[1:-1] - ext[:-2]) + self.vm * (ext[2:] - ext[1:-1])) / self.dx
        return tr + (np.asarray(nu)[:, None, None, None] / self.kn + shift) * z

    def source_iteration(self, A, rhs, nu, shift=0.0, rtol=1e-10, atol=0.0, maxiter=5000):
        """Solve A g = rhs by the source iteration S g^{l+1} = (S - A) g^l + rhs
        from g^0 = 0, S = sweep_operator (shift included in both S and A by
        the caller's A).  Stops at |rhs - A g| <= max(rtol |rhs|, atol).
        Returns (g, iterations, converged)."""
        g = np.zeros_like(rhs)
        target = max(rtol * self.norm(rhs), atol)
        for it in range(1, maxiter + 1):
            g = self.sweep(self.sweep_operator(g, nu, shift) - A(g) + rhs, nu, shift)
            if self.norm(rhs - A(g)) <= target:
                return g, it, True
        return g, maxiter, False

    def bordered_operator(self, params, f, jacobian="local_maxwellian"):
        """A'(g) = A g + e m(g) with e = f / m(f)."""
        A = self.exact_jacobian(f) if jacobian == "exact" else self.linear_operator(params)
        e = f / self.mass(f)

        def apply(g):
            return A(g) + e * self.mass(g)
        return apply

    def newton_step(self, f, total_mass, rtol=1e-10, restart=60, maxiter=400, shift=0.0,
                    jacobian="local_maxwellian", inner="gmres", nu_scale=1.0):
        """One modified Newton step: returns (f_new, g, |R(f)|).  GMRES on the
        bordered operator, preconditioned by the upwind sweep with
        nu_j = rho_j (Eq. (5.7)).  shift > 0 solves (A + shift I) g = R
        instead: one step of pseudo-transient continuation with
        dtau = 1/shift (a library extension; the paper's step has shift 0).
        jacobian="exact" uses exact_jacobian in place of the local-Maxwellian
        L_j (full Newton; also a library extension).  inner="source_iteration"
        solves the same system with the paper's source iteration instead
        (maxiter then caps its iterations); the sweep takes
        nu_j = nu_scale rho_j."""
        from scipy.sparse.linalg import LinearOperator, gmres
        R = self.residual(f)
        params = self.local_params(f)
        if self.inL is None and self.inR is None:
            A = self.bordered_operator(params, f, jacobian)
            rhs = R + (f / self.mass(f)) * (self.mass(f) - total_mass)
        else:
            # an inflow side fixes the incoming ghost values: no mass null
            # mode, and the mass in the slab is set by the boundary fluxes
            A = self.exact_jacobian(f) if jacobian == "exact" else self.linear_operator(params)
            rhs = R
        if shift:
            A0 = A
            A = lambda g: A0(g) + shift * g  # noqa: E731
        if inner == "source_iteration":
            g, _, _ = self.source_iteration(A, rhs, nu_scale * params[:, 0], shift, rtol=rtol, maxiter=maxiter)
            return f - g, g, self.norm(R)
        shape = f.shape
        n = R.size
        op = LinearOperator((n, n), matvec=lambda x: A(x.reshape(shape)).ravel(), dtype=np.float64)
        pre = LinearOperator((n, n), matvec=lambda x: self.sweep(x.reshape(shape), nu_scale * params[:, 0],
                                                                 shift).ravel(),
                             dtype=np.float64)
        x, info = gmres(op, rhs.ravel(), rtol=rtol, atol=0.0, restart=restart, maxiter=maxiter, M=pre)
        g = x.reshape(shape)
        return f - g, g, self.norm(R)


def initial_state(slab, total_mass=1.0, theta_left=1.0, theta_right=2.0):
    """Linear temperature profile between the walls, Eq. (S.initial):
    f_j = C/(x_R - x_L) (2 pi theta_j)^{-3/2} exp(-|v|^2/(2 theta_j))."""
    a = (np.arange(slab.n) - slab.n // 2) * slab.h
    v2 = a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2
    width = slab.nx * slab.dx
    out = []
    for x in slab.xc:
        w = (x - slab.xc[0] + 0.5 * slab.dx) / width
        th = (1 - w) * theta_left + w * theta_right
        out.append(total_mass / width * (2 * np.pi * th) ** -1.5 * np.exp(-v2 / (2 * th)))
    return np.stack(out)


class MixedSlab:
    """Slab whose cells carry different velocity grids n_j on the same box
    (the mixed-n shock workload; library extension).  Reading: the upwind
    difference of cell j uses its neighbours resampled to cell j's grid
    (resample.py: zero padding or truncation), so every cell's transport
    term lives on its own grid; collisions are cell-local with the tables
    of the cell's n.  Inflow sides only (the ghost of a Newton correction is
    zero, and there is no mass border).  States are lists of centred-order
    arrays, one per cell.
    """

    def __init__(self, ns, L, omega, x_left=-0.5, x_right=0.5, kn=1.0, hemisphere=None, q_mass_fix=None,
                 inflow_left=None, inflow_right=None):
        from .resample import resample_centred
        self.resample = resample_centred
        self.ns = [int(n) for n in ns]
        self.nx, self.L, self.kn = len(ns), L, kn
        self.dx = (x_right - x_left) / self.nx
        self.tabs = {n: Tables(n, L, omega, n) for n in sorted(set(self.ns))}
        self.sig, self.wm = hemisphere
        self.q_mass_fix = q_mass_fix

        def axes(n):
            a = (np.arange(n) - n // 2) * grid.spacing(n, L)
            return a

        def maxwell(st, n):
            rho, u1, u2, u3, th = st
            a = axes(n)
            return rho * (2 * np.pi * th) ** -1.5 * np.exp(
                -((a[:, None, None] - u1) ** 2 + (a[None, :, None] - u2) ** 2 + (a[None, None, :] - u3) ** 2)
                / (2 * th))
        self.v1 = {n: np.broadcast_to(axes(n)[:, None, None], (n, n, n)) for n in self.tabs}
        self.inL = maxwell(inflow_left, self.ns[0])
        self.inR = maxwell(inflow_right, self.ns[-1])

    def _on(self, x, n):
        return x if x.shape[0] == n else self.resample(x, n)

    def transport(self, f, linear=False):
        out = []
        for j, n in enumerate(self.ns):
            v1 = self.v1[n]
            left = (0.0 * f[j] if linear else self.inL) if j == 0 else self._on(f[j - 1], n)
            right = (0.0 * f[j] if linear else self.inR) if j == self.nx - 1 else self._on(f[j + 1], n)
            out.append((np.maximum(v1, 0.0) * (f[j] - left) + np.minimum(v1, 0.0) * (right - f[j])) / self.dx)
        return out

    def collision_q(self, f):
        return [grid.to_centred(quadratic_operator(self.tabs[n], grid.to_cyclic(f[j]), self.sig, self.wm,
                                                   mass_fix=self.q_mass_fix)) for j, n in enumerate(self.ns)]

    def residual(self, f):
        return [t - q / self.kn for t, q in zip(self.transport(f), self.collision_q(f))]

    def local_params(self, f):
        out = np.empty((self.nx, 5))
        for j, n in enumerate(self.ns):
            rho, u, th, _, _ = moments(grid.to_cyclic(f[j]), n, self.L)
            out[j] = (rho, u[0], u[1], u[2], th)
        return out

    def norm(self, r):
        """sqrt(dx sum_j h_j^3 sum r_j^2), the discrete L2 norm cell by cell."""
        return np.sqrt(self.dx * sum(grid.spacing(n, self.L) ** 3 * (x * x).sum() for n, x in zip(self.ns, r)))

    def operator(self, f, jacobian="local_maxwellian", shift=0.0):
        params = self.local_params(f)

        def coll(g):
            if jacobian == "exact":
                return [grid.to_centred(quadratic_operator(self.tabs[n], grid.to_cyclic(f[j]), self.sig, self.wm,
                                                           g=grid.to_cyclic(g[j]), mass_fix=self.q_mass_fix))
                        for j, n in enumerate(self.ns)]
            return [grid.to_centred(collision_operator(self.tabs[n], p[0], p[1:4], p[4], grid.to_cyclic(g[j])))
                    for j, (n, p) in enumerate(zip(self.ns, params))]

        def apply(g):
            return [t - c / self.kn + shift * x for t, c, x in zip(self.transport(g, linear=True), coll(g), g)]
        return apply

    def flatten(self, f):
        return np.concatenate([x.ravel() for x in f])

    def unflatten(self, x):
        out, o = [], 0
        for n in self.ns:
            out.append(x[o:o + n ** 3].reshape(n, n, n))
            o += n ** 3
        return out

    def newton_step(self, f, rtol=1e-10, restart=80, maxiter=400, shift=0.0, jacobian="local_maxwellian"):
        """One Newton step (modified or exact Jacobian, optional shift),
        unpreconditioned GMRES (scipy) on the flattened cells; returns
        (f_new, g, |R(f)|)."""
        from scipy.sparse.linalg import LinearOperator, gmres
        R = self.residual(f)
        A = self.operator(f, jacobian, shift)
        n = sum(x.size for x in f)
        op = LinearOperator((n, n), matvec=lambda x: self.flatten(A(self.unflatten(x))), dtype=np.float64)
        x, info = gmres(op, self.flatten(R), rtol=rtol, atol=0.0, restart=restart, maxiter=maxiter)
        g = self.unflatten(x)
        return [a - b for a, b in zip(f, g)], g, self.norm(R)
