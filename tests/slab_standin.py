"""A CPU stand-in for the per-block operations of the partitioned slab
solver (paper_2503_09580_gb300/distributed.py), in numpy on CPU torch
tensors, so that its host logic (halo exchange, wall ghosts, reductions
over ranks, the sweep chained across blocks, FGMRES) runs under gloo
without a GPU.

The transport, sweep, moments, wall flux and Maxwellian cell restate the
definitions the library's slab-block primitives implement (upwind
differences of Eq. (5.2), the sweep of Eq. (5.7), the moments of Sec. 2.1).
The collision operator is a stand-in, not the paper's: a BGK-type
relaxation that conserves the discrete mass, momentum and energy exactly,

    Q(f) = rho (P_{M[f]} f - f),

P_M g = M (a + b.v + c |v|^2) with the five discrete moments of g, and its
linearisation about the local Maxwellian L_M g = rho (P_M g - g) (so that
L_M[M] = 0, as for the true operator).
"""
import numpy as np
import torch


class NumpyBlock:
    def __init__(self, N, box):
        self.N, self.n3, self.h = N, N ** 3, 2.0 * box / N
        a = (np.arange(N) - N // 2) * self.h
        g = np.meshgrid(a, a, a, indexing="ij")
        self.v = np.stack([x.ravel() for x in g])          # (3, n3)
        self.v1 = self.v[0]
        self.phi = np.vstack([np.ones(self.n3), self.v, (self.v ** 2).sum(0)])  # (5, n3)
        self.device = "cpu"
        self.cached = None

    def zeros(self, *shape):
        return torch.zeros(*shape, dtype=torch.float64)

    # -- definitions -----------------------------------------------------------
    def maxwellian(self, rho, u, theta):
        d2 = ((self.v - np.asarray(u, float)[:, None]) ** 2).sum(0)
        return rho * (2 * np.pi * theta) ** -1.5 * np.exp(-d2 / (2 * theta))

    def cell_moments(self, x):
        h3 = self.h ** 3
        rho = h3 * x.sum()
        u = h3 * (self.v @ x) / rho
        e = h3 * ((self.v ** 2).sum(0) @ x)
        return rho, u, (e - rho * (u @ u)) / (3 * rho)

    def project(self, M, g):
        G = (self.phi * M) @ self.phi.T
        c = np.linalg.solve(G, self.phi @ g)
        return M * (c @ self.phi)

    # -- the block operations --------------------------------------------------
    def moments(self, f, nx, params, nu):
        F, P = f.numpy().reshape(nx, self.n3), params.numpy().reshape(nx, 5)
        for j in range(nx):
            rho, u, th = self.cell_moments(F[j])
            P[j] = (rho, u[0], u[1], u[2], th)
            nu.numpy()[j] = rho

    def quadratic(self, f, nx, out):
        F, O = f.numpy().reshape(nx, self.n3), out.numpy().reshape(nx, self.n3)
        for j in range(nx):
            rho, u, th = self.cell_moments(F[j])
            O[j] = rho * (self.project(self.maxwellian(rho, u, th), F[j]) - F[j])

    def linearized(self, params, v, nx, out):
        P, V, O = params.numpy().reshape(nx, 5), v.numpy().reshape(nx, self.n3), out.numpy().reshape(nx, self.n3)
        for j in range(nx):
            rho, u, th = P[j, 0], P[j, 1:4], P[j, 4]
            O[j] = rho * (self.project(self.maxwellian(rho, u, th), V[j]) - V[j])

    def cache(self, params, nx):
        self.cached = None if params is None else params.clone()

    def transport(self, v, gl, gr, out, nx, dx):
        V = v.numpy().reshape(nx, self.n3)
        left = np.vstack([np.zeros(self.n3) if gl is None else gl.numpy(), V[:-1]])
        right = np.vstack([V[1:], np.zeros(self.n3) if gr is None else gr.numpy()])
        p, m = np.maximum(self.v1, 0), np.minimum(self.v1, 0)
        out.numpy().reshape(nx, self.n3)[:] = (p * (V - left) + m * (right - V)) / dx

    def sweep(self, r, nu, il, ir, z, nx, dx, kn, shift, direction):
        R, Z, n = r.numpy().reshape(nx, self.n3), z.numpy().reshape(nx, self.n3), nu.numpy()
        c = np.abs(self.v1) / dx
        pos, neg = self.v1 >= 0, self.v1 < 0
        if direction >= 0:
            prev = np.zeros(self.n3) if il is None else il.numpy().copy()
            for j in range(nx):
                prev = np.where(pos, (R[j] + c * prev) / (c + n[j] / kn + shift), prev)
                Z[j, pos] = prev[pos]
        if direction <= 0:
            prev = np.zeros(self.n3) if ir is None else ir.numpy().copy()
            for j in range(nx - 1, -1, -1):
                prev = np.where(neg, (R[j] + c * prev) / (c + n[j] / kn + shift), prev)
                Z[j, neg] = prev[neg]

    def cell_flux(self, cell, side):
        w = np.minimum(self.v1, 0) if side == 0 else np.maximum(self.v1, 0)
        return float(self.h ** 3 * (w @ cell.numpy()))

    def maxwellian_cell(self, theta, u, scale, out):
        out.numpy()[:] = self.maxwellian(scale, u, theta)

    def dots(self, V, K, y):
        if V.dim() == 1:
            return np.array([V.numpy() @ y.numpy()])
        return V.numpy()[:K] @ y.numpy()

    def axpby(self, y, x, a, b):
        y.numpy()[:] = a * x.numpy() + b * y.numpy()

    def combination(self, y, V, K, c):
        y.numpy()[:] -= np.asarray(c[:K]) @ V.numpy()[:K]
