"""Modified Newton / flexible GMRES on the 1-D slab (Sec. 5) with the cells
split over several processes, one GPU each.  Rank r owns the contiguous
block of cells [c0, c0 + nx_r); every long-vector step runs on that block
in the library's kernels (the L and Q applications of its cells and the
slab-block primitives of include/lbo.h).  Between ranks travel:

* one boundary cell (N^3 doubles) to each neighbour per transport
  application: the upwind differences of Eq. (5.2) read the cell across
  the block edge (point to point);
* the incoming boundary values of the sweep preconditioner (Eq. (5.7)),
  passed downstream block by block: the v1 > 0 half from left to right and
  the v1 < 0 half from right to left, the two chains running at once;
* the K <= m + 1 dot products of each Gram-Schmidt pass, the norms and the
  mass of Eq. (5.3) (an all-reduce each).

The diffuse-wall ghost cells are formed on the two end ranks from their own
boundary cells.  The iteration is the single-GPU solver's, step for step
(bordered mass constraint, classical Gram-Schmidt with two passes, Givens
rotations, restart from the true residual, the same stopping tests), so a
single rank reproduces lbo_newton_step up to the order of its sums.

Scope: the modified Jacobian (L about each cell's local Maxwellian, Eqs.
(5.4), (5.6)), the NONE and SWEEP preconditioners, FGMRES, walls or inflow
on either side, pseudo-transient shift and nu_scale as in lbo_problem.

The communicator is torch.distributed (NCCL between GPUs, gloo on CPU); a
run without an initialised process group is a single rank.  A block object
supplies the per-block operations; GpuBlock runs them on this process's
GPU through lbo.Plan.
"""
import math

import numpy as np

try:
    import torch
    import torch.distributed as dist
except ImportError:  # pragma: no cover - torch is part of the stack
    torch = dist = None


def partition(nx, world):
    """Contiguous blocks of nx cells over world ranks: [(c0, count)], the
    first nx % world ranks one cell more; every rank gets at least one."""
    if world < 1 or nx < world:
        raise ValueError("need at least one cell per rank (nx=%d, world=%d)" % (nx, world))
    q, rem = divmod(nx, world)
    out, c0 = [], 0
    for r in range(world):
        n = q + (1 if r < rem else 0)
        out.append((c0, n))
        c0 += n
    return out


class Comm:
    """Point-to-point exchange and sums over torch.distributed; tensors for
    the collectives live on `device` (CUDA for NCCL, CPU for gloo)."""

    def __init__(self, device="cpu"):
        self.on = dist is not None and dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank() if self.on else 0
        self.world = dist.get_world_size() if self.on else 1
        self.device = device
        if self.world > 1:
            # every rank takes part in the group's first collective
            dist.barrier()

    def allreduce(self, values):
        a = np.asarray(values, dtype=np.float64).reshape(-1)
        if self.world == 1:
            return a
        t = torch.from_numpy(a.copy()).to(self.device)
        dist.all_reduce(t)
        return t.cpu().numpy()

    def exchange(self, sends, recvs):
        """sends, recvs: [(tensor, peer)]; returns when all have arrived."""
        ops = [dist.P2POp(dist.irecv, t, p) for t, p in recvs] + [dist.P2POp(dist.isend, t, p) for t, p in sends]
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()

    def isend(self, t, peer):
        return dist.isend(t, peer)

    def recv(self, t, peer):
        dist.recv(t, peer)


class GpuBlock:
    """The rank's cells on its GPU: the library's kernels through lbo.Plan
    (plan for L, rplan, if given, for the residual's Q)."""

    def __init__(self, plan, rplan=None):
        self.plan, self.rplan = plan, rplan or plan
        self.N = plan.N
        self.n3 = plan.N ** 3
        self.h = 2.0 * plan.box / plan.N
        self.device = torch.device("cuda", torch.cuda.current_device())

    def zeros(self, *shape):
        return torch.zeros(*shape, dtype=torch.float64, device=self.device)

    def moments(self, f, nx, params, nu):
        self.plan.block_moments(f, nx, params, nu)

    def quadratic(self, f, nx, out):
        N = self.N
        self.rplan.apply_quadratic(f.view(nx, N, N, N), out.view(nx, N, N, N))

    def linearized(self, params, v, nx, out):
        N = self.N
        self.plan.apply_linearized(params.view(nx, 5), v.view(nx, N, N, N), out.view(nx, N, N, N))

    def cache(self, params, nx):
        self.plan.cache_maxwellians(None if params is None else params.view(nx, 5))

    def transport(self, v, gl, gr, out, nx, dx):
        self.plan.block_transport(v, gl, gr, out, nx, dx)

    def sweep(self, r, nu, il, ir, z, nx, dx, kn, shift, direction):
        self.plan.block_sweep(r, nu, il, ir, z, nx, dx, kn, shift, direction)

    def cell_flux(self, cell, side):
        return self.plan.cell_flux(cell, side)

    def maxwellian_cell(self, theta, u, scale, out):
        self.plan.maxwellian_cell(theta, u, scale, out)

    def dots(self, V, K, y):
        return self.plan.vec_dots(V, V.stride(0) if V.dim() == 2 else V.numel(), K, y, y.numel())

    def axpby(self, y, x, a, b):
        self.plan.vec_axpby(y, x, a, b, y.numel())

    def combination(self, y, V, K, c):
        self.plan.vec_combination(y, V, V.stride(0), K, c, y.numel())


class DistributedSlab:
    """One rank's share of the slab solver.  The state f passed to
    newton_step is this rank's block (nx_r N^3 doubles, cells in order)."""

    def __init__(self, block, comm, nx, x_left=-0.5, x_right=0.5, kn=1.0, wall_left=(1.0, 0.0, 0.0, 0.0),
                 wall_right=(1.0, 0.0, 0.0, 0.0), total_mass=1.0, wall_flux="analytic", krylov_rtol=1e-3,
                 krylov_atol=1e-7, krylov_restart=30, krylov_maxit=300, precond="sweep", inflow_left=None,
                 inflow_right=None, pseudo_dt=0.0, nu_scale=1.0):
        if precond not in ("none", "sweep"):
            raise ValueError("the partitioned solver takes the none or sweep preconditioner")
        if not 1 <= krylov_restart <= 200:
            raise ValueError("krylov_restart must be in 1..200")
        self.b, self.comm = block, comm
        self.parts = partition(nx, comm.world)
        self.c0, self.nxl = self.parts[comm.rank]
        self.first, self.last = comm.rank == 0, comm.rank == comm.world - 1
        self.nx, self.kn, self.dx = nx, float(kn), (x_right - x_left) / nx
        self.h, self.n3 = block.h, block.n3
        self.len = self.nxl * self.n3
        self.wnorm = self.dx * self.h ** 3
        self.total_mass = float(total_mass)
        self.rtol, self.atol = float(krylov_rtol), float(krylov_atol)
        self.m, self.maxit = int(krylov_restart), int(krylov_maxit)
        self.precond, self.pseudo_dt, self.nu_scale = precond, float(pseudo_dt), float(nu_scale)
        self.inflow = (inflow_left is not None, inflow_right is not None)
        self.bordered = not (self.inflow[0] or self.inflow[1])
        self.shift, self.r_first = 0.0, 0.0
        z = block.zeros
        n3 = self.n3
        # wall (unit-density Maxwellian of the wall) or inflow (the given state) cells
        self.WL = self.WR = None
        self.kL = self.kR = 0.0
        for side, (wall, inflow, here) in enumerate(((wall_left, inflow_left, self.first),
                                                     (wall_right, inflow_right, self.last))):
            if not here:
                continue
            W = z(n3)
            if inflow is not None:
                block.maxwellian_cell(inflow[4], inflow[1:4], inflow[0], W)
            else:
                block.maxwellian_cell(wall[0], wall[1:4], 1.0, W)
            if side == 0:
                self.WL = W
            else:
                self.WR = W
            if inflow is None:
                if wall_flux == "discrete":
                    # normalise the discrete outgoing flux of the wall cell to one
                    flux = block.cell_flux(W, 1 if side == 0 else 0)
                    k = 1.0 / abs(flux)
                else:
                    k = math.sqrt(2.0 * math.pi / wall[0])
                if side == 0:
                    self.kL = k
                else:
                    self.kR = k
        L, m = self.len, self.m
        self.V, self.Z = z(m + 1, L), z(m, L)
        self.w, self.Lv, self.Qf, self.rhs, self.x, self.e = z(L), z(L), z(L), z(L), z(L), z(L)
        self.ones = z(L).fill_(1.0)
        self.params, self.nu = z(5 * self.nxl), z(self.nxl)
        self.gl, self.gr = z(n3), z(n3)          # neighbour or ghost cells of the transport
        self.sl, self.sr = z(n3), z(n3)          # incoming values of the sweep
        self.out_l, self.out_r = z(n3), z(n3)    # outgoing boundary cells of the sweep

    # -- reductions over all ranks -------------------------------------------
    def dot_all(self, V, K, y):
        return self.comm.allreduce(self.b.dots(V, K, y))

    def norm(self, v):
        return math.sqrt(max(float(self.dot_all(v, 1, v)[0]), 0.0))

    def mass(self, v):
        """dx h^3 sum v over all cells (the constraint of Eq. (5.3))."""
        return self.wnorm * float(self.dot_all(self.ones, 1, v)[0])

    # -- transport with neighbour and wall cells -------------------------------
    def transport(self, v, out, inflow_factor):
        """out = T v (upwind v1^+ D^- + v1^- D^+, Eq. (5.2)): neighbour cells
        exchanged, wall ghosts sigma W with the wall density sigma from v's
        outgoing flux, inflow ghosts inflow_factor x the inflow cell."""
        b, c, n3 = self.b, self.comm, self.n3
        sends, recvs = [], []
        if not self.first:
            sends.append((v[:n3], c.rank - 1))
            recvs.append((self.gl, c.rank - 1))
        if not self.last:
            sends.append((v[self.len - n3:], c.rank + 1))
            recvs.append((self.gr, c.rank + 1))
        if c.world > 1:
            c.exchange(sends, recvs)
        gl, gr = self.gl, self.gr
        if self.first:
            if self.inflow[0]:
                s = inflow_factor
            else:  # sigma_L = -kL h^3 sum v1^- v (first cell)
                s = -self.kL * b.cell_flux(v[:n3], 0)
            b.axpby(self.gl, self.WL, s, 0.0)
        if self.last:
            if self.inflow[1]:
                s = inflow_factor
            else:  # sigma_R = kR h^3 sum v1^+ v (last cell)
                s = self.kR * b.cell_flux(v[self.len - n3:], 1)
            b.axpby(self.gr, self.WR, s, 0.0)
        b.transport(v, gl, gr, out, self.nxl, self.dx)

    def residual(self, f, out):
        """R(f) = T f - Q(f, f) / Kn on this block; returns the weighted
        norm over all ranks."""
        self.b.quadratic(f, self.nxl, self.Qf)
        self.transport(f, out, 1.0)
        self.b.axpby(out, self.Qf, -1.0 / self.kn, 1.0)
        return self.norm(out) * math.sqrt(self.wnorm)

    def apply_op(self, v, out):
        """out = T v - L v / Kn + shift v + e m(v) (m(v) only between two walls)."""
        b = self.b
        b.linearized(self.params, v, self.nxl, self.Lv)
        self.transport(v, out, 0.0)
        b.axpby(out, self.Lv, -1.0 / self.kn, 1.0)
        if self.shift != 0.0:
            b.axpby(out, v, self.shift, 1.0)
        if self.bordered:
            b.axpby(out, self.e, self.mass(v), 1.0)

    # -- sweep preconditioner across the blocks --------------------------------
    def apply_precond(self, v, z):
        """z = S^-1 v, S the upwind transport plus nu_j/Kn + shift (Eq.
        (5.7)), zero incoming values at the two ends of the slab."""
        b, c, n3 = self.b, self.comm, self.n3
        if self.precond == "none":
            b.axpby(z, v, 1.0, 0.0)
            return
        args = (self.nxl, self.dx, self.kn, self.shift)
        if c.world == 1:
            b.sweep(v, self.nu, None, None, z, *args, 0)
            return
        pending = []

        def forward():  # v1 >= 0, left to right
            il = None
            if not self.first:
                c.recv(self.sl, c.rank - 1)
                il = self.sl
            b.sweep(v, self.nu, il, None, z, *args, 1)
            if not self.last:
                b.axpby(self.out_r, z[self.len - n3:], 1.0, 0.0)
                pending.append(c.isend(self.out_r, c.rank + 1))

        def backward():  # v1 < 0, right to left
            ir = None
            if not self.last:
                c.recv(self.sr, c.rank + 1)
                ir = self.sr
            b.sweep(v, self.nu, None, ir, z, *args, -1)
            if not self.first:
                b.axpby(self.out_l, z[:n3], 1.0, 0.0)
                pending.append(c.isend(self.out_l, c.rank - 1))

        # the left half of the ranks sits early on the forward chain, the
        # right half on the backward one: each does that direction first
        order = (forward, backward) if 2 * c.rank < c.world else (backward, forward)
        for fn in order:
            fn()
        for w in pending:
            w.wait()

    # -- flexible GMRES ----------------------------------------------------
    def fgmres(self, ns):
        """Restarted FGMRES(m) on A' x = rhs from x = 0, right-preconditioned."""
        b, m = self.b, self.m
        H = np.zeros((m + 1, m))
        cs, sn, gam = np.zeros(m), np.zeros(m), np.zeros(m + 1)
        b.axpby(self.x, self.x, 0.0, 0.0)
        rhs_norm = self.norm(self.rhs)
        ns["rhs_norm"] = rhs_norm * math.sqrt(self.wnorm)
        tol = max(self.rtol * rhs_norm, self.atol / math.sqrt(self.wnorm))
        if rhs_norm == 0.0:
            return
        if not math.isfinite(rhs_norm):
            ns["status"] = "nan"
            return
        V, Z = self.V, self.Z
        b.axpby(V[0], self.rhs, 1.0, 0.0)
        beta = rhs_norm
        done = False
        while not done:
            b.axpby(V[0], V[0], 1.0 / beta, 0.0)
            gam[:] = 0.0
            gam[0] = beta
            H[:] = 0.0
            k = 0
            while k < m:
                self.apply_precond(V[k], Z[k])
                self.apply_op(Z[k], self.w)
                for _ in range(2):  # classical Gram-Schmidt, two passes
                    hv = self.dot_all(V, k + 1, self.w)
                    b.combination(self.w, V, k + 1, hv)
                    H[:k + 1, k] += hv
                hn = self.norm(self.w)
                H[k + 1, k] = hn
                if not math.isfinite(hn):
                    ns["status"] = "nan"
                    return
                if hn > 0:
                    b.axpby(V[k + 1], self.w, 1.0 / hn, 0.0)
                for i in range(k):
                    a_, b_ = H[i, k], H[i + 1, k]
                    H[i, k] = cs[i] * a_ + sn[i] * b_
                    H[i + 1, k] = -sn[i] * a_ + cs[i] * b_
                a_, b_ = H[k, k], H[k + 1, k]
                rr = math.hypot(a_, b_)
                cs[k] = a_ / rr if rr > 0 else 1.0
                sn[k] = b_ / rr if rr > 0 else 0.0
                H[k, k], H[k + 1, k] = rr, 0.0
                gam[k + 1] = -sn[k] * gam[k]
                gam[k] = cs[k] * gam[k]
                ns["krylov_iterations"] += 1
                k += 1
                if abs(gam[k]) <= tol or hn == 0.0:
                    done = True
                    break
                if ns["krylov_iterations"] >= self.maxit:
                    done = True
                    ns["status"] = "not converged"
                    break
            # x += Z y with H[:k, :k] y = gam[:k]
            y = np.zeros(k)
            for i in range(k - 1, -1, -1):
                acc = gam[i] - H[i, i + 1:k] @ y[i + 1:k]
                y[i] = acc / H[i, i] if H[i, i] != 0 else 0.0
            b.combination(self.x, Z, k, -y)
            if done:
                break
            ns["restarts"] += 1
            self.apply_op(self.x, self.w)
            b.axpby(V[0], self.rhs, 1.0, 0.0)
            b.axpby(V[0], self.w, -1.0, 1.0)
            beta = self.norm(V[0])
            if beta <= tol:
                break

    # -- one modified Newton step ----------------------------------------------
    def prepare(self, f, ns):
        """The step's linear system A' g = rhs about f: the cells' local
        Maxwellians (cached for the Krylov products), rhs = R(f) (+ e (m(f)
        - C) between two walls), the pseudo-transient shift."""
        b = self.b
        b.moments(f, self.nxl, self.params, self.nu)
        if self.nu_scale > 0 and self.nu_scale != 1.0:
            b.axpby(self.nu, self.nu, self.nu_scale, 0.0)
        rn = self.residual(f, self.rhs)
        ns["residual_norm"] = rn
        self.shift = 0.0
        if self.pseudo_dt > 0 and rn > 0:
            if self.r_first <= 0:
                self.r_first = rn
            self.shift = rn / (self.pseudo_dt * self.r_first)
        ns["shift"] = self.shift
        if self.bordered:
            # e = f / m(f), rhs = R + e (m(f) - C)
            mf = self.mass(f)
            b.axpby(self.e, f, 1.0 / mf, 0.0)
            b.axpby(self.rhs, self.e, mf - self.total_mass, 1.0)
        b.cache(self.params, self.nxl)

    def newton_step(self, f):
        """f <- f - g with A' g = rhs (prepare); returns the step's statistics."""
        b = self.b
        ns = {"residual_norm": 0.0, "rhs_norm": 0.0, "linear_residual": 0.0, "krylov_iterations": 0,
              "restarts": 0, "status": "ok", "shift": 0.0}
        try:
            self.prepare(f, ns)
            self.fgmres(ns)
            if ns["status"] != "nan":
                self.apply_op(self.x, self.w)
                b.axpby(self.w, self.rhs, 1.0, -1.0)
                ns["linear_residual"] = self.norm(self.w) * math.sqrt(self.wnorm)
        finally:
            b.cache(None, self.nxl)
        if ns["status"] != "nan":
            b.axpby(f, self.x, -1.0, 1.0)
        return ns
