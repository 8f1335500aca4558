#!/usr/bin/env python3
"""Benchmark: batched applications of the linearized collision operator
L[g] (Algorithm 1) per second on one GB300, N = 32, batch 256, per-instance
background Maxwellians rho ~ U[0.5,2], u_i ~ U[-0.5,0.5], theta ~ U[0.5,2],
g = M * (quartic polynomial, N(0,1) coefficients) + 1e-3 N(0,1) grid noise.

One step = one lbo_apply_linearized call over the whole batch (every kernel
of the path).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
  python bench.py --impl reference   # the CPU oracle on the host cores

Multi-GPU (torchrun): each rank applies L to its own batch (instances are
independent; no data-path collective), value = all ranks' applications /
max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "L[g] applications/sec at N=32 (batch 256, per-instance Maxwellians)"
UNIT = "applications/s"
N_GRID, BOX, BATCH = 32, 8.0, 256
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
# ALU peaks derived from unit counts and the maximum SM clock:
#   FP64: 4 flop/clk/SM (2 DFMA/clk/SM, measured by an FMA probe) x 152 SMs x 2070 MHz
#   FP32: 256 flop/clk/SM (128 FFMA lanes) x 152 SMs x 2070 MHz
PEAK_TFLOPS = {"fp64": 4 * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12,
               "fp32": 256 * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12}
# DRAM bytes (read + write) per launch of the dominant kernel at the benchmark
# workload, from ncu (profiles/*.md); None when not captured for this build.
NCU_TRAFFIC = {("plane_inv_mh_fwd", 32, "fp64"): 82483456, ("f32_gain", 32, "fp32"): 370405376}


def transform_axis_flops(n):
    """Conventional flops of one axis pass of a real 3-D transform of n^3
    points: (2.5 n^3 log2(n^3)) / 3."""
    return 2.5 * n ** 3 * np.log2(n)


# Algorithmic flops per instance of each kernel of the generic path, in axis
# passes of a real 3-D transform (pointwise products counted separately).
KERNEL_AXIS_PASSES = {
    "plane_fwd_ratio": 2, "plane_fwd_u": 2, "plane_fwd_g": 2, "plane_fwd_maxw": 2,
    "plane_inv_mh_fwd": 4, "plane_inv": 2,
    "axis1_fwd": 1, "axis1_inv": 1, "axis1_fwd_mul_inv": 2, "axis1_fwd_acc": 1,
    "axis1_uhat_inv": 1,
}


def dct_pass_flops(n):
    """One pass of the octant DCT-I of u^_j: (n/2+1)^3 outputs, each n/4
    multiply-adds over the paired sums plus the pairing add."""
    hn, q4 = n // 2 + 1, n // 4
    return hn ** 3 * (2 * q4 + 1)


# u^_j kernels: their own work (the octant DCT passes and the weight build),
# not the FFT passes they replace
DCT_KERNELS = {
    "uhat_planes": lambda n, J: 2 * dct_pass_flops(n) + 4 * (n // 2 + 1) ** 3,      # one radial node
    "axis1_uhat_inv": lambda n, J: dct_pass_flops(n),                              # plus its FFT pass
    "f32_uhat": lambda n, J: J * (3 * dct_pass_flops(n) + 4 * (n // 2 + 1) ** 3),  # all radial nodes
}
KERNEL_POINTWISE = {  # flops per grid point per instance
    "plane_inv_mh_fwd": 2, "axis1_fwd_mul_inv": 3, "axis1_fwd_acc": 4, "axis1_uhat_inv": 3, "combine": 5,
}
# Fused FP32 kernels (N = 32): whole real 3-D transforms per instance.
#   head: r^ (1);  uhat: u^_j for every radial node (octant DCT-I, counted
#   by its own work in DCT_KERNELS);  gain: 2 per
#   radial node (psi_j, psi^_j) plus the loss term's 4 (g, M forward and
#   back);  tail: the inverse of L^+ (1).
FUSED_TRANSFORMS = {"f32_head": lambda J: 1, "f32_gain": lambda J: 2 * J + 4, "f32_tail": lambda J: 1}
FUSED_POINTWISE = {"f32_gain": lambda J: 10 * J}


def kernel_flops_per_instance(name, n, J=None):
    J = n if J is None else J
    extra = DCT_KERNELS[name](n, J) if name in DCT_KERNELS else 0
    if name == "f32_uhat":
        return extra
    if name in FUSED_TRANSFORMS:
        return (FUSED_TRANSFORMS[name](J) * 3 * transform_axis_flops(n)
                + FUSED_POINTWISE.get(name, lambda J: 0)(J) * n ** 3)
    return (KERNEL_AXIS_PASSES.get(name, 0) * transform_axis_flops(n)
            + KERNEL_POINTWISE.get(name, 0) * n ** 3 + extra)


def kernel_rooflines(prof, n, batch, peak):
    """Per kernel: average launch time (live CUDA events) and its own
    algorithmic rate against the pipe's peak (TFLOP/s)."""
    out = {}
    for name, (cnt, tot) in sorted(prof.items()):
        per = tot / max(cnt, 1)
        fl = kernel_flops_per_instance(name, n) * batch
        ach = fl / (per * 1e-3) / 1e12 if per > 0 else 0.0
        out[name] = {"launches": cnt, "ms_per_launch": per, "achieved_tflops": ach, "frac": ach / peak}
    return out


def apply_flops_per_instance(n, J):
    """(3J + 6) real 3-D transforms of n^3 points at 2.5 n^3 log2(n^3) flops."""
    return (3 * J + 6) * 3 * transform_axis_flops(n)


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            self.path = "/tmp/lbo_clocks_%d.csv" % os.getpid()
            f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sms.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def dist_setup(backend=None):
    """Rank, world size and local rank from the torchrun environment; for
    world > 1 a process group (NCCL on GPUs, gloo on the host)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(params, g, n, L, omega, seconds):
    """Time the CPU oracle (single process, as it stands) on the leading
    instances of the batch for about `seconds`; returns (outputs, apps/s)."""
    from oracle.linearized import Tables, apply_linearized
    t0 = time.perf_counter()
    tab = Tables(n, L, omega, n)
    outs = []
    b = 0
    while b < params.shape[0] and (b < 2 or time.perf_counter() - t0 < seconds):
        outs.append(apply_linearized(tab, params[b:b + 1], g[b:b + 1])[0])
        b += 1
    dt = time.perf_counter() - t0
    return np.stack(outs), len(outs) / dt


def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_2503_09580_gb300 import workloads
    params, g = workloads.batched_instances(N_GRID, BOX, batch=BATCH, seed=args.seed, noise=1e-3)
    from oracle.linearized import Tables, apply_linearized
    tab = Tables(N_GRID, BOX, args.omega, N_GRID)
    per_step = args.ref_instances
    for w in range(args.warmup):
        apply_linearized(tab, params[:1], g[:1])
    t0 = time.perf_counter()
    for k in range(args.steps):
        s = (k * per_step) % BATCH
        apply_linearized(tab, params[s:s + per_step], g[s:s + per_step])
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "batched L[g], N=32, batch 256 (sampled %d instances per step), "
                               "per-instance Maxwellians, quartic polynomial + 1e-3 noise" % per_step,
                   "N": N_GRID, "box": BOX, "vhs_omega": args.omega, "radial_nodes": N_GRID},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d instances per step, numpy FFT form of Algorithm 1" % per_step},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def newton_leg(precision, kn, nx=128, n=32, L=8.0, residual_precision=None):
    """One modified Newton step of the 1-D steady problem: x in [0, 1], nx
    cells, hard spheres, diffuse walls at theta 1 and 2, initial global
    Maxwellian rho = 1, u = 0, theta = 1.5, sweep-preconditioned FGMRES."""
    import torch
    from paper_2503_09580_gb300 import lbo
    a = (np.arange(n) - n // 2) * (2 * L / n)
    v2 = a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2
    f0 = np.broadcast_to((2 * np.pi * 1.5) ** -1.5 * np.exp(-v2 / 3.0), (nx, n, n, n)).copy()
    mass = (1.0 / nx) * (2 * L / n) ** 3 * f0.sum()
    plan = lbo.Plan(n, L, 0.5, n, precision=precision, hemisphere_p=4)
    solver = plan.solver(kind="slab", nx=nx, x_left=0.0, x_right=1.0, kn=kn, wall_left=(1.0, 0, 0, 0),
                         wall_right=(2.0, 0, 0, 0), total_mass=mass, krylov_rtol=1e-3, krylov_atol=1e-7,
                         krylov_restart=40, krylov_maxit=400, precond="sweep")
    rplan = None
    if residual_precision is not None:
        # the residual's Q(f,f) in its own precision, the Krylov operator in `precision`
        rplan = lbo.Plan(n, L, 0.5, n, precision=residual_precision, hemisphere_p=4)
        solver.set_residual_plan(rplan)
    f = torch.from_numpy(f0).cuda()
    # untimed step on a copy: workspaces, tables and the Q state are set up
    # on first use; the timed step then starts from the same state
    solver.newton_step(f.clone())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = solver.newton_step(f)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = {"ms": 1e3 * dt, "ms_residual": st["ms_residual"], "ms_linear": st["ms_linear"],
           "krylov_iterations": st["krylov_iterations"], "residual_before": st["residual_norm"],
           "linear_residual": st["linear_residual"]}
    solver.close()
    plan.close()
    if rplan is not None:
        rplan.close()
    return out


def newton_to_tol_leg(mode, tol=1e-10, nx=8, n=32, L=8.0):
    """Fourier-flow slab (x in [0, 1], nx cells, hard spheres, walls at theta
    1 and 2, Kn = 1, from a global Maxwellian theta = 1.5) solved to
    |R| < tol: modified Newton steps while they still gain, then
    exact-Jacobian steps.  mode 'fp64': everything FP64; 'mixed': the
    Krylov operator (L, and Q inside the exact Jacobian) in FP32 with the
    residual's Q in FP64."""
    import torch
    from paper_2503_09580_gb300 import lbo
    a = (np.arange(n) - n // 2) * (2 * L / n)
    v2 = a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2
    f0 = np.broadcast_to((2 * np.pi * 1.5) ** -1.5 * np.exp(-v2 / 3.0), (nx, n, n, n)).copy()
    mass = (1.0 / nx) * (2 * L / n) ** 3 * f0.sum()
    p64 = lbo.Plan(n, L, 0.5, n, hemisphere_p=2, mass_fix=1)
    pop = p64 if mode == "fp64" else lbo.Plan(n, L, 0.5, n, hemisphere_p=2, mass_fix=1, precision="fp32")
    kw = dict(kind="slab", nx=nx, x_left=0.0, x_right=1.0, kn=1.0, wall_left=(1.0, 0, 0, 0),
              wall_right=(2.0, 0, 0, 0), total_mass=mass, wall_flux="discrete", krylov_rtol=1e-3,
              krylov_atol=1e-16, krylov_restart=40, krylov_maxit=400, precond="sweep")
    mod = pop.solver(**kw)
    ex = pop.solver(**dict(kw, jacobian="exact", krylov_rtol=1e-6))
    if mode == "mixed":
        mod.set_residual_plan(p64)
        ex.set_residual_plan(p64)
    f = torch.from_numpy(f0).cuda()
    steps, its, prev = [], 0, None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(20):
        use_exact = prev is not None and (prev < 1e-4 or k >= 6)
        st = (ex if use_exact else mod).newton_step(f)
        r = st["residual_norm"]
        steps.append(("exact" if use_exact else "modified", r))
        its += st["krylov_iterations"]
        if r < tol:
            break
        prev = r
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    out = torch.empty_like(f)
    fp64_res = p64.solver(**kw)
    final = fp64_res.residual(f, out)
    for s in (mod, ex, fp64_res):
        s.close()
    return {"seconds": secs, "newton_steps": len(steps), "krylov_iterations": its,
            "final_residual_fp64": final, "history": [[k, float(r)] for k, r in steps]}


def shock_leg(precond, nx=128, n=32, L=8.0, tol=1e-10, coarse_operator="galerkin"):
    """Planar Mach-2 shock: x in [-1, 1], nx cells, hard spheres, Kn = 0.1,
    Rankine-Hugoniot inflow states (gamma = 5/3), tanh start; pseudo-
    transient continuation (dtau from 0.3) with exact-Jacobian Newton steps,
    Krylov operator in FP32 and residual in FP64, until |R| < tol."""
    import torch
    from paper_2503_09580_gb300 import lbo
    gam, mach = 5.0 / 3.0, 2.0
    u1 = mach * np.sqrt(gam)
    r = (gam + 1) * mach ** 2 / ((gam - 1) * mach ** 2 + 2)
    p2 = 1 + 2 * gam / (gam + 1) * (mach ** 2 - 1)
    up, down = (1.0, u1, 0.0, 0.0, 1.0), (r, u1 / r, 0.0, 0.0, p2 / r)
    x = -1.0 + (np.arange(nx) + 0.5) * (2.0 / nx)
    a = (np.arange(n) - n // 2) * (2 * L / n)
    f = []
    for wj in 0.5 * (1 + np.tanh(x / 0.15)):
        rho, uu, _, _, th = [(1 - wj) * p + wj * q for p, q in zip(up, down)]
        f.append(rho * (2 * np.pi * th) ** -1.5 * np.exp(-((a[:, None, None] - uu) ** 2 + a[None, :, None] ** 2
                                                           + a[None, None, :] ** 2) / (2 * th)))
    p32 = lbo.Plan(n, L, 0.5, n, hemisphere_p=2, precision="fp32", mass_fix=1)
    p64 = lbo.Plan(n, L, 0.5, n, hemisphere_p=2, mass_fix=1)
    solver = p32.solver(kind="slab", nx=nx, x_left=-1.0, x_right=1.0, kn=0.1, total_mass=1.0, inflow_left=up,
                        inflow_right=down, krylov_rtol=1e-3, krylov_atol=1e-14, krylov_restart=40,
                        krylov_maxit=600, precond=precond, pseudo_dt=0.3, jacobian="exact",
                        coarse_operator=coarse_operator)
    solver.set_residual_plan(p64)
    tf = torch.from_numpy(np.stack(f)).cuda()
    steps, its = [], 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(30):
        st = solver.newton_step(tf)
        steps.append(float(st["residual_norm"]))
        its += st["krylov_iterations"]
        if st["residual_norm"] < tol:
            break
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    solver.close()
    return {"seconds": secs, "newton_steps": len(steps), "krylov_iterations": its,
            "final_residual": steps[-1], "converged": steps[-1] < tol}


def shock_mixed_leg(nx=64, L=8.0, tol=1e-10, seed=5):
    """Mach-2 shock with a velocity grid per cell: N drawn from {24, 32, 48}
    with probabilities 0.5 / 0.35 / 0.15 (seeded), x in [-1, 1], Kn = 0.1,
    continuation + exact-Jacobian Newton, FP32 operator, FP64 residual per
    N, sweep on the finest grid, until |R| < tol."""
    import torch
    from paper_2503_09580_gb300 import lbo
    gam, mach = 5.0 / 3.0, 2.0
    u1 = mach * np.sqrt(gam)
    r = (gam + 1) * mach ** 2 / ((gam - 1) * mach ** 2 + 2)
    p2 = 1 + 2 * gam / (gam + 1) * (mach ** 2 - 1)
    up, down = (1.0, u1, 0.0, 0.0, 1.0), (r, u1 / r, 0.0, 0.0, p2 / r)
    Ns = (24, 32, 48)
    choice = np.random.default_rng(seed).choice(3, size=nx, p=[0.5, 0.35, 0.15])
    plans = [lbo.Plan(n, L, 0.5, n, hemisphere_p=2, precision="fp32", mass_fix=1) for n in Ns]
    rplans = [lbo.Plan(n, L, 0.5, n, hemisphere_p=2, mass_fix=1) for n in Ns]
    solver = lbo.mixed_solver(plans, list(choice), kind="slab", x_left=-1.0, x_right=1.0, kn=0.1,
                              inflow_left=up, inflow_right=down, krylov_rtol=1e-3, krylov_atol=1e-14,
                              krylov_restart=40, krylov_maxit=600, precond="sweep", pseudo_dt=0.3,
                              jacobian="exact")
    for p in rplans:
        solver.set_residual_plan(p)
    x = -1.0 + (np.arange(nx) + 0.5) * (2.0 / nx)
    cells = []
    for c, wj in zip(choice, 0.5 * (1 + np.tanh(x / 0.15))):
        n = Ns[c]
        rho, uu, _, _, th = [(1 - wj) * a + wj * b for a, b in zip(up, down)]
        a = (np.arange(n) - n // 2) * (2 * L / n)
        cells.append((rho * (2 * np.pi * th) ** -1.5 * np.exp(-((a[:, None, None] - uu) ** 2 + a[None, :, None] ** 2
                                                               + a[None, None, :] ** 2) / (2 * th))).ravel())
    tf = torch.from_numpy(np.concatenate(cells)).cuda()
    steps, its = [], 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(30):
        st = solver.newton_step(tf)
        steps.append(float(st["residual_norm"]))
        its += st["krylov_iterations"]
        if st["residual_norm"] < tol:
            break
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    solver.close()
    return {"workload": "Mach-2 planar shock, %d cells, N per cell from {24, 32, 48} (seeded 0.5/0.35/0.15: "
                        "%d/%d/%d), hard spheres, Kn=0.1; continuation + exact-Jacobian Newton, FP32 operator, "
                        "FP64 residual, sweep preconditioner" % ((nx,) + tuple(int((choice == k).sum()) for k in range(3))),
            "seconds": secs, "newton_steps": len(steps), "krylov_iterations": its, "final_residual": steps[-1],
            "converged": steps[-1] < tol}


def bkw_leg(precision, steps=1, n=64, L=8.0, dt=0.05):
    """Backward-Euler steps of the homogeneous equation with the quadratic
    operator (Maxwell molecules, BKW initial data at K = 0.6), Newton with the
    linearized operator; error against the BKW closed form."""
    import torch
    from paper_2503_09580_gb300 import lbo
    a = (np.arange(n) - n // 2) * (2 * L / n)
    v2 = a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2

    def bkw(t):
        K = 1 - np.exp(-t / 6)
        return ((2 * np.pi * K) ** -1.5 * np.exp(-v2 / (2 * K))
                * ((5 * K - 3) / (2 * K) + (1 - K) / (2 * K * K) * v2))
    t = 6 * np.log(2.5)
    plan = lbo.Plan(n, L, 1.0, n, hemisphere_p=4, precision=precision)
    solver = plan.solver(kind="homogeneous", nx=1, dt=dt, krylov_rtol=1e-10, krylov_atol=0.0,
                         krylov_restart=20, krylov_maxit=100, precond="none")
    fn = torch.from_numpy(bkw(t)[None]).cuda()
    f = fn.clone()
    newton_ms, iters = [], 0
    for _ in range(steps):
        for _ in range(4):
            st = solver.newton_step(f, fn)
            newton_ms.append(st["ms_residual"] + st["ms_linear"])
            iters += 1
        t += dt
        fn.copy_(f)
    ex = bkw(t)
    err = float(np.abs(f.cpu().numpy()[0] - ex).max() / np.abs(ex).max())
    solver.close()
    plan.close()
    return {"newton_step_ms": float(np.median(newton_ms)), "newton_iterations": iters, "steps": steps,
            "final_residual": st["residual_norm"], "rel_err_vs_bkw": err}


def n64_leg(with_oracle, batch=64, steps=3, L=8.0):
    """L[g] applications/s at N = 64 (J = 64, batch 64, benchmark recipe:
    per-instance Maxwellians, quartic polynomial + 1e-3 noise), FP32 and
    FP64; FP32 against FP64 on the whole batch and, with the oracle, both
    against the oracle on one instance."""
    import torch
    from paper_2503_09580_gb300 import lbo, workloads
    n = 64
    params, g = workloads.batched_instances(n, L, batch=batch, seed=7, noise=1e-3)
    tp, tg = torch.from_numpy(params).cuda(), torch.from_numpy(g).cuda()
    res, outs = {}, {}
    for prec in ("fp32", "fp64"):
        plan = lbo.Plan(n, L, 0.5, n, precision=prec)
        out = torch.empty_like(tg)
        for _ in range(2):
            plan.apply_linearized(tp, tg, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.apply_linearized(tp, tg, out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[prec] = {"value": batch / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms}
        outs[prec] = out.cpu().numpy()
        plan.close()
    a, b = outs["fp32"], outs["fp64"]
    res["fp32"]["rel_err_vs_fp64"] = float(max(np.abs(a[i] - b[i]).max() / np.abs(b[i]).max() for i in range(batch)))
    res["fp32"]["speedup_vs_fp64"] = res["fp32"]["value"] / res["fp64"]["value"]
    if with_oracle:
        from oracle.linearized import Tables, apply_linearized
        t0 = time.perf_counter()
        ref = apply_linearized(Tables(n, L, 0.5, n), params[:1], g[:1])[0]
        res["fp64"]["rel_err_vs_oracle"] = float(np.abs(b[0] - ref).max() / np.abs(ref).max())
        res["fp32"]["rel_err_vs_oracle"] = float(np.abs(a[0] - ref).max() / np.abs(ref).max())
        res["oracle_seconds_per_instance"] = time.perf_counter() - t0
    res["workload"] = "batched L[g], N=64, J=64, batch 64, per-instance Maxwellians, quartic + 1e-3 noise"
    return res


def mixed_leg(steps=5):
    """512 cells with N in {24, 32, 48} (about 50/35/15 %, seeded), FP32,
    one plan per N applied as a group replayed from a CUDA graph."""
    import torch
    from paper_2503_09580_gb300 import lbo, workloads
    rng = np.random.Generator(np.random.PCG64(7))
    sizes = rng.choice([24, 32, 48], size=512, p=[0.5, 0.35, 0.15])
    counts = {n: int((sizes == n).sum()) for n in (24, 32, 48)}
    plans, ps, gs, outs = [], [], [], []
    for i, n in enumerate((24, 32, 48)):
        p, g = workloads.batched_instances(n, 8.0, batch=counts[n], seed=100 + i, noise=1e-3)
        plans.append(lbo.Plan(n, 8.0, 0.5, n, precision="fp32"))
        ps.append(torch.from_numpy(p).cuda())
        gs.append(torch.from_numpy(g).cuda())
        outs.append(torch.empty_like(gs[-1]))
    grp = lbo.Group(plans, graph=True)
    for _ in range(3):
        grp.apply_linearized(ps, gs, outs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        grp.apply_linearized(ps, gs, outs)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    grp.close()
    return {"cells": 512, "counts": counts, "ms_per_step": ms, "value": 512 / (ms * 1e-3), "unit": UNIT,
            "precision": "fp32", "graph": True}


def run_ours(args, world, rank, local):
    import torch
    from paper_2503_09580_gb300 import lbo, workloads

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    params, g = workloads.batched_instances(N_GRID, BOX, batch=BATCH, seed=args.seed + rank, noise=1e-3)
    plan = lbo.Plan(N_GRID, BOX, args.omega, N_GRID, precision=args.precision)
    if args.eps is not None:
        plan.set("eps", args.eps)
    if args.moment_fix:
        plan.set("moment_fix", 1)
    tp = torch.from_numpy(params).to(dev)
    tg = torch.from_numpy(g).to(dev)
    out = torch.empty_like(tg)
    stream = torch.cuda.current_stream(dev)
    # radial-node groups per CTA of the fused FP32 kernel, timed on this batch
    jgroups = plan.autotune(tp, tg, out) if not args.no_autotune else 0
    for _ in range(args.warmup):
        plan.apply_linearized(tp, tg, out)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    plan.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        plan.apply_linearized(tp, tg, out)
        launches += plan.last_launches
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1) / args.steps
    prof = plan.profile_read()
    plan.profile(False)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, world)
    value = world * BATCH / (ms_max * 1e-3)

    # dominant kernel and its roofline
    name, (cnt, tot) = max(prof.items(), key=lambda kv: kv[1][1])
    per_launch_ms = tot / max(cnt, 1)
    flops = kernel_flops_per_instance(name, N_GRID) * BATCH
    achieved = flops / (per_launch_ms * 1e-3) / 1e12
    peak = PEAK_TFLOPS[args.precision]
    share = tot / sum(v[1] for v in prof.values())
    traffic = NCU_TRAFFIC.get((name, N_GRID, args.precision))

    # end to end through the same C-ABI call with pinned host buffers
    hp = torch.from_numpy(params).pin_memory()
    hg = torch.from_numpy(g).pin_memory()
    ho = torch.empty_like(hg).pin_memory()
    plan.apply_linearized(hp, hg, ho)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        plan.apply_linearized(hp, hg, ho)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_s = max_over_ranks(e2e_s, world)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": "batched L[g], N=32, batch 256 per GPU, per-instance Maxwellians, "
                               "quartic polynomial + 1e-3 noise",
                   "N": N_GRID, "box": BOX, "vhs_omega": args.omega, "radial_nodes": N_GRID,
                   "batch_per_gpu": BATCH, "precision": args.precision,
                   "eps": args.eps if args.eps is not None else 1e-9,
                   "jgroups": jgroups if jgroups else "default",
                   "parallelism": "replicas (instances sharded, no collective)" if world > 1 else "single GPU",
                   "l2": "inputs 67 MB + outputs 67 MB + workspace 0.41 GB per step > 129 MB L2"},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": "derived: flop/clk/SM x 152 SMs x 2070 MHz",
                     "kernel_share": share, "kernel_ms_per_launch": per_launch_ms,
                     "apply_flops_per_instance": apply_flops_per_instance(N_GRID, N_GRID)},
        "kernel_rooflines": kernel_rooflines(prof, N_GRID, BATCH, peak),
        "e2e": {"value": world * BATCH / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(params.nbytes + g.nbytes), "d2h_bytes_per_step": int(g.nbytes)},
    }
    if clk is not None:
        line["clocks"] = clk
    ref = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        got = out.cpu().numpy()
        ref, cpu_rate = oracle_sample(params, g, N_GRID, BOX, args.omega, args.cpu_seconds)
        k = ref.shape[0]
        err = float(np.abs(got[:k] - ref).max() / np.abs(ref).max())
        line["cpu_baseline"] = {"value": cpu_rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "first %d instances of the batch, numpy FFT form of "
                                          "Algorithm 1, single process" % k}
        line["rel_err_vs_oracle"] = {"value": err, "instances": k,
                                     "metric": "max|gpu - oracle| / max|oracle| over the sampled instances"}
    if args.precision != "fp64" and not args.no_fp64_leg:
        # the plain FP64 GPU path on the same inputs, same timing method
        p64 = lbo.Plan(N_GRID, BOX, args.omega, N_GRID, precision="fp64")
        out64 = torch.empty_like(tg)
        for _ in range(2):
            p64.apply_linearized(tp, tg, out64)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p64.profile(True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            p64.apply_linearized(tp, tg, out64)
        f1.record(stream)
        torch.cuda.synchronize()
        prof64 = p64.profile_read()
        p64.profile(False)
        ms64 = max_over_ranks(f0.elapsed_time(f1) / args.fp64_steps, world)
        line["fp64_plain"] = {"value": world * BATCH / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                              "speedup_of_value": value / (world * BATCH / (ms64 * 1e-3)),
                              "kernel_rooflines": kernel_rooflines(prof64, N_GRID, BATCH, PEAK_TFLOPS["fp64"])}
        if ref is not None:
            k = ref.shape[0]
            got64 = out64.cpu().numpy()[:k]
            line["fp64_plain"]["rel_err_vs_oracle"] = float(np.abs(got64 - ref).max() / np.abs(ref).max())
        p64.close()
    if rank == 0 and world == 1 and not args.no_extra:
        line["newton_step"] = {"workload": "1-D steady slab, 128 cells, N=32, hard spheres, walls theta 1/2, "
                                           "Kn=1, first step from a global Maxwellian theta=1.5",
                               "fp32": newton_leg("fp32", 1.0), "fp64": newton_leg("fp64", 1.0),
                               "fp32_operator_fp64_residual": newton_leg("fp32", 1.0, residual_precision="fp64")}
        line["newton_to_1e-10"] = {
            "workload": "1-D steady slab, 8 cells, N=32, hard spheres, walls theta 1/2, Kn=1, from a global "
                        "Maxwellian; modified steps, then exact-Jacobian steps, until |R| < 1e-10",
            "fp64": newton_to_tol_leg("fp64"), "fp32_operator_fp64_residual": newton_to_tol_leg("mixed")}
        line["shock_to_1e-10"] = {
            "workload": "Mach-2 planar shock, 128 cells, N=32, hard spheres, Kn=0.1, Rankine-Hugoniot inflow "
                        "states; continuation + exact-Jacobian Newton, FP32 operator, FP64 residual; "
                        "plain FGMRES (no preconditioner) does not converge on it",
            "sweep": shock_leg("sweep"), "moment_transport": shock_leg("moment", coarse_operator="transport")}
        if args.shock_cells > 0:
            line["shock_mixed_n_to_1e-10"] = shock_mixed_leg(nx=args.shock_cells)
        line["mixed_n"] = mixed_leg()
        line["n64"] = n64_leg(with_oracle=not args.no_cpu_baseline)
        line["bkw_n64"] = {"workload": "homogeneous BKW relaxation, Maxwell molecules, N=64, J=64, M=32, "
                                       "one backward-Euler step dt=0.05 (4 Newton iterations)",
                           "fp32": bkw_leg("fp32"), "fp64": bkw_leg("fp64")}
    line["kernels"] = {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items())}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32"])
    ap.add_argument("--no-fp64-leg", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--omega", type=float, default=0.5)
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--moment-fix", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default radial-node grouping")
    ap.add_argument("--shock-cells", type=int, default=0,
                    help="run the mixed-N shock leg with this many cells (64 cells: about 2.5 minutes)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-instances", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the Newton-step and mixed-N legs")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
