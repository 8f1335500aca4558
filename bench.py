#!/usr/bin/env python3
"""Benchmark: batched applications of the linearized collision operator
L[g] (Algorithm 1) per second on one GB300, N = 32, batch 256, per-instance
background Maxwellians rho ~ U[0.5,2], u_i ~ U[-0.5,0.5], theta ~ U[0.5,2],
g = M * (quartic polynomial, N(0,1) coefficients) + 1e-3 N(0,1) grid noise.

One step = one lbo_apply_linearized call over the whole batch (every kernel
of the path).  The headline value is the plain FP64 path (the paper's
arithmetic); the FP32 form, the VHS exponents 0.5 / 0.74 / 1.0 and the
solver and N = 64 workloads are reported beside it, each precision form
with its measured error against the oracle and its stated bound.  The ALU
peaks of the roofline fractions are measured in the run
(lbo_measure_alu_peaks); the HBM peak is the machine's measured copy bandwidth.
Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
  python bench.py --impl reference   # the CPU oracle on all host cores

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

METRIC = "L[g] applications/sec at N=32,64 vs plain FP64 GPU path at stated rel. error"
UNIT = "applications/s"
N_GRID, BOX, BATCH = 32, 8.0, 256
OMEGAS = (0.5, 0.74, 1.0)
U64, U32 = 2.0 ** -53, 2.0 ** -24
# unit roundoff of the transform arithmetic of each precision form
UNIT_ROUNDOFF = {"fp64": U64, "fp32": U32, "fp32x2": 2.0 ** -48, "fp64x2": 2.0 ** -105,
                 # effective unit of a split 16-bit transform on the tensor cores (BF16 parts; FP16 parts
                 # down to the FP32 accumulation floor)
                 "bf16_split": 2.0 ** -16, "fp16_split": 2.0 ** -21}
# The stated error bound of a precision form, per instance: the normwise
# relative error of the FFT form of Algorithm 1 grows with the size of the
# ratio r = g/M it transforms (Sec. 3.3); measured on the oracle's FFT form in
# FP32 and on the GPU paths, err <= ~0.6 u rms(r) with rms(r) over the whole
# grid (r = 0 where cut).  Stated bound: BOUND_FACTOR u rms(r).
BOUND_FACTOR = 4.0
HBM_FALLBACK_GBS = 6800.0
# Kernels bound by memory traffic, not by their arithmetic (rated in GB/s).
HBM_KERNELS = ("combine", "conservation_fix", "f32_head", "f32_tail", "tc_combine", "mh_table")
# DRAM bytes (read + write) per launch of a dominant kernel at the benchmark
# workload from one ncu capture, with the sha256 (first 16 hex digits) of the
# source files it was built from; reported as null once those sources change.
KERNEL_SOURCES = {
    "plane_inv_mh_fwd": ("lin_reg64.cuh", "fft_reg.cuh", "fft.cuh", "twiddles_hi.h"),
    "f32_gain": ("lin_fused32.cu", "fused32.cuh", "tmem.cuh"),
}
NCU_TRAFFIC = {
    # one capture of k_plane_mh_r64<8> at the benchmark workload: 138.75 MB read + 26.02 MB written
    ("plane_inv_mh_fwd", 32, "fp64"): (164766208, "c353d0056c0cbfeb"),
}


def sources_sha16(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, ()):
        with open(os.path.join(ROOT, "paper_2503_09580_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, n, precision):
    rec = NCU_TRAFFIC.get((kernel, n, precision))
    if rec is None or kernel not in KERNEL_SOURCES or rec[1] != sources_sha16(kernel):
        return None
    return rec[0]


def hbm_peak():
    """(GB/s, source) of the copy bandwidth measured on this machine's GPUs."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (copy bandwidth of this pool's GB300s)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback (one earlier GB300 measurement)"


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
    "axis1_uhat_inv": 1, "axis1_uhat_octant_inv": 1, "axis1_uhat_cached_inv": 1,
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
    "uhat_finish": lambda n, J: dct_pass_flops(n),                                 # axis 1 of the octant
    "uhat_octant": lambda n, J: 3 * dct_pass_flops(n) + 4 * (n // 2 + 1) ** 3,     # all three axes, one node
    "f32_uhat": lambda n, J: J * (3 * dct_pass_flops(n) + 4 * (n // 2 + 1) ** 3),  # all radial nodes
}
KERNEL_POINTWISE = {  # flops per grid point per instance
    "plane_inv_mh_fwd": 2, "axis1_fwd_mul_inv": 3, "axis1_fwd_acc": 4, "axis1_uhat_inv": 3, "combine": 5,
    "axis1_uhat_octant_inv": 3, "axis1_uhat_cached_inv": 3,
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


def kernel_bytes_per_instance(name, n, real_bytes, groups=1):
    """Compulsory HBM bytes per instance of the memory-bound kernels: what
    the kernel must read and write once (FP64 ABI arrays, intermediate
    fields in the transform precision)."""
    n3, h = n ** 3, n * n * (n // 2 + 1)
    if name == "combine":      # L+, u, w (transform precision) and g in; out
        return 3 * real_bytes * n3 + 16 * n3
    if name == "conservation_fix":  # out read and written, twice (moments, then the correction)
        return 32 * n3
    if name == "f32_head":     # g in (FP64); r^ out (FP32 half spectrum)
        return 8 * n3 + 8 * h
    if name == "f32_tail":     # G partial spectra and the FP32 loss field in; out (FP64)
        return groups * 8 * h + 4 * n3 + 8 * n3
    if name == "tc_combine":   # L+, u (FP64), w (FP32), g in; out
        return 8 * n3 * 4 + 4 * n3
    if name == "mh_table":     # M^h / 2 of the register plane kernel out (FP64)
        return 8 * n3
    return 0


def tensor_peak():
    """(TFLOP/s, source): the pool's measured cuBLAS bf16 rate, sustained (a
    tensor kernel timed inside a long step); FP16 has the same dense rate."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["bf16_tflops_sustained"]), "measured (sustained cuBLAS bf16 GEMM)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback (sustained bf16 GEMM of an earlier GB300 measurement)"


def kernel_rooflines(prof, n, batch, peak_tflops, hbm_gbs, real_bytes, groups=1):
    """Per kernel: average launch time (live CUDA events) and its own bound:
    algorithmic flops against the measured ALU peak, or compulsory bytes
    against the measured HBM bandwidth for the memory-bound kernels.  The
    tensor-core passes (tc_*): executed MMA flops (3 split products of the
    (2n x 2n) real DFT matrix per pencil of n complex values: 6 (2n)^2 per
    pencil, n^2 pencils per instance) against the measured sustained tensor
    peak, and their bytes (read and write of a complex FP32 field, plus the
    FP64 input or output of the first and last passes) against HBM."""
    out = {}
    tpk, _ = tensor_peak()
    for name, (cnt, tot) in sorted(prof.items()):
        per = tot / max(cnt, 1)
        rec = {"launches": cnt, "ms_per_launch": per}
        if name.startswith("tc_") and name != "tc_combine":
            fl = 6.0 * (2 * n) ** 2 * n * n * batch
            by = batch * n ** 3 * (8 + 8 + (8 if ("ratio" in name or "_g" in name or "real64" in name) else 0))
            ach = fl / (per * 1e-3) / 1e12 if per > 0 else 0.0
            gbs = by / (per * 1e-3) / 1e9 if per > 0 else 0.0
            rec.update({"bound": "tensor", "achieved_tflops": ach, "frac": ach / tpk, "achieved_gbs": gbs,
                        "frac_of_hbm": gbs / hbm_gbs})
            out[name] = rec
            continue
        if name in HBM_KERNELS:
            by = kernel_bytes_per_instance(name, n, real_bytes, groups) * batch
            ach = by / (per * 1e-3) / 1e9 if per > 0 else 0.0
            rec.update({"bound": "hbm", "achieved_gbs": ach, "frac": ach / hbm_gbs})
        else:
            fl = kernel_flops_per_instance(name, n) * batch
            ach = fl / (per * 1e-3) / 1e12 if per > 0 else 0.0
            rec.update({"bound": "alu", "achieved_tflops": ach, "frac": ach / peak_tflops})
        out[name] = rec
    return out


def apply_flops_per_instance(n, J):
    """(3J + 6) real 3-D transforms of n^3 points at 2.5 n^3 log2(n^3) flops."""
    return (3 * J + 6) * 3 * transform_axis_flops(n)


def ratio_rms(params, g, n, L, eps=1e-9):
    """Per instance: rms over the grid of r = g/M, 0 where the cut-off of
    Eq. (3.9) applies -- the size of what the FFT form transforms."""
    a = (np.arange(n) - n // 2) * (2 * L / n)
    out = []
    for b in range(params.shape[0]):
        rho, u1, u2, u3, th = params[b]
        d2 = (a[:, None, None] - u1) ** 2 + (a[None, :, None] - u2) ** 2 + (a[None, None, :] - u3) ** 2
        M = rho * (2 * np.pi * th) ** -1.5 * np.exp(-d2 / (2 * th))
        keep = d2 / (2 * th) <= np.log(1 / eps) - 1.5 * np.log(2 * np.pi * th)
        r = np.where(keep, g[b] / np.where(keep, M, 1.0), 0.0)
        out.append(float(np.sqrt(np.mean(r * r))))
    return np.array(out)


def error_report(got, ref, rms, unit):
    """Measured normwise relative error per instance against the oracle and
    the stated bound BOUND_FACTOR u rms(r) per instance."""
    k = ref.shape[0]
    errs = np.array([np.abs(got[b] - ref[b]).max() / np.abs(ref[b]).max() for b in range(k)])
    bounds = BOUND_FACTOR * unit * rms[:k]
    return {"rel_err_vs_oracle": float(errs.max()), "stated_bound": float(bounds.max()),
            "worst_err_over_bound": float((errs / bounds).max()), "within_bound": bool(np.all(errs <= bounds)),
            "instances": int(k),
            "metric": "max over instances of max|gpu - oracle| / max|oracle|; bound %g u rms(r) per instance"
                      % BOUND_FACTOR}


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


_W = {}


def _oracle_worker_init(n, L, omega, batch, seed, noise):
    """Pool worker: one numpy thread, the workload regenerated from its seed,
    the oracle's tables built once."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    sys.path.insert(0, ROOT)
    from oracle.linearized import Tables
    from paper_2503_09580_gb300 import workloads
    _W["params"], _W["g"] = workloads.batched_instances(n, L, batch=batch, seed=seed, noise=noise)
    _W["tab"] = Tables(n, L, omega, n)


def _oracle_worker_apply(b):
    from oracle.linearized import apply_linearized
    b = b % _W["params"].shape[0]
    apply_linearized(_W["tab"], _W["params"][b:b + 1], _W["g"][b:b + 1])
    return b


class OraclePool:
    """The oracle on every host core: a spawn-started process pool (no fork
    after CUDA initialisation), one instance per task."""

    def __init__(self, n, L, omega, batch, seed, noise):
        import multiprocessing as mp
        self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init,
                                                 initargs=(n, L, omega, batch, seed, noise))
        self.pool.map(_oracle_worker_apply, range(self.cores), chunksize=1)  # warm every worker

    def run(self, count):
        """Apply the oracle to `count` instances (cycling through the batch)
        on all cores; returns the wall time in seconds."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker_apply, range(count), chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def workload_config(omega, precision):
    return {"workload": "batched L[g], N=32, batch 256 per GPU, per-instance Maxwellians "
                        "rho~U[0.5,2], u_i~U[-0.5,0.5], theta~U[0.5,2], g = M * quartic (N(0,1) coefficients) "
                        "+ 1e-3 N(0,1) grid noise",
            "N": N_GRID, "box": BOX, "vhs_omega": omega, "radial_nodes": N_GRID, "batch_per_gpu": BATCH,
            "precision": precision, "eps": 1e-9}


def run_reference(args, world, rank):
    """The oracle (numpy FFT form of Algorithm 1, FP64) on all host cores,
    each step a bounded sample of the benchmark batch (one instance per
    core)."""
    if rank != 0:
        return
    pool = OraclePool(N_GRID, BOX, args.omega, BATCH, args.seed, 1e-3)
    per_step = pool.cores * args.ref_per_core
    for _ in range(args.warmup):
        pool.run(pool.cores)
    secs = 0.0
    for k in range(args.steps):
        secs += pool.run(per_step)
    pool.close()
    value = per_step * args.steps / secs
    sample = ("%d instances per step (%d per core, cycling through the batch), numpy FFT form of "
              "Algorithm 1 in FP64, one process per core" % (per_step, args.ref_per_core))
    cfg = workload_config(args.omega, "fp64")
    cfg["workload"] += " (sampled %d instances per step)" % per_step
    cfg["l2"] = "host"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_steps(plan, tp, tg, out, steps, stream, profile):
    """CUDA-event time per application of the whole batch on `stream`, the
    per-kernel event totals (profile) and the kernels launched."""
    import torch
    if profile:
        plan.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(steps):
        plan.apply_linearized(tp, tg, out)
        launches += plan.last_launches
    e1.record(stream)
    torch.cuda.synchronize()
    prof = {}
    if profile:
        prof = plan.profile_read()
        plan.profile(False)
    return e0.elapsed_time(e1) / steps, prof, launches


def dominant_roofline(prof, precision, peaks, hbm, hbm_src, groups=1):
    name, (cnt, tot) = max(prof.items(), key=lambda kv: kv[1][1])
    per = tot / max(cnt, 1)
    share = tot / sum(v[1] for v in prof.values())
    real_bytes = 4 if precision == "fp32" else 8
    if name in HBM_KERNELS:
        ach = kernel_bytes_per_instance(name, N_GRID, real_bytes, groups) * BATCH / (per * 1e-3) / 1e9
        rf = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "peak_source": hbm_src}
    else:
        ach = kernel_flops_per_instance(name, N_GRID) * BATCH / (per * 1e-3) / 1e12
        pk = peaks["fp64_tflops"] if precision == "fp64" else peaks["fp32_tflops"]
        rf = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
              "peak_source": "measured in this run (lbo_measure_alu_peaks: dense %s chains, %d SMs at %.0f MHz)"
                             % ("DFMA" if precision == "fp64" else "FFMA", peaks["sm_count"], peaks["sm_mhz"])}
    rf.update({"frac": rf["achieved"] / rf["peak"], "traffic": ncu_traffic(name, N_GRID, precision),
               "kernel": name, "kernel_share": share, "kernel_ms_per_launch": per,
               "apply_flops_per_instance": apply_flops_per_instance(N_GRID, N_GRID)})
    return rf


def variant_leg(precision, tp, tg, tpc, tgc, stream, steps, peaks, hbm, ref, ref_clean, rms, rms_clean, k_clean,
                kernel=0):
    """Another precision form (or kernel set) on the same inputs: apps/s
    (same event timing), its kernels' rooflines, and its error against the
    oracle with the stated bound, on the noisy benchmark batch and on its
    noise-free twin."""
    import torch
    from paper_2503_09580_gb300 import lbo
    plan = lbo.Plan(N_GRID, BOX, 0.5, N_GRID, precision=precision, kernel=kernel)
    out = torch.empty_like(tg)
    groups = plan.autotune(tp, tg, out) if precision == "fp32" else 0
    for _ in range(3):
        plan.apply_linearized(tp, tg, out)
    torch.cuda.synchronize()
    ms, prof, launches = time_steps(plan, tp, tg, out, steps, stream, True)
    unit = UNIT_ROUNDOFF[precision]
    real_bytes = 8 if precision in ("fp64", "fp32x2") else 4
    # the pairs of FP32 run on the FP32 pipe: their algorithmic (FP64-class)
    # flop rate is rated against the FFMA peak, and also shown against the
    # DFMA peak of the FP64 form they replace
    peak = peaks["fp64_tflops"] if precision == "fp64" else peaks["fp32_tflops"]
    kr = kernel_rooflines(prof, N_GRID, BATCH, peak, hbm, real_bytes, groups or 1)
    if precision == "fp32x2":
        for rec in kr.values():
            if "achieved_tflops" in rec:
                rec["frac_of_fp64_peak"] = rec["achieved_tflops"] / peaks["fp64_tflops"]
    res = {"value": BATCH / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "gpu_launches_per_step": launches // steps, "jgroups": groups or "n/a", "kernel_rooflines": kr}
    if ref is not None:
        got = out.cpu().numpy()
        res["accuracy_noisy"] = error_report(got, ref, rms, unit)
        outc = torch.empty_like(tgc)
        plan.apply_linearized(tpc, tgc, outc)
        torch.cuda.synchronize()
        res["accuracy_noise_free"] = error_report(outc.cpu().numpy()[:k_clean], ref_clean, rms_clean, unit)
    plan.close()
    return res


def omega_sweep(tp, tg, tpc, tgc, params, g, pc, gc, stream, steps, with_oracle, k=3):
    """The FP64 plain path at the three VHS exponents of the benchmark
    workload: apps/s and error against the oracle (noise-free twin: 1e-12
    bar; noisy input: stated bound), k sampled instances each."""
    import torch
    from paper_2503_09580_gb300 import lbo
    from oracle.linearized import Tables, apply_linearized
    res = {}
    rms = ratio_rms(params[:k], g[:k], N_GRID, BOX)
    for om in OMEGAS:
        plan = lbo.Plan(N_GRID, BOX, om, N_GRID)
        out = torch.empty_like(tg)
        for _ in range(2):
            plan.apply_linearized(tp, tg, out)
        torch.cuda.synchronize()
        ms, _, _ = time_steps(plan, tp, tg, out, steps, stream, False)
        rec = {"value": BATCH / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps}
        if with_oracle:
            tab = Tables(N_GRID, BOX, om, N_GRID)
            rec["accuracy_noisy"] = error_report(out.cpu().numpy()[:k], apply_linearized(tab, params[:k], g[:k]),
                                                 rms, U64)
            plan.apply_linearized(tpc, tgc, out)
            torch.cuda.synchronize()
            refc = apply_linearized(tab, pc[:k], gc[:k])
            errc = float(max(np.abs(out.cpu().numpy()[b] - refc[b]).max() / np.abs(refc[b]).max()
                             for b in range(k)))
            rec["rel_err_noise_free"] = errc
            rec["noise_free_within_1e-12"] = errc <= 1e-12
        res["omega=%g" % om] = rec
        plan.close()
    return res


def newton_leg(precision, kn, nx=128, n=32, L=8.0, residual_precision=None, device_krylov=False):
    """One modified Newton step of the 1-D steady problem: x in [0, 1], nx
    cells, hard spheres, diffuse walls at theta 1 and 2, initial global
    Maxwellian rho = 1, u = 0, theta = 1.5, sweep-preconditioned FGMRES
    (device_krylov: the Arnoldi kept on the device, cycles as CUDA graphs)."""
    import torch
    from paper_2503_09580_gb300 import lbo
    a = (np.arange(n) - n // 2) * (2 * L / n)
    v2 = a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2
    f0 = np.broadcast_to((2 * np.pi * 1.5) ** -1.5 * np.exp(-v2 / 3.0), (nx, n, n, n)).copy()
    mass = (1.0 / nx) * (2 * L / n) ** 3 * f0.sum()
    plan = lbo.Plan(n, L, 0.5, n, precision=precision, hemisphere_p=4)
    solver = plan.solver(kind="slab", nx=nx, x_left=0.0, x_right=1.0, kn=kn, wall_left=(1.0, 0, 0, 0),
                         wall_right=(2.0, 0, 0, 0), total_mass=mass, krylov_rtol=1e-3, krylov_atol=1e-7,
                         krylov_restart=40, krylov_maxit=400, precond="sweep", device_krylov=device_krylov)
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


def bkw_leg(op_precision, res_precision=None, steps=1, n=64, L=8.0, dt=0.05, tol=1e-10, max_newton=4):
    """Backward-Euler steps dt of the homogeneous equation with the quadratic
    operator (Maxwell molecules, N = 64, J = 64, M = 32; BKW initial data at
    K = 0.6), each solved by Newton with the linearized operator about the
    state's Maxwellian (op_precision; the residual's Q(f,f) in res_precision
    when given) until |F| < tol.  Error against the BKW closed form after
    every step (the time discretisation dominates it: O(dt))."""
    import torch
    from paper_2503_09580_gb300 import lbo
    a = (np.arange(n) - n // 2) * (2 * L / n)
    v2 = a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2

    def bkw(t):
        K = 1 - np.exp(-t / 6)
        return ((2 * np.pi * K) ** -1.5 * np.exp(-v2 / (2 * K))
                * ((5 * K - 3) / (2 * K) + (1 - K) / (2 * K * K) * v2))
    t = 6 * np.log(2.5)
    plan = lbo.Plan(n, L, 1.0, n, hemisphere_p=4, precision=op_precision)
    solver = plan.solver(kind="homogeneous", nx=1, dt=dt, krylov_rtol=1e-10, krylov_atol=0.0,
                         krylov_restart=20, krylov_maxit=100, precond="none")
    rplan = None
    if res_precision is not None:
        rplan = lbo.Plan(n, L, 1.0, n, hemisphere_p=4, precision=res_precision)
        solver.set_residual_plan(rplan)
    fn = torch.from_numpy(bkw(t)[None]).cuda()
    f = fn.clone()
    newton_ms, iters, errs, finals = [], [], [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        k = 0
        for k in range(1, max_newton + 1):
            st = solver.newton_step(f, fn)
            newton_ms.append(st["ms_residual"] + st["ms_linear"])
            if st["residual_norm"] < tol:
                break
        finals.append(st["residual_norm"])
        iters.append(k)
        t += dt
        fn.copy_(f)
        ex = bkw(t)
        errs.append(float(np.abs(f.cpu().numpy()[0] - ex).max() / np.abs(ex).max()))
    secs = time.perf_counter() - t0
    state = f.cpu().numpy()[0]
    solver.close()
    plan.close()
    if rplan is not None:
        rplan.close()
    marks = [i for i in (1, 10, 50, 100, 200) if i <= steps]
    return {"operator": op_precision, "residual": res_precision or op_precision, "steps": steps,
            "seconds": secs, "newton_iteration_ms": float(np.median(newton_ms)),
            "newton_iterations_per_step": float(np.mean(iters)), "max_residual_at_exit": float(max(finals)),
            "rel_err_vs_bkw_at_step": {str(i): errs[i - 1] for i in marks}, "max_rel_err_vs_bkw": max(errs),
            "_state": state}


def bkw_study(steps=200, ref_steps=20):
    """Config 3: 200 backward-Euler steps with an FP64-class residual (Q in
    pairs of FP32) and an FP32 or BF16-split (tensor-core) Jacobian; the
    all-FP64 run of the first ref_steps steps as the reference state."""
    out = {"workload": "homogeneous BKW relaxation, Maxwell molecules, N=64, J=64, M=32, backward Euler "
                       "dt=0.05 from K=0.6, Newton to |F| < 1e-10 (at most 4 iterations per step)"}
    ref = bkw_leg("fp64", steps=ref_steps)
    runs = {"fp32_operator_fp32x2_residual": bkw_leg("fp32", "fp32x2", steps=steps),
            "bf16_split_operator_fp32x2_residual": bkw_leg("bf16_split", "fp32x2", steps=ref_steps),
            "fp32_operator_fp32_residual": bkw_leg("fp32", steps=ref_steps)}
    r = ref.pop("_state")
    out["fp64"] = ref
    for k, v in runs.items():
        # the state after ref_steps steps (a short rerun for the long run)
        s = v["_state"] if v["steps"] == ref_steps else bkw_leg(v["operator"], v["residual"], steps=ref_steps)["_state"]
        v.pop("_state")
        v["rel_diff_vs_fp64_at_step_%d" % ref_steps] = float(np.abs(s - r).max() / np.abs(r).max())
        out[k] = v
    return out


def lin_vs_bin_leg(case, t_end=10.0, dt=0.1, ps=(2, 3, 4), fixes=True):
    """Sec. 4.2: df/dt = Q(f,f) and df/dt = L_M[f] (M the standard normal)
    by RK4 (dt = 0.1) from the paper's f^(1) (Case 1, Maxwell molecules) or
    f^(2) (Case 2, omega = 0.72), R = 6, N_p = 16, 17 radial nodes; Q with
    the product hemisphere rules of M = 2 p^2 points (the paper's Lebedev
    rules of 7 to 25 points are not available).  Reports E(t) (Eq. (4.3)),
    the L2 distances between the two solutions and to the Maxwellian at
    t_end, the mass drift, the mass-fixed variants of Sec. 4.2, and the time
    of 100 steps of each (Table 5's comparison)."""
    import torch
    from paper_2503_09580_gb300 import lbo, workloads
    n, R, J = 32, 6.0, 17
    L = (3 + np.sqrt(2)) * R / 4
    om = 1.0 if case == 1 else 0.72
    f0 = (workloads.paper_f1 if case == 1 else workloads.paper_f2)(n, L)[None]
    h3 = (2 * L / n) ** 3
    std = torch.tensor([[1.0, 0.0, 0.0, 0.0, 1.0]], dtype=torch.float64, device="cuda")
    a = workloads.velocity_axis(n, L)
    Mx = (2 * np.pi) ** -1.5 * np.exp(-(a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2) / 2)
    l2 = lambda x: float(np.sqrt(h3 * (x * x).sum()))
    nrec = int(round(t_end))
    per = int(round(1.0 / dt))

    def run(plan, mode):
        tf = torch.from_numpy(f0.copy()).cuda()
        snaps = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(nrec):
            plan.evolve(mode, tf, dt, per, params=std if mode == "linearized" else None)
            snaps.append(tf.cpu().numpy()[0])
        secs = time.perf_counter() - t0
        return snaps, secs * 100 / (nrec * per)  # seconds per 100 steps

    res = {"case": case, "omega": om, "N": n, "R": R, "L": L, "radial_nodes": J, "dt": dt, "t_end": t_end}
    lin, tl = run(lbo.Plan(n, L, om, J, R=R), "linearized")
    res["linearized"] = {"seconds_per_100_steps": tl, "l2_to_maxwellian": l2(lin[-1] - Mx),
                         "mass_drift": abs(h3 * lin[-1].sum() / (h3 * f0.sum()) - 1)}
    for p in ps:
        bins, tb = run(lbo.Plan(n, L, om, J, R=R, hemisphere_p=p), "quadratic")
        E = [l2(x - y) / l2(y) for x, y in zip(lin, bins)]
        res["quadratic_M%d" % (2 * p * p)] = {
            "seconds_per_100_steps": tb, "time_ratio_to_linearized": tb / tl,
            "l2_to_maxwellian": l2(bins[-1] - Mx), "mass_drift": abs(h3 * bins[-1].sum() / (h3 * f0.sum()) - 1),
            "l2_diff_to_linearized": [l2(x - y) for x, y in zip(lin, bins)], "E_t": E, "E_max": max(E)}
    if fixes:
        linf, _ = run(lbo.Plan(n, L, om, J, R=R, mass_fix=1), "linearized")
        res["linearized_mass_fix"] = {"mass_drift": abs(h3 * linf[-1].sum() / (h3 * f0.sum()) - 1),
                                      "l2_to_maxwellian": l2(linf[-1] - Mx)}
        for name, kw in (("zero_mode", {"mass_fix": 1}), ("sinc_quadrature", {"q_sinc_quadrature": 1})):
            p = ps[-1]
            bf, _ = run(lbo.Plan(n, L, om, J, R=R, hemisphere_p=p, **kw), "quadratic")
            res["quadratic_M%d_%s" % (2 * p * p, name)] = {
                "mass_drift": abs(h3 * bf[-1].sum() / (h3 * f0.sum()) - 1), "l2_to_maxwellian": l2(bf[-1] - Mx),
                "l2_diff_to_linearized_mass_fix": l2(bf[-1] - linf[-1])}
    return res


def steady_counts_leg(flow, kn, param, precision="fp64", nx=200, n=32, tol=1e-5, max_newton=12, p=4,
                      wall_flux="analytic", q_sinc=False, inner_solver="source_iteration", krylov_rtol=1e-3,
                      jacobian="local_maxwellian", box_factor=1.0, nu_scale=1.0):
    """Sec. 5.3: Newton iterations of the modified Newton method with the
    paper's source iteration (nu_j = rho_j, stop at 1e-7 absolute or 1e-3
    relative) to |R| < 1e-5 for the Couette flow (walls theta = 1 moving at
    -+u_W along v2; param = u_W) or the Fourier flow (theta_L = 1,
    theta_R = param, walls at rest); Maxwell molecules, x in [-0.5, 0.5],
    C = 1, 200 cells, N_p = 16, R = 3.5 (4 for theta_R >= 2.5), L =
    (3 + sqrt 2) R / 4, 17 radial nodes, initial guess of the supplement
    (the total density with the wall temperatures interpolated linearly).
    wall_flux: the wall density factor sqrt(2 pi / theta_w) of the
    supplement ("analytic") or the grid sum of the wall's flux ("discrete");
    q_sinc: Q with the sinc quadrature of Eq. (2.16) (exact discrete mass);
    box_factor: the velocity box L as a multiple of the smallest one the
    dealiasing condition of Sec. 2.3 allows, (3 + sqrt 2) R / 4."""
    import torch
    from paper_2503_09580_gb300 import lbo
    R = 4.0 if (flow == "fourier" and param >= 2.5) else 3.5
    L = box_factor * (3 + np.sqrt(2)) * R / 4
    if flow == "couette":
        wl, wr, thl, thr = (1.0, 0.0, -param, 0.0), (1.0, 0.0, param, 0.0), 1.0, 1.0
    else:
        wl, wr, thl, thr = (1.0, 0.0, 0.0, 0.0), (param, 0.0, 0.0, 0.0), 1.0, param
    xl, xr, C = -0.5, 0.5, 1.0
    x = xl + (np.arange(nx) + 0.5) * (xr - xl) / nx
    a = (np.arange(n) - n // 2) * (2 * L / n)
    v2 = a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2
    th = (xr - x) / (xr - xl) * thl + (x - xl) / (xr - xl) * thr
    f0 = np.stack([C / (xr - xl) * (2 * np.pi * t) ** -1.5 * np.exp(-v2 / (2 * t)) for t in th])
    plan = lbo.Plan(n, L, 1.0, 17, R=R, hemisphere_p=p, precision=precision, q_sinc_quadrature=int(q_sinc))
    solver = plan.solver(kind="slab", nx=nx, x_left=xl, x_right=xr, kn=kn, wall_left=wl, wall_right=wr,
                         total_mass=C, wall_flux=wall_flux, krylov_rtol=krylov_rtol, krylov_atol=1e-7, krylov_maxit=5000,
                         precond="sweep", inner=inner_solver, nu_scale=nu_scale, jacobian=jacobian)
    f = torch.from_numpy(f0).cuda()
    work = torch.empty_like(f)
    hist, inner, ms_res, ms_lin = [], [], 0.0, 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max_newton + 1):
        r = solver.residual(f, work)
        hist.append(r)
        if r < tol or len(inner) == max_newton:
            break
        st = solver.newton_step(f)
        inner.append(st["krylov_iterations"])
        ms_res += st["ms_residual"]
        ms_lin += st["ms_linear"]
    secs = time.perf_counter() - t0
    solver.close()
    plan.close()
    return {"flow": flow, "kn": kn, "param": param, "R": R, "wall_flux": wall_flux, "q_sinc": bool(q_sinc),
            "inner_solver": inner_solver, "krylov_rtol": krylov_rtol, "jacobian": jacobian, "p": p, "box": L,
            "nu_scale": nu_scale,
            "newton_iterations": len(inner),
            "converged": hist[-1] < tol, "residual_history": hist, "inner_iterations": inner,
            "seconds": secs, "share_residual_Q": ms_res / max(ms_res + ms_lin, 1e-9)}


def paper_newton_tables(precision="fp64", wall_flux="discrete", q_sinc=True, max_newton=8):
    """Tables 6 and 8 of Sec. 5.3 on the GPU.  By default with the wall
    flux summed on the grid and Q with the sinc quadrature of Eq. (2.16):
    the discrete problem then balances mass exactly, which the stopping
    threshold 1e-5 needs (with the printed factor sqrt(2 pi / theta_w) the
    grid sum of the wall's half-range flux is off by about h^2/12, and the
    residual stalls near 7e-4 at N_p = 16)."""
    out = {"precision": precision, "wall_flux": wall_flux, "q_sinc": q_sinc, "couette": {}, "fourier": {}}
    cases = [("couette", kn, uw) for kn in (0.1, 1.0, 10.0) for uw in (0.1, 0.2, 0.3, 0.4, 0.5)]
    cases += [("fourier", kn, tr) for kn in (0.1, 1.0, 10.0) for tr in (1.5, 2.0, 2.5, 3.0)]
    for flow, kn, prm in cases:
        key = ("Kn=%g,u_W=%g" if flow == "couette" else "Kn=%g,theta_R=%g") % (kn, prm)
        try:
            out[flow][key] = steady_counts_leg(flow, kn, prm, precision, max_newton=max_newton,
                                               wall_flux=wall_flux, q_sinc=q_sinc)
        except Exception as e:  # record the failure and go on with the next case
            out[flow][key] = {"error": str(e)}
        print(json.dumps({flow: {key: out[flow][key]}}), file=sys.stderr, flush=True)
    return out


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
    precs = ("fp32", "fp16_split", "bf16_split", "fp32x2", "fp64")
    for prec in precs:
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
    b = outs["fp64"]
    for prec in precs[:-1]:
        a = outs[prec]
        res[prec]["rel_err_vs_fp64"] = float(max(np.abs(a[i] - b[i]).max() / np.abs(b[i]).max() for i in range(batch)))
        res[prec]["speedup_vs_fp64"] = res[prec]["value"] / res["fp64"]["value"]
    if with_oracle:
        from oracle.linearized import Tables, apply_linearized
        t0 = time.perf_counter()
        ref = apply_linearized(Tables(n, L, 0.5, n), params[:1], g[:1])[0]
        res["oracle_seconds_per_instance"] = time.perf_counter() - t0
        rms = ratio_rms(params[:1], g[:1], n, L)[0]
        for prec in precs:
            res[prec]["rel_err_vs_oracle"] = float(np.abs(outs[prec][0] - ref).max() / np.abs(ref).max())
            res[prec]["stated_bound"] = BOUND_FACTOR * UNIT_ROUNDOFF[prec] * rms
    res["workload"] = "batched L[g], N=64, J=64, batch 64, per-instance Maxwellians, quartic + 1e-3 noise"
    return res


def quadratic_leg(precision, peaks, batch=128, steps=3, n=32, L=8.0, p=4, kernel=0):
    """Q(f,f) in the M-point form of Eq. (2.14) at N = 32, M = 2 p^2 = 32,
    J = N, hard spheres, on a batch of seeded g = M * quartic instances:
    evaluations/s and the rooflines of its two per-(j, m) kernels (their
    algorithmic work per radial and hemisphere node and instance:
    q_axis1_phase 2 axis passes + the phase products, q_plane_inv_prod 4 axis
    passes + the product)."""
    import torch
    from paper_2503_09580_gb300 import lbo, workloads
    _, g = workloads.batched_instances(n, L, batch=batch, seed=3, noise=0.0)
    tf = torch.from_numpy(g).cuda()
    out = torch.empty_like(tf)
    plan = lbo.Plan(n, L, 0.5, n, precision=precision, hemisphere_p=p, kernel=kernel)
    for _ in range(2):
        plan.apply_quadratic(tf, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.apply_quadratic(tf, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    plan.profile(True)
    plan.apply_quadratic(tf, out)
    torch.cuda.synchronize()
    prof = plan.profile_read()
    plan.profile(False)
    plan.close()
    M, J = 2 * p * p, n
    peak = peaks["fp64_tflops"] if precision == "fp64" else peaks["fp32_tflops"]
    work = {"q_axis1_phase": 2 * transform_axis_flops(n) + 9 * n ** 3,
            "q_plane_inv_prod": 4 * transform_axis_flops(n) + 2 * n ** 3}
    kr = {}
    for name, (cnt, tot) in sorted(prof.items()):
        per = tot / max(cnt, 1)
        rec = {"launches": cnt, "ms_per_launch": per}
        if name in work and precision != "fp32":
            fl = work[name] * batch * (J * M / cnt)  # (j, m) pairs per launch
            rec.update({"bound": "alu", "achieved_tflops": fl / (per * 1e-3) / 1e12})
            rec["frac"] = rec["achieved_tflops"] / peak
        kr[name] = rec
    return {"workload": "Q(f,f), N=32, M=32 hemisphere points, J=32, hard spheres, batch %d" % batch,
            "precision": precision, "kernel_set": {0: "fastest", 2: "shared-memory transforms"}.get(kernel, kernel),
            "ms_per_evaluation": ms, "value": batch / (ms * 1e-3), "unit": "Q evaluations/s",
            "kernel_rooflines": kr}


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
    prec = args.precision
    params, g = workloads.batched_instances(N_GRID, BOX, batch=BATCH, seed=args.seed + rank, noise=1e-3)
    tp, tg = torch.from_numpy(params).to(dev), torch.from_numpy(g).to(dev)
    stream = torch.cuda.current_stream(dev)
    peaks = lbo.measure_alu_peaks(stream)
    hbm, hbm_src = hbm_peak()
    plan = lbo.Plan(N_GRID, BOX, args.omega, N_GRID, precision=prec)
    if args.eps is not None:
        plan.set("eps", args.eps)
    if args.moment_fix:
        plan.set("moment_fix", 1)
    out = torch.empty_like(tg)
    # launch shape timed on this batch: radial-node groups per CTA of the
    # fused FP32 kernel, or planes per CTA of the FP64 register plane kernel
    shape = plan.autotune(tp, tg, out) if prec in ("fp32", "fp64") and not args.no_autotune else 0
    jgroups = shape if prec == "fp32" else 0
    for _ in range(args.warmup):
        plan.apply_linearized(tp, tg, out)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, prof, launches = time_steps(plan, tp, tg, out, args.steps, stream, True)
    barrier(world)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, world)
    value = world * BATCH / (ms_max * 1e-3)
    real_bytes = 4 if prec == "fp32" else 8
    peak = peaks["fp64_tflops"] if prec == "fp64" else peaks["fp32_tflops"]

    # end to end through the same C-ABI call with pinned host buffers
    hp = torch.from_numpy(params).pin_memory()
    hg = torch.from_numpy(g).pin_memory()
    ho = torch.empty_like(hg).pin_memory()
    plan.apply_linearized(hp, hg, ho)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        plan.apply_linearized(hp, hg, ho)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, world)

    cfg = workload_config(args.omega, prec)
    cfg.update({"eps": args.eps if args.eps is not None else 1e-9,
                "jgroups": jgroups if jgroups else "n/a",
                "planes_per_cta": shape if prec == "fp64" and shape else "n/a",
                "parallelism": "replicas (instances sharded, no collective)" if world > 1 else "single GPU",
                "l2": "inputs 67 MB + outputs 67 MB + workspace per step > 129 MB L2"})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp32x2": "f32x2"}[prec], "data": "synthetic",
        "config": cfg, "gpu_launches": launches,
        "roofline": dominant_roofline(prof, prec, peaks, hbm, hbm_src, jgroups or 1),
        "kernel_rooflines": kernel_rooflines(prof, N_GRID, BATCH, peak, hbm, real_bytes, jgroups or 1),
        "measured_peaks": dict(peaks, hbm_gbs=hbm, hbm_source=hbm_src),
        "e2e": {"value": world * BATCH / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(params.nbytes + g.nbytes), "d2h_bytes_per_step": int(g.nbytes)},
    }
    if clk is not None:
        line["clocks"] = clk
    solo = rank == 0 and world == 1
    ref = ref_c = rms = rms_c = None
    k_clean = 4
    pc, gc = workloads.batched_instances(N_GRID, BOX, batch=BATCH, seed=args.seed + rank, noise=0.0)
    tpc, tgc = torch.from_numpy(pc).to(dev), torch.from_numpy(gc).to(dev)
    if solo and not args.no_cpu_baseline:
        got = out.cpu().numpy()
        ref, rate1 = oracle_sample(params, g, N_GRID, BOX, args.omega, args.cpu_seconds)
        k = ref.shape[0]
        rms = ratio_rms(params[:k], g[:k], N_GRID, BOX)
        from oracle.linearized import Tables, apply_linearized
        ref_c = apply_linearized(Tables(N_GRID, BOX, args.omega, N_GRID), pc[:k_clean], gc[:k_clean])
        rms_c = ratio_rms(pc[:k_clean], gc[:k_clean], N_GRID, BOX)
        unit = UNIT_ROUNDOFF[prec]
        line["accuracy_noisy"] = error_report(got[:k], ref, rms, unit)
        outc = torch.empty_like(tgc)
        plan.apply_linearized(tpc, tgc, outc)
        torch.cuda.synchronize()
        acc_c = error_report(outc.cpu().numpy()[:k_clean], ref_c, rms_c, unit)
        if prec == "fp64":
            acc_c["within_1e-12"] = acc_c["rel_err_vs_oracle"] <= 1e-12
        line["accuracy_noise_free"] = acc_c
        pool = OraclePool(N_GRID, BOX, args.omega, BATCH, args.seed, 1e-3)
        count = max(pool.cores, int(rate1 * pool.cores * args.cpu_seconds))
        secs = pool.run(count)
        pool.close()
        line["cpu_baseline"] = {
            "value": count / secs, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": "%d instances of the benchmark batch (cycling), numpy FFT form of Algorithm 1 in FP64, "
                      "one process per host core" % count,
            "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                            "sample": "first %d instances of the batch, one process" % k}}
    if solo and not args.no_variants:
        line["variants"] = {}
        for vp in ("fp32x2", "fp32", "fp16_split", "bf16_split", "fp64"):
            if vp == prec:
                continue
            rec = variant_leg(vp, tp, tg, tpc, tgc, stream, args.steps, peaks, hbm, ref, ref_c, rms, rms_c,
                              k_clean)
            rec["speedup_vs_value"] = rec["value"] / value
            line["variants"][vp] = rec
        if prec == "fp64":
            # the same FP64 path with the two-stage shared-memory transforms
            # (LBO_OPT_KERNEL = 2) in place of the register kernels
            rec = variant_leg("fp64", tp, tg, tpc, tgc, stream, args.steps, peaks, hbm, ref, ref_c, rms, rms_c,
                              k_clean, kernel=2)
            rec["speedup_vs_value"] = rec["value"] / value
            line["variants"]["fp64_shared_memory_transforms"] = rec
        line["omega_sweep_fp64"] = omega_sweep(tp, tg, tpc, tgc, params, g, pc, gc, stream, min(args.steps, 10),
                                               not args.no_cpu_baseline)
    if solo and not args.no_extra:
        line["newton_step"] = {"workload": "1-D steady slab, 128 cells, N=32, hard spheres, walls theta 1/2, "
                                           "Kn=1, first step from a global Maxwellian theta=1.5",
                               "fp32": newton_leg("fp32", 1.0), "fp64": newton_leg("fp64", 1.0),
                               "fp32_operator_fp64_residual": newton_leg("fp32", 1.0, residual_precision="fp64"),
                               "fp32_operator_fp32x2_residual": newton_leg("fp32", 1.0, residual_precision="fp32x2"),
                               "fp32_device_krylov": newton_leg("fp32", 1.0, device_krylov=True),
                               "fp64_device_krylov": newton_leg("fp64", 1.0, device_krylov=True)}
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
        line["quadratic"] = {"fp64": quadratic_leg("fp64", peaks),
                             "fp64_shared_memory_transforms": quadratic_leg("fp64", peaks, kernel=2),
                             "fp32": quadratic_leg("fp32", peaks)}
        line["mixed_n"] = mixed_leg()
        line["n64"] = n64_leg(with_oracle=not args.no_cpu_baseline)
        if args.lin_vs_bin:
            line["lin_vs_bin"] = {"case1": lin_vs_bin_leg(1), "case2": lin_vs_bin_leg(2)}
        line["bkw_n64"] = bkw_study(steps=args.bkw_steps)
    line["kernels"] = {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items())}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fp32x2"],
                    help="precision of the headline value (the other forms are reported as variants)")
    ap.add_argument("--no-variants", action="store_true", help="skip the other precision forms and the omega sweep")
    ap.add_argument("--omega", type=float, default=0.5)
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--moment-fix", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default radial-node grouping")
    ap.add_argument("--shock-cells", type=int, default=0,
                    help="run the mixed-N shock leg with this many cells (64 cells: about 2.5 minutes)")
    ap.add_argument("--lin-vs-bin", action="store_true",
                    help="run the homogeneous linearized-vs-quadratic study of Sec. 4.2 (about a minute)")
    ap.add_argument("--bkw-steps", type=int, default=200, help="backward-Euler steps of the BKW leg")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-per-core", type=int, default=1, help="reference arm: instances per core per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the Newton-step and mixed-N legs")
    ap.add_argument("--q-only", action="store_true",
                    help="only the Q(f,f) leg (N=32, M=32, batch 128; FP64 and FP32), one JSON line")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.q_only:
        import torch
        from paper_2503_09580_gb300 import lbo
        peaks = lbo.measure_alu_peaks(torch.cuda.current_stream())
        print(json.dumps({"quadratic": {"fp64": quadratic_leg("fp64", peaks), "fp32": quadratic_leg("fp32", peaks)},
                          "measured_peaks": peaks}), flush=True)
        return
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
