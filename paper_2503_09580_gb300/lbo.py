"""Thin Python binding of liblbo.so (include/lbo.h): argument marshalling
only.  Every step of the operators runs in the library's CUDA kernels; if
the library is missing this module raises instead of computing anything.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays, float64,
C-contiguous.  CUDA tensors are passed as device pointers and the call is
asynchronous on torch's current stream; host arrays go through the
library's staged-copy path (the call returns with the result in host
memory).
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "liblbo.so")

LBO_OPT = {"R": 0, "C": 1, "eps": 2, "cutoff": 3, "mass_fix": 4, "moment_fix": 5,
           "hemisphere_p": 6, "precision": 7, "kernel": 8, "jgroups": 9, "q_sinc_quadrature": 10, "planes": 11}
PRECISION = {"fp64": 0, "fp32": 1, "fp32x2": 2, "fp64x2": 3, "bf16_split": 4, "fp16_split": 5}
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "not converged",
          5: "Krylov breakdown", 6: "non-finite value", 7: "unsupported configuration",
          8: "a kernel's bounded wait ran out"}

# Every symbol include/lbo.h declares (checked by the tests).
EXPORTS = ("lbo_plan_create", "lbo_plan_set", "lbo_plan_set_stream", "lbo_apply_linearized",
           "lbo_apply_quadratic", "lbo_plan_sync", "lbo_plan_last_launches", "lbo_plan_destroy",
           "lbo_status_string", "lbo_last_error", "lbo_plan_profile", "lbo_plan_profile_count",
           "lbo_plan_profile_get", "lbo_apply_linearized_noalloc", "lbo_noalloc_scratch_bytes",
           "lbo_noalloc_bytes_per_instance", "lbo_solver_create", "lbo_newton_step", "lbo_solver_residual",
           "lbo_solver_set_residual_plan", "lbo_solver_create_mixed", "lbo_solver_state_length",
           "lbo_solver_destroy", "lbo_network_param_count", "lbo_network_loss_grad", "lbo_solver_collect",
           "lbo_solver_pair_count", "lbo_solver_train_network", "lbo_solver_get_network", "lbo_solver_set_network",
           "lbo_solver_network_param_count", "lbo_plan_autotune", "lbo_group_create", "lbo_group_set_stream",
           "lbo_group_use_graph", "lbo_group_apply_linearized", "lbo_group_destroy", "lbo_measure_alu_peaks", "lbo_plan_cache_maxwellians",
           "lbo_dft_axis_tensor", "lbo_evolve_homogeneous", "lbo_slab_block_transport", "lbo_slab_block_sweep",
           "lbo_slab_block_moments", "lbo_slab_cell_flux", "lbo_slab_maxwellian_cell", "lbo_vec_dots",
           "lbo_vec_axpby", "lbo_vec_combination")

_lib = None


class Problem(ctypes.Structure):
    """lbo_problem"""
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("x_left", ctypes.c_double),
                ("x_right", ctypes.c_double), ("kn", ctypes.c_double), ("wall_left", ctypes.c_double * 4),
                ("wall_right", ctypes.c_double * 4), ("total_mass", ctypes.c_double), ("wall_flux", ctypes.c_int),
                ("dt", ctypes.c_double), ("krylov_rtol", ctypes.c_double), ("krylov_atol", ctypes.c_double),
                ("krylov_restart", ctypes.c_int), ("krylov_maxit", ctypes.c_int), ("precond", ctypes.c_int),
                ("bc_left", ctypes.c_int), ("bc_right", ctypes.c_int), ("inflow_left", ctypes.c_double * 5),
                ("inflow_right", ctypes.c_double * 5), ("line_search", ctypes.c_int),
                ("pseudo_dt", ctypes.c_double), ("coarse_moments", ctypes.c_int),
                ("jacobian", ctypes.c_int), ("coarse_operator", ctypes.c_int), ("inner_solver", ctypes.c_int),
                ("nu_scale", ctypes.c_double), ("device_krylov", ctypes.c_int)]


class NewtonStats(ctypes.Structure):
    """lbo_newton_stats"""
    _fields_ = [("residual_norm", ctypes.c_double), ("rhs_norm", ctypes.c_double),
                ("linear_residual", ctypes.c_double), ("krylov_iterations", ctypes.c_int),
                ("restarts", ctypes.c_int), ("fallbacks", ctypes.c_int), ("status", ctypes.c_int),
                ("ms_residual", ctypes.c_double),
                ("ms_linear", ctypes.c_double), ("step_length", ctypes.c_double),
                ("shift", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PROBLEM = {"slab": 0, "homogeneous": 1}
PRECOND = {"none": 0, "sweep": 1, "learned": 2, "moment": 3}
WALL_FLUX = {"analytic": 0, "discrete": 1}


class LboError(RuntimeError):
    def __init__(self, status, where):
        msg = "%s: %s" % (where, STATUS.get(status, "status %d" % status))
        detail = _lib.lbo_last_error().decode() if _lib is not None else ""
        if detail:
            msg += " (" + detail + ")"
        super().__init__(msg)
        self.status = status


def load():
    """Load liblbo.so (built by paper_2503_09580_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblbo.so not built (%s); run paper_2503_09580_gb300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int
    lib.lbo_plan_create.argtypes = [ip, ctypes.c_double, ctypes.c_double, ip, ctypes.POINTER(vp)]
    lib.lbo_plan_create.restype = ip
    lib.lbo_plan_set.argtypes = [vp, ip, ctypes.c_double]
    lib.lbo_plan_set.restype = ip
    lib.lbo_plan_set_stream.argtypes = [vp, vp]
    lib.lbo_plan_set_stream.restype = ip
    lib.lbo_apply_linearized.argtypes = [vp, dp, dp, dp, ip]
    lib.lbo_apply_linearized.restype = ip
    cd, sz, dpp = ctypes.c_double, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)
    lib.lbo_slab_block_transport.argtypes = [vp, vp, vp, vp, vp, ip, cd]
    lib.lbo_slab_block_sweep.argtypes = [vp, vp, vp, vp, vp, vp, ip, cd, cd, cd, ip]
    lib.lbo_slab_block_moments.argtypes = [vp, vp, ip, vp, vp]
    lib.lbo_slab_cell_flux.argtypes = [vp, vp, ip, dpp]
    lib.lbo_slab_maxwellian_cell.argtypes = [vp, cd, dpp, cd, vp]
    lib.lbo_vec_dots.argtypes = [vp, vp, sz, ip, vp, sz, dpp]
    lib.lbo_vec_axpby.argtypes = [vp, vp, vp, cd, cd, sz]
    lib.lbo_vec_combination.argtypes = [vp, vp, vp, sz, ip, dpp, sz]
    for fn in ("lbo_slab_block_transport", "lbo_slab_block_sweep", "lbo_slab_block_moments", "lbo_slab_cell_flux",
               "lbo_slab_maxwellian_cell", "lbo_vec_dots", "lbo_vec_axpby", "lbo_vec_combination"):
        getattr(lib, fn).restype = ip
    lib.lbo_evolve_homogeneous.argtypes = [vp, ip, dp, dp, ip, ctypes.c_double, ip]
    lib.lbo_evolve_homogeneous.restype = ip
    lib.lbo_dft_axis_tensor.argtypes = [ip, ip, ip, ip, vp, vp, ip, vp]
    lib.lbo_dft_axis_tensor.restype = ip
    lib.lbo_plan_cache_maxwellians.argtypes = [vp, dp, ip]
    lib.lbo_plan_cache_maxwellians.restype = ip
    lib.lbo_apply_quadratic.argtypes = [vp, dp, dp, ip]
    lib.lbo_apply_quadratic.restype = ip
    lib.lbo_plan_sync.argtypes = [vp]
    lib.lbo_plan_sync.restype = ip
    lib.lbo_plan_last_launches.argtypes = [vp]
    lib.lbo_plan_last_launches.restype = ip
    lib.lbo_plan_destroy.argtypes = [vp]
    lib.lbo_plan_destroy.restype = None
    lib.lbo_status_string.argtypes = [ip]
    lib.lbo_status_string.restype = ctypes.c_char_p
    lib.lbo_plan_profile.argtypes = [vp, ip]
    lib.lbo_plan_profile.restype = ip
    lib.lbo_plan_profile_count.argtypes = [vp]
    lib.lbo_plan_profile_count.restype = ip
    lib.lbo_plan_profile_get.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ip),
                                         ctypes.POINTER(ctypes.c_double)]
    lib.lbo_plan_profile_get.restype = ip
    lib.lbo_apply_linearized_noalloc.argtypes = [vp, dp, dp, dp, ip]
    lib.lbo_apply_linearized_noalloc.restype = ip
    lib.lbo_noalloc_scratch_bytes.argtypes = []
    lib.lbo_noalloc_scratch_bytes.restype = ctypes.c_size_t
    lib.lbo_noalloc_bytes_per_instance.argtypes = [vp]
    lib.lbo_noalloc_bytes_per_instance.restype = ctypes.c_size_t
    dpp = ctypes.POINTER(ctypes.c_double)
    lib.lbo_measure_alu_peaks.argtypes = [vp, dpp, dpp, ctypes.POINTER(ip), dpp]
    lib.lbo_measure_alu_peaks.restype = ip
    lib.lbo_solver_create.argtypes = [ctypes.POINTER(Problem), vp, ctypes.POINTER(vp)]
    lib.lbo_solver_create.restype = ip
    lib.lbo_newton_step.argtypes = [vp, dp, dp, ctypes.POINTER(NewtonStats)]
    lib.lbo_newton_step.restype = ip
    lib.lbo_solver_residual.argtypes = [vp, dp, dp, dp, ctypes.POINTER(ctypes.c_double)]
    lib.lbo_solver_residual.restype = ip
    lib.lbo_solver_set_residual_plan.argtypes = [vp, vp]
    lib.lbo_solver_set_residual_plan.restype = ip
    lib.lbo_solver_create_mixed.argtypes = [vp, vp, ip, vp, vp]
    lib.lbo_solver_create_mixed.restype = ip
    lib.lbo_solver_state_length.argtypes = [vp]
    lib.lbo_solver_state_length.restype = ctypes.c_size_t
    lib.lbo_solver_destroy.argtypes = [vp]
    lib.lbo_solver_destroy.restype = None
    lib.lbo_network_param_count.argtypes = [ip]
    lib.lbo_network_param_count.restype = ip
    lib.lbo_network_loss_grad.argtypes = [ip, vp, vp, vp, ip, ip, ctypes.POINTER(ctypes.c_double), vp]
    lib.lbo_network_loss_grad.restype = ip
    lib.lbo_solver_collect.argtypes = [vp, ip]
    lib.lbo_solver_collect.restype = ip
    lib.lbo_solver_pair_count.argtypes = [vp]
    lib.lbo_solver_pair_count.restype = ip
    lib.lbo_solver_train_network.argtypes = [vp, ip, ip, ctypes.c_double, ctypes.c_uint,
                                             ctypes.POINTER(ctypes.c_double)]
    lib.lbo_solver_train_network.restype = ip
    lib.lbo_solver_get_network.argtypes = [vp, ctypes.POINTER(ip), vp, vp]
    lib.lbo_solver_get_network.restype = ip
    lib.lbo_solver_set_network.argtypes = [vp, ip, vp, vp]
    lib.lbo_solver_set_network.restype = ip
    lib.lbo_solver_network_param_count.argtypes = [vp, ip]
    lib.lbo_solver_network_param_count.restype = ip
    lib.lbo_plan_autotune.argtypes = [vp, dp, dp, dp, ip, ctypes.POINTER(ip)]
    lib.lbo_plan_autotune.restype = ip
    lib.lbo_group_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp)]
    lib.lbo_group_create.restype = ip
    lib.lbo_group_set_stream.argtypes = [vp, vp]
    lib.lbo_group_set_stream.restype = ip
    lib.lbo_group_use_graph.argtypes = [vp, ip]
    lib.lbo_group_use_graph.restype = ip
    lib.lbo_group_apply_linearized.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                               ctypes.POINTER(ip)]
    lib.lbo_group_apply_linearized.restype = ip
    lib.lbo_group_destroy.argtypes = [vp]
    lib.lbo_group_destroy.restype = None
    lib.lbo_last_error.argtypes = []
    lib.lbo_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(a):
    """Data pointer of a float64 C-contiguous torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        return ctypes.c_void_p(a.data_ptr())
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous float64 array")
    return ctypes.c_void_p(a.ctypes.data)


def _optr(a):
    return None if a is None else _ptr(a)


def _check(st, where):
    if st != 0:
        raise LboError(st, where)


def _current_stream(*arrays):
    for a in arrays:
        if hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return None


def dft_axis_tensor(N, precision, inverse, axis, x, out):
    """lbo_dft_axis_tensor: one axis pass of a batched 3-D DFT on the tensor
    cores; x, out: CUDA float32 tensors [batch, N, N, N, 2] (re, im)."""
    import torch
    for a in (x, out):
        if a.dtype != torch.float32 or not a.is_contiguous() or not a.is_cuda:
            raise TypeError("expected contiguous float32 CUDA tensors")
    batch = int(x.shape[0])
    _check(load().lbo_dft_axis_tensor(int(N), PRECISION[precision], int(inverse), int(axis),
                                      ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      batch, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
           "lbo_dft_axis_tensor")
    return out


def measure_alu_peaks(stream=None):
    """lbo_measure_alu_peaks on the current device: {"fp32_tflops",
    "fp64_tflops", "sm_count", "sm_mhz"} (stream: a torch.cuda.Stream or
    None for torch's current stream)."""
    lib = load()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    f32, f64, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    sms = ctypes.c_int()
    _check(lib.lbo_measure_alu_peaks(ctypes.c_void_p(stream.cuda_stream), ctypes.byref(f32), ctypes.byref(f64),
                                     ctypes.byref(sms), ctypes.byref(mhz)), "lbo_measure_alu_peaks")
    return {"fp32_tflops": f32.value, "fp64_tflops": f64.value, "sm_count": sms.value, "sm_mhz": mhz.value}


class Plan:
    """lbo_plan: N^3 grid on [-box, box]^3, VHS exponent, radial nodes."""

    def __init__(self, N, box, vhs_omega, radial_nodes, **options):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.lbo_plan_create(int(N), float(box), float(vhs_omega), int(radial_nodes), ctypes.byref(h)),
               "lbo_plan_create")
        self._h = h
        self.N, self.box, self.vhs_omega, self.J = int(N), float(box), float(vhs_omega), int(radial_nodes)
        for k, v in options.items():
            self.set(k, v)

    def set(self, key, value):
        if key == "precision" and isinstance(value, str):
            value = PRECISION[value]
        _check(load().lbo_plan_set(self._h, LBO_OPT[key], float(value)), "lbo_plan_set(%s)" % key)

    def _stream(self, *arrays):
        s = _current_stream(*arrays)
        _check(load().lbo_plan_set_stream(self._h, s), "lbo_plan_set_stream")

    def apply_linearized(self, params, g, out):
        """out[b] = L_b[g[b]] (Algorithm 1); params (B,5), g/out (B,N,N,N)."""
        batch = int(params.shape[0]) if len(params.shape) == 2 else 1
        self._stream(params, g, out)
        _check(load().lbo_apply_linearized(self._h, _ptr(params), _ptr(g), _ptr(out), batch),
               "lbo_apply_linearized")
        return out

    def cache_maxwellians(self, params):
        """lbo_plan_cache_maxwellians: precompute the Maxwellian-dependent
        factors for these (device) params; None drops the cache."""
        if params is None:
            _check(load().lbo_plan_cache_maxwellians(self._h, None, 0), "lbo_plan_cache_maxwellians")
            return
        batch = int(params.shape[0]) if len(params.shape) == 2 else 1
        self._stream(params)
        _check(load().lbo_plan_cache_maxwellians(self._h, _ptr(params), batch), "lbo_plan_cache_maxwellians")

    def apply_linearized_noalloc(self, params, g, out):
        """lbo_apply_linearized_noalloc: same operator, scratch from the
        library's static device array (device tensors only)."""
        batch = int(params.shape[0]) if len(params.shape) == 2 else 1
        self._stream(params, g, out)
        _check(load().lbo_apply_linearized_noalloc(self._h, _ptr(params), _ptr(g), _ptr(out), batch),
               "lbo_apply_linearized_noalloc")
        return out

    def noalloc_max_batch(self):
        lib = load()
        return lib.lbo_noalloc_scratch_bytes() // lib.lbo_noalloc_bytes_per_instance(self._h)

    def evolve(self, mode, f, dt, nsteps, params=None):
        """lbo_evolve_homogeneous: RK4 steps of df/dt = Q(f,f) (mode
        "quadratic") or L_M[f] (mode "linearized", params the Maxwellians),
        in place on the device tensor f."""
        batch = int(f.shape[0]) if len(f.shape) == 4 else 1
        m = {"quadratic": 0, "linearized": 1}[mode]
        self._stream(f)
        _check(load().lbo_evolve_homogeneous(self._h, m, None if params is None else _ptr(params), _ptr(f), batch,
                                             float(dt), int(nsteps)), "lbo_evolve_homogeneous")
        return f

    def apply_quadratic(self, f, out):
        batch = int(f.shape[0]) if len(f.shape) == 4 else 1
        self._stream(f, out)
        _check(load().lbo_apply_quadratic(self._h, _ptr(f), _ptr(out), batch), "lbo_apply_quadratic")
        return out

    def sync(self):
        _check(load().lbo_plan_sync(self._h), "lbo_plan_sync")

    # Primitives on one block of slab cells (device tensors, flat or shaped;
    # distributed.py composes them).  None stands for a zero boundary cell.
    def block_transport(self, v, ghost_left, ghost_right, out, nx, dx):
        self._stream(v, out)
        _check(load().lbo_slab_block_transport(self._h, _ptr(v), _optr(ghost_left), _optr(ghost_right), _ptr(out),
                                               int(nx), float(dx)), "lbo_slab_block_transport")
        return out

    def block_sweep(self, r, nu, in_left, in_right, z, nx, dx, kn, shift=0.0, direction=0):
        self._stream(r, z)
        _check(load().lbo_slab_block_sweep(self._h, _ptr(r), _ptr(nu), _optr(in_left), _optr(in_right), _ptr(z),
                                           int(nx), float(dx), float(kn), float(shift), int(direction)),
               "lbo_slab_block_sweep")
        return z

    def block_moments(self, f, nx, params, nu=None):
        self._stream(f, params)
        _check(load().lbo_slab_block_moments(self._h, _ptr(f), int(nx), _ptr(params), _optr(nu)),
               "lbo_slab_block_moments")
        return params

    def cell_flux(self, cell, side):
        out = ctypes.c_double()
        self._stream(cell)
        _check(load().lbo_slab_cell_flux(self._h, _ptr(cell), int(side), ctypes.byref(out)), "lbo_slab_cell_flux")
        return out.value

    def maxwellian_cell(self, theta, u, scale, out):
        uu = (ctypes.c_double * 3)(*[float(x) for x in u])
        self._stream(out)
        _check(load().lbo_slab_maxwellian_cell(self._h, float(theta), uu, float(scale), _ptr(out)),
               "lbo_slab_maxwellian_cell")
        return out

    def vec_dots(self, V, ld, K, y, length):
        """[<V + k ld, y> for k < K] over length doubles (host floats)."""
        out = (ctypes.c_double * int(K))()
        self._stream(V, y)
        _check(load().lbo_vec_dots(self._h, _ptr(V), int(ld), int(K), _ptr(y), int(length), out), "lbo_vec_dots")
        return np.frombuffer(out, dtype=np.float64).copy()

    def vec_axpby(self, y, x, a, b, length):
        self._stream(y, x)
        _check(load().lbo_vec_axpby(self._h, _ptr(y), _ptr(x), float(a), float(b), int(length)), "lbo_vec_axpby")
        return y

    def vec_combination(self, y, V, ld, K, c, length):
        """y -= sum_k c[k] (V + k ld), k < K."""
        cc = (ctypes.c_double * int(K))(*[float(x) for x in c[:K]])
        self._stream(y, V)
        _check(load().lbo_vec_combination(self._h, _ptr(y), _ptr(V), int(ld), int(K), cc, int(length)),
               "lbo_vec_combination")
        return y

    def autotune(self, params, g, out):
        """lbo_plan_autotune on device tensors; returns the chosen shape."""
        batch = int(params.shape[0])
        ch = ctypes.c_int()
        self._stream(params, g, out)
        _check(load().lbo_plan_autotune(self._h, _ptr(params), _ptr(g), _ptr(out), batch, ctypes.byref(ch)),
               "lbo_plan_autotune")
        return ch.value

    def solver(self, **kw):
        return Solver(self, **kw)

    def profile(self, enable=True):
        """Start (clearing counters) or stop per-kernel event timing."""
        _check(load().lbo_plan_profile(self._h, 1 if enable else 0), "lbo_plan_profile")

    def profile_read(self):
        """{kernel name: (launches, total ms)} since profiling started."""
        lib = load()
        n = lib.lbo_plan_profile_count(self._h)
        out = {}
        for i in range(n):
            name, cnt, ms = ctypes.c_char_p(), ctypes.c_int(), ctypes.c_double()
            _check(lib.lbo_plan_profile_get(self._h, i, ctypes.byref(name), ctypes.byref(cnt), ctypes.byref(ms)),
                   "lbo_plan_profile_get")
            out[name.value.decode()] = (cnt.value, ms.value)
        return out

    @property
    def last_launches(self):
        return load().lbo_plan_last_launches(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lbo_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """lbo_solver: Newton steps whose linear systems are solved by flexible
    GMRES (inner="fgmres") or the paper's source iteration
    (inner="source_iteration"); nu_scale sets nu_j = nu_scale rho_j in the
    sweep of Eq. (5.7)."""

    def __init__(self, plan, kind="slab", nx=1, x_left=-0.5, x_right=0.5, kn=1.0,
                 wall_left=(1.0, 0.0, 0.0, 0.0), wall_right=(1.0, 0.0, 0.0, 0.0), total_mass=1.0,
                 wall_flux="analytic", dt=0.0, krylov_rtol=1e-3, krylov_atol=1e-7, krylov_restart=30,
                 krylov_maxit=300, precond="sweep", inflow_left=None, inflow_right=None, line_search=0,
                 pseudo_dt=0.0, coarse_moments=5, jacobian="local_maxwellian",
                 coarse_operator="galerkin", inner="fgmres", nu_scale=1.0, device_krylov=False, _mixed=None):
        lib = load()
        pb = Problem()
        pb.kind = PROBLEM[kind]
        pb.nx = int(nx)
        pb.x_left, pb.x_right, pb.kn = float(x_left), float(x_right), float(kn)
        for i in range(4):
            pb.wall_left[i] = float(wall_left[i])
            pb.wall_right[i] = float(wall_right[i])
        pb.total_mass = float(total_mass)
        pb.wall_flux = WALL_FLUX[wall_flux]
        pb.dt = float(dt)
        pb.krylov_rtol, pb.krylov_atol = float(krylov_rtol), float(krylov_atol)
        pb.krylov_restart, pb.krylov_maxit = int(krylov_restart), int(krylov_maxit)
        pb.precond = PRECOND[precond]
        # inflow_left / inflow_right: (rho, u1, u2, u3, theta) replaces the wall on that side
        pb.bc_left = 0 if inflow_left is None else 1
        pb.bc_right = 0 if inflow_right is None else 1
        for i in range(5):
            pb.inflow_left[i] = 0.0 if inflow_left is None else float(inflow_left[i])
            pb.inflow_right[i] = 0.0 if inflow_right is None else float(inflow_right[i])
        pb.line_search = int(line_search)
        pb.pseudo_dt = float(pseudo_dt)
        pb.coarse_moments = int(coarse_moments)
        pb.jacobian = {"local_maxwellian": 0, "exact": 1}[jacobian]
        pb.coarse_operator = {"galerkin": 0, "transport": 1}[coarse_operator]
        pb.inner_solver = {"fgmres": 0, "source_iteration": 1}[inner]
        pb.nu_scale = float(nu_scale)
        pb.device_krylov = 1 if device_krylov else 0
        h = ctypes.c_void_p()
        if _mixed is None:
            _check(lib.lbo_solver_create(ctypes.byref(pb), plan._h, ctypes.byref(h)), "lbo_solver_create")
        else:
            plans, cell_plan = _mixed
            arr = (ctypes.c_void_p * len(plans))(*[q._h.value for q in plans])
            cp = (ctypes.c_int * len(cell_plan))(*[int(c) for c in cell_plan])
            _check(lib.lbo_solver_create_mixed(ctypes.byref(pb), arr, len(plans), cp, ctypes.byref(h)),
                   "lbo_solver_create_mixed")
            self._plans = list(plans)  # kept alive with the solver
        self._h, self.plan, self.problem = h, plan, pb

    def state_length(self):
        """Doubles in the state vector (sum of the cells' N^3)."""
        return int(load().lbo_solver_state_length(self._h))

    def newton_step(self, f, f_prev=None):
        """One Newton step (modified or exact Jacobian, as the problem sets it) in place on the
        device tensor f; returns the stats dict (converged_inner False when the inner solve hit
        its cap: the step is applied all the same)."""
        st = NewtonStats()
        self.plan._stream(f)
        rc = load().lbo_newton_step(self._h, _ptr(f), None if f_prev is None else _ptr(f_prev), ctypes.byref(st))
        if rc not in (0, 4):
            _check(rc, "lbo_newton_step")
        d = st.as_dict()
        d["converged_inner"] = rc == 0
        return d

    def residual(self, f, out, f_prev=None):
        nrm = ctypes.c_double()
        self.plan._stream(f)
        _check(load().lbo_solver_residual(self._h, _ptr(f), None if f_prev is None else _ptr(f_prev), _ptr(out),
                                          ctypes.byref(nrm)), "lbo_solver_residual")
        return nrm.value

    def collect(self, max_pairs):
        """Keep up to max_pairs (A z_k, z_k) training pairs from the next solves."""
        _check(load().lbo_solver_collect(self._h, int(max_pairs)), "lbo_solver_collect")

    @property
    def pair_count(self):
        return load().lbo_solver_pair_count(self._h)

    def train_network(self, hidden=32, epochs=500, lr=3e-3, seed=0):
        loss = ctypes.c_double()
        _check(load().lbo_solver_train_network(self._h, int(hidden), int(epochs), float(lr), int(seed),
                                               ctypes.byref(loss)), "lbo_solver_train_network")
        return loss.value

    def get_network(self):
        lib = load()
        hid = ctypes.c_int()
        _check(lib.lbo_solver_get_network(self._h, ctypes.byref(hid), None, None), "lbo_solver_get_network")
        if hid.value < 0:
            return None
        params = np.empty(lib.lbo_solver_network_param_count(self._h, hid.value), dtype=np.float32)
        scales = np.empty(31, dtype=np.float32)
        _check(lib.lbo_solver_get_network(self._h, ctypes.byref(hid), params.ctypes.data_as(ctypes.c_void_p),
                                          scales.ctypes.data_as(ctypes.c_void_p)), "lbo_solver_get_network")
        return hid.value, params, scales

    def set_network(self, hidden, params, scales):
        params = np.ascontiguousarray(params, dtype=np.float32)
        scales = np.ascontiguousarray(scales, dtype=np.float32)
        _check(load().lbo_solver_set_network(self._h, int(hidden), params.ctypes.data_as(ctypes.c_void_p),
                                             scales.ctypes.data_as(ctypes.c_void_p)), "lbo_solver_set_network")

    def set_residual_plan(self, plan):
        """Evaluate the residual's Q(f,f) with `plan` (e.g. FP64) while the
        Krylov operator keeps the solver's plan; None undoes it."""
        _check(load().lbo_solver_set_residual_plan(self._h, None if plan is None else plan._h),
               "lbo_solver_set_residual_plan")
        self._rplan = plan  # kept alive with the solver

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lbo_solver_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def network_loss_grad(hidden, theta, x, t):
    """lbo_network_loss_grad on CUDA float32 tensors; returns (loss, grad tensor)."""
    import torch
    grad = torch.empty_like(theta)
    loss = ctypes.c_double()
    _check(load().lbo_network_loss_grad(int(hidden), ctypes.c_void_p(theta.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(t.data_ptr()), int(x.shape[0]), int(x.shape[1]),
                                        ctypes.byref(loss), ctypes.c_void_p(grad.data_ptr())), "lbo_network_loss_grad")
    return loss.value, grad


class Group:
    """lbo_group: plans (e.g. of different N) applied together, optionally
    replayed from a CUDA graph."""

    def __init__(self, plans, graph=False):
        lib = load()
        arr = (ctypes.c_void_p * len(plans))(*[p._h.value for p in plans])
        h = ctypes.c_void_p()
        _check(lib.lbo_group_create(arr, len(plans), ctypes.byref(h)), "lbo_group_create")
        self._h, self.plans = h, list(plans)
        _check(lib.lbo_group_use_graph(h, 1 if graph else 0), "lbo_group_use_graph")

    def apply_linearized(self, params, gs, outs):
        import torch
        n = len(self.plans)
        lib = load()
        _check(lib.lbo_group_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
               "lbo_group_set_stream")
        P = (ctypes.c_void_p * n)(*[_ptr(x).value for x in params])
        G = (ctypes.c_void_p * n)(*[_ptr(x).value for x in gs])
        O = (ctypes.c_void_p * n)(*[_ptr(x).value for x in outs])
        B = (ctypes.c_int * n)(*[int(x.shape[0]) for x in params])
        _check(lib.lbo_group_apply_linearized(self._h, P, G, O, B), "lbo_group_apply_linearized")
        return outs

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lbo_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mixed_solver(plans, cell_plan, **problem):
    """lbo_solver_create_mixed: a slab whose cell j uses plans[cell_plan[j]]
    (one plan per N, the same box); `problem` as for Plan.solver (kind
    'slab', inflow sides).  The state is the cells' fields concatenated, cell
    j as N_j^3 doubles in centred order."""
    problem = dict(problem)
    problem["nx"] = len(cell_plan)
    return Solver(plans[0], _mixed=(plans, cell_plan), **problem)
