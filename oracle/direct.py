"""ctypes binding of the O(J n^6) direct-sum oracle in ``direct.c``.
Oracle: test infrastructure only.  ``build()`` compiles it with gcc."""
import ctypes
import os
import subprocess

import numpy as np

from . import grid
from .quadrature import vhs_kernel

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_SRC_LD = os.path.join(_HERE, "direct_ld.c")
_LIB = os.path.join(_HERE, "_direct.so")
_lib = None


def build(force=False):
    """Compile direct.c (double) and direct_ld.c (long double) into
    oracle/_direct.so (plain C, -O2, no contraction of a*b+c into FMAs, so
    that every operation is rounded as written)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_LD))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", _LIB, _SRC, _SRC_LD,
                               "-lm"])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        for sfx in ("", "_ld"):
            getattr(_lib, "lbo_direct_linearized" + sfx).argtypes = [
                ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp,
                ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, dp]
            getattr(_lib, "lbo_direct_quadratic" + sfx).argtypes = [
                ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, dp, dp, ctypes.c_int, dp, dp,
                dp, dp, dp]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def direct_linearized(tab, rho, u, theta, f_cyc, cutoff=True, eps=1e-9, extended=False):
    """L[f] by direct sums (cyclic order in and out); same readings as
    ``linearized.collision_operator`` with ``nyquist='standard'``.
    extended=True sums in long double (the cut-off decision stays FP64)."""
    lib = _load()
    fn = lib.lbo_direct_linearized_ld if extended else lib.lbo_direct_linearized
    n = tab.n
    f = np.ascontiguousarray(f_cyc, dtype=np.float64)
    out = np.zeros((n, n, n))
    g = np.ascontiguousarray(tab.g)
    w = np.ascontiguousarray(tab.w)
    B = np.ascontiguousarray(vhs_kernel(tab.g, tab.omega_vhs, tab.C))
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    rc = fn(n, tab.L, tab.J, _p(g), _p(w), _p(B), float(rho), _p(uu),
                                   float(theta), int(cutoff), float(eps), _p(f), _p(out))
    if rc:
        raise MemoryError("direct oracle allocation failed")
    return out


def direct_quadratic(tab, f_cyc, sig, wm, g_cyc=None, extended=False):
    """Q(f,f) (or Q(f,g)+Q(g,f)) by direct Fourier-space sums, cyclic order;
    extended=True sums in long double."""
    lib = _load()
    fn = lib.lbo_direct_quadratic_ld if extended else lib.lbo_direct_quadratic
    n = tab.n
    f = np.ascontiguousarray(f_cyc, dtype=np.float64)
    gg = None if g_cyc is None else np.ascontiguousarray(g_cyc, dtype=np.float64)
    out = np.zeros((n, n, n))
    gj = np.ascontiguousarray(tab.g)
    w = np.ascontiguousarray(tab.w)
    B = np.ascontiguousarray(vhs_kernel(tab.g, tab.omega_vhs, tab.C))
    s = np.ascontiguousarray(sig, dtype=np.float64)
    ww = np.ascontiguousarray(wm, dtype=np.float64)
    rc = fn(n, tab.L, tab.J, _p(gj), _p(w), _p(B), len(ww), _p(s), _p(ww),
                                  _p(f), None if gg is None else _p(gg), _p(out))
    if rc:
        raise MemoryError("direct oracle allocation failed")
    return out
