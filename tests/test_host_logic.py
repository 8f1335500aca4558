"""Host-side logic inside the CUDA sources, checked on the CPU by small
nvcc-built harnesses that run no kernel (tests/host/): the banded LU with an
arrow border of the moment coarse correction, the resampling matrices of
the mixed-N solver against the oracle's FFT-based resampling, and the
register-resident 32-point transform of the FP64 kernels against a direct
DFT."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.resample import resample_axis

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HOST = os.path.join(ROOT, "tests", "host")
NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def _build(name, tmp_path):
    if not os.path.exists(NVCC):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / name)
    subprocess.check_call([NVCC, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2503_09580_gb300", "csrc"), "-o", exe,
                           os.path.join(HOST, name + ".cu")])
    return exe


def test_banded_lu_with_arrow_border(tmp_path):
    out = subprocess.run([_build("banded_lu", tmp_path)], check=True, capture_output=True, text=True).stdout
    rows = [line.split() for line in out.strip().splitlines()]
    assert len(rows) == 5
    for nb, nx, border, err in rows:
        assert err != "factor_failed", (nb, nx, border)
        assert float(err) < 1e-11, (nb, nx, border, err)


def test_resampling_matrices_match_the_oracle(tmp_path):
    pairs = [(16, 24), (24, 16), (32, 48), (48, 24), (24, 32), (64, 32)]
    L = 8.0
    inp = "".join("%d %d\n" % p for p in pairs)
    out = subprocess.run([_build("resample_matrix", tmp_path), str(L)], input=inp, check=True,
                         capture_output=True, text=True).stdout
    vals = np.array([float(x) for x in out.split()])
    o = 0
    for na, nb in pairs:
        R = vals[o:o + na * nb].reshape(nb, na)
        o += na * nb
        # the oracle resamples centred-order unit vectors (cyclic order inside)
        E = np.eye(na)
        cols = []
        for a in range(na):
            e = np.fft.ifftshift(E[a])
            cols.append(np.fft.fftshift(resample_axis(e, nb, 0)))
        ref = np.array(cols).T
        assert np.abs(R - ref).max() <= 1e-13, (na, nb, np.abs(R - ref).max())
    assert o == vals.size


def test_register_fft32_against_a_direct_dft(tmp_path):
    """The 32-point transform of the FP64 register kernels (scaled-twiddle
    radix-2, fft_reg.cuh) against a direct DFT in long double: a few units
    of the working precision's roundoff, forward and inverse, and the scaled
    twiddles reproduce W_32^m to about one unit of double roundoff."""
    out = subprocess.run([_build("fft_reg", tmp_path)], check=True, capture_output=True, text=True).stdout
    res = {" ".join(line.split()[:-1]): float(line.split()[-1]) for line in out.strip().splitlines()}
    assert res["double forward"] <= 8 * 2.0 ** -53 and res["double inverse"] <= 8 * 2.0 ** -53
    assert res["float forward"] <= 8 * 2.0 ** -24 and res["float inverse"] <= 8 * 2.0 ** -24
    assert res["twiddle"] <= 4 * 2.0 ** -53
