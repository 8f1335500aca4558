"""Writes noisy_n16_extended.txt: L[g] of one noisy N = 16 instance by the
oracle's extended-precision direct sums (Algorithm 1 written as cyclic
convolutions, oracle/direct.c compiled with long double; the cut-off of
Eq. (3.9) decided in FP64).  Input: the seeded benchmark recipe,
workloads.batched_instances(16, 8.0, batch=1, seed=31, noise=1e-3), VHS
omega = 0.5, J = 16 Gauss-Legendre radial nodes, eps = 1e-9.  Stored: max
|L[g]|, max |g/M| over the points the cut-off keeps, and 257 sampled values
(centred-order flat index, value): the largest |L[g]| and 256 seeded draws.
Run from the repository root:  python tests/golden/make_noisy_n16_extended.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import grid  # noqa: E402
from oracle.direct import direct_linearized  # noqa: E402
from oracle.linearized import Tables  # noqa: E402
from paper_2503_09580_gb300 import workloads  # noqa: E402

N, L, OMEGA, SEED = 16, 8.0, 0.5, 31


def main():
    params, g = workloads.batched_instances(N, L, batch=1, seed=SEED, noise=1e-3)
    rho, u1, u2, u3, th = params[0]
    ref = grid.to_centred(direct_linearized(Tables(N, L, OMEGA, N), rho, (u1, u2, u3), th,
                                            grid.to_cyclic(g[0]), extended=True)).ravel()
    a = workloads.velocity_axis(N, L)
    d2 = (a[:, None, None] - u1) ** 2 + (a[None, :, None] - u2) ** 2 + (a[None, None, :] - u3) ** 2
    M = rho * (2 * np.pi * th) ** -1.5 * np.exp(-d2 / (2 * th))
    keep = d2 / (2 * th) <= np.log(1e9) - 1.5 * np.log(2 * np.pi * th)
    rmax = np.abs(g[0][keep] / M[keep]).max()
    idx = [int(np.abs(ref).argmax())] + sorted(np.random.default_rng(0).choice(ref.size, 256, replace=False).tolist())
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "noisy_n16_extended.txt")
    with open(path, "w") as fh:
        fh.write("# L[g] by extended-precision direct sums (Algorithm 1 as cyclic convolutions);\n")
        fh.write("# written by tests/golden/make_noisy_n16_extended.py (oracle only).\n")
        fh.write("# input: workloads.batched_instances(16, 8.0, batch=1, seed=31, noise=1e-3), omega 0.5, J 16\n")
        fh.write("max_abs %.17e\nmax_ratio %.17e\n" % (np.abs(ref).max(), rmax))
        for i in idx:
            fh.write("%d %.17e\n" % (i, ref[i]))


if __name__ == "__main__":
    main()
