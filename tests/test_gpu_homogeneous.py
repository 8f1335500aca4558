"""lbo_evolve_homogeneous (RK4 of Sec. 4.2) against the oracle's RK4 with its
own operators, for the paper's two cases: Case 1, Maxwell molecules
(B_1 = 1/(4 pi)) from f^(1); Case 2, B_2 = g^0.56/(4 pi) (omega = 0.72) from
f^(2); R = 6 with L = (3 + sqrt 2) R / 4 (Sec. 2.3), N_p = 16 (N = 32),
17 radial nodes (exact to degree 33 >= 2 N_p), dt = 0.1."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.evolve import rk4
from oracle.linearized import Tables, apply_linearized
from oracle.quadratic import apply_quadratic
from oracle.quadrature import hemisphere_rule
from paper_2503_09580_gb300 import lbo, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N, R, J, DT = 32, 6.0, 17, 0.1
L = (3 + np.sqrt(2)) * R / 4
STD = np.array([[1.0, 0.0, 0.0, 0.0, 1.0]])


def relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_linearized_rk4_case1_matches_oracle():
    f0 = workloads.paper_f1(N, L)[None]
    tab = Tables(N, L, 1.0, J, R=R)
    ref = rk4(lambda f: apply_linearized(tab, STD, f), f0, DT, 3)
    plan = lbo.Plan(N, L, 1.0, J, R=R)
    tf = torch.from_numpy(f0.copy()).to(DEV)
    plan.evolve("linearized", tf, DT, 3, params=torch.from_numpy(STD).to(DEV))
    got = tf.cpu().numpy()
    assert relerr(got, ref) <= 1e-12
    assert relerr(got, f0) > 1e-3  # it did evolve


@pytest.mark.parametrize("fix", [None, "sinc_quadrature"])
def test_quadratic_rk4_case2_matches_oracle(fix):
    f0 = workloads.paper_f2(N, L)[None]
    tab = Tables(N, L, 0.72, J, R=R)
    sig, w = hemisphere_rule(2)
    ref = rk4(lambda f: apply_quadratic(tab, f, sig, w, mass_fix=fix), f0, DT, 2)
    plan = lbo.Plan(N, L, 0.72, J, R=R, hemisphere_p=2, q_sinc_quadrature=1 if fix else 0)
    tf = torch.from_numpy(f0.copy()).to(DEV)
    plan.evolve("quadratic", tf, DT, 2)
    got = tf.cpu().numpy()
    assert relerr(got, ref) <= 1e-12
    h3 = (2 * L / N) ** 3
    m0, m2 = h3 * f0.sum(), h3 * got.sum()
    if fix:
        assert abs(m2 / m0 - 1) < 1e-13  # Eq. (2.16): mass kept to rounding
