"""Pins of the oracle's ROK4E coefficient table (Sec. 4.1-4.2).

The coefficients are compared with the printed table (tests/golden/rok4e_table.txt)
and checked against the nine order conditions of Eq. order_cond_ros_k, the
embedded order-3 conditions, L-stability of the stability function
(Eq. stability_exact_jac) and the shared stage-3/4 argument.
"""

import os

import numpy as np
import pytest

from oracle import rok4e

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rok4e_table.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        out[k] = float(v)
    return out


def _conditions(b, g, A, G):
    """Residuals of the nine order-4 conditions (a)-(i) of Eq. order_cond_ros_k."""
    beta = A + G  # beta_ij = alpha_ij + gamma_ij (strictly lower part)
    al = A.sum(axis=1)  # alpha_i
    bp = beta.sum(axis=1)  # beta'_i
    r = []
    r.append(b.sum() - 1)
    r.append(b[1] * bp[1] + b[2] * bp[2] + b[3] * bp[3] - (0.5 - g))
    r.append(b[1] * al[1] ** 2 + b[2] * al[2] ** 2 + b[3] * al[3] ** 2 - 1 / 3)
    r.append(b[2] * beta[2, 1] * bp[1] + b[3] * (beta[3, 1] * bp[1] + beta[3, 2] * bp[2])
             - (1 / 6 - g + g**2))
    r.append(b[1] * al[1] ** 3 + b[2] * al[2] ** 3 + b[3] * al[3] ** 3 - 0.25)
    r.append(b[2] * al[2] * A[2, 1] * bp[1] + b[3] * al[3] * (A[3, 1] * bp[1] + A[3, 2] * bp[2])
             - (1 / 8 - g / 3))
    r.append(b[2] * A[2, 1] * al[1] ** 2 + b[3] * (A[3, 1] * al[1] ** 2 + A[3, 2] * al[2] ** 2) - 1 / 12)
    r.append(b[2] * G[2, 1] * al[1] ** 2 + b[3] * (G[3, 1] * al[1] ** 2 + G[3, 2] * al[2] ** 2) + g / 3)
    r.append(b[3] * beta[3, 2] * beta[2, 1] * bp[1] - (1 / 24 - g / 2 + 1.5 * g**2 - g**3))
    return np.array(r)


def test_table_matches_printed_values():
    gd = _golden()
    assert rok4e.GAMMA == gd["gamma"]
    for i in range(4):
        for j in range(i):
            assert rok4e.GAMMA_IJ[i, j] == gd[f"gamma{i+1}{j+1}"]
            assert rok4e.ALPHA_IJ[i, j] == gd[f"alpha{i+1}{j+1}"]
    for j in range(4):
        assert rok4e.B[j] == gd[f"b{j+1}"]
        assert rok4e.BHAT[j] == gd[f"bhat{j+1}"]


def test_nine_order_conditions():
    r = _conditions(rok4e.B, rok4e.GAMMA, rok4e.ALPHA_IJ, rok4e.GAMMA_IJ)
    assert np.max(np.abs(r)) < 1e-14, r


def test_embedded_formula_is_order_three():
    r = _conditions(rok4e.BHAT, rok4e.GAMMA, rok4e.ALPHA_IJ, rok4e.GAMMA_IJ)
    assert np.max(np.abs(r[:4])) < 1e-14, r[:4]  # conditions (a)-(d)
    assert np.max(np.abs(r[4:])) > 1e-3  # and genuinely not order 4


def test_alternative_reading_of_garbled_rows_fails():
    # the printed bhat row read literally (0.1865 in the slot after bhat2 labelled
    # "bhat_2", i.e. bhat4) breaks condition (b)
    bhat_alt = np.array([-0.217819895945721, 1.03130847478467, 0.0, 0.186511421161047])
    r = _conditions(bhat_alt, rok4e.GAMMA, rok4e.ALPHA_IJ, rok4e.GAMMA_IJ)
    assert abs(r[1]) > 0.05
    b_alt = np.array([0.194335256262729, 0.0, 0.483167813989227, 0.322496929748044])
    assert np.max(np.abs(_conditions(b_alt, rok4e.GAMMA, rok4e.ALPHA_IJ, rok4e.GAMMA_IJ))) > 1e-2


def _stability(z, b):
    beta = rok4e.ALPHA_IJ + rok4e.GAMMA_IJ + rok4e.GAMMA * np.eye(4)
    one = np.ones(4)
    return 1 + z * b @ np.linalg.solve(np.eye(4) - z * beta, one)


def test_l_stability():
    beta = rok4e.ALPHA_IJ + rok4e.GAMMA_IJ + rok4e.GAMMA * np.eye(4)
    r_inf = 1 - rok4e.B @ np.linalg.solve(beta, np.ones(4))
    assert abs(r_inf) < 1e-13
    assert abs(rok4e.GAMMA - 0.573) < 5e-4  # the text's rounded value
    rng = np.random.default_rng(0)
    z = -rng.exponential(10.0, 4000) + 1j * rng.normal(0, 30.0, 4000)
    vals = np.array([abs(_stability(zz, rok4e.B)) for zz in z])
    assert np.all(vals <= 1 + 1e-12)
    # imaginary axis (A-stability boundary)
    for y in np.linspace(-1e3, 1e3, 2001):
        assert abs(_stability(1j * y, rok4e.B)) <= 1 + 1e-12


def test_stability_function_is_exp_to_order_four():
    # R(z) - e^z = O(z^5): the ratio of errors at z and z/2 is close to 32
    e1 = abs(_stability(-0.02, rok4e.B) - np.exp(-0.02))
    e2 = abs(_stability(-0.01, rok4e.B) - np.exp(-0.01))
    assert 25 < e1 / e2 < 40


def test_stages_three_and_four_share_the_argument():
    assert np.array_equal(rok4e.ALPHA_IJ[3, :2], rok4e.ALPHA_IJ[2, :2])
    assert rok4e.ALPHA_IJ[3, 2] == 0.0
    assert rok4e.B[2] == 0.0


@pytest.mark.parametrize("err_prev,err,expect", [(1.0, 0.0, 5.0), (1.0, 1e12, 0.2), (1.0, np.nan, 0.2),
                                                 (1.0, 1.0, 0.8)])
def test_pi_factor_limits(err_prev, err, expect):
    assert rok4e.pi_factor(err, err_prev) == pytest.approx(expect)
