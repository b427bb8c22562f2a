"""Pins of the relaxation parameter (Sec. 2.3.3, Algorithm 2) in the oracle.

Cases with a known answer: a residual that shrinks geometrically, f_new = c f_old,
gives alpha = -alpha_k / (c - 1) exactly (Aitken's extrapolation of a linear
sequence); a residual that grows in the same direction gives a negative value,
reset to 1; the cap du_max / ||g||_inf; no f_old or equal residuals keep alpha_k.
"""

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def f():
    return np.random.default_rng(3).normal(0, 1, (2, 7, 4, 3))


def test_geometric_residual(f):
    for c, ak in ((0.5, 1.0), (0.25, 0.6), (-0.5, 2.0)):
        alpha = oracle.relax_alpha(c * f, f, [ak, ak], np.zeros((2, 5, 4, 3)))
        np.testing.assert_allclose(alpha, -ak / (c - 1.0), rtol=1e-14)


def test_negative_is_reset(f):
    alpha = oracle.relax_alpha(2.0 * f, f, [1.0, 3.0], np.zeros((2, 5, 4, 3)))  # -1 and -3
    np.testing.assert_array_equal(alpha, [1.0, 1.0])


def test_cap_and_no_old(f):
    g = np.zeros((2, 5, 4, 3))
    g[0, 1, 2, 0] = -3.0
    g[1, 0, 0, 2] = 0.5
    alpha = oracle.relax_alpha(f, None, [2.0, 2.0], g, du_max=1.0)
    # rhs 0: |2 * 3| > 1 -> 1/3; rhs 1: |2 * 0.5| = 1 is not above the bound -> kept
    np.testing.assert_allclose(alpha, [1.0 / 3.0, 2.0], rtol=1e-15)


def test_equal_residuals_keep_alpha(f):
    alpha = oracle.relax_alpha(f, f.copy(), [0.7, 1.3], np.zeros((2, 5, 4, 3)))
    np.testing.assert_array_equal(alpha, [0.7, 1.3])


def test_general_case_by_hand(f):
    rng = np.random.default_rng(8)
    f_old = rng.normal(0, 1, f.shape)
    alpha = oracle.relax_alpha(f, f_old, [1.5, 0.5], np.zeros((2, 5, 4, 3)))
    for r in range(2):
        d = f[r] - f_old[r]
        want = -[1.5, 0.5][r] * np.sum(f_old[r] * d) / np.sum(d * d)
        assert alpha[r] == pytest.approx(want if want >= 0 else 1.0, rel=1e-13)
