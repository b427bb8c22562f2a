"""Pins of the oracle's continuum Green function (Sec. 3.1, Eq. 33).

None of these retypes the oracle's formula: each checks a property that the
mathematics fixes -- two independent representations agreeing, the
equilibrium of a unit point force, the Navier equation, symmetry,
homogeneity and the rotation rule.
"""

import numpy as np
import pytest

from conftest import CUBIC, ISO

NU = ISO["nu"]
LAM = 2.0 * ISO["mu"] * NU / (1.0 - 2.0 * NU)
# a cubic medium whose constants satisfy C11 - C12 = 2 C44 is isotropic
CUBIC_AS_ISO = {"kind": "cubic", "C11": LAM + 2.0, "C12": LAM, "C44": 1.0}


def _stiffness(material):
    if material["kind"] == "isotropic":
        mu, nu = material["mu"], material["nu"]
        lam = 2 * mu * nu / (1 - 2 * nu)
        C11, C12, C44 = lam + 2 * mu, lam, mu
    else:
        C11, C12, C44 = material["C11"], material["C12"], material["C44"]
    C = np.zeros((3, 3, 3, 3))
    d = np.eye(3)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[i, j, k, l] = (C12 * d[i, j] * d[k, l] + C44 * (d[i, k] * d[j, l] + d[i, l] * d[j, k])
                                     + (C11 - C12 - 2 * C44) * (i == j == k == l))
    return C


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def test_barnett_reduces_to_kelvin(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(20):
        r = rng.standard_normal(3) * rng.uniform(0.5, 50.0)
        Gk = oracle_mod.green(ISO, r)
        Gb = oracle_mod.green(CUBIC_AS_ISO, r)
        assert np.abs(Gb - Gk).max() <= 1e-14 * np.abs(Gk).max()


@pytest.mark.parametrize("material", [ISO, CUBIC], ids=["kelvin", "barnett"])
def test_symmetry_evenness_homogeneity(oracle_mod, material):
    rng = np.random.default_rng(2)
    for _ in range(10):
        r = rng.standard_normal(3) * 3.0
        G = oracle_mod.green(material, r)
        assert np.abs(G - G.T).max() <= 1e-15 * np.abs(G).max()
        assert np.abs(oracle_mod.green(material, -r) - G).max() <= 1e-15 * np.abs(G).max()
        lam = 7.25
        assert np.abs(oracle_mod.green(material, lam * r) * lam - G).max() <= 4e-15 * np.abs(G).max()
        # positive definite (the medium is stable)
        assert np.linalg.eigvalsh(0.5 * (G + G.T)).min() > 0


@pytest.mark.parametrize("material", [ISO, CUBIC], ids=["kelvin", "barnett"])
def test_point_force_equilibrium(oracle_mod, material):
    """The tractions of the unit point-force solution balance the force.

    For u = G e_k, the stress sigma_ij = C_ijpq d_q u_p integrated over a
    sphere around the origin must give -delta_ik (the surface carries the
    reaction to the unit force).  This pins the normalisation and the sign.
    """
    C = _stiffness(material)
    nth, nph = 24, 48
    xg, wg = np.polynomial.legendre.leggauss(nth)
    total = np.zeros((3, 3))
    h = 1e-4
    for ct, wt in zip(xg, wg):
        st = np.sqrt(1 - ct * ct)
        for jp in range(nph):
            ph = 2 * np.pi * jp / nph
            n = np.array([st * np.cos(ph), st * np.sin(ph), ct])
            # dG[q] = d G / d x_q by a fourth-order central difference
            dG = np.zeros((3, 3, 3))
            for q in range(3):
                e = np.zeros(3)
                e[q] = h
                dG[q] = (8 * (oracle_mod.green(material, n + e) - oracle_mod.green(material, n - e))
                         - (oracle_mod.green(material, n + 2 * e) - oracle_mod.green(material, n - 2 * e))) / (12 * h)
            # sigma_ij for load direction k: C_ijpq dG[q][p, k]
            sig = np.einsum("ijpq,qpk->ijk", C, dG)
            total += np.einsum("ijk,j->ik", sig, n) * wt * (2 * np.pi / nph)
    # the angular product rule resolves the anisotropic integrand to ~1e-7
    assert np.abs(total + np.eye(3)).max() < 1e-6


@pytest.mark.parametrize("material", [ISO, CUBIC], ids=["kelvin", "barnett"])
def test_navier_residual(oracle_mod, material):
    """Away from the origin, C_ijkl d_j d_l G_km = 0 (the Navier equation)."""
    C = _stiffness(material)
    rng = np.random.default_rng(3)
    h = 2e-3
    for _ in range(3):
        r = rng.standard_normal(3)
        r *= 2.5 / np.linalg.norm(r)
        H = np.zeros((3, 3, 3, 3))  # H[j, l] = d_j d_l G
        E = np.eye(3) * h
        for j in range(3):
            for l in range(3):
                H[j, l] = (oracle_mod.green(material, r + E[j] + E[l]) - oracle_mod.green(material, r + E[j] - E[l])
                           - oracle_mod.green(material, r - E[j] + E[l])
                           + oracle_mod.green(material, r - E[j] - E[l])) / (4 * h * h)
        res = np.einsum("ijkl,jlkm->im", C, H)
        scale = np.abs(np.einsum("ijkl,jlkm->ijlm", np.abs(C), np.abs(H))).max()
        assert np.abs(res).max() < 1e-5 * scale


def test_barnett_quadrature_converged(oracle_mod):
    rng = np.random.default_rng(4)
    for _ in range(5):
        r = rng.standard_normal(3)
        a = oracle_mod.green(CUBIC, r, nquad=96)
        b = oracle_mod.green(CUBIC, r, nquad=192)
        assert np.abs(a - b).max() <= 2e-15 * np.abs(b).max()


def test_rotation_rule(oracle_mod):
    """With r_crystal = Q r, the computational-frame function is Q^T G(Q r) Q."""
    Q = _rot([1.0, 2.0, 0.5], 0.7)
    mat = dict(CUBIC, Q=Q)
    rng = np.random.default_rng(5)
    for _ in range(5):
        r = rng.standard_normal(3)
        Gq = oracle_mod.green(mat, r)
        ref = Q.T @ oracle_mod.green(CUBIC, Q @ r) @ Q
        assert np.abs(Gq - ref).max() <= 1e-14 * np.abs(ref).max()


def test_invalid_inputs_rejected(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.green(ISO, [0.0, 0.0, 0.0])
    with pytest.raises(ValueError):
        oracle_mod.green({"kind": "isotropic", "mu": -1.0, "nu": 0.3}, [1.0, 0.0, 0.0])
