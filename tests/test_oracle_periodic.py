"""Pins of the oracle's periodic kernel and its per-mode tables.

* Richardson's weights (Sec. 3.1, Eq. 36) reproduce the limit of any sequence
  that is exactly a polynomial of degree N in 1/n (Eq. 35).
* The extrapolated image sum agrees with a brute-force direct sum over tens of
  thousands of images whose tail is removed by a two-point 1/J^2 fit -- no
  Richardson code is involved on that side.
* The tabulated kernel is symmetric, even and mirror-symmetric.
* The k = 0 mode is the full lattice line sum, which approaches the 2D
  plane-strain / antiplane line-force solution divided by c (differences
  between sites cancel the regularisation constant).
* Modes k >= 1 of an isotropic medium follow from Poisson summation of the
  Kelvin kernel's Fourier transform along the line (modified Bessel K0, K1).
"""

import math

import numpy as np
import pytest
from scipy import special

from conftest import CUBIC, ISO

M_MIRROR = np.diag([1.0, 1.0, -1.0])


def test_richardson_weights_exact_on_polynomials(oracle_mod):
    rng = np.random.default_rng(7)
    for n, N in [(1, 5), (4, 6), (2, 8), (8, 8)]:
        w = oracle_mod.richardson_weights(n, N)
        assert abs(w.sum() - 1.0) < 1e-12 * np.abs(w).sum()
        Qs = rng.standard_normal(N + 1)
        seq = [sum(Qs[j] * float(m) ** (-j) for j in range(N + 1)) for m in range(n, n + N + 1)]
        est = float(np.dot(w, seq))
        assert abs(est - Qs[0]) < 1e-13 * np.abs(w).sum() * np.abs(Qs).max()
        # a term of degree N + 1 leaves exactly (-1)^N / (n (n+1) ... (n+N))
        seq2 = [s + float(m) ** (-(N + 1)) for s, m in zip(seq, range(n, n + N + 1))]
        resid = float(np.dot(w, seq2)) - Qs[0]
        want = (-1.0) ** N / math.prod(range(n, n + N + 1))
        assert abs(resid - want) < 1e-13 * np.abs(w).sum() * np.abs(Qs).max()


def _brute_force_periodic(oracle_mod, material, l3, r, J):
    """sum_{i=-J..J} [G(r + i l3 e3) - G(0,0,i l3)] (i = 0 subtraction skipped)."""
    total = oracle_mod.green(material, r).copy()
    for i in range(1, J + 1):
        total += oracle_mod.green(material, [r[0], r[1], r[2] + i * l3])
        total += oracle_mod.green(material, [r[0], r[1], r[2] - i * l3])
        total -= oracle_mod.green(material, [0.0, 0.0, i * l3])
        total -= oracle_mod.green(material, [0.0, 0.0, -i * l3])
    return total


@pytest.mark.parametrize("material,l3,r", [
    (ISO, 16.0, [5.0, -3.0, 6.0]),
    (ISO, 256.0, [60.0, 60.0, 100.0]),
    (CUBIC, 16.0, [4.0, 2.0, -7.0]),
], ids=["iso-short", "iso-long", "cubic"])
def test_richardson_matches_brute_force(oracle_mod, material, l3, r):
    J = 4000 if material is ISO else 1000
    S1 = _brute_force_periodic(oracle_mod, material, l3, r, J)
    S2 = S1 + (_brute_force_periodic(oracle_mod, material, l3, r, 2 * J) - S1)
    # tail of the paired sum decays like J^-2: remove it with a two-point fit
    lim = S2 + (S2 - S1) / 3.0
    q = oracle_mod.periodic(material, l3, r, n=8, N=8)
    scale = np.abs(lim).max()
    assert np.abs(q - lim).max() < 5e-8 * scale


def _longest_difference(xy_i, xy_p):
    """The pad-minus-interface difference of largest length (chunked over pad columns)."""
    best, arg = -1, None
    xi = xy_i.astype(np.int64)
    for lo in range(0, len(xy_p), 1000):
        D = xy_p[lo:lo + 1000, None, :].astype(np.int64) - xi[None, :, :]
        r2 = (D * D).sum(-1)
        j = int(np.argmax(r2))
        if r2.flat[j] > best:
            best, arg = int(r2.flat[j]), D.reshape(-1, 2)[j]
    return arg


# Truncation of Eq. 36 against the exact image sum of Eq. 32 at each workload's longest difference
# (the largest |d| / l3, where Richardson's truncation is worst): the default order (n, N) = (4, 6)
# and (8, 8), the most accurate order at all three sizes (larger n or N amplify the rounding of the
# image terms more than they remove truncation).  Bounds: the measured values rounded up.
@pytest.mark.parametrize("name,tol46,tol88", [
    ("ring200x300_L16_iso", 3.5e-6, 3e-9),
    ("ring4000x6000_L256_cubic", 6e-8, 1.5e-10),
    ("ring8000x12000_L1024_rhs64_iso", 1e-8, 1e-11),
], ids=["L16", "L256-cubic", "L1024"])
def test_default_order_truncation_at_the_workloads(oracle_mod, name, tol46, tol88):
    from paper_2105_08798_gb300 import inputs

    w = inputs.WORKLOADS[name]
    xy_i, xy_p = w.geometry()
    d = _longest_difference(xy_i, xy_p)
    l3 = w.L * w.c
    J = 4000 if w.material["kind"] == "isotropic" else 600
    worst46 = worst88 = 0.0
    for s in (0.0, l3 / 4, l3 / 2):
        r = [float(d[0]), float(d[1]), s]
        S1 = _brute_force_periodic(oracle_mod, w.material, l3, r, J)
        S2 = _brute_force_periodic(oracle_mod, w.material, l3, r, 2 * J)
        lim = S2 + (S2 - S1) / 3.0
        scale = np.abs(lim).max()
        worst46 = max(worst46, np.abs(oracle_mod.periodic(w.material, l3, r) - lim).max() / scale)
        worst88 = max(worst88, np.abs(oracle_mod.periodic(w.material, l3, r, n=8, N=8) - lim).max() / scale)
    assert worst46 < tol46, worst46
    assert worst88 < tol88, worst88
    # the default order is not needlessly loose either: its truncation is visible at this |d| / l3
    assert worst46 > 10 * worst88


def test_richardson_converges_in_n(oracle_mod):
    r = [24.0, 3.0, 8.0]
    ref = oracle_mod.periodic(ISO, 16.0, r, n=16, N=8)
    errs = [np.abs(oracle_mod.periodic(ISO, 16.0, r, n=n, N=6) - ref).max() for n in (1, 2, 4, 8)]
    assert all(b < a for a, b in zip(errs, errs[1:]))


@pytest.mark.parametrize("material", [ISO, CUBIC], ids=["iso", "cubic"])
def test_table_symmetries(oracle_mod, material):
    L = 16
    d = np.array([[3, 1], [-3, -1], [0, 5], [0, -5], [7, -2], [-7, 2]], dtype=np.int32)
    T = oracle_mod.kernel_table(material, L, 1.0, d, nquad=64 if material is CUBIC else None)
    for a in range(0, len(d), 2):
        for s in range(L):
            G = T[a, s]
            scale = np.abs(G).max()
            # Kelvin's form is exactly even and symmetric in floating point; Barnett's
            # quadrature is so only up to rounding, which Eq. 36's weights (sum |w| ~ 1.6e4
            # at n = 4, N = 6) amplify to a few 1e-14 of the entry
            tol = 1e-15 if material is ISO else 2e-13
            assert np.abs(G - G.T).max() <= tol * scale
            # evenness: G~(-d, -s) = G~(d, s)
            assert np.abs(T[a + 1, (-s) % L] - G).max() <= tol * scale
            # mirror z -> -z of both media: G~(d, -s) = M G~(d, s) M
            assert np.abs(T[a, (-s) % L] - M_MIRROR @ G @ M_MIRROR).max() <= tol * scale


@pytest.mark.parametrize("material", [ISO, CUBIC], ids=["iso", "cubic"])
def test_mode_table_structure(oracle_mod, material):
    L = 16
    d = np.array([[3, 1], [-3, -1], [6, -4]], dtype=np.int32)
    T = oracle_mod.kernel_table(material, L, 1.0, d, nquad=64 if material is CUBIC else None)
    g = oracle_mod.mode_table(T)
    scale = np.abs(g).max()
    tol = 1e-14 if material is ISO else 2e-13
    # complex-symmetric
    assert np.abs(g - np.swapaxes(g, -1, -2)).max() <= tol * scale
    # mirror symmetry: 11, 12, 22, 33 real; 13, 23 imaginary
    even = [(0, 0), (0, 1), (1, 1), (2, 2), (1, 0)]
    odd = [(0, 2), (1, 2), (2, 0), (2, 1)]
    for (i, j) in even:
        assert np.abs(g[..., i, j].imag).max() <= tol * scale
    for (i, j) in odd:
        assert np.abs(g[..., i, j].real).max() <= tol * scale
    # g^k(-d) = conj g^k(d)
    assert np.abs(g[1] - np.conj(g[0])).max() <= tol * scale
    # k = 0 and k = L/2 modes are real
    assert np.abs(g[:, 0].imag).max() <= tol * scale
    assert np.abs(g[:, -1].imag).max() <= tol * scale


def _line_force_2d(d, mu, nu):
    """2D isotropic line-force solution (unit force per unit length)."""
    x = np.asarray(d, dtype=np.float64)
    r2 = float(x @ x)
    G = np.zeros((3, 3))
    pre = 1.0 / (8.0 * math.pi * mu * (1.0 - nu))
    for a in range(2):
        for b in range(2):
            G[a, b] = pre * (-(3.0 - 4.0 * nu) * 0.5 * math.log(r2) * (a == b) + x[a] * x[b] / r2)
    G[2, 2] = -0.5 * math.log(r2) / (2.0 * math.pi * mu)
    return G


def test_k0_mode_matches_plane_strain_and_antiplane(oracle_mod):
    mu, nu = ISO["mu"], ISO["nu"]
    L, c = 16, 1.0
    d = np.array([[6, 0], [0, 7], [5, 6], [9, -4], [-8, 8]], dtype=np.int32)
    T = oracle_mod.kernel_table(ISO, L, c, d, n=8, N=8)
    g0 = oracle_mod.mode_table(T)[:, 0].real
    ref = [_line_force_2d(x, mu, nu) / c for x in d]
    for a in range(1, len(d)):
        got = g0[a] - g0[0]
        want = ref[a] - ref[0]
        assert np.abs(got - want).max() < 2e-8 * np.abs(want).max()


def _kelvin_line_ft(d, q, mu, nu):
    """Fourier transform along z of the Kelvin kernel, q != 0:
    int G(d, z) exp(-i q z) dz, from FT[1/R] = 2 K0, FT[1/R^3] = 2|q| K1 / rho,
    FT[z/R^3] = -2 i q K0 and z^2/R^3 = 1/R - rho^2/R^3."""
    rho = float(np.hypot(d[0], d[1]))
    aq = abs(q)
    k0 = special.k0(aq * rho)
    k1 = special.k1(aq * rho)
    ft_inv_r = 2.0 * k0
    ft_inv_r3 = 2.0 * aq * k1 / rho
    ft_z_r3 = -2j * q * k0
    pre = 1.0 / (16.0 * math.pi * mu * (1.0 - nu))
    G = np.zeros((3, 3), dtype=complex)
    for a in range(2):
        for b in range(2):
            G[a, b] = pre * ((3.0 - 4.0 * nu) * ft_inv_r * (a == b) + d[a] * d[b] * ft_inv_r3)
        G[a, 2] = G[2, a] = pre * d[a] * ft_z_r3
    G[2, 2] = pre * ((3.0 - 4.0 * nu) * ft_inv_r + ft_inv_r - rho * rho * ft_inv_r3)
    return G


def test_kge1_modes_match_bessel_poisson_sum(oracle_mod):
    mu, nu = ISO["mu"], ISO["nu"]
    L, c = 16, 1.0
    d = np.array([[1, 0], [2, 3], [6, -5], [12, 1]], dtype=np.int32)
    T = oracle_mod.kernel_table(ISO, L, c, d, n=8, N=8)
    g = oracle_mod.mode_table(T)
    for a, x in enumerate(d):
        # high modes at large |d| decay like exp(-q |d|) below the rounding of the
        # table, so the error is measured against the largest mode of this d
        scale = np.abs(g[a, 1:]).max()
        for k in range(1, L // 2 + 1):
            th = 2.0 * math.pi * k / L
            ref = sum(_kelvin_line_ft(x, (th + 2.0 * math.pi * m) / c, mu, nu) for m in range(-12, 13)) / c
            # Richardson truncation at (n, N) = (8, 8) is ~2e-9 when |d| ~ L
            assert np.abs(g[a, k] - ref).max() < 5e-9 * scale, (x, k)
