"""Pins of the lattice Green function oracle (App., the inverse transform of the inverted symbol).

* the stencil applied to the Green function gives the unit impulse (exactly, on the zone grid's
  n-periodic lattice; for k = 0 minus the uniform 1/n^2 the zero-mean function carries);
* the mirror structure of the six-real mode layout: the in-plane and diagonal entries are real,
  the 13 and 23 entries imaginary, a_ij even and b_i3 odd in d;
* the far field is the continuum Green function of the medium the spring model stands for
  (C11 = k1 + 2 k2, C12 = C44 = k2 for c = 1), computed by the oracle's own image sums: within
  1 % in the long-wave modes and for differences of the k = 0 mode.
"""

import itertools

import numpy as np
import pytest

from oracle import harmonic

K1, K2, L = 1.0, 0.4, 64


@pytest.fixture(scope="module")
def K():
    return harmonic.spring_blocks(K1, K2, 1.0)


@pytest.mark.parametrize("k", [0, 1, 5])
def test_stencil_applied_to_green_function_is_an_impulse(K, k):
    n = 48
    Kb = np.asarray(K).reshape(27, 3, 3)
    targets = [(0, 0), (1, 0), (3, -2)]
    offs = [o for o in itertools.product((-1, 0, 1), repeat=3)]
    need = sorted({(dx + nx, dy + ny) for dx, dy in targets for nx, ny, _ in offs})
    g = harmonic.lattice_mode_table(K, 8, need, [k], n)[:, 0]
    at = {d: g[i] for i, d in enumerate(need)}
    for d in targets:
        acc = np.zeros((3, 3), dtype=complex)
        for j, (nx, ny, nz) in enumerate(offs):
            acc += np.exp(2j * np.pi * k * nz / 8) * Kb[j] @ at[(d[0] + nx, d[1] + ny)]
        want = (np.eye(3) if d == (0, 0) else 0.0) - (np.eye(3) / n**2 if k == 0 else 0.0)
        assert np.abs(acc - want).max() <= 1e-12, (d, k)


@pytest.mark.parametrize("L", [4, 8])
def test_real_space_table_is_the_periodic_lattice_green_function(K, L):
    """In real space along the line: sum_n K(n) G(d + n_xy, s + n_z) = delta(d) delta(s) I - I / (n^2 L)
    (the unit impulse on the n x n x L periodic lattice, minus the uniform mode that is left out)."""
    n = 32
    Kb = np.asarray(K).reshape(27, 3, 3)
    targets = [(0, 0), (1, 0), (2, -3)]
    offs = [o for o in itertools.product((-1, 0, 1), repeat=3)]
    need = sorted({(dx + nx, dy + ny) for dx, dy in targets for nx, ny, _ in offs})
    G = harmonic.lattice_kernel_table(K, L, need, n)
    at = {d: G[i] for i, d in enumerate(need)}
    for d in targets:
        for s in range(L):
            acc = np.zeros((3, 3))
            for j, (nx, ny, nz) in enumerate(offs):
                acc += Kb[j] @ at[(d[0] + nx, d[1] + ny)][(s + nz) % L]
            want = (np.eye(3) if d == (0, 0) and s == 0 else 0.0) - np.eye(3) / (n * n * L)
            assert np.abs(acc - want).max() <= 1e-12, (d, s)
    # symmetric blocks, even in (d, s), mirror-symmetric along the line
    G2 = harmonic.lattice_kernel_table(K, L, [(2, -3), (-2, 3)], n)
    M = np.diag([1.0, 1.0, -1.0])
    for s in range(L):
        assert np.abs(G2[0, s] - G2[0, s].T).max() <= 1e-14
        assert np.abs(G2[1, (-s) % L] - G2[0, s]).max() <= 1e-14
        assert np.abs(G2[0, (-s) % L] - M @ G2[0, s] @ M).max() <= 1e-14


def test_real_space_update_matches_mode_space_update(K, oracle_mod):
    """The two oracle forms of the update with the lattice Green function agree (the real-space double
    sum in C against numpy's real FFTs and per-mode products)."""
    from paper_2105_08798_gb300 import inputs

    Ls = 8
    xy_i, xy_p = inputs.ring_geometry(24, 30)
    f = inputs.forces(2, len(xy_i), Ls, seed=5)
    d = np.unique((xy_p[:, None, :] - xy_i[None, :, :]).reshape(-1, 2), axis=0)
    g = harmonic.lattice_mode_table(K, Ls, d, list(range(Ls // 2 + 1)), 48)
    gk = {tuple(x): g[i] for i, x in enumerate(d.tolist())}
    u_modes = oracle_mod.mode_space_update(xy_i, xy_p, Ls, f, lambda dd: gk[dd])
    u_real = oracle_mod.real_space_update(xy_i, xy_p, Ls, f, lambda dl: harmonic.lattice_kernel_table(K, Ls, dl, 48))
    assert np.linalg.norm(u_real - u_modes) <= 1e-13 * np.linalg.norm(u_modes)


def test_mirror_structure(K):
    ds = [(2, 1), (-2, -1), (0, 3), (4, -1)]
    g = harmonic.lattice_mode_table(K, 16, ds, [1, 3], 64)
    scale = np.abs(g).max()
    for a, b in ((0, 0), (0, 1), (1, 1), (2, 2)):
        assert np.abs(g[..., a, b].imag).max() <= 1e-14 * scale
    for a, b in ((0, 2), (1, 2)):
        assert np.abs(g[..., a, b].real).max() <= 1e-14 * scale
    # a_ij even, b_i3 odd under d -> -d
    np.testing.assert_allclose(g[1, :, 0, 0], g[0, :, 0, 0], atol=1e-14 * scale)
    np.testing.assert_allclose(g[1, :, 0, 2], -g[0, :, 0, 2], atol=1e-14 * scale)


def test_far_field_is_the_continuum_green_function(K, oracle_mod):
    mat = {"kind": "cubic", "C11": K1 + 2 * K2, "C12": K2, "C44": K2}
    ds = [(8, 3), (12, 5), (16, 0), (20, 0)]
    gl = harmonic.lattice_mode_table(K, L, ds, [0, 1, 2], 512)
    gc = oracle_mod.mode_table(oracle_mod.kernel_table(mat, L, 1.0, np.array(ds)))[:, :3]
    for i in range(3):
        for k in (1, 2):
            rel = np.linalg.norm(gl[i, k] - gc[i, k]) / np.linalg.norm(gc[i, k])
            assert rel < 1e-2, (ds[i], k, rel)
        # k = 0: both are defined up to a constant; compare differences to the farthest point
        a, b = gl[i, 0] - gl[3, 0], gc[i, 0] - gc[3, 0]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-2, ds[i]


def test_golden_regression():
    """The stored values written by tests/golden/make_golden_lattice.py (oracle only)."""
    import json
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "spring_lattice_modes_L16_n64.json")
    gold = json.load(open(path))
    K = harmonic.spring_blocks(gold["k1"], gold["k2"], gold["c"])
    g = harmonic.lattice_mode_table(K, gold["L"], gold["d"], gold["k"], gold["n_zone"])
    six = np.stack([g[..., 0, 0].real, g[..., 0, 1].real, g[..., 1, 1].real, g[..., 2, 2].real,
                    g[..., 0, 2].imag, g[..., 1, 2].imag], axis=-1)
    ref = np.array(gold["g"])
    assert np.abs(six - ref).max() <= 1e-13 * np.abs(ref).max()
