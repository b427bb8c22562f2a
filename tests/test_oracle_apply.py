"""Pins of the oracle's real-space pad update (Sec. 1, Eq. 1; Sec. 3.2, Eqs. 37-38).

* A numpy brute-force double sum over (b, q) with its own indexing agrees.
* One pad column against one interface column is a circular convolution along
  the line, which numpy's FFT evaluates independently.
* Linearity; rolling the forces along the line rolls the result exactly.
* Adding a constant tensor to the kernel leaves u unchanged once the forces are
  neutral (the regularisation of Eq. 32 is a constant shift).
* The projection leaves zero net force; the zero-mean step (Eq. 23) leaves
  zero mean pad displacement; sampled and full evaluations agree.
* A golden regression file, written by ``tests/golden/make_golden.py`` from the
  oracle alone, guards the oracle against drift across hosts.
"""

import json
import os

import numpy as np
import pytest

from conftest import CUBIC, ISO
from paper_2105_08798_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_case(n_i=3, n_p=4, L=16, seed=11):
    rng = np.random.default_rng(seed)
    xy_i = np.array([[5, 1], [-4, 3], [2, -6]], dtype=np.int32)[:n_i]
    xy_p = np.array([[9, 0], [0, 9], [-8, -3], [6, 7]], dtype=np.int32)[:n_p]
    f = rng.standard_normal((2, n_i, L, 3))
    return xy_i, xy_p, L, f


def test_brute_force_numpy_double_sum(oracle_mod):
    xy_i, xy_p, L, f = _small_case()
    u = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, CUBIC, f, project=False, nquad=64)
    d_list, d_index = oracle_mod.difference_index(xy_i, xy_p)
    T = oracle_mod.kernel_table(CUBIC, L, 1.0, d_list, nquad=64)
    ref = np.zeros_like(u)
    for r in range(f.shape[0]):
        for a in range(len(xy_p)):
            for p in range(L):
                acc = np.zeros(3)
                for b in range(len(xy_i)):
                    d = xy_p[a] - xy_i[b]
                    row = np.flatnonzero((d_list == d).all(axis=1))[0]
                    for q in range(L):
                        acc += T[row, (p - q) % L] @ f[r, b, q]
                ref[r, a, p] = acc
    assert np.abs(u - ref).max() <= 1e-14 * np.abs(ref).max()


def test_single_pair_is_circular_convolution(oracle_mod):
    L = 32
    xy_i = np.array([[3, -2]], dtype=np.int32)
    xy_p = np.array([[-5, 4]], dtype=np.int32)
    f = np.random.default_rng(3).standard_normal((1, 1, L, 3))
    u = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f, project=False)[0, 0]
    T = oracle_mod.kernel_table(ISO, L, 1.0, (xy_p - xy_i))[0]  # [L][3][3]
    That = np.fft.fft(T, axis=0)
    Fhat = np.fft.fft(f[0, 0], axis=0)
    ref = np.fft.ifft(np.einsum("kij,kj->ki", That, Fhat), axis=0).real
    assert np.abs(u - ref).max() <= 1e-13 * np.abs(ref).max()


def test_linearity_and_roll(oracle_mod):
    xy_i, xy_p = inputs.ring_geometry(40, 50)
    L = 16
    f = inputs.forces(2, 40, L, seed=5)
    u = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f)
    u1 = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f[:1])
    u2 = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f[1:])
    ua = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, 2.5 * f[:1] - 0.75 * f[1:])
    assert np.abs(ua - (2.5 * u1 - 0.75 * u2)).max() <= 1e-13 * np.abs(ua).max()
    assert np.abs(u[:1] - u1).max() == 0.0
    ur = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, np.roll(f, 3, axis=2))
    assert np.abs(ur - np.roll(u, 3, axis=2)).max() <= 1e-13 * np.abs(u).max()


def test_constant_kernel_shift_is_invisible_after_projection(oracle_mod):
    xy_i, xy_p = inputs.ring_geometry(30, 40)
    L = 16
    f = oracle_mod.project_neutral(inputs.forces(1, 30, L, seed=9))
    d_list, d_index = oracle_mod.difference_index(xy_i, xy_p)
    T = oracle_mod.kernel_table(ISO, L, 1.0, d_list)
    cols = np.repeat(np.arange(len(xy_p)), L)
    ps = np.tile(np.arange(L), len(xy_p))
    u = oracle_mod.real_space_sum(d_index, T, f, cols, ps)
    C = np.array([[1.0, 0.2, -0.3], [0.2, -0.7, 0.1], [-0.3, 0.1, 0.4]])
    u_shift = oracle_mod.real_space_sum(d_index, T + C, f, cols, ps)
    assert np.abs(u_shift - u).max() < 1e-13 * np.abs(u).max()
    # without neutrality the shift is visible
    fr = inputs.forces(1, 30, L, seed=9)
    v = oracle_mod.real_space_sum(d_index, T, fr, cols, ps)
    v_shift = oracle_mod.real_space_sum(d_index, T + C, fr, cols, ps)
    assert np.abs(v_shift - v).max() > 1e-3 * np.abs(v).max()


def test_projection_and_zero_mean(oracle_mod):
    f = inputs.forces(3, 50, 16, seed=2) + 0.7
    fp = oracle_mod.project_neutral(f)
    assert np.abs(fp.sum(axis=(1, 2))).max() < 1e-12
    assert np.abs(oracle_mod.project_neutral(fp) - fp).max() < 1e-15
    u = np.random.default_rng(1).standard_normal((2, 20, 16, 3)) + 3.0
    uz = oracle_mod.zero_mean(u)
    assert np.abs(uz.mean(axis=(1, 2))).max() < 1e-15
    assert np.abs((u - uz) - (u - uz)[:, :1, :1, :]).max() < 1e-14


def test_samples_match_full_and_update_form(oracle_mod):
    xy_i, xy_p = inputs.ring_geometry(60, 80)
    L = 16
    f = inputs.forces(1, 60, L, seed=4)
    u0 = np.random.default_rng(8).standard_normal((1, 80, L, 3))
    full = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f, alpha=-0.6, beta=1.0, u0=u0)
    rng = np.random.default_rng(0)
    samples = np.stack([rng.integers(0, 80, 25), rng.integers(0, L, 25)], axis=1)
    part = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f, alpha=-0.6, beta=1.0, u0=u0, samples=samples)
    assert np.abs(part[0] - full[0, samples[:, 0], samples[:, 1]]).max() == 0.0


def test_golden_regression(oracle_mod):
    with open(os.path.join(GOLDEN, "ring200x300_L16_iso_samples.json")) as fh:
        g = json.load(fh)
    w = inputs.WORKLOADS["ring200x300_L16_iso"]
    xy_i, xy_p = w.geometry()
    f = w.forces()
    samples = np.asarray(g["samples"], dtype=np.int64)
    u = oracle_mod.pad_update(xy_i, xy_p, w.L, w.c, w.material, f, samples=samples,
                              n=g["rich_n"], N=g["rich_N"])
    ref = np.asarray(g["u"], dtype=np.float64)
    assert np.abs(u[0] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_mode_space_update_matches_real_space_sum(oracle_mod):
    """The mode-by-mode update with the continuum mode table (convolution theorem along the line)
    equals the real-space sum over all pairs and repeats."""
    from conftest import ISO
    from paper_2105_08798_gb300 import inputs

    xy_i, xy_p = inputs.ring_geometry(60, 90)
    L = 8
    f = inputs.forces(2, 60, L, seed=3)
    d = np.unique((xy_p[:, None, :] - xy_i[None, :, :]).reshape(-1, 2), axis=0)
    cont = oracle_mod.mode_table(oracle_mod.kernel_table(ISO, L, 1.0, d))
    gk = {tuple(x): cont[i] for i, x in enumerate(d.tolist())}
    a = oracle_mod.mode_space_update(xy_i, xy_p, L, f, lambda dd: gk[dd])
    b = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-13
