"""Pins of the incompatibility-force oracle (Sec. 2.3.2, Eq. 21) against physics and hand values.

* a rigid translation of every site gives no force;
* a homogeneous in-plane strain gives no force on any interface site (inversion
  symmetry of the Bravais lattice: the bond forces cancel pairwise);
* one displaced atom: the forces on its interface neighbour at the three planes it
  reaches, worked out by hand from the spring directions;
* long-wave limit: for c = 1 the spring model is the cubic medium C11 = k1 + 2 k2,
  C12 = C44 = k2, so a plane wave of small wave vector theta sees
  f = Gamma(theta) u with Gamma the Christoffel matrix C_ijkl theta_j theta_l,
  up to O(|theta|^2) relative;
* the block-stencil definition with the C library's spring blocks equals the
  bond-force form (the library's host-only block builder, no device needed);
* the stencil builder rejects a missing neighbour and a doubly listed site before
  it allocates anything (no device needed).
"""

import numpy as np
import pytest

from oracle import harmonic
from paper_2105_08798_gb300 import inputs

N_I, N_P = 200, 300


@pytest.fixture(scope="module")
def geom():
    xy_i, xy_p = inputs.ring_geometry(N_I, N_P)
    return inputs.core_sites(N_I), xy_i, xy_p


def _sources(geom, fill):
    xy_c, xy_i, xy_p = geom
    return [(xy, fill(xy)) for xy in (xy_c, xy_i, xy_p)]


def test_rigid_translation(geom):
    L = 8
    shift = np.array([[0.3, -1.2, 2.0], [1.0, 0.5, -0.25]])  # one per right-hand side
    src = _sources(geom, lambda xy: np.broadcast_to(shift[:, None, None, :], (2, len(xy), L, 3)).copy())
    f = harmonic.spring_incompat_force(geom[1], src, L, 1.3, 2.0, 0.7)
    assert np.abs(f).max() <= 1e-14


def test_homogeneous_in_plane_strain(geom):
    L = 6
    E = np.array([[0.02, -0.01], [0.005, 0.03], [-0.04, 0.015]])  # u = E (x, y), all three components
    src = _sources(geom, lambda xy: np.broadcast_to((xy.astype(float) @ E.T)[None, :, None, :],
                                                    (1, len(xy), L, 3)).copy())
    f = harmonic.spring_incompat_force(geom[1], src, L, 1.5, 1.0, 0.4)
    assert np.abs(f).max() <= 1e-13
    assert np.abs(src[1][1]).max() > 0.1  # the field itself is not small


def test_single_displaced_atom_by_hand():
    # interface site (0, 0) with its eight in-plane neighbours as atoms
    L, c, k1, k2 = 5, 1.5, 2.0, 0.5
    xy_i = np.array([[0, 0]])
    xy_a = np.array([[dx, dy] for dx in (-1, 0, 1) for dy in (-1, 0, 1) if (dx, dy) != (0, 0)])
    u_a = np.zeros((1, len(xy_a), L, 3))
    j = int(np.flatnonzero((xy_a[:, 0] == 1) & (xy_a[:, 1] == 0))[0])
    u_a[0, j, 0] = [1.0, 2.0, 3.0]  # atom (1, 0) displaced at plane 0 only
    src = [(xy_a, u_a), (xy_i, np.zeros((1, 1, L, 3)))]
    f = harmonic.spring_incompat_force(xy_i, src, L, c, k1, k2)[0, 0]
    # plane 0: bond (1,0,0), k1 along x: -2 * (1, 0, 0)
    np.testing.assert_allclose(f[0], [-2.0, 0.0, 0.0], atol=1e-15)
    # plane L-1 reaches plane 0 through bond (1,0,+1), v = (1, 0, 1.5), |v|^2 = 3.25, v.e = 5.5
    np.testing.assert_allclose(f[L - 1], [-0.5 * 5.5 / 3.25, 0.0, -0.5 * 5.5 / 3.25 * 1.5], atol=1e-15)
    # plane 1 through bond (1,0,-1), v = (1, 0, -1.5), v.e = -3.5
    np.testing.assert_allclose(f[1], [0.5 * 3.5 / 3.25, 0.0, -0.5 * 3.5 / 3.25 * 1.5], atol=1e-15)
    assert np.abs(f[2:L - 1]).max() == 0.0


def test_long_wave_limit_is_cubic_elasticity(geom):
    L, k1, k2 = 128, 1.0, 0.35
    C11, C12, C44 = k1 + 2 * k2, k2, k2
    th = np.array([0.031, -0.022, 2 * np.pi / L])
    w = np.array([0.7, -0.2, 0.5])

    def wave(xy):
        q = np.arange(L)
        ph = th[0] * xy[:, 0, None] + th[1] * xy[:, 1, None] + th[2] * q[None, :]
        return (np.cos(ph)[..., None] * w)[None]

    src = _sources(geom, wave)
    f = harmonic.spring_incompat_force(geom[1], src, L, 1.0, k1, k2)
    G = np.empty((3, 3))  # Christoffel matrix of the cubic medium
    for i in range(3):
        for k in range(3):
            if i == k:
                G[i, i] = C11 * th[i] ** 2 + C44 * (th @ th - th[i] ** 2)
            else:
                G[i, k] = (C12 + C44) * th[i] * th[k]
    pred = src[1][1] @ G.T
    rel = np.linalg.norm(f - pred) / np.linalg.norm(pred)
    assert rel < 5e-3, rel


def test_library_spring_blocks_match_bond_form(geom):
    from paper_2105_08798_gb300 import build, fbc

    build.build()
    fbc.load()
    L, c, k1, k2 = 7, 1.25, 1.6, 0.45
    K = fbc.fbc_spring_constants(k1, k2, c)
    assert np.abs(K.reshape(27, 9).sum(axis=0)).max() <= 1e-15  # rows of L_h sum to zero
    assert np.allclose(K, K.transpose(0, 2, 1))
    rng = np.random.default_rng(3)
    src = _sources(geom, lambda xy: rng.normal(0, 1, (2, len(xy), L, 3)))
    a = harmonic.stencil_apply(geom[1], src, L, K)
    b = harmonic.spring_incompat_force(geom[1], src, L, c, k1, k2)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
    # the oracle's own blocks: the same operator as the bond form, and the same numbers as the library's
    Ko = harmonic.spring_blocks(k1, k2, c)
    a2 = harmonic.stencil_apply(geom[1], src, L, Ko)
    assert np.abs(a2 - b).max() <= 1e-13 * np.abs(b).max()
    np.testing.assert_allclose(K, Ko, rtol=0, atol=1e-15)


def test_stencil_builder_rejects_bad_geometry(geom):
    from paper_2105_08798_gb300 import build, fbc

    build.build()
    fbc.load()
    xy_c, xy_i, xy_p = geom
    K = fbc.fbc_spring_constants(1.0, 0.5, 1.0)
    with pytest.raises(fbc.FBCError, match="in no source set"):
        fbc.fbc_stencil_create(xy_i, [xy_c, xy_i, xy_p[:20]], 8, K)  # pad too thin
    with pytest.raises(fbc.FBCError, match="appears twice"):
        fbc.fbc_stencil_create(xy_i, [xy_c, xy_i, np.concatenate([xy_p, xy_i[:1]])], 8, K)
    with pytest.raises(fbc.FBCError):
        fbc.fbc_stencil_create(xy_i, [xy_c, xy_i, xy_p], 0, K)
