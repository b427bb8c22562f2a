"""Oracle of the incompatibility force (Sec. 2.3.2, Eq. 21; Algorithm 1).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy, FP64,
written from the definitions:

* ``stencil_apply`` -- the harmonic operator as a local block stencil,
  ``f(a, q) = sum_n K(n) u(x_a + (n_x, n_y), (q + n_z) mod L)``, rows restricted
  to the interface columns, each neighbour's displacement taken from the site
  set that holds it (the relaxed atoms with u_{k+1}, the continuum nodes with
  u_k), which is ``L^{i+|i}[u_{k+1}] + L^{i+|i++}[u_k]``.
* ``spring_incompat_force`` -- the same quantity for the synthetic spring
  model written as a sum of pair forces, ``f(a) = sum_bonds k v v^T / |v|^2
  (u(a) - u(a + n))`` (the stiffness acting on the interface site), without
  any block table.
* ``spring_bonds`` -- the model's bonds: central springs k1 to the neighbours
  with |n|_1 = 1 and k2 to those with |n|_1 = 2 on the lattice with in-plane
  spacing 1 and plane spacing c; ``spring_blocks`` -- the same as a block
  stencil.
* ``symbol`` and ``lattice_mode_table`` -- the lattice Green function of the
  stencil (App., the inverse transform of the inverted Fourier symbol), in
  the modes of the line-periodic lattice, by the zone grid's trapezoid rule.
"""

from __future__ import annotations

import itertools

import numpy as np


def spring_bonds(k1: float, k2: float, c: float):
    """[(n, k, v)] for the 18 bonds of a site: n integer offset, k stiffness, v = (n_x, n_y, c n_z)."""
    out = []
    for n in itertools.product((-1, 0, 1), repeat=3):
        l1 = sum(abs(t) for t in n)
        if l1 in (1, 2):
            out.append((n, k1 if l1 == 1 else k2, np.array([n[0], n[1], c * n[2]], dtype=np.float64)))
    return out


def spring_blocks(k1: float, k2: float, c: float) -> np.ndarray:
    """The spring model as a block stencil K [27][3][3] (offset index (n_x+1)*9 + (n_y+1)*3 + (n_z+1)):
    K(n) = -k v v^T / |v|^2 for each bond, K(0) = minus the sum of the others."""
    K = np.zeros((27, 3, 3))
    for n, k, v in spring_bonds(k1, k2, c):
        blk = k * np.outer(v, v) / float(v @ v)
        K[(n[0] + 1) * 9 + (n[1] + 1) * 3 + (n[2] + 1)] -= blk
        K[13] += blk
    return K


def _site_lookup(sources):
    where = {}
    for s, (xy, _) in enumerate(sources):
        for t, (x, y) in enumerate(np.asarray(xy).reshape(-1, 2)):
            key = (int(x), int(y))
            if key in where:
                raise ValueError(f"site {key} is in two source sets")
            where[key] = (s, t)
    return where


def _column(sources, where, x: int, y: int):
    """u[:, column, :, :] of the site (x, y): [R][L][3]."""
    if (x, y) not in where:
        raise ValueError(f"site {(x, y)} is in no source set")
    s, t = where[(x, y)]
    return np.asarray(sources[s][1], dtype=np.float64)[:, t]


def stencil_apply(xy_i, sources, L: int, K) -> np.ndarray:
    """f [R][n_i][L][3] = sum over the 27 offsets of K(n) u(x_a + n_xy, q + n_z); ``sources`` is a list of
    (xy [n][2], u [R][n][L][3]); K [27][3][3] with offset index (n_x+1)*9 + (n_y+1)*3 + (n_z+1)."""
    K = np.asarray(K, dtype=np.float64).reshape(27, 3, 3)
    where = _site_lookup(sources)
    xy_i = np.asarray(xy_i).reshape(-1, 2)
    R = np.asarray(sources[0][1]).shape[0]
    f = np.zeros((R, len(xy_i), L, 3))
    for a, (x, y) in enumerate(xy_i):
        for nx, ny, nz in itertools.product((-1, 0, 1), repeat=3):
            Kn = K[(nx + 1) * 9 + (ny + 1) * 3 + (nz + 1)]
            if not Kn.any():
                continue
            col = _column(sources, where, int(x) + nx, int(y) + ny)  # [R][L][3]
            shifted = np.roll(col, -nz, axis=1)  # shifted[:, q] = col[:, (q + nz) mod L]
            f[:, a] += shifted @ Kn.T
    return f


def spring_incompat_force(xy_i, sources, L: int, c: float, k1: float, k2: float) -> np.ndarray:
    """f [R][n_i][L][3] of the spring model as a sum of bond forces on each interface site."""
    where = _site_lookup(sources)
    xy_i = np.asarray(xy_i).reshape(-1, 2)
    R = np.asarray(sources[0][1]).shape[0]
    f = np.zeros((R, len(xy_i), L, 3))
    bonds = spring_bonds(k1, k2, c)
    for a, (x, y) in enumerate(xy_i):
        u_a = _column(sources, where, int(x), int(y))
        for n, k, v in bonds:
            u_b = np.roll(_column(sources, where, int(x) + n[0], int(y) + n[1]), -n[2], axis=1)
            stretch = (u_a - u_b) @ v  # [R][L]: bond elongation times |v|
            f[:, a] += (k / float(v @ v)) * stretch[..., None] * v
    return f


def symbol(K, theta) -> np.ndarray:
    """Fourier symbol of the block stencil, D(theta) = sum_n K(n) exp(-i theta . n), theta [..., 3]
    (App., the transform of the lattice Green function); returns complex [..., 3, 3]."""
    K = np.asarray(K, dtype=np.float64).reshape(27, 3, 3)
    theta = np.asarray(theta, dtype=np.float64)
    D = np.zeros(theta.shape[:-1] + (3, 3), dtype=np.complex128)
    for j, (nx, ny, nz) in enumerate(itertools.product((-1, 0, 1), repeat=3)):
        if K[j].any():
            ph = np.exp(-1j * (theta[..., 0] * nx + theta[..., 1] * ny + theta[..., 2] * nz))
            D += ph[..., None, None] * K[j]
    return D


def lattice_mode_table(K, L: int, d_list, ks, n: int) -> np.ndarray:
    """Lattice Green function of the stencil in the modes of the line-periodic lattice (App., the
    inverse transform of the inverted symbol), complex [len(d_list)][len(ks)][3][3]:

        g^k(d) = (1 / n^2) sum_{theta in the n x n zone grid} D(theta_x, theta_y, 2 pi k / L)^-1
                 exp(i theta . d),   theta_x, theta_y = 2 pi j / n.

    This is the trapezoid rule for the zone integral (2 pi)^-2 int D^-1 exp(i theta . d), and the
    exact Green function of the lattice made n-periodic in the plane.  For k = 0 the symbol is
    singular at theta = 0; that term is left out (the zero-mean periodic Green function, defined up
    to the constant every Green function of the plane carries)."""
    d_list = np.asarray(d_list).reshape(-1, 2)
    th = 2.0 * np.pi * np.arange(n) / n
    TX, TY = np.meshgrid(th, th, indexing="ij")
    out = np.zeros((len(d_list), len(ks), 3, 3), dtype=np.complex128)
    for ik, k in enumerate(ks):
        theta = np.stack([TX, TY, np.full_like(TX, 2.0 * np.pi * k / L)], axis=-1)
        D = symbol(K, theta)
        if k % L == 0:
            D[0, 0] = np.eye(3)  # placeholder, its inverse is zeroed below
        Dinv = np.linalg.inv(D)
        if k % L == 0:
            Dinv[0, 0] = 0.0
        for idd, (dx, dy) in enumerate(d_list):
            ph = np.exp(1j * (TX * dx + TY * dy))
            out[idd, ik] = np.einsum("xy,xyij->ij", ph, Dinv) / (n * n)
    return out


def lattice_kernel_table(K, L: int, d_list, n: int) -> np.ndarray:
    """The lattice Green function of the stencil in real space along the line (App.), float64
    [len(d_list)][L][3][3]:

        G_lat(d, s) = (1 / L) sum_{k = 0}^{L - 1} g^k(d) exp(2 pi i k s / L),

    with g^k(d) the zone sums of ``lattice_mode_table`` and g^{L - k} = conj g^k (the symbol is real
    and even, so the Green function is real).  This is the Green function of the stencil on the
    n x n x L periodic lattice with the uniform mode left out: applying the stencil gives the unit
    impulse minus I / (n^2 L).  The inverse DFT is written out as a plain sum over k."""
    d_list = np.asarray(d_list).reshape(-1, 2)
    Kh = L // 2 + 1
    g = lattice_mode_table(K, L, d_list, list(range(Kh)), n)  # [nd][Kh][3][3]
    full = np.empty((len(d_list), L, 3, 3), dtype=np.complex128)
    full[:, :Kh] = g
    for k in range(Kh, L):
        full[:, k] = np.conj(g[:, L - k])
    out = np.zeros((len(d_list), L, 3, 3), dtype=np.complex128)
    for s in range(L):
        for k in range(L):
            out[:, s] += full[:, k] * np.exp(2j * np.pi * k * s / L)
    out /= L
    if np.abs(out.imag).max() > 1e-12 * max(np.abs(out.real).max(), 1e-300):
        raise ValueError("lattice Green function is not real: the stencil's symbol is not real and even")
    return out.real.copy()
