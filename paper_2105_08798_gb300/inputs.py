"""Seeded synthetic workloads for the flexible-boundary-condition pad update.

This module only *generates inputs*: integer column sites and random force
vectors.  It holds none of the method's arithmetic (no Green function, no
projection, no transform), so the CUDA path and the CPU oracle can both be fed
from it without sharing any computation.

Geometry (Sec. 2.1, the line-periodic slab of a Bravais lattice): every atom
column sits at an integer in-plane site ``x in Z^2`` and repeats ``L`` times
along the line with spacing ``c``.  The interface set (sources, the paper's
``Lambda^{i+}``) and the pad set (targets, ``Lambda^p``) are concentric rings
around the dislocation core:

* ``R_I = 10 * sqrt(N_I / 200)``;
* interface = the ``N_I`` sites with ``|x| <= R_I`` that lie farthest out;
* pad = the ``N_P`` sites with ``|x| > R_I`` that lie closest in;
* ties are broken by ``(|x|^2, atan2(y, x), x, y)``.

The two sets are disjoint, so no pair has ``x_a - x_b = 0``.

Forces: i.i.d. standard normal in 3 components per atom from
``numpy.random.Generator(PCG64(seed))``, laid out ``[n_rhs][N_I][L][3]``.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "ring_geometry",
    "core_sites",
    "forces",
    "Workload",
    "WORKLOADS",
    "batch_instances",
]


def _sites_sorted(r2_max: int) -> np.ndarray:
    """All integer sites with ``x^2 + y^2 <= r2_max``, sorted by the tie rule."""
    R = int(math.isqrt(r2_max)) + 1
    ax = np.arange(-R, R + 1, dtype=np.int64)
    X, Y = np.meshgrid(ax, ax, indexing="ij")
    X = X.ravel()
    Y = Y.ravel()
    r2 = X * X + Y * Y
    keep = r2 <= r2_max
    X, Y, r2 = X[keep], Y[keep], r2[keep]
    ang = np.arctan2(Y.astype(np.float64), X.astype(np.float64))
    order = np.lexsort((Y, X, ang, r2))  # last key is the primary key
    return np.stack([X[order], Y[order]], axis=1), r2[order]


def ring_geometry(n_i: int, n_p: int) -> tuple[np.ndarray, np.ndarray]:
    """Interface and pad column sites, ``int32 [n][2]`` each.

    ``|x| <= R_I`` is tested exactly as ``200 |x|^2 <= 100 N_I``, i.e.
    ``2 |x|^2 <= N_I``.
    """
    if n_i <= 0 or n_p <= 0:
        raise ValueError("n_i and n_p must be positive")
    # enough sites for both rings: area ~ pi r^2 per unit cell
    need = n_i + n_p
    r2_max = int(math.ceil((n_i / 2.0) + need / math.pi * 1.3 + 64))
    while True:
        xy, r2 = _sites_sorted(r2_max)
        inner = 2 * r2 <= n_i
        n_inner = int(inner.sum())
        n_outer = len(xy) - n_inner
        if n_inner >= n_i and n_outer >= n_p:
            break
        r2_max *= 2
    xy_inner = xy[inner]
    xy_outer = xy[~inner]
    xy_i = xy_inner[n_inner - n_i:]
    xy_p = xy_outer[:n_p]
    return np.ascontiguousarray(xy_i, dtype=np.int32), np.ascontiguousarray(xy_p, dtype=np.int32)


def core_sites(n_i: int) -> np.ndarray:
    """The sites inside the interface ring (the atomistic core, ``Lambda^a``), ``int32 [n][2]``:
    every site with ``2 |x|^2 <= N_I`` that ``ring_geometry`` does not put in the interface, in
    the same tie order.  Together with the interface and a pad of at least two site layers they
    contain every site within one lattice step (in x and y) of an interface site."""
    r2_max = int(math.ceil(n_i / 2.0)) + 1
    xy, r2 = _sites_sorted(r2_max)
    inner = 2 * r2 <= n_i
    n_inner = int(inner.sum())
    if n_inner < n_i:
        raise ValueError("fewer sites inside the ring than interface sites")
    return np.ascontiguousarray(xy[inner][: n_inner - n_i], dtype=np.int32)


def forces(n_rhs: int, n_i: int, L: int, seed: int, decay: float | None = None) -> np.ndarray:
    """Random interface forces ``float64 [n_rhs][n_i][L][3]``.

    With ``decay`` set, right-hand side ``j`` is scaled by ``decay**j`` (the
    successive residuals of a relaxation, each smaller than the last).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    f = rng.standard_normal((n_rhs, n_i, L, 3))
    if decay is not None:
        f *= (decay ** np.arange(n_rhs, dtype=np.float64))[:, None, None, None]
    return f


@dataclass(frozen=True)
class Workload:
    """One named workload: ring sizes, line repeats, material and seed."""

    name: str
    n_i: int
    n_p: int
    L: int
    n_rhs: int
    material: dict = field(default_factory=dict)
    seed: int = 0
    c: float = 1.0

    @property
    def pair_modes(self) -> int:
        """Pad column x interface column x mode (k = 0..L/2) x right-hand side."""
        return self.n_p * self.n_i * (self.L // 2 + 1) * self.n_rhs

    def geometry(self):
        return ring_geometry(self.n_i, self.n_p)

    def forces(self, seed: int | None = None):
        return forces(self.n_rhs, self.n_i, self.L, self.seed if seed is None else seed)


ISO = {"kind": "isotropic", "mu": 1.0, "nu": 0.3}
CUBIC = {"kind": "cubic", "C11": 1.5, "C12": 1.0, "C44": 0.9}

WORKLOADS = {
    # tiny isotropic case the oracle evaluates in full
    "ring200x300_L16_iso": Workload("ring200x300_L16_iso", 200, 300, 16, 1, ISO, 0),
    # paper-scale single instance, cubic medium (Zener ratio 3.6)
    "ring4000x6000_L256_cubic": Workload("ring4000x6000_L256_cubic", 4000, 6000, 256, 1, CUBIC, 1),
    # precision sweep size: 64 right-hand sides, isotropic
    "ring8000x12000_L1024_rhs64_iso": Workload("ring8000x12000_L1024_rhs64_iso", 8000, 12000, 1024, 64, ISO, 4),
    # the same kind of case at a size a profiler capture can hold (a few GB on the device)
    "ring4000x6000_L256_rhs64_iso": Workload("ring4000x6000_L256_rhs64_iso", 4000, 6000, 256, 64, ISO, 5),
    # the H-matrix comparison: 96 000 pad atoms, where the H-matrix at eps = 1e-5 (about 19 GB of
    # FP32 factors) fits on one GPU; at 4000 x 6000, L = 256 it does not
    "ring1000x1500_L64_iso": Workload("ring1000x1500_L64_iso", 1000, 1500, 64, 1, ISO, 6),
}


def batch_instances(n_inst: int = 64, n_rhs: int = 16, base_seed: int = 1000):
    """The batched workload: uneven instances drawn from a seeded generator.

    ``N_I ~ U[500, 8000]``, ``N_P = 1.5 N_I`` (rounded), ``L`` uniform over
    {32, 64, 128, 256, 512}; instance ``i`` draws its forces with seed
    ``base_seed + i`` and right-hand side ``j`` is scaled by ``0.5**j``.
    """
    rng = np.random.Generator(np.random.PCG64(base_seed))
    out = []
    for i in range(n_inst):
        n_i = int(rng.integers(500, 8001))
        n_p = int(round(1.5 * n_i))
        L = int(rng.choice([32, 64, 128, 256, 512]))
        out.append(dict(index=i, n_i=n_i, n_p=n_p, L=L, n_rhs=n_rhs, seed=base_seed + i, material=ISO))
    return out
