"""Oracle of the hierarchical-matrix (H-matrix) form of the pad update (Sec. 3.2; App., the
construction of the H-matrix approximation of the Green matrix).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy, FP64, written from the
paper's three construction steps and used to check the device H-matrix:

* The Green matrix (Sec. 3.2) has 3 x 3 blocks G~(x_a - x_b, (p - q) c).  Its rows are the pad
  atoms (a, p) and its columns the interface atoms (b, q).  Every atom is a site (x, y) of its
  column at height z = p c, and z is periodic with period L c.
* ``cluster_tree`` (Step 1) does geometric clustering by binary space partitioning.  A cluster
  with more than ``b_min`` atoms is split at the midpoint of the longest side of its bounding
  box.  Atoms on the midpoint go to the first child, and each child keeps the atoms' order.
* ``partition`` (Step 2) uses the admissibility criterion with the periodic neighbours s+ and s-
  (the same cluster one period up and down).  A block t x s is admissible when
  min(diam t, diam s') <= gamma dist(t, s') holds for every s' in {s, s+, s-}.  diam is the
  diagonal of the cluster's bounding box and dist is the distance between the centroids.  An
  admissible block is a low-rank leaf.  A block of two leaves that is not admissible is dense.
  Otherwise the non-leaf clusters are split and the children are examined.
* ``aca`` (Step 3) is adaptive cross approximation with partial pivoting (the linear-cost
  heuristic: a row is chosen, then the largest entry of that row's residual).  It pivots on
  atoms (3 x 3 blocks): see below.
* ``HMatrix.matvec``: u = G_H f.

Readings, where the paper leaves a choice to its library:

1. Pivots are atoms, not single rows.  The residual rows of the pivot atom are computed.  The
   column atom is the one whose 3 x 3 residual block has the largest Frobenius norm.  Up to
   three rank-1 terms are then taken from that 3 x 3 block by elimination with full pivoting.
   A pivot smaller than ``PIVOT_DROP`` times the block's first pivot ends the step: that is the
   scale of the rounding left in the residual by the stored terms (FP32 on the device), and a
   pivot at that level adds noise and can fill the rank of a small block.  Scalar
   pivoting stalls on this kernel: the z rows decouple from the in-plane rows at s = 0 and
   s = L/2, and the partial search then misses whole components.
2. The stopping rule is the paper's "norm of R^k - R^(k-1) below eps", taken relative.  The
   Frobenius norm of the step's terms must be <= eps ||S||_F, where S is the approximation so
   far, on ``STOP_STEPS`` consecutive steps.  One small step alone sometimes stops the scalar
   and the atom-pivoted forms early.
3. The next pivot atom is the unused row atom where the step's new column vectors have the
   largest norm.  The first pivot atom is the block's first row atom.
4. ``b_min`` counts atoms, so a leaf block has at most 3 b_min x 3 b_min entries.
"""

from __future__ import annotations

import numpy as np

PIVOT_DROP = 1e-6
STOP_STEPS = 3


# ----------------------------------------------------------------------------- Step 1

class ClusterTree:
    """Binary space partitioning of integer atom positions (x, y, p); z = p c.

    ``perm[k]`` is the atom in cluster order position k.  Node n covers positions
    ``start[n] .. start[n] + count[n] - 1``.  ``kids[n]`` is () or (left, right).  Nodes are
    numbered in pre-order.
    """

    def __init__(self, pts: np.ndarray, c: float, b_min: int):
        pts = np.asarray(pts, dtype=np.int64)
        self.c = float(c)
        self.perm = np.arange(len(pts), dtype=np.int64)
        self.start, self.count, self.lo, self.hi, self.sum, self.kids = [], [], [], [], [], []
        self._pts = pts
        self._b_min = int(b_min)
        self._build(0, len(pts))
        del self._pts

    def _build(self, start: int, count: int) -> int:
        idx = self.perm[start:start + count]
        p = self._pts[idx]
        lo, hi = p.min(0), p.max(0)
        me = len(self.start)
        self.start.append(start)
        self.count.append(count)
        self.lo.append(lo)
        self.hi.append(hi)
        self.sum.append(p.sum(0))
        self.kids.append(())
        if count > self._b_min:
            ext = [float(hi[0] - lo[0]), float(hi[1] - lo[1]), float(hi[2] - lo[2]) * self.c]
            ax = int(np.argmax(ext))  # the first longest side
            first = 2 * p[:, ax] <= lo[ax] + hi[ax]  # on or below the midpoint
            n1 = int(first.sum())
            if 0 < n1 < count:
                self.perm[start:start + count] = np.concatenate([idx[first], idx[~first]])
                a = self._build(start, n1)
                b = self._build(start + n1, count - n1)
                self.kids[me] = (a, b)
        return me

    def is_leaf(self, n: int) -> bool:
        return not self.kids[n]

    def centroid(self, n: int) -> tuple[float, float, float]:
        s, k = self.sum[n], self.count[n]
        return (float(s[0]) / k, float(s[1]) / k, (float(s[2]) / k) * self.c)

    def diam2(self, n: int) -> float:
        dx = float(self.hi[n][0] - self.lo[n][0])
        dy = float(self.hi[n][1] - self.lo[n][1])
        dz = float(self.hi[n][2] - self.lo[n][2]) * self.c
        return (dx * dx + dy * dy) + dz * dz


def atom_positions(xy: np.ndarray, L: int) -> np.ndarray:
    """Atoms of a column set in the layout order of [n][L]: (x_a, y_a, p) for a, then p."""
    xy = np.asarray(xy, dtype=np.int64)
    return np.c_[np.repeat(xy, L, axis=0), np.tile(np.arange(L, dtype=np.int64), len(xy))]


def cluster_tree(xy: np.ndarray, L: int, c: float, b_min: int) -> ClusterTree:
    """Step 1: the cluster tree of a column set's atoms."""
    return ClusterTree(atom_positions(xy, L), c, b_min)


# ----------------------------------------------------------------------------- Step 2

def admissible(Tt: ClusterTree, t: int, Ts: ClusterTree, s: int, gamma: float, period: float) -> bool:
    """min(diam t, diam s') <= gamma dist(t, s') for s' in {s, s+, s-} (compared as squares)."""
    ct, cs = Tt.centroid(t), Ts.centroid(s)
    m = min(Tt.diam2(t), Ts.diam2(s))
    g2 = gamma * gamma
    for shift in (0.0, period, -period):
        dx = ct[0] - cs[0]
        dy = ct[1] - cs[1]
        dz = ct[2] - (cs[2] + shift)
        if not (m <= g2 * ((dx * dx + dy * dy) + dz * dz)):
            return False
    return True


def partition(Tt: ClusterTree, Ts: ClusterTree, gamma: float, period: float) -> np.ndarray:
    """Step 2: the blocks as int64 rows (row start, row count, col start, col count, low rank),
    in atoms of cluster order, sorted by (row start, col start)."""
    out = []
    stack = [(0, 0)]
    while stack:
        t, s = stack.pop()
        if admissible(Tt, t, Ts, s, gamma, period):
            out.append((Tt.start[t], Tt.count[t], Ts.start[s], Ts.count[s], 1))
            continue
        lt, ls = Tt.is_leaf(t), Ts.is_leaf(s)
        if lt and ls:
            out.append((Tt.start[t], Tt.count[t], Ts.start[s], Ts.count[s], 0))
            continue
        for a in ((t,) if lt else Tt.kids[t]):
            for b in ((s,) if ls else Ts.kids[s]):
                stack.append((a, b))
    out.sort()
    return np.array(out, dtype=np.int64).reshape(-1, 5)


# ----------------------------------------------------------------------------- Step 3

def aca(rows, cols, n_t: int, n_s: int, eps: float, max_rank: int | None = None):
    """Adaptive cross approximation of an (3 n_t) x (3 n_s) block M = U V.

    ``rows(i)`` returns M's three rows of row atom i (3 x 3 n_s).  ``cols(j)`` returns the three
    columns of column atom j (3 n_t x 3).  Returns (U [3 n_t][k], V [k][3 n_s], capped), where
    capped means a rank limit below full rank was reached before the stopping rule held.
    """
    nt3, ns3 = 3 * n_t, 3 * n_s
    full = min(nt3, ns3)
    max_rank = full if max_rank is None else min(max_rank, full)
    U = np.zeros((nt3, 0))
    V = np.zeros((0, ns3))
    used = np.zeros(n_t, dtype=bool)
    ia, S2, small, capped = 0, 0.0, 0, False
    p0 = None  # the block's first pivot: the scale of the drop rule
    while True:
        R = rows(ia) - U[3 * ia:3 * ia + 3] @ V  # residual rows of the pivot atom
        used[ia] = True
        bn = (R.reshape(3, n_s, 3) ** 2).sum(axis=(0, 2))
        ja = int(np.argmax(bn))
        if bn[ja] == 0.0:  # the row atom is represented exactly: take the next unused one
            if used.all():
                break
            ia = int(np.argmin(used))
            continue
        C = cols(ja) - U @ V[:, 3 * ja:3 * ja + 3]  # residual columns of the pivot column atom
        new_u, new_v = [], []
        for _ in range(3):
            P = R[:, 3 * ja:3 * ja + 3]
            a, b = np.unravel_index(int(np.argmax(np.abs(P))), P.shape)
            piv = P[a, b]
            if p0 is None:
                p0 = abs(piv)
            if not (abs(piv) > PIVOT_DROP * p0):
                break
            u = C[:, b] / piv
            v = R[a, :].copy()
            new_u.append(u)
            new_v.append(v)
            R = R - np.outer(u[3 * ia:3 * ia + 3], v)
            C = C - np.outer(u, v[3 * ja:3 * ja + 3])
        Un = np.array(new_u).reshape(len(new_u), nt3).T
        Vn = np.array(new_v).reshape(len(new_v), ns3)
        cross = float(np.sum((U.T @ Un) * (V @ Vn.T)))
        step2 = float(np.sum((Un.T @ Un) * (Vn @ Vn.T)))
        S2 += 2.0 * cross + step2
        U = np.c_[U, Un]
        V = np.r_[V, Vn]
        small = small + 1 if np.sqrt(step2) <= eps * np.sqrt(S2) else 0
        if small >= STOP_STEPS or used.all():
            break
        if U.shape[1] >= max_rank:
            capped = max_rank < full  # a full-rank factorisation is exact
            break
        if not new_u:  # nothing above the drop level in this row atom: the first unused one next
            ia = int(np.argmin(used))
            continue
        w = (Un.reshape(n_t, 3, -1) ** 2).sum(axis=(1, 2))
        w[used] = -1.0
        ia = int(np.argmax(w))
    return U, V, capped


# ----------------------------------------------------------------------------- the H-matrix

class HMatrix:
    """H-matrix approximation of the Green matrix G~^{p|i+} (Sec. 3.2) from a real-space kernel
    table.  ``table_of_d(d_list)`` returns G~(d, s) as [n_d][L][3][3] for the in-plane
    differences d = x_a - x_b (the oracle's ``kernel_table``)."""

    def __init__(self, xy_i, xy_p, L: int, c: float, table_of_d, eps: float = 1e-5, gamma: float = 2.0,
                 b_min: int = 20, max_rank: int | None = None):
        self.xy_i = np.asarray(xy_i, dtype=np.int64)
        self.xy_p = np.asarray(xy_p, dtype=np.int64)
        self.L, self.c = int(L), float(c)
        self.Tp = cluster_tree(self.xy_p, L, c, b_min)
        self.Ti = cluster_tree(self.xy_i, L, c, b_min)
        self.blocks = partition(self.Tp, self.Ti, gamma, L * c)
        d = (self.xy_p[:, None, :] - self.xy_i[None, :, :]).reshape(-1, 2)
        self.d_list, inv = np.unique(d, axis=0, return_inverse=True)
        self.d_of = inv.reshape(len(self.xy_p), len(self.xy_i))
        self.table = np.asarray(table_of_d(self.d_list))
        self.factors = []
        self.capped = 0
        for r0, nr, c0, nc, lowrank in self.blocks:
            if lowrank:
                U, V, cap = aca(lambda i, r0=r0, c0=c0, nc=nc: self.entries(r0 + i, 1, c0, nc),
                                lambda j, r0=r0, nr=nr, c0=c0: self.entries(r0, nr, c0 + j, 1),
                                int(nr), int(nc), eps, max_rank)
                self.capped += int(cap)
                self.factors.append((U, V))
            else:
                self.factors.append(self.entries(r0, nr, c0, nc))

    def entries(self, r0: int, nr: int, c0: int, nc: int) -> np.ndarray:
        """Rows r0 .. r0+nr-1 and columns c0 .. c0+nc-1 (cluster order, atoms) as a dense
        (3 nr) x (3 nc) matrix."""
        ra = self.Tp.perm[r0:r0 + nr]
        ca = self.Ti.perm[c0:c0 + nc]
        a, p = np.divmod(ra, self.L)
        b, q = np.divmod(ca, self.L)
        G = self.table[self.d_of[a[:, None], b[None, :]], (p[:, None] - q[None, :]) % self.L]
        return G.transpose(0, 2, 1, 3).reshape(3 * nr, 3 * nc)

    def ranks(self) -> np.ndarray:
        return np.array([f[0].shape[1] for f, blk in zip(self.factors, self.blocks) if blk[4]], dtype=np.int64)

    def matvec(self, f: np.ndarray) -> np.ndarray:
        """u = G_H f for f [n_rhs][n_i][L][3] (no projection); returns [n_rhs][n_p][L][3]."""
        f = np.asarray(f, dtype=np.float64)
        R = f.shape[0]
        x = f.reshape(R, -1, 3)[:, self.Ti.perm].reshape(R, -1)
        y = np.zeros((R, 3 * len(self.Tp.perm)))
        for (r0, nr, c0, nc, lowrank), fac in zip(self.blocks, self.factors):
            xs = x[:, 3 * c0:3 * (c0 + nc)]
            if lowrank:
                U, V = fac
                y[:, 3 * r0:3 * (r0 + nr)] += (xs @ V.T) @ U.T
            else:
                y[:, 3 * r0:3 * (r0 + nr)] += xs @ fac.T
        u = np.zeros_like(y).reshape(R, -1, 3)
        u[:, self.Tp.perm] = y.reshape(R, -1, 3)
        return u.reshape(R, len(self.xy_p), self.L, 3)

    def frobenius_error(self) -> float:
        """||G - G_H||_F / ||G||_F over the whole matrix (block by block)."""
        e2 = n2 = 0.0
        for (r0, nr, c0, nc, lowrank), fac in zip(self.blocks, self.factors):
            M = self.entries(r0, nr, c0, nc)
            n2 += float((M * M).sum())
            if lowrank:
                D = M - fac[0] @ fac[1]
                e2 += float((D * D).sum())
        return float(np.sqrt(e2 / n2))
