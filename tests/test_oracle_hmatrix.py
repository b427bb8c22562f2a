"""Pins of the H-matrix oracle (Sec. 3.2; App., the H-matrix construction), against facts that do
not come from the oracle itself.

* Step 1: the leaves cover every atom once, hold at most b_min atoms, and each split lies at
  the midpoint of the longest side of the parent's bounding box (recomputed from the atoms).
* Step 2: the blocks cover every (pad atom, interface atom) pair exactly once (brute-force
  count).  Every low-rank block meets the admissibility criterion, recomputed from its atoms
  with the periodic neighbours.  Every dense block is a pair of leaves that fails it.
* Step 3: cross approximation reproduces a matrix of known rank exactly (to rounding) with
  that rank, and on a block of the Green matrix it lands within a small factor of the SVD's
  error at the same rank.
* The whole H-matrix: its Frobenius error is of the order of eps, as the paper states, and
  u = G_H f agrees with the exact real-space update (Eq. 1) to that order.  A looser eps gives
  a larger error.
"""

import numpy as np
import pytest

import oracle
from oracle import hmatrix
from paper_2105_08798_gb300 import inputs
from paper_2105_08798_gb300.inputs import ISO


def table_fn(L):
    return lambda d: oracle.kernel_table(ISO, L, 1.0, d)


@pytest.fixture(scope="module")
def tiny():
    xy_i, xy_p = inputs.ring_geometry(12, 18)
    return xy_i, xy_p, 8


def test_cluster_tree_bisection(tiny):
    xy_i, xy_p, L = tiny
    pts = hmatrix.atom_positions(xy_p, L)
    T = hmatrix.cluster_tree(xy_p, L, 1.0, 5)
    leaves = [n for n in range(len(T.start)) if T.is_leaf(n)]
    cover = np.zeros(len(pts), dtype=int)
    for n in leaves:
        assert T.count[n] <= 5
        cover[T.perm[T.start[n]:T.start[n] + T.count[n]]] += 1
    assert (cover == 1).all()
    assert sorted(T.perm.tolist()) == list(range(len(pts)))
    for n in range(len(T.start)):
        p = pts[T.perm[T.start[n]:T.start[n] + T.count[n]]]
        assert (p.min(0) == T.lo[n]).all() and (p.max(0) == T.hi[n]).all()
        if T.is_leaf(n):
            continue
        a, b = T.kids[n]
        ext = p.max(0) - p.min(0)
        ax = int(np.argmax(ext))
        mid2 = p.min(0)[ax] + p.max(0)[ax]
        pa = pts[T.perm[T.start[a]:T.start[a] + T.count[a]]]
        pb = pts[T.perm[T.start[b]:T.start[b] + T.count[b]]]
        assert (2 * pa[:, ax] <= mid2).all() and (2 * pb[:, ax] > mid2).all()
        assert T.start[a] == T.start[n] and T.start[b] == T.start[n] + T.count[a]
    # every split keeps the atoms' order, so each leaf lists its atoms in increasing order
    for n in leaves:
        assert (np.diff(T.perm[T.start[n]:T.start[n] + T.count[n]]) > 0).all()


@pytest.mark.parametrize("gamma", [2.0, 0.5])
def test_partition_covers_each_pair_once_and_is_admissible(tiny, gamma):
    xy_i, xy_p, L = tiny
    Tp = hmatrix.cluster_tree(xy_p, L, 1.0, 4)
    Ti = hmatrix.cluster_tree(xy_i, L, 1.0, 4)
    blocks = hmatrix.partition(Tp, Ti, gamma, float(L))
    pp, pi = hmatrix.atom_positions(xy_p, L).astype(float), hmatrix.atom_positions(xy_i, L).astype(float)
    cover = np.zeros((len(pp), len(pi)), dtype=int)
    leaf_sets = {(Tp.start[n], Tp.count[n]) for n in range(len(Tp.start)) if Tp.is_leaf(n)}
    leaf_seti = {(Ti.start[n], Ti.count[n]) for n in range(len(Ti.start)) if Ti.is_leaf(n)}

    def adm(A, B):  # from the atoms: bounding-box diagonal, centroid distance, periodic images
        m = min(np.linalg.norm(A.max(0) - A.min(0)), np.linalg.norm(B.max(0) - B.min(0)))
        return all(m <= gamma * np.linalg.norm(A.mean(0) - (B.mean(0) + [0, 0, sh])) for sh in (0, L, -L))

    n_dense = 0
    for r0, nr, c0, nc, lowrank in blocks:
        ra, ca = Tp.perm[r0:r0 + nr], Ti.perm[c0:c0 + nc]
        cover[np.ix_(ra, ca)] += 1
        if lowrank:
            assert adm(pp[ra], pi[ca])
        else:
            n_dense += 1
            assert (r0, nr) in leaf_sets and (c0, nc) in leaf_seti
            assert not adm(pp[ra], pi[ca])
    assert (cover == 1).all()
    if gamma < 1.0:
        assert n_dense > 0  # the strict criterion leaves dense near-field blocks


def test_aca_reproduces_a_matrix_of_known_rank():
    rng = np.random.default_rng(7)
    n_t, n_s, r = 40, 30, 5
    # M[(a,i),(b,j)] = sum_m phi_m(a) psi_m(b) B_m[i][j]: rank <= 3 r
    phi, psi = rng.standard_normal((r, n_t)), rng.standard_normal((r, n_s))
    B = rng.standard_normal((r, 3, 3))
    M = np.einsum("ma,mb,mij->aibj", phi, psi, B).reshape(3 * n_t, 3 * n_s)
    U, V, capped = hmatrix.aca(lambda i: M[3 * i:3 * i + 3], lambda j: M[:, 3 * j:3 * j + 3], n_t, n_s, 1e-5)
    assert not capped
    assert np.linalg.norm(M - U @ V) <= 1e-12 * np.linalg.norm(M)
    assert np.linalg.matrix_rank(M) == 3 * r
    assert 3 * r <= U.shape[1] <= 3 * r + 3 * hmatrix.STOP_STEPS


def test_aca_on_a_green_block_is_near_the_svd():
    L = 16
    xy_i, xy_p = inputs.ring_geometry(60, 90)
    H = hmatrix.HMatrix(xy_i, xy_p, L, 1.0, table_fn(L), eps=1e-5)
    lr = [k for k, b in enumerate(H.blocks) if b[4]]
    sizes = [H.blocks[k][1] * H.blocks[k][3] for k in lr]
    k = lr[int(np.argmax(sizes))]  # the largest low-rank block
    r0, nr, c0, nc, _ = H.blocks[k]
    M = H.entries(r0, nr, c0, nc)
    U, V = H.factors[k]
    e_aca = np.linalg.norm(M - U @ V) / np.linalg.norm(M)
    sv = np.linalg.svd(M, compute_uv=False)
    rank = U.shape[1]
    assert e_aca <= 2e-5
    # the best rank-k error (Eckart-Young) for every k; the SVD's rank for the error ACA reached
    tail = np.sqrt(np.append(np.cumsum((sv ** 2)[::-1])[::-1], 0.0)) / np.linalg.norm(sv)
    k_svd = int(np.argmax(tail <= e_aca))
    assert k_svd <= rank <= 2 * k_svd + 3 * hmatrix.STOP_STEPS, (rank, k_svd)


def test_hmatrix_error_is_of_the_order_of_eps():
    L = 16
    xy_i, xy_p = inputs.ring_geometry(60, 90)
    H = hmatrix.HMatrix(xy_i, xy_p, L, 1.0, table_fn(L), eps=1e-5)
    assert H.capped == 0
    e = H.frobenius_error()
    assert 1e-8 < e <= 1e-5
    f = inputs.forces(2, len(xy_i), L, seed=11)
    ref = oracle.pad_update(xy_i, xy_p, L, 1.0, ISO, f)
    u = H.matvec(oracle.project_neutral(f))
    assert np.linalg.norm(u - ref) <= 2e-5 * np.linalg.norm(ref)
    # a looser tolerance gives a larger error and a smaller matrix
    H3 = hmatrix.HMatrix(xy_i, xy_p, L, 1.0, table_fn(L), eps=1e-3)
    e3 = H3.frobenius_error()
    assert e < e3 <= 1e-3
    assert H3.ranks().sum() < H.ranks().sum()


def test_hmatrix_update_at_the_small_ring():
    """200 interface and 300 pad columns, L = 16 (the small isotropic workload)."""
    L = 16
    xy_i, xy_p = inputs.ring_geometry(200, 300)
    H = hmatrix.HMatrix(xy_i, xy_p, L, 1.0, table_fn(L), eps=1e-5)
    f = inputs.forces(1, len(xy_i), L, seed=0)
    ref = oracle.pad_update(xy_i, xy_p, L, 1.0, ISO, f)
    u = H.matvec(oracle.project_neutral(f))
    assert np.linalg.norm(u - ref) <= 2e-5 * np.linalg.norm(ref)
