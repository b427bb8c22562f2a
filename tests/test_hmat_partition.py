"""Steps 1 and 2 of the H-matrix construction (Sec. 3.2; App., cluster trees and the admissible
partition) in the library's host code, against the oracle: the cluster orders and the block lists
agree bit for bit (both take the same integer and double-precision steps).  No GPU needed."""

import numpy as np
import pytest

from oracle import hmatrix
from paper_2105_08798_gb300 import build as fbc_build
from paper_2105_08798_gb300 import fbc, inputs

CASES = [
    (12, 18, 8, 1.0, 2.0, 4),
    (12, 18, 8, 1.0, 0.5, 4),     # strict criterion: dense near-field blocks
    (60, 90, 16, 1.0, 2.0, 20),
    (200, 300, 16, 1.0, 2.0, 20),  # the small isotropic workload, the paper's settings
    (150, 220, 32, 0.7, 1.3, 9),   # spacing c != 1, non-integer gamma
    (1000, 1500, 64, 1.0, 2.0, 20),
]


@pytest.fixture(scope="module")
def lib():
    fbc_build.build()
    return fbc.load()


@pytest.mark.parametrize("n_i,n_p,L,c,gamma,b_min", CASES)
def test_partition_matches_the_oracle(lib, n_i, n_p, L, c, gamma, b_min):
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    blocks, perm_p, perm_i = fbc.fbc_hmat_partition(xy_i, xy_p, L, c, gamma, b_min)
    Tp = hmatrix.cluster_tree(xy_p, L, c, b_min)
    Ti = hmatrix.cluster_tree(xy_i, L, c, b_min)
    ref = hmatrix.partition(Tp, Ti, gamma, L * c)
    assert np.array_equal(perm_p, Tp.perm) and np.array_equal(perm_i, Ti.perm)
    assert np.array_equal(blocks, ref)
    # every (pad atom, interface atom) pair once: the block areas add up to the matrix
    assert int((blocks[:, 1] * blocks[:, 3]).sum()) == n_p * L * n_i * L
