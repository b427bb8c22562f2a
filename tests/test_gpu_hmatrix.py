"""The device H-matrix (Sec. 3.2; App., the H-matrix construction) through the C ABI.

* Its partition and cluster orders are the oracle's, bit for bit.  Its ranks are within a small
  factor of the oracle's FP64 cross approximation, though the pivot choices are not unique.
* u = G_H f agrees with the oracle's exact real-space update (Eq. 1) to the order of eps, and
  with the oracle's own H-matrix product to the same order.  This holds on the small isotropic
  ring (the paper's settings), a cubic medium, a strict gamma (dense near-field blocks) and 6
  right-hand sides (two passes of four).
* The update form beta u + alpha G_H f with the zero mean matches the oracle.  Results are
  deterministic, and a build split into many waves gives the same bits.
* A looser eps gives a larger error and smaller ranks.  A rank cap is reported.  Plans whose
  kernel is not the periodic continuum one are refused.
* At 1000 x 1500 columns, L = 64, every repeat of four pad columns matches the oracle.
"""

import numpy as np
import pytest

import oracle
from oracle import hmatrix
from paper_2105_08798_gb300 import inputs
from paper_2105_08798_gb300.inputs import CUBIC, ISO

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def fbc():
    from paper_2105_08798_gb300 import build, fbc as binding

    build.build()
    binding.load()
    return binding


def make(fbc, n_i, n_p, L, material=ISO, **kw):
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    plan = fbc.Plan(xy_i, xy_p, L, material)
    H = fbc.HMatrix(plan, **kw)
    return xy_i, xy_p, plan, H


def test_small_ring_against_the_oracle(fbc):
    L, R = 16, 2
    xy_i, xy_p, plan, H = make(fbc, 200, 300, L)
    info = H.info()
    blocks, ranks = H.blocks()
    orc = hmatrix.HMatrix(xy_i, xy_p, L, 1.0, lambda d: oracle.kernel_table(ISO, L, 1.0, d))
    assert np.array_equal(blocks, orc.blocks)
    assert info["n_capped"] == 0 and info["n_dense"] == 0
    assert info["n_rows"] == 3 * 300 * L and info["n_cols"] == 3 * 200 * L
    lr = blocks[:, 4] == 1
    r_dev, r_orc = ranks[lr].astype(float), orc.ranks().astype(float)
    assert 0.5 <= r_dev.sum() / r_orc.sum() <= 2.0
    f = inputs.forces(R, 200, L, seed=3)
    fd = torch.from_numpy(f).cuda()
    u = torch.full((R, 300, L, 3), float("nan"), dtype=torch.float64, device="cuda")
    H.apply(fd, u)
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    ref = oracle.pad_update(xy_i, xy_p, L, 1.0, ISO, f)
    assert rel(got, ref) <= 2e-5
    assert rel(got, orc.matvec(oracle.project_neutral(f))) <= 2e-5
    # deterministic
    u2 = torch.zeros_like(u)
    H.apply(fd, u2)
    torch.cuda.synchronize()
    assert torch.equal(u, u2)
    # u <- beta u0 + alpha G_H f, then the zero mean
    u0 = np.random.default_rng(1).standard_normal((R, 300, L, 3))
    u3 = torch.from_numpy(u0).cuda()
    H.apply(fd, u3, alpha=-0.5, beta=2.0, zero_mean=True)
    torch.cuda.synchronize()
    want = oracle.zero_mean(2.0 * u0 - 0.5 * ref)
    assert rel(u3.cpu().numpy(), want) <= 2e-5
    # without the projection: the same as the projected forces given already neutral
    fp = torch.from_numpy(oracle.project_neutral(f)).cuda()
    u4 = torch.zeros_like(u)
    H.apply(fp, u4, project=False)
    torch.cuda.synchronize()
    assert rel(u4.cpu().numpy(), ref) <= 2e-5
    H.close()
    plan.close()


def test_dense_blocks_cubic_and_many_rhs(fbc):
    L, R = 16, 6
    xy_i, xy_p, plan, H = make(fbc, 60, 90, L, CUBIC, gamma=0.5, b_min=8)
    info = H.info()
    assert info["n_dense"] > 0 and info["dense_bytes"] > 0
    blocks, _ = H.blocks()
    Tp = hmatrix.cluster_tree(xy_p, L, 1.0, 8)
    Ti = hmatrix.cluster_tree(xy_i, L, 1.0, 8)
    assert np.array_equal(blocks, hmatrix.partition(Tp, Ti, 0.5, float(L)))
    f = inputs.forces(R, 60, L, seed=9)
    u = torch.zeros((R, 90, L, 3), dtype=torch.float64, device="cuda")
    H.apply(torch.from_numpy(f).cuda(), u)
    torch.cuda.synchronize()
    ref = oracle.pad_update(xy_i, xy_p, L, 1.0, CUBIC, f)
    got = u.cpu().numpy()
    for r in range(R):
        assert rel(got[r], ref[r]) <= 2e-5, r
    H.close()
    plan.close()


def test_tolerance_rank_cap_and_waves(fbc):
    L = 16
    xy_i, xy_p = inputs.ring_geometry(60, 90)
    f = inputs.forces(1, 60, L, seed=4)
    ref = oracle.pad_update(xy_i, xy_p, L, 1.0, ISO, f)
    fd = torch.from_numpy(f).cuda()
    out = {}
    with fbc.Plan(xy_i, xy_p, L, ISO) as plan:
        for key, kw in {"e5": {}, "e3": {"eps": 1e-3}, "cap": {"max_rank": 6},
                        "waves": {"scratch_bytes": 1 << 16}}.items():
            with fbc.HMatrix(plan, **kw) as H:
                u = torch.zeros((1, 90, L, 3), dtype=torch.float64, device="cuda")
                H.apply(fd, u)
                torch.cuda.synchronize()
                out[key] = (u.cpu().numpy(), H.info())
    e5, e3, ecap = rel(out["e5"][0], ref), rel(out["e3"][0], ref), rel(out["cap"][0], ref)
    assert e5 <= 2e-5 and e5 < e3 <= 3e-3
    assert out["e3"][1]["rank_sum"] < out["e5"][1]["rank_sum"]
    assert out["cap"][1]["n_capped"] > 0 and out["cap"][1]["rank_max"] <= 6 + 2 and ecap > e5
    assert out["waves"][1]["n_waves"] > 1
    assert np.array_equal(out["waves"][0], out["e5"][0])


def test_refusals(fbc):
    xy_i, xy_p = inputs.ring_geometry(60, 90)
    with fbc.Plan(xy_i, xy_p, 16, ISO) as plan:
        with pytest.raises(fbc.FBCError) as ei:
            fbc.HMatrix(plan, eps=1e-7)
        assert ei.value.status == fbc.FBC_ERR_INVALID_ARG
        with fbc.HMatrix(plan) as H:
            with pytest.raises(ValueError):
                H.apply(torch.zeros((1, 60, 16, 3), dtype=torch.float64, device="cuda"),
                        torch.zeros((1, 89, 16, 3), dtype=torch.float64, device="cuda"))
    # interface sites inside the pad (self-terms): the kernel there is the lattice one
    pad = np.concatenate([xy_p, xy_i[:5]])
    with fbc.Plan(xy_i, pad, 16, ISO, self_terms=True) as plan:
        with pytest.raises(fbc.FBCError) as ei:
            fbc.HMatrix(plan)
        assert ei.value.status == fbc.FBC_ERR_UNSUPPORTED


def test_mid_size_at_sampled_columns(fbc):
    """1000 x 1500 columns, L = 64 (96 000 pad atoms): every repeat of the two innermost and the two
    outermost pad columns against the oracle's real-space sum."""
    L, R = 64, 2
    xy_i, xy_p, plan, H = make(fbc, 1000, 1500, L)
    info = H.info()
    assert info["n_capped"] == 0
    f = inputs.forces(R, 1000, L, seed=12)
    u = torch.zeros((R, 1500, L, 3), dtype=torch.float64, device="cuda")
    H.apply(torch.from_numpy(f).cuda(), u)
    torch.cuda.synchronize()
    cols = np.array([0, 1, 1498, 1499])
    fp = oracle.project_neutral(f)
    d_list, d_index = oracle.difference_index(xy_i, xy_p[cols])
    table = oracle.kernel_table(ISO, L, 1.0, d_list)
    samp_col = np.repeat(np.arange(len(cols)), L).astype(np.int32)
    samp_p = np.tile(np.arange(L), len(cols)).astype(np.int32)
    ref = oracle.real_space_sum(d_index, table, fp, samp_col, samp_p).reshape(R, len(cols), L, 3)
    got = u.cpu().numpy()[:, cols]
    assert rel(got, ref) <= 3e-5
    # storage: far below the dense matrix (9 n_p n_i L^2 FP32 numbers)
    assert info["factor_bytes"] + info["dense_bytes"] < 0.2 * 4 * 9 * 1500 * 1000 * L * L
    H.close()
    plan.close()
