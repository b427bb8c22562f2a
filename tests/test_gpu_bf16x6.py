"""FP64-accurate tensor-core form (FBC_PREC_BF16X6): fixed-point bf16 slices with exact FP32
accumulation per diagonal, k = 0 in double-float, FP64 line transforms.

Its error is that of the double-float form: below 1e-13 relative L2 against the oracle's plain
real-space sum (Eq. 1; Sec. 3.2, Eqs. 37-38) and against the dense FP64 GPU form.  The cases span
several pad tiles (128 columns), several interface tiles (64 columns, one accumulation group each)
with a ragged last tile, one and several groups of 16 right-hand sides with a ragged last group,
isotropic and cubic media, and forces scaled far from 1 (the power-of-two scales must follow).
"""

import numpy as np
import pytest

from conftest import CUBIC, ISO
from paper_2105_08798_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.fixture(scope="module")
def fbc():
    from paper_2105_08798_gb300 import build, fbc as binding

    build.build()
    binding.load()
    return binding


def _apply(fbc, plan, f, R, n_p, L, prec, alpha=1.0, beta=0.0, u0=None, zero_mean=False):
    plan.set_precision(prec)
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    ud = (torch.from_numpy(u0).cuda() if u0 is not None
          else torch.full((R, n_p, L, 3), float("nan"), dtype=torch.float64, device="cuda"))
    plan.apply(fd, ud, alpha=alpha, beta=beta, zero_mean=zero_mean)
    torch.cuda.synchronize()
    plan.sync_status()
    return ud.cpu().numpy()


# (n_i, n_p, L, R, material): ragged interface tiles everywhere; 20 and 37 rhs make two and three
# rhs groups with ragged last groups; 1500 x 2000 has 24 interface tiles and 16 pad tiles
CASES = [(300, 450, 32, 16, ISO), (150, 220, 16, 3, CUBIC), (100, 140, 8, 20, ISO), (1500, 2000, 8, 8, ISO),
         (260, 390, 64, 37, CUBIC)]


@pytest.mark.parametrize("n_i,n_p,L,R,mat", CASES)
def test_bf16x6_against_oracle_and_fp64(fbc, oracle_mod, n_i, n_p, L, R, mat):
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    f = inputs.forces(R, n_i, L, seed=n_i + 7 * R)
    with fbc.Plan(xy_i, xy_p, L, mat, precision="fp64", max_rhs=R) as plan:
        plan.tabulate()
        u64 = _apply(fbc, plan, f, R, n_p, L, "fp64")
        ux6 = _apply(fbc, plan, f, R, n_p, L, "bf16x6")
    assert np.isfinite(ux6).all()
    assert rel_l2(ux6, u64) <= TOL
    # the oracle for the first and the last right-hand side
    rs = [0, R - 1] if R > 1 else [0]
    ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, mat, f[rs])
    assert rel_l2(ux6[rs], ref) <= TOL
    for j, r in enumerate(rs):
        assert rel_l2(ux6[r], ref[j]) <= TOL, r


def test_bf16x6_scales_follow_the_forces(fbc):
    """Forces of 1e-20 and 1e+20 (and one rhs of zeros next to them): the per-column power-of-two
    scales keep the relative error, and a zero right-hand side gives zeros."""
    xy_i, xy_p = inputs.ring_geometry(200, 300)
    L, R = 16, 18
    f = inputs.forces(R, 200, L, seed=5)
    f[1] *= 1e-20
    f[2] *= 1e20
    f[17] = 0.0
    with fbc.Plan(xy_i, xy_p, L, ISO, max_rhs=R) as plan:
        plan.tabulate()
        u64 = _apply(fbc, plan, f, R, 300, L, "fp64")
        ux6 = _apply(fbc, plan, f, R, 300, L, "bf16x6")
    for r in range(R - 1):
        assert rel_l2(ux6[r], u64[r]) <= TOL, r
    assert np.all(ux6[R - 1] == 0.0)


def test_bf16x6_update_form(fbc, oracle_mod):
    """beta u0 + alpha G f with the zero mean, against the oracle."""
    xy_i, xy_p = inputs.ring_geometry(120, 170)
    L, R = 16, 5
    f = inputs.forces(R, 120, L, seed=9)
    u0 = np.random.default_rng(4).standard_normal((R, 170, L, 3))
    with fbc.Plan(xy_i, xy_p, L, ISO, max_rhs=R) as plan:
        plan.tabulate()
        got = _apply(fbc, plan, f, R, 170, L, "bf16x6", alpha=-0.7, beta=0.3, u0=u0.copy(), zero_mean=True)
    ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f, alpha=-0.7, beta=0.3, u0=u0, zero_mean_u=True)
    assert rel_l2(got, ref) <= TOL


def test_bf16x6_is_deterministic(fbc):
    """Exact sums in a fixed order: two applies give the same bits."""
    xy_i, xy_p = inputs.ring_geometry(300, 450)
    L, R = 16, 16
    f = inputs.forces(R, 300, L, seed=2)
    with fbc.Plan(xy_i, xy_p, L, ISO, precision="bf16x6", max_rhs=R) as plan:
        plan.tabulate()
        a = _apply(fbc, plan, f, R, 450, L, "bf16x6")
        b = _apply(fbc, plan, f, R, 450, L, "bf16x6")
    assert np.array_equal(a, b)
