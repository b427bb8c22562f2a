"""Host logic of the plan (no GPU): tiling, the difference box and a replay of
the contraction kernel's index arithmetic against its buffers.

A host-only plan (``FBC_PLAN_HOST_ONLY``) runs the same validation and tiling
as a real one without touching the device; its layout is read back with
``fbc_plan_layout`` and every shared-memory and table index the contraction
and line-transform kernels compute is checked to stay inside its buffer.
"""

import numpy as np
import pytest

from paper_2105_08798_gb300 import build as fbc_build
from paper_2105_08798_gb300 import fbc, inputs

ISO = {"kind": "isotropic", "mu": 1.0, "nu": 0.3}


@pytest.fixture(scope="module", autouse=True)
def lib():
    fbc_build.build()
    return fbc.load()


def line_cols(L):
    return int(min(64, max(2, 2048 // L)))


CASES = [(200, 300, 16), (4000, 6000, 256), (8000, 12000, 1024), (1, 1, 2), (65, 129, 16), (777, 1165, 512)]


@pytest.mark.parametrize("n_i,n_p,L", CASES)
def test_layout_and_kernel_indices(n_i, n_p, L):
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    with fbc.Plan(xy_i, xy_p, L, ISO, host_only=True) as plan:
        info = plan.info()
        lay = plan.layout()
    TA, TB = info["tile_a"], info["tile_b"]
    nta, ntb = info["n_tiles_a"], info["n_tiles_b"]
    W, H = info["sub_w"], info["sub_h"]
    x0, y0, Dx, Dy = info["box_x0"], info["box_y0"], info["box_nx"], info["box_ny"]
    NIpad, NPpad = ntb * TB, nta * TA
    # permutations: every real column exactly once, padding only at the end
    for perm, n, T in ((lay["perm_i"], n_i, TB), (lay["perm_p"], n_p, TA)):
        real = perm[perm >= 0]
        assert sorted(real.tolist()) == list(range(n))
        assert (perm[:n] >= 0).all() and (perm[n:] == -1).all()
        assert len(perm) % T == 0
    # sorted sites are the original sites
    assert np.array_equal(lay["xy_i"][:n_i], xy_i[lay["perm_i"][:n_i]])
    assert np.array_equal(lay["xy_p"][:n_p], xy_p[lay["perm_p"][:n_p]])
    # line-transform blocking divides the padded column counts
    assert NIpad % line_cols(L) == 0 and NPpad % line_cols(L) == 0
    # tile bounding boxes as the kernel sees them (padding repeats the first site)
    def bboxes(xy, T, nt):
        t = xy.reshape(nt, T, 2)
        return t[:, :, 0].min(1), t[:, :, 0].max(1), t[:, :, 1].min(1), t[:, :, 1].max(1)
    aminx, amaxx, aminy, amaxy = bboxes(lay["xy_p"], TA, nta)
    bminx, bmaxx, bminy, bmaxy = bboxes(lay["xy_i"], TB, ntb)
    assert (amaxx - aminx + 1).max() + (bmaxx - bminx + 1).max() - 1 <= W
    assert (amaxy - aminy + 1).max() + (bmaxy - bminy + 1).max() - 1 <= H
    # shared-memory gather index idx = base_a - off_b for every slot pair of every tile pair
    xa = lay["xy_p"].reshape(nta, TA, 2)
    xb = lay["xy_i"].reshape(ntb, TB, 2)
    off_b = xb[:, :, 0] + W * xb[:, :, 1]  # [ntb][TB]
    for ta in range(nta):
        ox = aminx[ta] - bmaxx  # [ntb]
        oy = aminy[ta] - bmaxy
        assert (ox - x0 >= 0).all() and (oy - y0 >= 0).all()  # staged table loads start inside the box
        base = (xa[ta, :, 0][None, :] - ox[:, None]) + W * (xa[ta, :, 1][None, :] - oy[:, None])  # [ntb][TA]
        idx = base[:, :, None] - off_b[:, None, :]  # [ntb][TA][TB]
        assert idx.min() >= 0 and idx.max() < W * H
        ix = xa[ta, :, 0][None, :, None] - xb[:, None, :, 0] - ox[:, None, None]
        assert ix.min() >= 0 and ix.max() < W
    # every realised difference lies in the table box; count the distinct ones on a bitmap
    used = np.zeros((Dy, Dx), dtype=bool)
    for a0 in range(0, n_p, 512):
        d = xy_p[a0:a0 + 512, None, :].astype(np.int64) - xy_i[None, :, :]
        assert d[..., 0].min() >= x0 and d[..., 0].max() < x0 + Dx
        assert d[..., 1].min() >= y0 and d[..., 1].max() < y0 + Dy
        used[d[..., 1] - y0, d[..., 0] - x0] = True
    assert info["n_used_d"] == int(used.sum())
    if 0 <= -y0 < Dy and 0 <= -x0 < Dx:
        assert not used[-y0, -x0]  # d = 0 never occurs


def test_tiles_are_compact():
    xy_i, xy_p = inputs.ring_geometry(4000, 6000)
    with fbc.Plan(xy_i, xy_p, 256, ISO, host_only=True) as plan:
        info = plan.info()
    # a 128-site tile at unit density spans about 11 x 11; the sub-box stays small
    assert info["sub_w"] * info["sub_h"] <= 40 * 40


def test_host_only_plan_refuses_device_work():
    xy_i, xy_p = inputs.ring_geometry(20, 30)
    with fbc.Plan(xy_i, xy_p, 16, ISO, host_only=True) as plan:
        with pytest.raises(fbc.FBCError) as ei:
            plan.tabulate()
        assert ei.value.status == fbc.FBC_ERR_INVALID_ARG
