"""In-plane FFT form of the per-mode contraction (FBC_PREC_FFT64) through the C ABI.

The per-mode sum over interface columns is a 2D lattice convolution; the FFT form
evaluates it exactly (circular convolution on a grid of at least 2 max|d| + 1 points
per side), so it must agree with the oracle and with the dense FP64 contraction to
FP64 rounding: 1e-12 relative L2.  Also checked: several right-hand sides with the
projection, zero mean, alpha and beta; switching precisions back and forth on one
plan; a case whose (rhs, mode) items need several workspace chunks; the cubic medium.
"""

import numpy as np
import pytest

from conftest import CUBIC, ISO
from paper_2105_08798_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.fixture(scope="module")
def fbc():
    from paper_2105_08798_gb300 import build, fbc as binding

    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("material", [ISO, CUBIC], ids=["iso", "cubic"])
def test_fft_against_oracle(fbc, oracle_mod, material):
    n_i, n_p, L = 200, 300, 16
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    f = inputs.forces(1, n_i, L, seed=21)
    ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, material, f)
    with fbc.Plan(xy_i, xy_p, L, material, precision="fft64") as plan:
        plan.tabulate()
        u = torch.full((1, n_p, L, 3), float("nan"), dtype=torch.float64, device="cuda")
        plan.apply(torch.from_numpy(f).cuda(), u)
        torch.cuda.synchronize()
        plan.sync_status()
        got = u.cpu().numpy()
    assert rel_l2(got, ref) <= 1e-12


def _both(fbc, xy_i, xy_p, L, R, seed, **kw):
    n_i, n_p = len(xy_i), len(xy_p)
    f = torch.from_numpy(inputs.forces(R, n_i, L, seed=seed)).cuda()
    u0 = torch.from_numpy(np.random.default_rng(seed).normal(0, 1, (R, n_p, L, 3))).cuda()
    out = {}
    with fbc.Plan(xy_i, xy_p, L, ISO, max_rhs=R) as plan:
        plan.tabulate()
        for prec in ("fp64", "fft64", "f32x2", "fft64"):
            plan.set_precision(prec)
            u = u0.clone()
            plan.apply(f, u, **kw)
            torch.cuda.synchronize()
            plan.sync_status()
            out.setdefault(prec, []).append(u.cpu().numpy())
            if prec == "fft64":
                out["info"] = plan.info()
    return out


def test_fft_multi_rhs_flags_and_switching(fbc):
    xy_i, xy_p = inputs.ring_geometry(300, 450)
    out = _both(fbc, xy_i, xy_p, 8, 3, 5, alpha=-0.7, beta=1.0, project=True, zero_mean=True)
    ref = out["fp64"][0]
    for got in out["fft64"]:
        assert rel_l2(got, ref) <= 1e-12
    np.testing.assert_array_equal(out["fft64"][0], out["fft64"][1])  # rebuilt transform, same bits
    assert rel_l2(out["f32x2"][0], ref) <= 1e-12


def test_fft_chunked_workspace(fbc):
    # 8000 x 12000 columns: differences span 305 per side, a 320 x 320 grid (radices 5, 8, 8), about
    # 4.7 MB of workspace per (rhs, mode) item, so the 2 x 129 items run in two chunks
    xy_i, xy_p = inputs.ring_geometry(8000, 12000)
    out = _both(fbc, xy_i, xy_p, 256, 2, 8)
    assert rel_l2(out["fft64"][0], out["fp64"][0]) <= 1e-12
    assert out["info"]["fft_mx"] == 320 and out["info"]["fft_chunk_items"] < 2 * 129, out["info"]


def test_fft_rejected_for_batches(fbc):
    xy_i, xy_p = inputs.ring_geometry(100, 150)
    f = torch.from_numpy(inputs.forces(1, 100, 8, seed=1)).cuda()
    u = torch.zeros((1, 150, 8, 3), dtype=torch.float64, device="cuda")
    with fbc.Plan(xy_i, xy_p, 8, ISO, precision="fft64") as plan:
        plan.tabulate()
        with pytest.raises(fbc.FBCError):
            fbc.Batch([plan], [f], [u])


@pytest.mark.parametrize("n_i,n_p,L,R", [(200, 300, 16, 1), (300, 450, 8, 3), (1500, 2000, 8, 2)])
def test_fft32_against_fp64(fbc, n_i, n_p, L, R):
    """FP32 transforms for k >= 1 (error at the FP32 level, as the dense FP32 form), FP64 for k = 0."""
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    f = torch.from_numpy(inputs.forces(R, n_i, L, seed=n_i + R)).cuda()
    out = {}
    with fbc.Plan(xy_i, xy_p, L, ISO, max_rhs=R) as plan:
        plan.tabulate()
        for prec in ("fp64", "fft32", "fp32"):
            plan.set_precision(prec)
            u = torch.full((R, n_p, L, 3), float("nan"), dtype=torch.float64, device="cuda")
            plan.apply(f, u)
            torch.cuda.synchronize()
            plan.sync_status()
            out[prec] = u.cpu().numpy()
    ref = out["fp64"]
    assert np.isfinite(out["fft32"]).all()
    assert rel_l2(out["fft32"], ref) <= 1e-5, rel_l2(out["fft32"], ref)
    # the k = 0 band (the mean along the line) keeps FP64 accuracy
    assert rel_l2(out["fft32"].mean(axis=2), ref.mean(axis=2)) <= 1e-11


def test_fft_host_entry_point(fbc):
    """fbc_apply_host on an FFT plan: the same bits as the device entry point."""
    xy_i, xy_p = inputs.ring_geometry(150, 220)
    L, R = 8, 2
    f = inputs.forces(R, 150, L, seed=3)
    u0 = np.random.default_rng(4).normal(0, 1, (R, 220, L, 3))
    with fbc.Plan(xy_i, xy_p, L, CUBIC, precision="fft64", max_rhs=R) as plan:
        plan.tabulate()
        ud = torch.from_numpy(u0.copy()).cuda()
        plan.apply(torch.from_numpy(f).cuda(), ud, alpha=0.5, beta=2.0)
        torch.cuda.synchronize()
        uh = u0.copy()
        plan.apply_host(f, uh, alpha=0.5, beta=2.0)
        plan.sync_status()
    np.testing.assert_array_equal(uh, ud.cpu().numpy())


@pytest.mark.parametrize("n_i,n_p,L", [(1, 1, 2), (2, 3, 4), (5, 7, 8), (13, 20, 2)])
def test_fft_degenerate_geometries(fbc, oracle_mod, n_i, n_p, L):
    """One or a few columns and the shortest lines: grid sides of 2 to 9 points (single passes of
    radix 2, 3, 5 and mixed lengths), K = 2 modes."""
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    f = inputs.forces(1, n_i, L, seed=n_i)
    ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f)
    for prec, tol in (("fft64", 1e-12), ("fft32", 1e-5)):
        with fbc.Plan(xy_i, xy_p, L, ISO, precision=prec) as plan:
            plan.tabulate()
            u = torch.full((1, n_p, L, 3), float("nan"), dtype=torch.float64, device="cuda")
            plan.apply(torch.from_numpy(f).cuda(), u)
            torch.cuda.synchronize()
            plan.sync_status()
            got = u.cpu().numpy()
        assert rel_l2(got, ref) <= tol, (prec, rel_l2(got, ref))
