"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every test feeds the same seeded inputs to both sides.  The bar for the FP64
and the double-float (F32X2) contractions is a relative L2 error of 1e-12
against the oracle; the FP32 contraction's error is measured and bounded at
the level FP32 rounding of 3 N_I terms per output allows (stated below).
"""

import numpy as np
import pytest

from conftest import CUBIC, ISO
from paper_2105_08798_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12
TOL_FP32 = 5e-6  # FP32 products, sums of a few thousand terms per output


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def fbc():
    from paper_2105_08798_gb300 import build, fbc as binding

    build.build()
    binding.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def gpu_update(fbc, xy_i, xy_p, L, material, f, precision="fp64", alpha=1.0, beta=0.0, u0=None, project=True,
               zero_mean=False, plan=None, **plan_kw):
    n_rhs = f.shape[0]
    own = plan is None
    if own:
        plan = fbc.Plan(xy_i, xy_p, L, material, precision=precision, max_rhs=n_rhs, **plan_kw)
        plan.tabulate()
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    if u0 is None:
        ud = torch.full((n_rhs, len(xy_p), L, 3), float("nan"), dtype=torch.float64, device="cuda")
    else:
        ud = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    plan.apply(fd, ud, alpha=alpha, beta=beta, project=project, zero_mean=zero_mean)
    torch.cuda.synchronize()
    plan.sync_status()
    out = ud.cpu().numpy()
    if own:
        plan.close()
    return out


def test_tiny_ring_full_parity_fp64(fbc, oracle_mod):
    w = inputs.WORKLOADS["ring200x300_L16_iso"]
    xy_i, xy_p = w.geometry()
    f = w.forces()
    ref = oracle_mod.pad_update(xy_i, xy_p, w.L, w.c, w.material, f)
    got = gpu_update(fbc, xy_i, xy_p, w.L, w.material, f)
    assert np.isfinite(got).all()
    assert rel_l2(got, ref) <= TOL_FP64


@pytest.mark.parametrize("material,L", [(ISO, 16), (CUBIC, 32)], ids=["iso-L16", "cubic-L32"])
def test_mode_table_parity(fbc, oracle_mod, material, L):
    xy_i, xy_p = inputs.ring_geometry(90, 130)
    plan = fbc.Plan(xy_i, xy_p, L, material)
    plan.tabulate()
    d_all, _ = oracle_mod.difference_index(xy_i, xy_p)
    rng = np.random.default_rng(0)
    d = d_all[rng.choice(len(d_all), 40, replace=False)]
    got = plan.mode_table(d)  # [nd][K][6]
    plan.close()
    g = oracle_mod.mode_table(oracle_mod.kernel_table(material, L, 1.0, d, nquad=64))
    ref = np.stack([g[..., 0, 0].real, g[..., 0, 1].real, g[..., 1, 1].real, g[..., 2, 2].real,
                    g[..., 0, 2].imag, g[..., 1, 2].imag], axis=-1)
    for a in range(len(d)):
        scale = np.abs(ref[a]).max()
        assert np.abs(got[a] - ref[a]).max() <= 1e-12 * scale, d[a]


def test_cubic_ring_parity(fbc, oracle_mod):
    xy_i, xy_p = inputs.ring_geometry(150, 220)
    L = 32
    f = inputs.forces(1, 150, L, seed=21)
    ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, CUBIC, f, nquad=64)
    got = gpu_update(fbc, xy_i, xy_p, L, CUBIC, f)
    assert rel_l2(got, ref) <= TOL_FP64


@pytest.mark.parametrize("n_i,n_p,L", [(1, 1, 2), (1, 3, 4), (3, 1, 8), (65, 129, 16), (64, 128, 64), (7, 300, 2)])
def test_edge_sizes(fbc, oracle_mod, n_i, n_p, L):
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    f = inputs.forces(2, n_i, L, seed=n_i + n_p + L)
    for project in (True, False):
        ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f, project=project)
        got = gpu_update(fbc, xy_i, xy_p, L, ISO, f, project=project)
        assert rel_l2(got, ref) <= TOL_FP64, (n_i, n_p, L, project)


def test_update_form_and_zero_mean(fbc, oracle_mod):
    xy_i, xy_p = inputs.ring_geometry(120, 170)
    L = 32
    f = inputs.forces(2, 120, L, seed=3)
    u0 = np.random.default_rng(5).standard_normal((2, 170, L, 3))
    ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f, alpha=-0.7, beta=1.0, u0=u0, zero_mean_u=True)
    got = gpu_update(fbc, xy_i, xy_p, L, ISO, f, alpha=-0.7, beta=1.0, u0=u0, zero_mean=True)
    assert rel_l2(got, ref) <= TOL_FP64
    assert np.abs(got.mean(axis=(1, 2))).max() < 1e-14


def test_precisions(fbc, oracle_mod):
    xy_i, xy_p = inputs.ring_geometry(300, 450)
    L = 64
    f = inputs.forces(1, 300, L, seed=8)
    ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f)
    plan = fbc.Plan(xy_i, xy_p, L, ISO)
    plan.tabulate()
    errs = {}
    for prec in ("fp64", "f32x2", "fp32"):
        plan.set_precision(prec)
        errs[prec] = rel_l2(gpu_update(fbc, xy_i, xy_p, L, ISO, f, plan=plan), ref)
    plan.close()
    assert errs["fp64"] <= TOL_FP64
    assert errs["f32x2"] <= TOL_FP64
    assert errs["fp32"] <= TOL_FP32
    assert errs["fp32"] > 1e-9  # really ran in single precision


def test_invariants_on_gpu(fbc):
    xy_i, xy_p = inputs.ring_geometry(100, 140)
    L = 32
    f = inputs.forces(2, 100, L, seed=4)
    plan = fbc.Plan(xy_i, xy_p, L, ISO, max_rhs=2)
    plan.tabulate()
    u = gpu_update(fbc, xy_i, xy_p, L, ISO, f, plan=plan)
    # roll along the line
    ur = gpu_update(fbc, xy_i, xy_p, L, ISO, np.roll(f, 5, axis=2), plan=plan)
    assert rel_l2(ur, np.roll(u, 5, axis=2)) <= 1e-14
    # linearity
    comb = 1.5 * f[:1] - 0.25 * f[1:]
    uc = gpu_update(fbc, xy_i, xy_p, L, ISO, comb, plan=plan)
    assert rel_l2(uc, 1.5 * u[:1] - 0.25 * u[1:]) <= 1e-13
    # deterministic: the same call gives the same bits
    u2 = gpu_update(fbc, xy_i, xy_p, L, ISO, f, plan=plan)
    assert np.array_equal(u, u2)
    plan.close()


def test_host_entry_point_matches_device(fbc):
    xy_i, xy_p = inputs.ring_geometry(80, 100)
    L = 16
    f = inputs.forces(1, 80, L, seed=6)
    plan = fbc.Plan(xy_i, xy_p, L, ISO)
    plan.tabulate()
    dev = gpu_update(fbc, xy_i, xy_p, L, ISO, f, plan=plan, alpha=-1.0, beta=1.0, u0=np.ones((1, 100, L, 3)))
    host_u = np.ones((1, 100, L, 3))
    plan.apply_host(np.ascontiguousarray(f), host_u, alpha=-1.0, beta=1.0)
    plan.close()
    assert np.array_equal(dev, host_u)


def test_host_entry_point_in_chunks(fbc):
    """fbc_apply_host with 22 right-hand sides runs the CUDA-core forms in chunks (5 of 5, 5, 5, 5, 2)
    whose copies overlap the applies of the others, and the tensor-core forms in chunks of whole
    right-hand-side groups (here one).  Every right-hand side gets the bits of one device apply of all
    22 (the CUDA-core forms and BF16X6; BF16X2 within 1e-14), with beta u0, the zero mean and the
    ragged last chunk."""
    xy_i, xy_p = inputs.ring_geometry(80, 100)
    L, R = 16, 22
    f = inputs.forces(R, 80, L, seed=16)
    u0 = np.random.default_rng(5).standard_normal((R, 100, L, 3))
    for prec in ("f32x2", "fp64", "bf16x2", "bf16x6"):
        with fbc.Plan(xy_i, xy_p, L, ISO, precision=prec, max_rhs=R) as plan:
            plan.tabulate()
            dev = gpu_update(fbc, xy_i, xy_p, L, ISO, f, plan=plan, alpha=-1.0, beta=0.5, u0=u0, zero_mean=True)
            host_u = u0.copy()
            plan.apply_host(np.ascontiguousarray(f), host_u, alpha=-1.0, beta=0.5, zero_mean=True)
            plan.sync_status()
        if prec == "bf16x2":
            assert rel_l2(host_u, dev) <= 1e-14
        else:
            assert np.array_equal(dev, host_u), prec


def test_errors_are_reported(fbc):
    xy_i, xy_p = inputs.ring_geometry(10, 12)
    plan = fbc.Plan(xy_i, xy_p, 8, ISO, max_rhs=1)
    f = torch.zeros((1, 10, 8, 3), dtype=torch.float64, device="cuda")
    u = torch.zeros((1, 12, 8, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(fbc.FBCError) as ei:
        plan.apply(f, u)
    assert ei.value.status == fbc.FBC_ERR_NOT_TABULATED
    plan.tabulate()
    with pytest.raises(fbc.FBCError) as ei:
        fbc.fbc_apply(plan.handle, f.data_ptr(), u.data_ptr(), 2, 1.0, 0.0, 0, None)
    assert ei.value.status == fbc.FBC_ERR_INVALID_ARG
    with pytest.raises(fbc.FBCError) as ei:
        fbc.fbc_apply(plan.handle, f.data_ptr(), f.data_ptr(), 1, 1.0, 0.0, 0, None)
    assert ei.value.status == fbc.FBC_ERR_INVALID_ARG  # f and u overlap
    plan.close()


def test_paper_scale_cubic_sampled(fbc, oracle_mod):
    """Full-size cubic instance (N_I = 4000, N_P = 6000, L = 256) in the
    configuration the benchmark times, checked at sampled pad atoms."""
    w = inputs.WORKLOADS["ring4000x6000_L256_cubic"]
    xy_i, xy_p = w.geometry()
    f = w.forces()
    r2 = (xy_p.astype(np.int64) ** 2).sum(axis=1)
    cols = [int(np.argmin(r2)), int(np.argmax(r2))]
    samples = np.array([[a, p] for a in cols for p in (0, 17, 128, 255)], dtype=np.int64)
    ref = oracle_mod.pad_update(xy_i, xy_p, w.L, w.c, w.material, f, samples=samples, nquad=64)[0]
    plan = fbc.Plan(xy_i, xy_p, w.L, w.material)
    plan.tabulate()
    for prec in ("fp64", "f32x2"):
        plan.set_precision(prec)
        got = gpu_update(fbc, xy_i, xy_p, w.L, w.material, f, plan=plan)
        sel = got[0, samples[:, 0], samples[:, 1]]
        assert rel_l2(sel, ref) <= TOL_FP64, prec
    plan.close()


@pytest.mark.parametrize("R,n_i,n_p,L", [(7, 200, 300, 16), (64, 130, 260, 8)], ids=["R7-ragged", "R64"])
def test_multi_rhs_double_float_tile_bits(fbc, oracle_mod, R, n_i, n_p, L):
    """The multi-rhs double-float tile (several right-hand sides per thread, used for n_rhs >= 2) gives every
    right-hand side the same bits as an apply of that right-hand side alone (one-rhs tile): the products,
    their order and the fold per interface tile are the same.  Also for the k = 0 one-mode launch of the
    FP32 and tensor-core forms.  Right-hand side 0 against the oracle at 1e-12; a ragged last group."""
    torch_ = pytest.importorskip("torch")
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    f = inputs.forces(R, n_i, L, seed=41)
    fd = torch_.from_numpy(f).cuda()
    for prec in ("f32x2", "bf16x2"):
        with fbc.Plan(xy_i, xy_p, L, ISO, precision=prec, max_rhs=R) as plan:
            plan.tabulate()
            u = torch_.zeros((R, n_p, L, 3), dtype=torch_.float64, device="cuda")
            plan.apply(fd, u)
            torch_.cuda.synchronize()
            plan.sync_status()
            many = u.cpu().numpy()
            one = np.empty_like(many)
            for r in range(R):
                u1 = torch_.zeros((1, n_p, L, 3), dtype=torch_.float64, device="cuda")
                plan.apply(fd[r:r + 1].contiguous(), u1)
                torch_.cuda.synchronize()
                one[r] = u1[0].cpu().numpy()
            plan.sync_status()
        if prec == "f32x2":
            assert np.array_equal(many, one)
            ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f[:1])
            assert rel_l2(many[:1], ref) <= 1e-12
        else:
            # the k = 0 mode comes from the double-float tile in both cases: equal bits in that band
            k0_many = many.sum(axis=2)
            k0_one = one.sum(axis=2)
            assert np.abs(k0_many - k0_one).max() <= 1e-12 * np.abs(k0_one).max()


def test_double_float_wide_sub_box(fbc, oracle_mod):
    """Two rows of columns, the pad row three sites apart: the sub-box of a tile pair is 445 x 1 table
    entries, a line of 445 x 48 bytes, over the 256 8-byte elements of a tensor copy's box line, so the
    double-float tile stages it with its threads instead of one TMA copy.  That staging against the
    oracle at 1e-12 (the ring geometries of the other tests take the TMA copy)."""
    n_i, n_p, L, R = 200, 300, 8, 3
    xy_i = np.stack([np.arange(n_i), np.zeros(n_i, dtype=np.int64)], axis=1).astype(np.int32)
    xy_p = np.stack([3 * np.arange(n_p), np.full(n_p, 2)], axis=1).astype(np.int32)
    f = inputs.forces(R, n_i, L, seed=23)
    ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f)
    with fbc.Plan(xy_i, xy_p, L, ISO, precision="f32x2", max_rhs=R) as plan:
        info = plan.info()
        assert 6 * info["sub_w"] > 256
        plan.tabulate()
        for n in (1, R):  # the one-rhs and the multi-rhs tiles
            got = gpu_update(fbc, xy_i, xy_p, L, ISO, f[:n], plan=plan)
            assert rel_l2(got, ref[:n]) <= TOL_FP64, n
