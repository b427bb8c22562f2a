"""Learned mode-table surrogate: kernels against the FP64 reference, training,
and the streamed pad update with and without it (ablation).

* forward pass and loss gradient of the CUDA MLP against ``oracle/mlp.py``
  (FP64, pinned by finite differences), element by element;
* training lowers the loss, is reproducible for a seed, and the trained
  network's table entries approach the exact FP64 mode table;
* the streamed contraction (one mode slice at a time) with every difference
  served exactly reproduces the K-slice table path of the same precision;
* with the surrogate serving |d| >= r_min, the update's error against FP64,
  its memory and the release of the K-slice tables.
"""

import numpy as np
import pytest

from conftest import ISO
from oracle import mlp
from paper_2105_08798_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


# BF16-weight inference: widths 32..128 (multiples of 32) run the fused
# tensor-core kernel, whose activations carry ~16 mantissa bits (hi + lo bf16
# pieces) -> a few 1e-6 per layer; other widths the FP32 GEMM path.
FUSED = {32, 64, 96, 128}


@pytest.mark.parametrize("H,n", [(8, 5), (32, 129), (64, 1000), (96, 77), (128, 333), (128, 70000)])
def test_forward_matches_fp64(fbc, H, n):
    with fbc.Surrogate(width=H, seed=H) as S:
        p = S.params()
        assert p.size == mlp.n_params(H) == S.n_params
        x = np.random.default_rng(n).normal(0, 1, (n, 4)).astype(np.float32)
        xd = torch.from_numpy(x).cuda()
        y = S.forward(xd).cpu().numpy()
        yb = S.forward(xd, bf16_weights=True).cpu().numpy()
        S.sync_status()
        ref, _ = mlp.forward(p, H, x)
        refb, _ = mlp.forward(mlp.round_bf16(p), H, x)
        assert rel_l2(y, ref) <= 1e-5
        eb = rel_l2(yb, refb)
        assert eb <= (5e-5 if H in FUSED else 1e-5), eb
        assert rel_l2(yb, ref) > 10 * eb  # the BF16 weights really are rounded


@pytest.mark.parametrize("H,n", [(8, 7), (64, 777), (128, 4096)])
def test_loss_gradient_matches_fp64(fbc, H, n):
    rng = np.random.default_rng(H + n)
    with fbc.Surrogate(width=H, seed=7) as S:
        p = rng.normal(0, 0.3, S.n_params).astype(np.float32)
        S.set_params(p)
        np.testing.assert_array_equal(S.params(), p)
        x = rng.normal(0, 1, (n, 4)).astype(np.float32)
        t = rng.normal(0, 1, (n, 6)).astype(np.float32)
        loss, g = S.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
        ref_loss, ref_g = mlp.loss_grad(p, H, x, t)
        assert loss == pytest.approx(ref_loss, rel=1e-5)
        assert rel_l2(g, ref_g) <= 1e-5
        # every block of the parameter vector (each weight and bias) on its own
        o = 0
        for blk in mlp.unpack(ref_g, H):
            sl = slice(o, o + blk.size)
            assert rel_l2(g[sl], ref_g[sl]) <= 1e-4, (o, blk.shape)
            o += blk.size


@pytest.fixture(scope="module")
def trained(fbc):
    xy_i, xy_p = inputs.ring_geometry(300, 450)
    L = 64
    plan = fbc.Plan(xy_i, xy_p, L, ISO, precision="fp32", max_rhs=4)
    plan.tabulate()
    S = fbc.Surrogate(width=64, seed=11)
    first = S.train(plan, n_samples=1 << 14, r_min=8.0, epochs=1, batch=1024, lr=3e-3, seed=1)
    last = S.train(plan, n_samples=1 << 16, r_min=8.0, epochs=40, batch=1024, lr=3e-3, seed=2)
    yield plan, S, first, last, xy_i, xy_p, L
    plan.close()
    S.close()


def _far_samples(xy_i, xy_p, L, r_min, n, seed):
    used = np.unique((xy_p[:, None, :] - xy_i[None, :, :]).reshape(-1, 2), axis=0)
    r = np.hypot(used[:, 0], used[:, 1])
    far = used[r >= r_min]
    rng = np.random.default_rng(seed)
    d = far[rng.integers(0, len(far), n)]
    k = rng.integers(1, L // 2 + 1, n)
    return d, k


def test_training_reduces_loss_and_fits_the_table(fbc, trained):
    plan, S, first, last, xy_i, xy_p, L = trained
    print(f"\nsurrogate loss: first epoch {first:.3e}, after 40 epochs {last:.3e}")
    assert np.isfinite(first) and np.isfinite(last)
    assert last < 0.1 * first
    d, k = _far_samples(xy_i, xy_p, L, 8.0, 2000, seed=4)
    sur = S.table(plan, d, k)
    exact = plan.mode_table(d)[np.arange(len(k)), k]
    sc = mlp.scale(d, k, L)
    keep = sc > 0
    err = np.linalg.norm((sur - exact)[keep] / sc[keep, None]) / np.linalg.norm(exact[keep] / sc[keep, None])
    print(f"surrogate table error (scaled units, {keep.sum()} samples): {err:.3e}")
    assert err <= 5e-2
    assert np.all(sur[~keep] == 0.0)


def test_training_is_reproducible(fbc, trained):
    plan = trained[0]
    ps = []
    for _ in range(2):
        with fbc.Surrogate(width=16, seed=3) as S:
            S.train(plan, n_samples=4096, r_min=8.0, epochs=3, batch=512, lr=1e-3, seed=9)
            ps.append(S.params())
    np.testing.assert_array_equal(ps[0], ps[1])


def _apply(plan, f):
    fd = torch.from_numpy(f).cuda()
    ud = torch.full((f.shape[0], plan.n_p, plan.L, 3), float("nan"), dtype=torch.float64, device="cuda")
    plan.apply(fd, ud)
    torch.cuda.synchronize()
    plan.sync_status()
    return ud.cpu().numpy()


@pytest.mark.parametrize("precision,R", [("fp32", 1), ("fp32", 4), ("tf32", 16), ("bf16x3", 16)])
def test_streamed_exact_slices_match_table_path(fbc, precision, R):
    xy_i, xy_p = inputs.ring_geometry(200, 300)
    L = 32
    f = inputs.forces(R, 200, L, seed=R)
    with fbc.Plan(xy_i, xy_p, L, ISO, precision=precision, max_rhs=R) as plan, fbc.Surrogate(width=32) as S:
        plan.tabulate()
        ref = _apply(plan, f)
        plan.attach_surrogate(S, r_min=1e9)  # every difference is near: exact slices
        info = plan.info()
        assert info["surrogate_attached"] == 1 and info["n_far_d"] == 0
        got = _apply(plan, f)
        assert np.isfinite(got).all()
        assert rel_l2(got, ref) <= 1e-12
        plan.attach_surrogate(None)
        assert plan.info()["surrogate_attached"] == 0
        np.testing.assert_array_equal(_apply(plan, f), ref)


def _six_to_complex(six):
    """[..., 6] mode-table reals -> complex-symmetric [..., 3, 3] (11, 12, 22, 33 real; 13, 23 imaginary)."""
    A11, A12, A22, A33, B13, B23 = np.moveaxis(six, -1, 0)
    g = np.zeros(six.shape[:-1] + (3, 3), dtype=complex)
    g[..., 0, 0], g[..., 0, 1], g[..., 1, 0], g[..., 1, 1], g[..., 2, 2] = A11, A12, A12, A22, A33
    g[..., 0, 2] = g[..., 2, 0] = 1j * B13
    g[..., 1, 2] = g[..., 2, 1] = 1j * B23
    return g


def _mode_domain_update(oracle_mod, xy_i, xy_p, L, f, table):
    """u = G f evaluated in the mode domain with a given mode table (numpy FFT along the line)."""
    F = np.fft.fft(oracle_mod.project_neutral(f), axis=2)  # [R][n_i][L][3]
    dd = (xy_p[:, None, :] - xy_i[None, :, :]).reshape(-1, 2)
    uniq, inv = np.unique(dd, axis=0, return_inverse=True)
    g = _six_to_complex(table(uniq))  # [nu][K][3][3]
    U = np.zeros((f.shape[0], len(xy_p), L, 3), dtype=complex)
    for k in range(L):
        gk = g[:, k] if k <= L // 2 else np.conj(g[:, L - k])
        G = gk[inv.ravel()].reshape(len(xy_p), len(xy_i), 3, 3)
        U[:, :, k, :] = np.einsum("abij,rbj->rai", G, F[:, :, k, :])
    return np.fft.ifft(U, axis=2).real


def test_streamed_surrogate_slices(fbc, oracle_mod, trained):
    """The fused kernel's slices against the network's row outputs, through a whole update."""
    _, S, _, _, _, _, _ = trained
    xy_i, xy_p = inputs.ring_geometry(200, 300)
    L, R, r_min = 32, 3, 6.0
    f = inputs.forces(R, 200, L, seed=17)
    K = L // 2 + 1
    with fbc.Plan(xy_i, xy_p, L, ISO, precision="fp32", max_rhs=R) as plan:
        plan.tabulate()
        exact = lambda d: plan.mode_table(d)
        u_tab = _apply(plan, f)
        ref_tab = _mode_domain_update(oracle_mod, xy_i, xy_p, L, f, exact)
        assert rel_l2(u_tab, ref_tab) <= 1e-5  # the reference itself, on the exact table

        def hybrid(d):
            t = exact(d)
            far = np.hypot(d[:, 0], d[:, 1]) >= r_min
            df = np.repeat(d[far], K - 1, axis=0)
            kf = np.tile(np.arange(1, K), far.sum())
            t[far, 1:] = S.table(plan, df, kf).reshape(far.sum(), K - 1, 6)
            return t

        plan.attach_surrogate(S, r_min=r_min)
        u_sur = _apply(plan, f)
        ref_sur = _mode_domain_update(oracle_mod, xy_i, xy_p, L, f, hybrid)
        e = rel_l2(u_sur, ref_sur)
        print(f"\nstreamed surrogate update vs mode-domain reference: {e:.2e}; vs exact table {rel_l2(u_sur, u_tab):.2e}")
        assert e <= 1e-5


def test_surrogate_update_ablation(fbc, trained):
    plan, S, _, _, xy_i, xy_p, L = trained
    f = inputs.forces(4, len(xy_i), L, seed=21)
    u32 = _apply(plan, f)
    with fbc.Plan(xy_i, xy_p, L, ISO, precision="fp64", max_rhs=4) as p64:
        p64.tabulate()
        u64 = _apply(p64, f)
    plan.attach_surrogate(S, r_min=8.0)
    info = plan.info()
    u_sur = _apply(plan, f)
    plan.attach_surrogate(None)
    e32, esur = rel_l2(u32, u64), rel_l2(u_sur, u64)
    print(f"\nablation: fp32 table {e32:.3e}, surrogate (r >= 8) {esur:.3e}; far differences "
          f"{info['n_far_d']} of {info['n_used_d']}; surrogate buffers {info['surrogate_bytes']} B, "
          f"FP64 table {info['table_bytes']} B")
    assert info["n_far_d"] > 0
    assert np.isfinite(u_sur).all()
    assert esur <= 5e-2
    assert esur > e32  # the learned far field is the larger error


def test_released_tables(fbc, trained):
    _, S, _, _, xy_i, xy_p, L = trained
    f = inputs.forces(2, len(xy_i), L, seed=5)
    with fbc.Plan(xy_i, xy_p, L, ISO, precision="fp32", max_rhs=2) as plan:
        plan.tabulate()
        before = plan.info()
        plan.attach_surrogate(S, r_min=8.0)
        keep = _apply(plan, f)
        plan.attach_surrogate(S, r_min=8.0, release_tables=True)
        after = plan.info()
        np.testing.assert_array_equal(_apply(plan, f), keep)
        assert after["table_bytes"] == 0
        assert after["workspace_bytes"] + after["surrogate_bytes"] < before["workspace_bytes"] + before["table_bytes"]
        for call in (lambda: plan.mode_table([[1, 0]]), lambda: plan.set_precision("fp64"), plan.tabulate,
                     lambda: plan.attach_surrogate(None)):
            with pytest.raises(fbc.FBCError):
                call()


def test_attach_validation(fbc):
    xy_i, xy_p = inputs.ring_geometry(100, 140)
    with fbc.Surrogate(width=8) as S8, fbc.Plan(xy_i, xy_p, 8, ISO, precision="fp32") as plan:
        plan.tabulate()
        with pytest.raises(fbc.FBCError):
            plan.attach_surrogate(S8, r_min=4.0)  # no fused inference kernel for this width
    with fbc.Surrogate(width=32) as S:
        with fbc.Plan(xy_i, xy_p, 8, ISO, precision="fp64") as plan:
            plan.tabulate()
            with pytest.raises(fbc.FBCError):
                plan.attach_surrogate(S, r_min=8.0)  # FP64 plans keep the exact table
        with fbc.Plan(xy_i, xy_p, 8, ISO, precision="fp32") as plan:
            with pytest.raises(fbc.FBCError):
                plan.attach_surrogate(S, r_min=8.0)  # not tabulated
            plan.tabulate()
            with pytest.raises(fbc.FBCError):
                plan.attach_surrogate(S, r_min=0.0)
            plan.attach_surrogate(S, r_min=4.0)
            with pytest.raises(fbc.FBCError):
                plan.set_precision("f32x2")  # the surrogate serves FP32 and tensor-core plans
            plan.set_precision("bf16x2")
    with pytest.raises(fbc.FBCError):
        fbc.Surrogate(width=12)
