"""Tensor-core (tcgen05) contraction for plans with several right-hand sides.

The TF32, BF16x2 and BF16x3 forms (k >= 1 on the tensor cores with FP32
accumulation in tensor memory, k = 0 in FP64) are compared with the FP64 GPU
path, which is itself at 1e-12 of the oracle.  Expected accuracy from the
operand precision and FP32 accumulation over 3 N_I terms: TF32 ~1e-3,
BF16x2 ~1e-5, BF16x3 ~1e-6.  Also checked: ragged right-hand-side counts
(padding of the GEMM's N dimension), more than 64 right-hand sides (two CTA
groups along N), and agreement with the oracle on one right-hand side.
"""

import numpy as np
import pytest

from conftest import ISO
from paper_2105_08798_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUNDS = {"tf32": 5e-3, "bf16x2": 1e-4, "bf16x3": 1e-5}


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.fixture(scope="module")
def fbc():
    from paper_2105_08798_gb300 import build, fbc as binding

    build.build()
    binding.load()
    return binding


def _run_all(fbc, n_i, n_p, L, R, seed):
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    f = inputs.forces(R, n_i, L, seed=seed)
    out = {}
    with fbc.Plan(xy_i, xy_p, L, ISO, max_rhs=R) as plan:
        plan.tabulate()
        fd = torch.from_numpy(f).cuda()
        for prec in ("fp64", "tf32", "bf16x2", "bf16x3"):
            plan.set_precision(prec)
            ud = torch.full((R, n_p, L, 3), float("nan"), dtype=torch.float64, device="cuda")
            plan.apply(fd, ud)
            torch.cuda.synchronize()
            plan.sync_status()
            out[prec] = ud.cpu().numpy()
    return xy_i, xy_p, f, out


# (1500, 2000): more than 1024 interface columns, so the accumulators are drained mid-sum
@pytest.mark.parametrize("n_i,n_p,L,R", [(300, 450, 32, 16), (150, 220, 16, 3), (100, 140, 8, 70), (1500, 2000, 8, 8)])
def test_tensor_forms_against_fp64(fbc, n_i, n_p, L, R):
    _, _, _, out = _run_all(fbc, n_i, n_p, L, R, seed=n_i + R)
    assert np.isfinite(out["fp64"]).all()
    errs = {}
    for prec, bound in BOUNDS.items():
        assert np.isfinite(out[prec]).all(), prec
        errs[prec] = rel_l2(out[prec], out["fp64"])
        assert errs[prec] <= bound, (prec, errs[prec])
    assert errs["bf16x3"] < errs["bf16x2"] < errs["tf32"], errs


def test_tensor_form_against_oracle(fbc, oracle_mod):
    xy_i, xy_p, f, out = _run_all(fbc, 200, 300, 16, 8, seed=3)
    ref = oracle_mod.pad_update(xy_i, xy_p, 16, 1.0, ISO, f[:1])
    assert rel_l2(out["fp64"][:1], ref) <= 1e-12
    assert rel_l2(out["bf16x3"][:1], ref) <= BOUNDS["bf16x3"]


def test_k0_band_stays_fp64(fbc):
    """The k = 0 mode runs in double-float and the FP32 line transforms keep it in FP64:
    the mean along the line of every pad column matches the FP64 path to rounding."""
    _, _, _, out = _run_all(fbc, 300, 450, 64, 8, seed=11)
    ref = np.fft.rfft(out["fp64"], axis=2)[:, :, 0]
    for prec in BOUNDS:
        got = np.fft.rfft(out[prec], axis=2)[:, :, 0]
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-11, (prec, err)


def test_fast_accumulate_flag(fbc):
    """More than 1024 interface columns: the default splits the tensor-memory accumulation
    into groups; FBC_PLAN_TC_FAST_ACCUMULATE keeps one group.  Both stay within the BF16x2
    bound against FP64, and they differ (the flag changes the summation)."""
    n_i, n_p, L, R = 1500, 2000, 8, 8
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    f = torch.from_numpy(inputs.forces(R, n_i, L, seed=2)).cuda()
    out = {}
    for name, prec, fast in (("fp64", "fp64", False), ("grouped", "bf16x2", False), ("one", "bf16x2", True)):
        with fbc.Plan(xy_i, xy_p, L, ISO, precision=prec, max_rhs=R, tc_fast_accumulate=fast) as plan:
            plan.tabulate()
            ud = torch.full((R, n_p, L, 3), float("nan"), dtype=torch.float64, device="cuda")
            plan.apply(f, ud)
            torch.cuda.synchronize()
            plan.sync_status()
            out[name] = ud.cpu().numpy()
    for name in ("grouped", "one"):
        assert rel_l2(out[name], out["fp64"]) <= BOUNDS["bf16x2"], name
    assert not np.array_equal(out["grouped"], out["one"])
