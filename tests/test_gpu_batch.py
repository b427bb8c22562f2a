"""Multi-right-hand-side and batched updates on the GPU (through the C ABI).

* The register-blocked FP32 contraction (8 right-hand sides per thread, a
  ragged last block) matches the oracle at the FP32 tolerance and the FP64
  GPU path.
* A batch of uneven instances, applied by one persistent contraction launch
  (directly and replayed from a CUDA graph), reproduces each plan's own
  fbc_apply bit for bit, and the oracle within the FP64 tolerance; graph
  replays are deterministic; the autotuner keeps results unchanged.
* The same for the tensor-core forms (one persistent tcgen05 launch over the
  items of all instances, k = 0 in double-float), including the autotuner's
  choice of the rhs group (right-hand sides per work item).
"""

import numpy as np
import pytest

from conftest import ISO
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


def test_multi_rhs_fp32_blocks(fbc, oracle_mod):
    xy_i, xy_p = inputs.ring_geometry(140, 200)
    L, R = 32, 10
    f = inputs.forces(R, 140, L, seed=31, decay=0.7)
    ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, f)
    with fbc.Plan(xy_i, xy_p, L, ISO, max_rhs=R) as plan:
        plan.tabulate()
        fd = torch.from_numpy(f).cuda()
        out = {}
        for prec in ("fp32", "fp64"):
            plan.set_precision(prec)
            ud = torch.full((R, 200, L, 3), float("nan"), dtype=torch.float64, device="cuda")
            plan.apply(fd, ud)
            torch.cuda.synchronize()
            out[prec] = ud.cpu().numpy()
    assert rel_l2(out["fp64"], ref) <= 1e-12
    for r in range(R):
        assert rel_l2(out["fp32"][r], ref[r]) <= 5e-6, r


CASES = [(60, 90, 16, 2), (150, 220, 32, 3), (90, 130, 64, 1), (30, 45, 8, 9)]


def _make(fbc, prec):
    plans, fs, us, ref_u = [], [], [], []
    for idx, (n_i, n_p, L, R) in enumerate(CASES):
        xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
        p = fbc.Plan(xy_i, xy_p, L, ISO, precision=prec, max_rhs=R)
        p.tabulate()
        f = torch.from_numpy(inputs.forces(R, n_i, L, seed=100 + idx, decay=0.5)).cuda()
        u0 = torch.from_numpy(np.random.default_rng(idx).standard_normal((R, n_p, L, 3))).cuda()
        plans.append(p)
        fs.append(f)
        us.append(u0)
        ref_u.append(u0.clone())
    return plans, fs, us, ref_u


@pytest.mark.parametrize("prec", ["fp64", "f32x2", "fp32", "bf16x2", "tf32", "bf16x3"])
def test_batch_matches_per_plan_apply(fbc, prec):
    plans, fs, us, ref_u = _make(fbc, prec)
    for p, f, u in zip(plans, fs, ref_u):
        p.apply(f, u, alpha=-0.5, beta=1.0, zero_mean=True)
    u_direct = [u.clone() for u in us]
    with fbc.Batch(plans, fs, u_direct) as b:
        b.apply(alpha=-0.5, beta=1.0, zero_mean=True, graph=False)
    u_graph = [u.clone() for u in us]
    with fbc.Batch(plans, fs, u_graph) as b:
        b.apply(alpha=-0.5, beta=1.0, zero_mean=True, graph=True)
        torch.cuda.synchronize()
        info = b.info()
    torch.cuda.synchronize()
    for r, d, g in zip(ref_u, u_direct, u_graph):
        assert torch.equal(r, d)
        assert torch.equal(r, g)
    assert info["n_plans"] == len(CASES) and info["n_contract_items"] > 0
    for p in plans:
        p.close()


def test_batch_graph_replay_and_autotune(fbc, oracle_mod):
    plans, fs, us, _ = _make(fbc, "fp64")
    outs = [torch.zeros_like(u) for u in us]
    with fbc.Batch(plans, fs, outs) as b:
        b.apply()
        torch.cuda.synchronize()
        first = [o.clone() for o in outs]
        b.apply()  # replay (beta = 0: same result)
        torch.cuda.synchronize()
        assert all(torch.equal(a, o) for a, o in zip(first, outs))
        ms = b.autotune()
        assert ms > 0
        b.apply()
        torch.cuda.synchronize()
        assert all(torch.equal(a, o) for a, o in zip(first, outs))
    # one instance against the oracle
    n_i, n_p, L, R = CASES[1]
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, fs[1].cpu().numpy())
    assert rel_l2(first[1].cpu().numpy(), ref) <= 1e-12
    for p in plans:
        p.close()


def test_batch_rejects_bad_input(fbc):
    plans, fs, us, _ = _make(fbc, "fp64")
    with pytest.raises(fbc.FBCError):
        fbc.Batch([plans[0], plans[0]], [fs[0], fs[0]], [us[0], us[0]])  # same plan twice
    plans[1].set_precision("fp32")
    with pytest.raises(fbc.FBCError):
        fbc.Batch(plans[:2], fs[:2], us[:2])  # mixed precisions
    for p in plans:
        p.close()


def test_tensor_batch_autotune_and_oracle(fbc, oracle_mod):
    cases = [(200, 300, 32, 16), (120, 180, 16, 16), (260, 390, 64, 16)]
    plans, fs, outs = [], [], []
    for idx, (n_i, n_p, L, R) in enumerate(cases):
        xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
        p = fbc.Plan(xy_i, xy_p, L, ISO, precision="bf16x2", max_rhs=R)
        p.tabulate()
        plans.append(p)
        fs.append(torch.from_numpy(inputs.forces(R, n_i, L, seed=200 + idx, decay=0.5)).cuda())
        outs.append(torch.zeros((R, n_p, L, 3), dtype=torch.float64, device="cuda"))
    with fbc.Batch(plans, fs, outs) as b:
        b.apply()
        torch.cuda.synchronize()
        first = [o.clone() for o in outs]
        ms = b.autotune()
        assert ms > 0
        info = b.info()
        assert info["rhs_per_cta"] in (16, 8)
        assert info["launch_form"] in (0, 1)
        b.apply()
        torch.cuda.synchronize()
        assert all(torch.equal(a, o) for a, o in zip(first, outs))
        plans[0].sync_status()
    # each instance against its own apply, and one against the oracle (BF16x2 level; k = 0 FP64-accurate)
    for p, f, o in zip(plans, fs, first):
        u = torch.zeros_like(o)
        p.apply(f, u)
        torch.cuda.synchronize()
        assert torch.equal(u, o)
    n_i, n_p, L, R = cases[0]
    xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
    ref = oracle_mod.pad_update(xy_i, xy_p, L, 1.0, ISO, fs[0][:2].cpu().numpy())
    assert rel_l2(first[0][:2].cpu().numpy(), ref) <= 1e-4
    for p in plans:
        p.close()
