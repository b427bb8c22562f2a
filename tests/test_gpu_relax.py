"""Relaxed FBC update (Algorithm 1 with the relaxation of Algorithm 2) through the C ABI.

The device computes alpha from the residuals and ||G f||_inf and applies
u <- u - alpha G f; the oracle does the same in FP64 on the CPU
(``oracle.relaxed_update``).  Checked: the Aitken step with and without the cap,
no previous residual, the zero mean, two iterations in a row (alpha carried on
the device), and a tensor-core plan against the FP64 plan.
"""

import numpy as np
import pytest

from conftest import ISO
from paper_2105_08798_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_I, N_P, L, R = 200, 300, 16, 3


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.fixture(scope="module")
def fbc():
    from paper_2105_08798_gb300 import build, fbc as binding

    build.build()
    binding.load()
    return binding


@pytest.fixture(scope="module")
def case():
    xy_i, xy_p = inputs.ring_geometry(N_I, N_P)
    rng = np.random.default_rng(12)
    f_old = inputs.forces(R, N_I, L, seed=4)
    f_new = 0.6 * f_old + 0.3 * inputs.forces(R, N_I, L, seed=5)  # a shrinking residual
    u0 = rng.normal(0, 1, (R, N_P, L, 3))
    return xy_i, xy_p, f_old, f_new, u0


def _gpu(fbc, plan, f_new, f_old, u0, alpha_k, du_max, zero_mean=False):
    fn = torch.from_numpy(f_new).cuda()
    fo = None if f_old is None else torch.from_numpy(f_old).cuda()
    u = torch.from_numpy(u0.copy()).cuda()
    a = torch.tensor(alpha_k, dtype=torch.float64, device="cuda")
    plan.apply_relaxed(fn, fo, u, a, du_max=du_max, zero_mean=zero_mean)
    torch.cuda.synchronize()
    plan.sync_status()
    return u.cpu().numpy(), a.cpu().numpy()


# du_max = 1 caps some right-hand sides and not others; 1e-2 caps all of them
@pytest.mark.parametrize("du_max,zero_mean,use_old", [(0.0, False, True), (1.0, False, True), (1e-2, False, True),
                                                      (0.0, True, False), (1.0, True, False)])
def test_relaxed_update_matches_oracle(fbc, oracle_mod, case, du_max, zero_mean, use_old):
    xy_i, xy_p, f_old, f_new, u0 = case
    alpha_k = [1.0, 0.7, 2.5]
    fo = f_old if use_old else None
    ref_u, ref_a = oracle_mod.relaxed_update(xy_i, xy_p, L, 1.0, ISO, f_new, fo, u0, alpha_k, du_max=du_max,
                                             zero_mean_u=zero_mean)
    with fbc.Plan(xy_i, xy_p, L, ISO, precision="fp64", max_rhs=R) as plan:
        plan.tabulate()
        u, a = _gpu(fbc, plan, f_new, fo, u0, alpha_k, du_max, zero_mean)
    np.testing.assert_allclose(a, ref_a, rtol=1e-12)
    assert rel_l2(u, ref_u) <= 1e-12
    if du_max == 1.0:
        _, free = oracle_mod.relaxed_update(xy_i, xy_p, L, 1.0, ISO, f_new, fo, u0, alpha_k)
        capped = ref_a < free
        assert capped.any() and not capped.all(), (ref_a, free)


def test_two_iterations(fbc, oracle_mod, case):
    """alpha stays on the device between calls; the second step uses the first step's alpha."""
    xy_i, xy_p, f_old, f_new, u0 = case
    f_next = 0.5 * f_new + 0.1 * f_old
    with fbc.Plan(xy_i, xy_p, L, ISO, precision="f32x2", max_rhs=R) as plan:
        plan.tabulate()
        fn, fo, fx = (torch.from_numpy(x).cuda() for x in (f_new, f_old, f_next))
        u = torch.from_numpy(u0.copy()).cuda()
        a = torch.ones(R, dtype=torch.float64, device="cuda")
        plan.apply_relaxed(fn, fo, u, a, du_max=0.05)
        plan.apply_relaxed(fx, fn, u, a, du_max=0.05)
        torch.cuda.synchronize()
        plan.sync_status()
        u, a = u.cpu().numpy(), a.cpu().numpy()
    u1, a1 = oracle_mod.relaxed_update(xy_i, xy_p, L, 1.0, ISO, f_new, f_old, u0, np.ones(R), du_max=0.05)
    u2, a2 = oracle_mod.relaxed_update(xy_i, xy_p, L, 1.0, ISO, f_next, f_new, u1, a1, du_max=0.05)
    np.testing.assert_allclose(a, a2, rtol=1e-12)
    assert rel_l2(u, u2) <= 1e-12


@pytest.mark.parametrize("prec,tol", [("bf16x2", 1e-4), ("fft32", 1e-5), ("fft64", 1e-12)])
def test_other_forms(fbc, case, prec, tol):
    """Tensor-core and in-plane FFT plans: alpha from the same FP64 dot products, ||G f|| from the form's
    own inverse transform (FP32 for the tensor-core and FP32 FFT forms)."""
    xy_i, xy_p, f_old, f_new, u0 = case
    out = {}
    for p in ("fp64", prec):
        with fbc.Plan(xy_i, xy_p, L, ISO, precision=p, max_rhs=R) as plan:
            plan.tabulate()
            out[p] = _gpu(fbc, plan, f_new, f_old, u0, [1.0, 1.0, 1.0], 1e-2)
    np.testing.assert_allclose(out[prec][1], out["fp64"][1], rtol=tol)
    assert rel_l2(out[prec][0] - u0, out["fp64"][0] - u0) <= tol


def test_rejects_bad_arguments(fbc, case):
    xy_i, xy_p, f_old, f_new, u0 = case
    with fbc.Plan(xy_i, xy_p, L, ISO, precision="fp64", max_rhs=R) as plan:
        plan.tabulate()
        fn = torch.from_numpy(f_new).cuda()
        u = torch.from_numpy(u0.copy()).cuda()
        a = torch.ones(R, dtype=torch.float64, device="cuda")
        with pytest.raises(fbc.FBCError):
            plan.apply_relaxed(fn, fn, u, a)  # f_old is f_new
        with pytest.raises(fbc.FBCError):
            plan.apply_relaxed(fn, None, u, a, du_max=-1.0)


def test_iteration_captured_in_a_cuda_graph(fbc, case):
    """alpha lives on the device, so an iteration (incompatibility force, then the relaxed update)
    needs no host round trip: captured once in a CUDA graph and replayed, it gives the same bits as
    the same calls made directly."""
    from paper_2105_08798_gb300 import inputs as inp

    xy_i, xy_p, f_old, f_new, u0 = case
    xy_c = inp.core_sites(N_I)
    K = fbc.fbc_spring_constants(1.0, 0.4, 1.0)
    rng = np.random.default_rng(21)
    u_c = torch.from_numpy(0.05 * rng.normal(0, 1, (R, len(xy_c), L, 3))).cuda()
    u_i = torch.from_numpy(0.05 * rng.normal(0, 1, (R, N_I, L, 3))).cuda()
    outs = []
    with fbc.Plan(xy_i, xy_p, L, ISO, precision="f32x2", max_rhs=R) as plan, \
            fbc.Stencil(xy_i, [xy_c, xy_i, xy_p], L, K) as st:
        plan.tabulate()
        for mode in ("direct", "graph"):
            up = torch.from_numpy(u0.copy()).cuda()
            fs = [torch.zeros((R, N_I, L, 3), dtype=torch.float64, device="cuda") for _ in range(2)]
            a = torch.ones(R, dtype=torch.float64, device="cuda")

            def step(i):
                st.incompat_force([u_c, u_i, up], f=fs[i % 2])
                plan.apply_relaxed(fs[i % 2], fs[(i + 1) % 2], up, a, du_max=0.05, zero_mean=True)

            step(0)  # first iteration (no previous residual in fs[1]: zeros, alpha kept) made directly
            torch.cuda.synchronize()
            if mode == "direct":
                for i in range(1, 5):
                    step(i)
            else:
                graphs = []
                for parity in (1, 2):  # the two residual buffers alternate: one graph per parity
                    g = torch.cuda.CUDAGraph()
                    side = torch.cuda.Stream()
                    side.wait_stream(torch.cuda.current_stream())
                    with torch.cuda.graph(g, stream=side):
                        step(parity)
                    graphs.append(g)
                # capture does not run the work: replay in order 1, 2, 3, 4
                up.copy_(torch.from_numpy(u0.copy()).cuda())
                a.fill_(1.0)
                for t in fs:
                    t.zero_()
                step(0)
                for i in range(1, 5):
                    graphs[(i - 1) % 2].replay()
            torch.cuda.synchronize()
            plan.sync_status()
            outs.append((up.cpu().numpy(), a.cpu().numpy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
