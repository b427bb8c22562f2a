"""Error paths of the boundary on the device: a bounded wait that runs out, and allocations that fail.

* Timeout: the tensor-core contraction's pipeline waits are bounded by the plan's wait limit
  (fbc_plan_set_wait_limit).  With one poll per wait the first hand-off between the builder warps
  and the MMA thread cannot be ready in time, so the kernel stops, records the device status word
  and frees its tensor memory; fbc_plan_sync_status reports FBC_ERR_TIMEOUT.  With the default
  restored, the same plan gives the same bits as before the stop.  No wait here is unbounded and
  nothing faults: the stop is the kernel's own bounded give-up.
* Allocation failures: FBC_TEST_FAIL_ALLOC=<name> makes the named device allocation fail on the
  host before cudaMalloc is called.  Every named allocation of plan creation (and of the derived
  tables and staging buffers) then returns FBC_ERR_OOM with a NULL plan and releases what was
  already allocated.
"""

import ctypes
import os

import numpy as np
import pytest

from paper_2105_08798_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ISO = {"kind": "isotropic", "mu": 1.0, "nu": 0.3}


@pytest.fixture(scope="module")
def fbc():
    from paper_2105_08798_gb300 import build, fbc as fbc_mod

    build.build()
    fbc_mod.load()
    assert torch.cuda.is_available()
    return fbc_mod


@pytest.mark.parametrize("prec", ["bf16x2", "tf32", "bf16x3", "bf16x6"])
def test_wait_limit_timeout_then_recovery(fbc, prec):
    xy_i, xy_p = inputs.ring_geometry(200, 300)
    L, R = 16, 16
    f = torch.from_numpy(inputs.forces(R, len(xy_i), L, seed=3)).cuda()
    u = torch.zeros((R, len(xy_p), L, 3), dtype=torch.float64, device="cuda")
    with fbc.Plan(xy_i, xy_p, L, ISO, precision=prec, max_rhs=R) as plan:
        plan.tabulate()
        plan.apply(f, u)
        plan.sync_status()
        ref = u.cpu().numpy()
        plan.set_wait_limit(1)
        u.zero_()
        plan.apply(f, u)
        with pytest.raises(fbc.FBCError) as ei:
            plan.sync_status()
        assert ei.value.status == fbc.FBC_ERR_TIMEOUT
        plan.sync_status()  # the status word was cleared by the report
        plan.set_wait_limit(0)
        u.zero_()
        plan.apply(f, u)
        plan.sync_status()
        got = u.cpu().numpy()
    assert np.array_equal(got, ref)


def test_wait_limit_argument_checks(fbc):
    lib = fbc.load()
    assert lib.fbc_plan_set_wait_limit(None, 0) == fbc.FBC_ERR_INVALID_ARG
    xy_i, xy_p = inputs.ring_geometry(20, 30)
    with fbc.Plan(xy_i, xy_p, 8, ISO, host_only=True) as plan:
        assert lib.fbc_plan_set_wait_limit(plan.handle, -1) == fbc.FBC_ERR_INVALID_ARG
        assert lib.fbc_plan_set_wait_limit(plan.handle, (1 << 24) + 1) == fbc.FBC_ERR_INVALID_ARG
        assert lib.fbc_plan_set_wait_limit(plan.handle, 5) == fbc.FBC_OK
        assert lib.fbc_plan_set_wait_limit(plan.handle, 0) == fbc.FBC_OK


# (allocation name, precision whose plan allocates it)
ALLOCS = [(n, "fp64") for n in ("xy_p", "off_i", "bbox_a", "bbox_b", "perm_i", "perm_p", "used", "twiddles",
                                "table_twiddles", "line_twiddles", "table", "fh", "uh", "partials", "relaxation",
                                "status")] + [
    ("table32", "fp32"), ("table_x2_k0", "fp32"), ("tensor force operand", "bf16x2"), ("uh32", "bf16x2"),
    ("table_x2", "f32x2")]


def _create(fbc, xy_i, xy_p, L, prec, max_rhs):
    g = fbc.fbc_geometry(len(xy_i), len(xy_p), L, 1.0, xy_i.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                         xy_p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    o = fbc.fbc_default_options()
    o.precision = fbc.PRECISIONS[prec]
    o.max_rhs = max_rhs
    h = ctypes.c_void_p(12345)
    st = fbc.load().fbc_plan_create(ctypes.byref(g), ctypes.byref(fbc.material_struct(ISO)), ctypes.byref(o),
                                    ctypes.byref(h))
    return st, h.value


def test_injected_allocation_failures(fbc):
    xy_i, xy_p = inputs.ring_geometry(300, 450)
    xy_i, xy_p = np.ascontiguousarray(xy_i, np.int32), np.ascontiguousarray(xy_p, np.int32)
    L, R = 32, 16
    torch.cuda.synchronize()
    # one plan of each kind first, so that lazily loaded modules do not count as a leak
    for prec in ("fp64", "fp32", "bf16x2", "f32x2"):
        st, h = _create(fbc, xy_i, xy_p, L, prec, R)
        assert st == fbc.FBC_OK
        fbc.fbc_destroy(h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for name, prec in ALLOCS:
            os.environ["FBC_TEST_FAIL_ALLOC"] = name
            st, h = _create(fbc, xy_i, xy_p, L, prec, R)
            msg = fbc.fbc_last_error()
            assert st == fbc.FBC_ERR_OOM, (name, st, msg)
            assert h is None, name
            assert name in msg, (name, msg)
        # the host-apply staging buffers: the call fails, the plan stays usable
        for name in ("stage_f", "stage_u"):
            os.environ.pop("FBC_TEST_FAIL_ALLOC", None)
            with fbc.Plan(xy_i, xy_p, L, ISO, max_rhs=1) as plan:
                plan.tabulate()
                f = inputs.forces(1, len(xy_i), L, seed=1)
                u = np.zeros((1, len(xy_p), L, 3))
                os.environ["FBC_TEST_FAIL_ALLOC"] = name
                with pytest.raises(fbc.FBCError) as ei:
                    plan.apply_host(f, u)
                assert ei.value.status == fbc.FBC_ERR_OOM
                os.environ.pop("FBC_TEST_FAIL_ALLOC", None)
                plan.apply_host(f, u)
                assert np.abs(u).max() > 0
    finally:
        os.environ.pop("FBC_TEST_FAIL_ALLOC", None)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0 - (8 << 20), (free0, free1)
