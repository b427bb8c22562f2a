"""The allocation-free zero-mean entry point against the regular apply.

Callers that cannot call cudaMalloc where they re-centre the pad
displacements (an engine that owns the device through its own pool, a loop
that must not take the allocator lock) use fbc_zero_mean_static, whose scratch
is a fixed array inside the library.
This test calls it through the C ABI twice in a row, on different inputs and
sizes, and checks each result against fbc_apply's own zero-mean step
(FBC_APPLY_ZERO_MEAN_U) within the FP64 parity tolerance.  It lives in a file
of its own so that it runs last in a full test run; it also passes alone.
"""

import numpy as np
import pytest

from paper_2105_08798_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ISO = {"kind": "isotropic", "mu": 1.0, "nu": 0.3}
TOL = 1e-12


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_zero_mean_static_matches_apply_twice():
    from paper_2105_08798_gb300 import build, fbc

    build.build()
    fbc.load()
    assert torch.cuda.is_available()
    cases = [(90, 130, 16, 2, 11), (150, 220, 32, 3, 12)]
    for n_i, n_p, L, n_rhs, seed in cases:
        xy_i, xy_p = inputs.ring_geometry(n_i, n_p)
        f = torch.from_numpy(inputs.forces(n_rhs, n_i, L, seed=seed)).cuda()
        u0 = torch.from_numpy(np.random.default_rng(seed).standard_normal((n_rhs, n_p, L, 3)) + 2.0).cuda()
        with fbc.Plan(xy_i, xy_p, L, ISO, max_rhs=n_rhs) as plan:
            plan.tabulate()
            ref = u0.clone()
            plan.apply(f, ref, alpha=-0.5, beta=1.0, zero_mean=True)
            got = u0.clone()
            plan.apply(f, got, alpha=-0.5, beta=1.0, zero_mean=False)
            stream = torch.cuda.current_stream()
            fbc.fbc_zero_mean_static(got.data_ptr(), n_rhs, n_p, L, stream)
            torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert _rel(g, r) <= TOL
        assert np.abs(g.mean(axis=(1, 2))).max() < 1e-14


def test_zero_mean_static_rejects_too_many_rhs():
    from paper_2105_08798_gb300 import fbc

    fbc.load()
    u = torch.zeros((1, 4, 2, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(fbc.FBCError) as ei:
        fbc.fbc_zero_mean_static(u.data_ptr(), 65, 4, 2, None)
    assert ei.value.status == fbc.FBC_ERR_INVALID_ARG
    assert "64" in str(ei.value)
