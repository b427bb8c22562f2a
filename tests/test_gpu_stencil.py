"""Incompatibility force on the device (Sec. 2.3.2, Eq. 21) against the oracle, through the C ABI.

* the synthetic spring model (library blocks) against the oracle's bond-force form;
* arbitrary blocks at all 27 offsets against the block-stencil definition, with the
  degenerate line lengths L = 1, 2, 3 (the plane neighbours q - 1 and q + 1 coincide
  or wrap onto q) and an empty source set;
* the harmonic half of Algorithm 1 for two iterations: f_in from the stencil, the
  relaxed pad update, and the updated pad displacements feeding the next f_in.
"""

import numpy as np
import pytest

from conftest import CUBIC
from oracle import harmonic
from paper_2105_08798_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_I, N_P = 200, 300


@pytest.fixture(scope="module")
def fbc():
    from paper_2105_08798_gb300 import build, fbc as binding

    build.build()
    binding.load()
    return binding


@pytest.fixture(scope="module")
def geom():
    xy_i, xy_p = inputs.ring_geometry(N_I, N_P)
    return inputs.core_sites(N_I), xy_i, xy_p


def _gpu_force(fbc, xy_i, sites, us, L, K):
    with fbc.Stencil(xy_i, sites, L, K) as st:
        f = st.incompat_force([torch.from_numpy(np.ascontiguousarray(u)).cuda() for u in us])
        torch.cuda.synchronize()
    return f.cpu().numpy()


@pytest.mark.parametrize("L,c,R", [(16, 1.0, 3), (8, 1.3, 1)])
def test_spring_model(fbc, geom, L, c, R):
    k1, k2 = 1.7, 0.6
    rng = np.random.default_rng(L + R)
    us = [rng.normal(0, 1, (R, len(xy), L, 3)) for xy in geom]
    ref = harmonic.spring_incompat_force(geom[1], list(zip(geom, us)), L, c, k1, k2)
    got = _gpu_force(fbc, geom[1], list(geom), us, L, fbc.fbc_spring_constants(k1, k2, c))
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("L,R", [(1, 2), (2, 1), (3, 2), (16, 1)])
def test_arbitrary_blocks(fbc, geom, L, R):
    rng = np.random.default_rng(100 + L)
    K = rng.normal(0, 1, (27, 3, 3))
    K[5] = 0.0  # one all-zero block is skipped
    xy_c, xy_i, xy_p = geom
    sites = [xy_c, xy_i, xy_p, np.zeros((0, 2), dtype=np.int32)]
    us = [rng.normal(0, 1, (R, len(xy), L, 3)) for xy in sites]
    ref = harmonic.stencil_apply(xy_i, list(zip(sites, us)), L, K)
    got = _gpu_force(fbc, xy_i, sites, us, L, K)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_two_fbc_iterations(fbc, oracle_mod, geom):
    """u_p <- u_p - alpha G f_in with f_in = L_h^{i+|.}[u] and alpha from Algorithm 2, twice."""
    xy_c, xy_i, xy_p = geom
    L, c, R, k1, k2 = 16, 1.0, 2, 1.0, 0.4
    mat = dict(CUBIC, C11=k1 + 2 * k2, C12=k2, C44=k2)  # the spring model's long-wave medium
    rng = np.random.default_rng(9)
    u_atoms = [0.05 * rng.normal(0, 1, (R, len(xy_c), L, 3)) for _ in range(2)]  # two atomistic solves
    u_int = 0.05 * rng.normal(0, 1, (R, len(xy_i), L, 3))
    u_pad0 = 0.05 * rng.normal(0, 1, (R, len(xy_p), L, 3))
    du_max = 0.02
    # oracle
    u_pad, alpha, f_prev = u_pad0.copy(), np.ones(R), None
    for it in range(2):
        f = harmonic.spring_incompat_force(xy_i, [(xy_c, u_atoms[it]), (xy_i, u_int), (xy_p, u_pad)], L, c, k1, k2)
        u_pad, alpha = oracle_mod.relaxed_update(xy_i, xy_p, L, c, mat, f, f_prev, u_pad, alpha, du_max=du_max,
                                                 zero_mean_u=True)
        f_prev = f
    # device
    K = fbc.fbc_spring_constants(k1, k2, c)
    with fbc.Plan(xy_i, xy_p, L, mat, c=c, precision="fp64", max_rhs=R) as plan, \
            fbc.Stencil(xy_i, [xy_c, xy_i, xy_p], L, K) as st:
        plan.tabulate()
        ua = [torch.from_numpy(u).cuda() for u in u_atoms]
        ui = torch.from_numpy(u_int).cuda()
        up = torch.from_numpy(u_pad0.copy()).cuda()
        a = torch.ones(R, dtype=torch.float64, device="cuda")
        fs = [torch.empty((R, N_I, L, 3), dtype=torch.float64, device="cuda") for _ in range(2)]
        for it in range(2):
            st.incompat_force([ua[it], ui, up], f=fs[it])
            plan.apply_relaxed(fs[it], fs[it - 1] if it else None, up, a, du_max=du_max, zero_mean=True)
        torch.cuda.synchronize()
        plan.sync_status()
        got_u, got_a = up.cpu().numpy(), a.cpu().numpy()
    np.testing.assert_allclose(got_a, alpha, rtol=1e-12)
    assert np.linalg.norm(got_u - u_pad) <= 1e-12 * np.linalg.norm(u_pad)
