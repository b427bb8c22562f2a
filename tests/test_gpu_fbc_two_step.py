"""The FBC iteration on the device converges in two steps when the atomistic model is the harmonic
one (Sec. 2.3.1, Remark 1): interface sites inside the pad (FBC_PLAN_SELF_TERMS), a table that is
the lattice Green function of the spring model throughout (fbc_plan_lattice_near_field, no
blending constant), the incompatibility force from the stencil (fbc_incompat_force) and the pad
update u_p <- u_p - G f_in (fbc_apply).  The atomistic problem itself is solved on the host (the
set-up, the exact solution and the solver are those of the oracle-level test).
"""

import numpy as np
import pytest

from oracle import harmonic
from test_oracle_fbc_two_step import L, N_ZONE, atomistic_solve, fbc_geometry

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAT = {"kind": "cubic", "C11": 1.8, "C12": 0.4, "C44": 0.4}  # the spring model's long-wave medium


@pytest.fixture(scope="module")
def fbc():
    from paper_2105_08798_gb300 import build, fbc as binding

    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("prec", ["fp64", "fft64"])
def test_two_step_convergence_on_device(fbc, oracle_mod, prec):
    K = fbc.fbc_spring_constants(1.0, 0.4, 1.0)  # the device's blocks
    Kb = harmonic.spring_blocks(1.0, 0.4, 1.0)  # the oracle's blocks: exact solution and atomistic model
    atoms, ip, pad = fbc_geometry()
    x0 = (0, 0)
    fext = np.zeros((len(atoms), L, 3))
    fext[atoms.index(x0), :, 0] = np.cos(2 * np.pi * np.arange(L) / L)
    need = sorted({(p[0] - q[0], p[1] - q[1]) for p in atoms + pad for q in [x0]})
    g = harmonic.lattice_mode_table(Kb, L, need, list(range(L // 2 + 1)), N_ZONE)
    gk = {d: g[i] for i, d in enumerate(need)}
    # the exact solution u* = G_lat f_ext: the real-space sum with the lattice Green function in real space
    exact = oracle_mod.real_space_update(np.array([x0]), np.array(atoms + pad), L, fext[None, [atoms.index(x0)]],
                                         lambda dl: harmonic.lattice_kernel_table(Kb, L, dl, N_ZONE),
                                         project=False)[0]
    cross = oracle_mod.mode_space_update(np.array([x0]), np.array(atoms + pad), L,
                                         fext[None, [atoms.index(x0)]], lambda d: gk[d], project=False)[0]
    assert np.linalg.norm(cross - exact) <= 1e-13 * np.linalg.norm(exact)
    ua_star = exact[:len(atoms)]
    with fbc.Plan(np.array(ip), np.array(pad), L, MAT, precision=prec, self_terms=True) as plan, \
            fbc.Stencil(np.array(ip), [np.array(atoms), np.array(pad)], L, K) as st:
        plan.tabulate()
        up = torch.zeros((1, len(pad), L, 3), dtype=torch.float64, device="cuda")
        fin = torch.zeros((1, len(ip), L, 3), dtype=torch.float64, device="cuda")
        with pytest.raises(fbc.FBCError):
            plan.apply(fin, up)  # the self-terms are not in the table yet
        plan.lattice_near_field(K, 1e3, (0, 0), N_ZONE)  # the lattice Green function throughout
        errs = []
        for _ in range(3):
            ua = atomistic_solve(Kb, atoms, pad, up[0].cpu().numpy(), fext)
            errs.append(np.linalg.norm(ua - ua_star) / np.linalg.norm(ua_star))
            st.incompat_force([torch.from_numpy(ua[None]).cuda(), up], f=fin)
            plan.apply(fin, up, alpha=-1.0, beta=1.0, project=False)
        torch.cuda.synchronize()
        plan.sync_status()
    assert errs[0] > 1e-3
    assert errs[1] <= 1e-12 and errs[2] <= 1e-12, errs
