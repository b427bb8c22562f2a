"""Lattice Green function near field (App.) through the C ABI, against the oracle.

The plan's table entries with |d| <= r_cut become the lattice Green function of the synthetic
spring model, computed on the GPU by 2D FFTs over the zone grid; the oracle computes the same
zone sums directly.  The k = 0 mode is shifted by the blending constant at the reference
difference.  Checked: the near entries (1e-12), the far entries unchanged (bit for bit), the
update with the modified table against the oracle's real-space sum with the blended real-space
kernel (1e-12; the oracle's mode-space form as a cross-check), the double-float and in-plane FFT
forms on the same plan, and the argument checks.
"""

import numpy as np
import pytest

from oracle import harmonic
from paper_2105_08798_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K1, K2 = 1.0, 0.4
MAT = {"kind": "cubic", "C11": K1 + 2 * K2, "C12": K2, "C44": K2}  # the spring model's long-wave medium
N_I, N_P, L, N_ZONE, R_CUT, R_REF = 120, 180, 16, 64, 5.0, 10.0


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def six(g):
    """complex [..., 3, 3] -> the six-real layout [Re g11, Re g12, Re g22, Re g33, Im g13, Im g23]"""
    return np.stack([g[..., 0, 0].real, g[..., 0, 1].real, g[..., 1, 1].real, g[..., 2, 2].real,
                     g[..., 0, 2].imag, g[..., 1, 2].imag], axis=-1)


def from_six(v):
    a11, a12, a22, a33, b13, b23 = (v[..., i] for i in range(6))
    g = np.zeros(v.shape[:-1] + (3, 3), dtype=np.complex128)
    g[..., 0, 0], g[..., 0, 1], g[..., 1, 0], g[..., 1, 1], g[..., 2, 2] = a11, a12, a12, a22, a33
    g[..., 0, 2] = g[..., 2, 0] = 1j * b13
    g[..., 1, 2] = g[..., 2, 1] = 1j * b23
    return g


@pytest.fixture(scope="module")
def fbc():
    from paper_2105_08798_gb300 import build, fbc as binding

    build.build()
    binding.load()
    return binding


@pytest.fixture(scope="module")
def geom():
    xy_i, xy_p = inputs.ring_geometry(N_I, N_P)
    d = np.unique((xy_p[:, None, :] - xy_i[None, :, :]).reshape(-1, 2), axis=0)
    r = np.hypot(d[:, 0], d[:, 1])
    near = d[r <= R_CUT]
    far = d[r > R_CUT]
    ref = far[np.argmin(np.abs(np.hypot(far[:, 0], far[:, 1]) - R_REF))]
    return xy_i, xy_p, d, near, far, ref


def check_near_entries(got, lat, before_ref_k0):
    """got, lat: [n_near + 1 (the reference last for lat)][K][6].  Modes k >= 1 equal the oracle's zone
    sums; the k = 0 entries differ from them by one common constant, C = lat(d_ref) - table(d_ref)."""
    lat_near = lat[:-1]
    scale = np.abs(lat_near).max()
    assert np.abs(got[:, 1:] - lat_near[:, 1:]).max() <= 1e-12 * scale
    shift = lat_near[:, 0] - got[:, 0]  # [n_near][6]
    assert np.abs(shift - shift[0]).max() <= 1e-12 * scale  # one constant for every near difference
    assert np.abs(shift[0] - (lat[-1, 0] - before_ref_k0)).max() <= 1e-12 * scale


def test_near_entries_and_far_entries(fbc, geom):
    xy_i, xy_p, d, near, far, ref = geom
    K = fbc.fbc_spring_constants(K1, K2, 1.0)
    K_modes = L // 2 + 1
    with fbc.Plan(xy_i, xy_p, L, MAT) as plan:
        plan.tabulate()
        before = plan.mode_table(d)
        plan.lattice_near_field(K, R_CUT, ref, N_ZONE)
        after = plan.mode_table(d)
    idx = {tuple(x): i for i, x in enumerate(d.tolist())}
    Ko = harmonic.spring_blocks(K1, K2, 1.0)  # the oracle's own blocks
    lat = six(harmonic.lattice_mode_table(Ko, L, np.vstack([near, ref[None]]), list(range(K_modes)), N_ZONE))
    got = np.array([after[idx[tuple(x)]] for x in near.tolist()])
    assert len(near) > 0
    check_near_entries(got, lat, before[idx[tuple(ref)], 0])
    fi = [idx[tuple(x)] for x in far.tolist()]
    np.testing.assert_array_equal(after[fi], before[fi])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("f32x2", 1e-12), ("fft64", 1e-12), ("fft32", 1e-5)])
def test_update_with_near_field(fbc, oracle_mod, geom, prec, tol):
    xy_i, xy_p, d, near, far, ref = geom
    K = fbc.fbc_spring_constants(K1, K2, 1.0)
    f = inputs.forces(1, N_I, L, seed=31)
    with fbc.Plan(xy_i, xy_p, L, MAT, precision=prec) as plan:
        plan.tabulate()
        table = plan.mode_table(d)  # continuum
        plan.lattice_near_field(K, R_CUT, ref, N_ZONE)
        table_near = plan.mode_table(near)
        u = torch.full((1, N_P, L, 3), float("nan"), dtype=torch.float64, device="cuda")
        plan.apply(torch.from_numpy(f).cuda(), u)
        torch.cuda.synchronize()
        plan.sync_status()
        got = u.cpu().numpy()
    # the oracle's table: its own continuum modes, near entries from its own zone sums
    K_modes = L // 2 + 1
    cont = oracle_mod.mode_table(oracle_mod.kernel_table(MAT, L, 1.0, d))
    idx = {tuple(x): i for i, x in enumerate(d.tolist())}
    Ko = harmonic.spring_blocks(K1, K2, 1.0)  # the oracle's own blocks
    lat = harmonic.lattice_mode_table(Ko, L, np.vstack([near, ref[None]]), list(range(K_modes)), N_ZONE)
    C = lat[-1, 0] - cont[idx[tuple(ref)], 0]
    gk = {tuple(x): cont[i] for i, x in enumerate(d.tolist())}
    for j, x in enumerate(near.tolist()):
        g = lat[j].copy()
        g[0] -= C
        gk[tuple(x)] = g
    # the real-space oracle: the continuum kernel G~(d, s) beyond r_cut, the lattice Green function in real
    # space (plain inverse DFT of the zone sums along the line) within, shifted by the blending constant
    # (C in the k = 0 mode is C / L at every repeat s); then the plain double sum over (b, q)
    near_set = {tuple(x) for x in near.tolist()}
    lat_rs = harmonic.lattice_kernel_table(Ko, L, np.vstack([near, ref[None]]), N_ZONE)
    lat_at = {tuple(x): lat_rs[j] for j, x in enumerate(near.tolist())}

    def blended(d_list):
        cont_rs = oracle_mod.kernel_table(MAT, L, 1.0, d_list)
        iref = [j for j, x in enumerate(d_list.tolist()) if tuple(x) == tuple(ref)]
        C_rs = lat_rs[-1].sum(axis=0) - (cont_rs[iref[0]].sum(axis=0) if iref else
                                         oracle_mod.kernel_table(MAT, L, 1.0, ref[None])[0].sum(axis=0))
        for j, x in enumerate(d_list.tolist()):
            if tuple(x) in near_set:
                cont_rs[j] = lat_at[tuple(x)] - C_rs / L
        return cont_rs

    ref_real = oracle_mod.real_space_update(xy_i, xy_p, L, f, blended)
    assert rel_l2(got, ref_real) <= tol, (prec, rel_l2(got, ref_real))
    # cross-check: the oracle's mode-by-mode form of the same update
    ref_modes = oracle_mod.mode_space_update(xy_i, xy_p, L, f, lambda dd: gk[dd])
    assert rel_l2(ref_modes, ref_real) <= 1e-13
    assert np.abs(from_six(table_near)).max() > 0  # the near field is in use


def test_argument_checks(fbc, geom):
    xy_i, xy_p, d, near, far, ref = geom
    K = fbc.fbc_spring_constants(K1, K2, 1.0)
    with fbc.Plan(xy_i, xy_p, L, MAT) as plan:
        with pytest.raises(fbc.FBCError):
            plan.lattice_near_field(K, R_CUT, ref, N_ZONE)  # not tabulated
        plan.tabulate()
        with pytest.raises(fbc.FBCError):
            plan.lattice_near_field(K, R_CUT, near[0], N_ZONE)  # reference inside the cut-off
        bad = K.copy()
        bad[1, 0, 2] += 0.1  # breaks K(-n) = K(n) and the mirror symmetry
        with pytest.raises(fbc.FBCError):
            plan.lattice_near_field(bad, R_CUT, ref, N_ZONE)
        # K(-n) = K(n) and the mirror symmetry hold, but the blocks of n = (+-1, 0, 0) are not symmetric
        skew = K.copy()
        skew[22, 0, 1] += 0.1
        skew[4, 0, 1] += 0.1
        with pytest.raises(fbc.FBCError, match="symmetric"):
            plan.lattice_near_field(skew, R_CUT, ref, N_ZONE)
        with pytest.raises(fbc.FBCError):
            plan.lattice_near_field(K, R_CUT, ref, 16)  # zone grid too small for the reference
        with pytest.raises(fbc.FBCError):
            plan.lattice_near_field(K, R_CUT, (1000, 0), N_ZONE)  # not a difference of the table
