"""Host-side checks of the C ABI (no GPU needed).

* ``build()`` cross-compiles the library for sm_103a and it loads;
* every entry point declared in ``include/fbc.h`` is exported;
* the ctypes structures have the C layout (sizes and offsets, checked against
  a C program compiled from the header);
* argument validation rejects bad input before any device work.
"""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2105_08798_gb300 import build as fbc_build
from paper_2105_08798_gb300 import fbc, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fbc.h")


@pytest.fixture(scope="module")
def lib():
    fbc_build.build()
    return fbc.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fbc_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fbc_plan_create", "fbc_tabulate_kernel", "fbc_apply", "fbc_destroy", "fbc_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert fbc.fbc_version().startswith("fbc-gb300")


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "fbc.h"
#define P(T, f) printf("%s.%s %zu\n", #T, #f, offsetof(T, f));
int main(void) {
  printf("fbc_geometry %zu\nfbc_material %zu\nfbc_options %zu\nfbc_plan_info %zu\nfbc_batch_info %zu\n",
         sizeof(fbc_geometry), sizeof(fbc_material), sizeof(fbc_options), sizeof(fbc_plan_info),
         sizeof(fbc_batch_info));
  printf("fbc_hmat_options %zu\nfbc_hmat_info %zu\n", sizeof(fbc_hmat_options), sizeof(fbc_hmat_info));
  P(fbc_hmat_options, b_min) P(fbc_hmat_options, scratch_bytes)
  P(fbc_hmat_info, rank_max) P(fbc_hmat_info, factor_bytes) P(fbc_hmat_info, n_waves) P(fbc_hmat_info, build_ms)
  P(fbc_batch_info, smem_contract) P(fbc_batch_info, pair_modes) P(fbc_batch_info, rhs_per_cta)
  P(fbc_geometry, c) P(fbc_geometry, xy_i) P(fbc_geometry, xy_p)
  P(fbc_material, mu) P(fbc_material, C44) P(fbc_material, Q)
  P(fbc_options, max_rhs) P(fbc_options, flags)
  P(fbc_plan_info, pair_modes_per_rhs) P(fbc_plan_info, table_bytes) P(fbc_plan_info, workspace_bytes)
  P(fbc_plan_info, fft_mx) P(fbc_plan_info, fft_chunk_items) P(fbc_plan_info, reserved2)
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["cc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    vals = dict(line.split() for line in out if line.strip())
    assert int(vals["fbc_geometry"]) == ctypes.sizeof(fbc.fbc_geometry)
    assert int(vals["fbc_material"]) == ctypes.sizeof(fbc.fbc_material)
    assert int(vals["fbc_options"]) == ctypes.sizeof(fbc.fbc_options)
    assert int(vals["fbc_plan_info"]) == ctypes.sizeof(fbc.fbc_plan_info)
    assert int(vals["fbc_batch_info"]) == ctypes.sizeof(fbc.fbc_batch_info)
    assert int(vals["fbc_hmat_options"]) == ctypes.sizeof(fbc.fbc_hmat_options)
    assert int(vals["fbc_hmat_info"]) == ctypes.sizeof(fbc.fbc_hmat_info)
    for key, v in vals.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(getattr(fbc, t), f).offset == int(v), key


def test_default_options(lib):
    o = fbc.fbc_default_options()
    assert (o.precision, o.rich_n, o.rich_N, o.quad, o.max_rhs, o.flags) == (0, 4, 6, 64, 1, 0)


def _try_create(xy_i, xy_p, L, material, **kw):
    with pytest.raises(fbc.FBCError) as ei:
        fbc.Plan(xy_i, xy_p, L, material, **kw)
    return ei.value.status


ISO = {"kind": "isotropic", "mu": 1.0, "nu": 0.3}


def test_validation_rejects_bad_input(lib):
    xy_i, xy_p = inputs.ring_geometry(20, 30)
    assert _try_create(xy_i, xy_p, 12, ISO) == fbc.FBC_ERR_INVALID_ARG  # L not a power of two
    assert _try_create(xy_i, xy_p, 8192, ISO) == fbc.FBC_ERR_INVALID_ARG
    dup = np.concatenate([xy_i, xy_i[:1]])
    assert _try_create(dup, xy_p, 16, ISO) == fbc.FBC_ERR_INVALID_ARG  # duplicate site
    clash = np.concatenate([xy_i, xy_p[:1]])
    assert _try_create(clash, xy_p, 16, ISO) == fbc.FBC_ERR_INVALID_ARG  # d = 0
    assert _try_create(xy_i, xy_p, 16, {"kind": "isotropic", "mu": 1.0, "nu": 0.5}) == fbc.FBC_ERR_INVALID_ARG
    assert _try_create(xy_i, xy_p, 16, {"kind": "cubic", "C11": 1.0, "C12": 1.5, "C44": 0.9}) == \
        fbc.FBC_ERR_INVALID_ARG  # unstable
    tilt = np.array([[1, 0, 0], [0, np.cos(0.3), -np.sin(0.3)], [0, np.sin(0.3), np.cos(0.3)]])
    assert _try_create(xy_i, xy_p, 16, {"kind": "cubic", "C11": 1.5, "C12": 1.0, "C44": 0.9, "Q": tilt}) == \
        fbc.FBC_ERR_UNSUPPORTED
    assert _try_create(xy_i, xy_p, 16, ISO, max_rhs=0) == fbc.FBC_ERR_INVALID_ARG
    assert _try_create(xy_i, xy_p, 16, ISO, rich_n=0) == fbc.FBC_ERR_INVALID_ARG
    assert _try_create(xy_i, xy_p, 16, ISO, precision=fbc.FBC_PREC_BF16X6 + 1) == fbc.FBC_ERR_INVALID_ARG
    assert "power of two" in fbc.fbc_last_error() or fbc.fbc_last_error() != ""


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.fbc_plan_create(None, None, None, ctypes.byref(h)) == fbc.FBC_ERR_INVALID_ARG
    assert h.value is None
    assert lib.fbc_apply(None, None, None, 1, 1.0, 0.0, 0, None) == fbc.FBC_ERR_INVALID_ARG
    assert lib.fbc_tabulate_kernel(None, None) == fbc.FBC_ERR_INVALID_ARG
    lib.fbc_destroy(None)


def test_new_entry_points_validate_before_device_work(lib):
    """Relaxed apply, stencil and lattice near field: NULL handles, host-only plans and bad scalars are
    rejected with a status and a message, without any device work (no GPU here)."""
    assert lib.fbc_apply_relaxed(None, None, None, None, 1, None, 0.0, 0, None) == fbc.FBC_ERR_INVALID_ARG
    assert lib.fbc_incompat_force(None, None, None, 1, None) == fbc.FBC_ERR_INVALID_ARG
    assert lib.fbc_stencil_destroy(None) == fbc.FBC_OK
    K = (ctypes.c_double * 243)()
    assert lib.fbc_spring_constants(1.0, 0.4, 0.0, K) == fbc.FBC_ERR_INVALID_ARG  # c must be > 0
    assert lib.fbc_spring_constants(1.0, 0.4, 1.0, None) == fbc.FBC_ERR_INVALID_ARG
    assert lib.fbc_plan_lattice_near_field(None, K, 5.0, 12, 0, 64) == fbc.FBC_ERR_INVALID_ARG
    xy_i, xy_p = inputs.ring_geometry(20, 30)
    with fbc.Plan(xy_i, xy_p, 8, {"kind": "isotropic", "mu": 1.0, "nu": 0.3}, host_only=True) as plan:
        with pytest.raises(fbc.FBCError, match="host-only"):
            fbc.fbc_apply_relaxed(plan.handle, 1, None, 2, 1, 3, 0.0, 0, None)
        with pytest.raises(fbc.FBCError, match="host-only"):
            fbc.fbc_plan_lattice_near_field(plan.handle, fbc.fbc_spring_constants(1.0, 0.4, 1.0), 5.0, (12, 0), 64)
    # interface sites inside the pad: accepted only with the self-terms flag
    pad = np.concatenate([xy_i[:5], xy_p])
    with fbc.Plan(xy_i, pad, 8, {"kind": "isotropic", "mu": 1.0, "nu": 0.3}, host_only=True, self_terms=True):
        pass
    with pytest.raises(fbc.FBCError, match="coincides"):
        fbc.Plan(xy_i, pad, 8, {"kind": "isotropic", "mu": 1.0, "nu": 0.3}, host_only=True)


def test_hmat_entry_points_validate_before_device_work(lib):
    """H-matrix: bad options, NULL handles and host-only plans are rejected without device work."""
    h = ctypes.c_void_p()
    bad = [fbc.fbc_hmat_options(1e-7, 2.0, 20, 0, 0), fbc.fbc_hmat_options(1e-5, 0.0, 20, 0, 0),
           fbc.fbc_hmat_options(1e-5, 2.0, 0, 0, 0), fbc.fbc_hmat_options(1e-5, 2.0, 20, 7000, 0),
           fbc.fbc_hmat_options(1e-5, 2.0, 20, 0, -1)]
    for opt in bad:
        assert lib.fbc_hmat_create(None, ctypes.byref(opt), None, ctypes.byref(h)) == fbc.FBC_ERR_INVALID_ARG
        assert h.value is None
    assert lib.fbc_hmat_create(None, None, None, ctypes.byref(h)) == fbc.FBC_ERR_INVALID_ARG
    assert lib.fbc_measure_fma_peak(0, None, None) == fbc.FBC_ERR_INVALID_ARG
    assert lib.fbc_hmat_apply(None, None, None, 1, 1.0, 0.0, 0, None) == fbc.FBC_ERR_INVALID_ARG
    assert lib.fbc_hmat_get_info(None, None) == fbc.FBC_ERR_INVALID_ARG
    lib.fbc_hmat_destroy(None)
    xy_i, xy_p = inputs.ring_geometry(20, 30)
    with fbc.Plan(xy_i, xy_p, 8, {"kind": "isotropic", "mu": 1.0, "nu": 0.3}, host_only=True) as plan:
        with pytest.raises(fbc.FBCError, match="host-only"):
            fbc.fbc_hmat_create(plan.handle, 1e-5, 2.0, 20, 0, 0)
    n = ctypes.c_int64(0)
    xi = np.ascontiguousarray(xy_i, dtype=np.int32)
    xp = np.ascontiguousarray(xy_p, dtype=np.int32)
    i32 = ctypes.POINTER(ctypes.c_int32)
    assert lib.fbc_hmat_partition(xi.ctypes.data_as(i32), len(xi), xp.ctypes.data_as(i32), len(xp), 8, 1.0, 2.0, 0,
                                  ctypes.byref(n), None, 0, None, None) == fbc.FBC_ERR_INVALID_ARG
    assert lib.fbc_hmat_partition(xi.ctypes.data_as(i32), len(xi), xp.ctypes.data_as(i32), len(xp), 8, 1.0, 2.0, 20,
                                  ctypes.byref(n), None, 0, None, None) == fbc.FBC_OK
    blk = (ctypes.c_int64 * 5)()
    if n.value > 1:
        assert lib.fbc_hmat_partition(xi.ctypes.data_as(i32), len(xi), xp.ctypes.data_as(i32), len(xp), 8, 1.0, 2.0, 20,
                                      ctypes.byref(n), blk, 1, None, None) == fbc.FBC_ERR_INVALID_ARG
