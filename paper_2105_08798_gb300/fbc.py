"""Thin ctypes binding of ``libfbc.so`` (the C ABI declared in ``include/fbc.h``).

Every entry point of the header has a function of the same name here that
only marshals arguments (structures, raw device pointers, the CUDA stream
handle) and turns a non-zero status into ``FBCError``.  All arithmetic runs in
the library's CUDA kernels; there is no CPU fallback: ``load()`` raises if the
library is missing, and every call raises if it fails.

``Plan`` is a convenience wrapper over the same calls that accepts torch
tensors (device memory, ``data_ptr``) and numpy arrays (host memory).
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfbc.so")

FBC_OK = 0
FBC_ERR_INVALID_ARG = 1
FBC_ERR_OOM = 2
FBC_ERR_CUDA = 3
FBC_ERR_NOT_TABULATED = 4
FBC_ERR_TIMEOUT = 5
FBC_ERR_UNSUPPORTED = 6

FBC_MATERIAL_ISOTROPIC = 0
FBC_MATERIAL_CUBIC = 1

FBC_PREC_FP64 = 0
FBC_PREC_FP32 = 1
FBC_PREC_F32X2 = 2
FBC_PREC_TF32 = 3
FBC_PREC_BF16X2 = 4
FBC_PREC_BF16X3 = 5
FBC_PREC_FFT64 = 6
FBC_PREC_FFT32 = 7
FBC_PREC_BF16X6 = 8
PRECISIONS = {"fp64": FBC_PREC_FP64, "fp32": FBC_PREC_FP32, "f32x2": FBC_PREC_F32X2, "tf32": FBC_PREC_TF32,
              "bf16x2": FBC_PREC_BF16X2, "bf16x3": FBC_PREC_BF16X3, "fft64": FBC_PREC_FFT64,
              "fft32": FBC_PREC_FFT32, "bf16x6": FBC_PREC_BF16X6}

FBC_PLAN_HOST_ONLY = 1
FBC_PLAN_SELF_TERMS = 4
FBC_PLAN_TC_FAST_ACCUMULATE = 2

FBC_APPLY_PROJECT_NEUTRAL = 1
FBC_APPLY_ZERO_MEAN_U = 2
FBC_APPLY_NO_GRAPH = 4


class FBCError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where} failed with status {status}: {message}")
        self.status = status


class fbc_geometry(ctypes.Structure):
    _fields_ = [("n_i", ctypes.c_int32), ("n_p", ctypes.c_int32), ("L", ctypes.c_int32), ("c", ctypes.c_double),
                ("xy_i", ctypes.POINTER(ctypes.c_int32)), ("xy_p", ctypes.POINTER(ctypes.c_int32))]


class fbc_material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("mu", ctypes.c_double), ("nu", ctypes.c_double),
                ("C11", ctypes.c_double), ("C12", ctypes.c_double), ("C44", ctypes.c_double),
                ("Q", ctypes.c_double * 9)]


class fbc_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("rich_n", ctypes.c_int32), ("rich_N", ctypes.c_int32),
                ("quad", ctypes.c_int32), ("max_rhs", ctypes.c_int32), ("flags", ctypes.c_int32)]


class fbc_plan_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("n_i", "n_p", "L", "K", "max_rhs", "precision", "tile_a", "tile_b",
                                              "n_tiles_a", "n_tiles_b", "box_x0", "box_y0", "box_nx", "box_ny",
                                              "sub_w", "sub_h", "n_used_d", "tabulated")] + [
        ("pair_modes_per_rhs", ctypes.c_double), ("table_bytes", ctypes.c_size_t),
        ("workspace_bytes", ctypes.c_size_t), ("surrogate_bytes", ctypes.c_size_t),
        ("surrogate_attached", ctypes.c_int32), ("n_far_d", ctypes.c_int32), ("surrogate_chunk", ctypes.c_int32),
        ("reserved", ctypes.c_int32)] + [(n, ctypes.c_int32) for n in ("fft_mx", "fft_my", "fft_rows_i", "fft_rows_p",
                                                                     "fft_chunk_items", "reserved2")]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class fbc_batch_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("n_plans", "precision", "n_contract_items", "grid", "occupancy",
                                              "lpt_order", "kernel_launches")] + [
        ("smem_contract", ctypes.c_size_t), ("pair_modes", ctypes.c_double), ("rhs_per_cta", ctypes.c_int32),
        ("launch_form", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class fbc_hmat_options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("gamma", ctypes.c_double), ("b_min", ctypes.c_int32),
                ("max_rank", ctypes.c_int32), ("scratch_bytes", ctypes.c_int64)]


class fbc_hmat_info(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("n_lowrank", ctypes.c_int64),
                ("n_dense", ctypes.c_int64), ("rank_sum", ctypes.c_int64), ("rank_max", ctypes.c_int32),
                ("n_capped", ctypes.c_int32), ("factor_bytes", ctypes.c_int64), ("dense_bytes", ctypes.c_int64),
                ("n_row_leaves", ctypes.c_int32), ("n_col_leaves", ctypes.c_int32), ("n_waves", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("build_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


_lock = threading.Lock()
_lib = None

_P = ctypes.POINTER
_vp = ctypes.c_void_p
_SIGNATURES = {
    "fbc_default_options": (None, [_P(fbc_options)]),
    "fbc_plan_create": (ctypes.c_int, [_P(fbc_geometry), _P(fbc_material), _P(fbc_options), _P(_vp)]),
    "fbc_tabulate_kernel": (ctypes.c_int, [_vp, _vp]),
    "fbc_apply": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_uint32,
                                 _vp]),
    "fbc_apply_host": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_uint32, _vp]),
    "fbc_apply_relaxed": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int32, _vp, ctypes.c_double, ctypes.c_uint32,
                                         _vp]),
    "fbc_plan_set_precision": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "fbc_plan_info_get": (ctypes.c_int, [_vp, _P(fbc_plan_info)]),
    "fbc_get_mode_table": (ctypes.c_int, [_vp, _P(ctypes.c_int32), ctypes.c_int32, _P(ctypes.c_double)]),
    "fbc_plan_layout": (ctypes.c_int, [_vp, _P(ctypes.c_int32), _P(ctypes.c_int32), _P(ctypes.c_int32),
                                       _P(ctypes.c_int32)]),
    "fbc_plan_sync_status": (ctypes.c_int, [_vp, _vp]),
    "fbc_plan_set_timing": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "fbc_plan_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "fbc_plan_stage_times": (ctypes.c_int, [_vp, _P(ctypes.c_float)]),
    "fbc_destroy": (None, [_vp]),
    "fbc_last_error": (ctypes.c_char_p, []),
    "fbc_version": (ctypes.c_char_p, []),
    "fbc_zero_mean_static": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp]),
    "fbc_spring_constants": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, _P(ctypes.c_double)]),
    "fbc_stencil_create": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_int32), ctypes.c_int32, _P(_P(ctypes.c_int32)),
                                          _P(ctypes.c_int32), ctypes.c_int32, _P(ctypes.c_double), _P(_vp)]),
    "fbc_incompat_force": (ctypes.c_int, [_vp, _P(_vp), _vp, ctypes.c_int32, _vp]),
    "fbc_stencil_destroy": (ctypes.c_int, [_vp]),
    "fbc_plan_lattice_near_field": (ctypes.c_int, [_vp, _P(ctypes.c_double), ctypes.c_double, ctypes.c_int32,
                                                   ctypes.c_int32, ctypes.c_int32]),
    "fbc_batch_create": (ctypes.c_int, [_P(_vp), ctypes.c_int32, _P(_vp), _P(_vp), _P(ctypes.c_int32), _P(_vp)]),
    "fbc_batch_apply": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_uint32, _vp]),
    "fbc_batch_autotune": (ctypes.c_int, [_vp, _vp, _P(ctypes.c_double)]),
    "fbc_batch_info_get": (ctypes.c_int, [_vp, _P(fbc_batch_info)]),
    "fbc_batch_destroy": (None, [_vp]),
    "fbc_surrogate_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint64, _P(_vp)]),
    "fbc_surrogate_n_params": (ctypes.c_int, [_vp]),
    "fbc_surrogate_params": (ctypes.c_int, [_vp, _vp, _vp]),
    "fbc_surrogate_forward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp]),
    "fbc_surrogate_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, _P(ctypes.c_double), _vp, _vp]),
    "fbc_surrogate_train": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_uint64, _vp, _P(ctypes.c_double)]),
    "fbc_surrogate_eval_table": (ctypes.c_int, [_vp, _vp, _P(ctypes.c_int32), _P(ctypes.c_int32), ctypes.c_int32,
                                                _P(ctypes.c_double)]),
    "fbc_plan_attach_surrogate": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_int32]),
    "fbc_surrogate_sync_status": (ctypes.c_int, [_vp, _vp]),
    "fbc_surrogate_destroy": (None, [_vp]),
    "fbc_hmat_partition": (ctypes.c_int, [_P(ctypes.c_int32), ctypes.c_int32, _P(ctypes.c_int32), ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                          _P(ctypes.c_int64), _P(ctypes.c_int64), ctypes.c_int64, _P(ctypes.c_int64),
                                          _P(ctypes.c_int64)]),
    "fbc_hmat_create": (ctypes.c_int, [_vp, _P(fbc_hmat_options), _vp, _P(_vp)]),
    "fbc_hmat_apply": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_uint32, _vp]),
    "fbc_hmat_get_info": (ctypes.c_int, [_vp, _P(fbc_hmat_info)]),
    "fbc_hmat_blocks": (ctypes.c_int, [_vp, _P(ctypes.c_int64), _P(ctypes.c_int32), ctypes.c_int64]),
    "fbc_hmat_destroy": (None, [_vp]),
    "fbc_measure_fma_peak": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_double), _vp]),
}


def load(path: str | None = None) -> ctypes.CDLL:
    """Load ``libfbc.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise FBCError(-1, "load", f"{p} is missing: run `python -m paper_2105_08798_gb300.build`")
            lib = ctypes.CDLL(p)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != FBC_OK:
        raise FBCError(status, where, load().fbc_last_error().decode(errors="replace"))


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


# ---- same-name wrappers of the C ABI ---------------------------------------
def fbc_default_options() -> fbc_options:
    o = fbc_options()
    load().fbc_default_options(ctypes.byref(o))
    return o


def fbc_plan_create(geom: fbc_geometry, mat: fbc_material, opt: fbc_options | None) -> int:
    h = _vp()
    _check(load().fbc_plan_create(ctypes.byref(geom), ctypes.byref(mat), ctypes.byref(opt) if opt else None,
                                  ctypes.byref(h)), "fbc_plan_create")
    return h.value


def fbc_tabulate_kernel(plan: int, stream=None):
    _check(load().fbc_tabulate_kernel(plan, _stream_handle(stream)), "fbc_tabulate_kernel")


def fbc_apply(plan: int, f_ptr: int, u_ptr: int, n_rhs: int, alpha: float, beta: float, flags: int, stream=None):
    _check(load().fbc_apply(plan, f_ptr, u_ptr, n_rhs, alpha, beta, flags, _stream_handle(stream)), "fbc_apply")


def fbc_apply_host(plan: int, f_ptr: int, u_ptr: int, n_rhs: int, alpha: float, beta: float, flags: int,
                   stream=None):
    _check(load().fbc_apply_host(plan, f_ptr, u_ptr, n_rhs, alpha, beta, flags, _stream_handle(stream)),
           "fbc_apply_host")


def fbc_apply_relaxed(plan: int, f_new_ptr: int, f_old_ptr: int | None, u_ptr: int, n_rhs: int, alpha_ptr: int,
                      du_max: float, flags: int, stream=None):
    _check(load().fbc_apply_relaxed(plan, f_new_ptr, f_old_ptr, u_ptr, n_rhs, alpha_ptr, du_max, flags,
                                    _stream_handle(stream)), "fbc_apply_relaxed")


def fbc_plan_set_precision(plan: int, precision: int):
    _check(load().fbc_plan_set_precision(plan, precision), "fbc_plan_set_precision")


def fbc_plan_info_get(plan: int) -> fbc_plan_info:
    info = fbc_plan_info()
    _check(load().fbc_plan_info_get(plan, ctypes.byref(info)), "fbc_plan_info_get")
    return info


def fbc_plan_layout(plan: int) -> dict:
    info = fbc_plan_info_get(plan)
    nip, npp = info.n_tiles_b * info.tile_b, info.n_tiles_a * info.tile_a
    perm_i = np.zeros(nip, np.int32)
    perm_p = np.zeros(npp, np.int32)
    xy_i = np.zeros((nip, 2), np.int32)
    xy_p = np.zeros((npp, 2), np.int32)
    P32 = _P(ctypes.c_int32)
    _check(load().fbc_plan_layout(plan, perm_i.ctypes.data_as(P32), perm_p.ctypes.data_as(P32),
                                  xy_i.ctypes.data_as(P32), xy_p.ctypes.data_as(P32)), "fbc_plan_layout")
    return {"perm_i": perm_i, "perm_p": perm_p, "xy_i": xy_i, "xy_p": xy_p}


def fbc_get_mode_table(plan: int, d: np.ndarray, K: int) -> np.ndarray:
    d = np.ascontiguousarray(d, dtype=np.int32).reshape(-1, 2)
    out = np.zeros((len(d), K, 6))
    _check(load().fbc_get_mode_table(plan, d.ctypes.data_as(_P(ctypes.c_int32)), len(d),
                                     out.ctypes.data_as(_P(ctypes.c_double))), "fbc_get_mode_table")
    return out


def fbc_plan_sync_status(plan: int, stream=None):
    _check(load().fbc_plan_sync_status(plan, _stream_handle(stream)), "fbc_plan_sync_status")


def fbc_plan_set_wait_limit(plan: int, polls: int):
    _check(load().fbc_plan_set_wait_limit(plan, int(polls)), "fbc_plan_set_wait_limit")


def fbc_plan_set_timing(plan: int, enable: bool):
    _check(load().fbc_plan_set_timing(plan, 1 if enable else 0), "fbc_plan_set_timing")


def fbc_plan_stage_times(plan: int) -> list[float]:
    ms = (ctypes.c_float * 3)()
    _check(load().fbc_plan_stage_times(plan, ms), "fbc_plan_stage_times")
    return [float(x) for x in ms]


def fbc_destroy(plan: int):
    load().fbc_destroy(plan)


def fbc_last_error() -> str:
    return load().fbc_last_error().decode(errors="replace")


def fbc_version() -> str:
    return load().fbc_version().decode()


def fbc_zero_mean_static(u_ptr: int, n_rhs: int, n_p: int, L: int, stream=None):
    _check(load().fbc_zero_mean_static(u_ptr, n_rhs, n_p, L, _stream_handle(stream)), "fbc_zero_mean_static")


def fbc_spring_constants(k1: float, k2: float, c: float = 1.0) -> np.ndarray:
    """Force-constant blocks K [27][3][3] of the synthetic spring model (host only)."""
    K = np.empty((27, 3, 3), dtype=np.float64)
    _check(load().fbc_spring_constants(k1, k2, c, K.ctypes.data_as(_P(ctypes.c_double))), "fbc_spring_constants")
    return K


def fbc_stencil_create(xy_i: np.ndarray, sources: list[np.ndarray], L: int, K: np.ndarray) -> int:
    xy_i = np.ascontiguousarray(xy_i, dtype=np.int32)
    srcs = [np.ascontiguousarray(x, dtype=np.int32).reshape(-1, 2) for x in sources]
    ptrs = (_P(ctypes.c_int32) * len(srcs))(*[x.ctypes.data_as(_P(ctypes.c_int32)) for x in srcs])
    counts = (ctypes.c_int32 * len(srcs))(*[len(x) for x in srcs])
    K = np.ascontiguousarray(K, dtype=np.float64)
    if K.size != 27 * 9:
        raise ValueError("K must hold 27 blocks of 3x3")
    h = _vp()
    _check(load().fbc_stencil_create(len(xy_i), xy_i.ctypes.data_as(_P(ctypes.c_int32)), len(srcs), ptrs, counts,
                                     int(L), K.ctypes.data_as(_P(ctypes.c_double)), ctypes.byref(h)),
           "fbc_stencil_create")
    return h.value


def fbc_incompat_force(st: int, u_ptrs: list[int | None], f_ptr: int, n_rhs: int, stream=None):
    arr = (_vp * len(u_ptrs))(*u_ptrs)
    _check(load().fbc_incompat_force(st, arr, f_ptr, n_rhs, _stream_handle(stream)), "fbc_incompat_force")


def fbc_plan_lattice_near_field(plan: int, K: np.ndarray, r_cut: float, d_ref, n_zone: int):
    K = np.ascontiguousarray(K, dtype=np.float64)
    if K.size != 27 * 9:
        raise ValueError("K must hold 27 blocks of 3x3")
    _check(load().fbc_plan_lattice_near_field(plan, K.ctypes.data_as(_P(ctypes.c_double)), r_cut, int(d_ref[0]),
                                              int(d_ref[1]), n_zone), "fbc_plan_lattice_near_field")


def fbc_stencil_destroy(st: int):
    _check(load().fbc_stencil_destroy(st), "fbc_stencil_destroy")


def fbc_batch_create(plans: list[int], f_ptrs: list[int], u_ptrs: list[int], n_rhs: list[int]) -> int:
    n = len(plans)
    P = (_vp * n)(*plans)
    F = (_vp * n)(*f_ptrs)
    U = (_vp * n)(*u_ptrs)
    R = (ctypes.c_int32 * n)(*n_rhs)
    h = _vp()
    _check(load().fbc_batch_create(P, n, F, U, R, ctypes.byref(h)), "fbc_batch_create")
    return h.value


def fbc_batch_apply(batch: int, alpha: float, beta: float, flags: int, stream=None):
    _check(load().fbc_batch_apply(batch, alpha, beta, flags, _stream_handle(stream)), "fbc_batch_apply")


def fbc_batch_autotune(batch: int, stream=None) -> float:
    best = ctypes.c_double()
    _check(load().fbc_batch_autotune(batch, _stream_handle(stream), ctypes.byref(best)), "fbc_batch_autotune")
    return best.value


def fbc_batch_info_get(batch: int) -> dict:
    info = fbc_batch_info()
    _check(load().fbc_batch_info_get(batch, ctypes.byref(info)), "fbc_batch_info_get")
    return info.as_dict()


def fbc_batch_destroy(batch: int):
    load().fbc_batch_destroy(batch)


def fbc_surrogate_create(width: int, seed: int) -> int:
    h = _vp()
    _check(load().fbc_surrogate_create(width, seed, ctypes.byref(h)), "fbc_surrogate_create")
    return h.value


def fbc_surrogate_n_params(sur: int) -> int:
    return load().fbc_surrogate_n_params(sur)


def fbc_surrogate_params(sur: int, host_out: np.ndarray | None, host_in: np.ndarray | None):
    for a in (host_out, host_in):
        if a is not None and (a.dtype != np.float32 or not a.flags.c_contiguous or a.size != fbc_surrogate_n_params(sur)):
            raise ValueError("parameter arrays must be contiguous float32 of n_params")
    _check(load().fbc_surrogate_params(sur, None if host_out is None else host_out.ctypes.data,
                                       None if host_in is None else host_in.ctypes.data), "fbc_surrogate_params")


def fbc_surrogate_forward(sur: int, x_ptr: int, y_ptr: int, n: int, bf16_weights: bool, stream=None):
    _check(load().fbc_surrogate_forward(sur, x_ptr, y_ptr, n, int(bf16_weights), _stream_handle(stream)),
           "fbc_surrogate_forward")


def fbc_surrogate_loss_grad(sur: int, x_ptr: int, t_ptr: int, n: int, stream=None) -> tuple[float, np.ndarray]:
    loss = ctypes.c_double()
    g = np.empty(fbc_surrogate_n_params(sur), dtype=np.float32)
    _check(load().fbc_surrogate_loss_grad(sur, x_ptr, t_ptr, n, ctypes.byref(loss), g.ctypes.data,
                                          _stream_handle(stream)), "fbc_surrogate_loss_grad")
    return loss.value, g


def fbc_surrogate_train(sur: int, plan: int, n_samples: int, r_min: float, epochs: int, batch: int, lr: float,
                        seed: int, stream=None) -> float:
    loss = ctypes.c_double()
    _check(load().fbc_surrogate_train(sur, plan, n_samples, r_min, epochs, batch, lr, seed, _stream_handle(stream),
                                      ctypes.byref(loss)), "fbc_surrogate_train")
    return loss.value


def fbc_surrogate_eval_table(sur: int, plan: int, d: np.ndarray, k: np.ndarray) -> np.ndarray:
    d = np.ascontiguousarray(d, dtype=np.int32).reshape(-1, 2)
    k = np.ascontiguousarray(k, dtype=np.int32).reshape(-1)
    if d.shape[0] != k.shape[0]:
        raise ValueError("d and k differ in length")
    out = np.empty((k.shape[0], 6), dtype=np.float64)
    _check(load().fbc_surrogate_eval_table(sur, plan, d.ctypes.data_as(_P(ctypes.c_int32)),
                                           k.ctypes.data_as(_P(ctypes.c_int32)), k.shape[0],
                                           out.ctypes.data_as(_P(ctypes.c_double))), "fbc_surrogate_eval_table")
    return out


def fbc_plan_attach_surrogate(plan: int, sur: int | None, r_min: float, release_tables: bool):
    _check(load().fbc_plan_attach_surrogate(plan, sur, r_min, int(release_tables)), "fbc_plan_attach_surrogate")


def fbc_surrogate_sync_status(sur: int, stream=None):
    _check(load().fbc_surrogate_sync_status(sur, _stream_handle(stream)), "fbc_surrogate_sync_status")


def fbc_surrogate_destroy(sur: int):
    load().fbc_surrogate_destroy(sur)


# ---- convenience wrapper -----------------------------------------------------
def fbc_measure_fma_peak(fp64: bool, stream=None) -> float:
    """Measured FP32 (or FP64) fused multiply-add rate of this GPU in TFLOP/s."""
    t = ctypes.c_double(0.0)
    _check(load().fbc_measure_fma_peak(1 if fp64 else 0, ctypes.byref(t), _stream_handle(stream)),
           "fbc_measure_fma_peak")
    return t.value


def fbc_hmat_partition(xy_i: np.ndarray, xy_p: np.ndarray, L: int, c: float = 1.0, gamma: float = 2.0,
                       b_min: int = 20) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Steps 1-2 of the H-matrix construction on the host: (blocks [n][5], perm_p, perm_i)."""
    lib = load()
    xi = np.ascontiguousarray(xy_i, dtype=np.int32).reshape(-1, 2)
    xp = np.ascontiguousarray(xy_p, dtype=np.int32).reshape(-1, 2)
    n = ctypes.c_int64(0)
    i32 = _P(ctypes.c_int32)
    i64 = _P(ctypes.c_int64)
    _check(lib.fbc_hmat_partition(xi.ctypes.data_as(i32), len(xi), xp.ctypes.data_as(i32), len(xp), L, c, gamma, b_min,
                                  ctypes.byref(n), None, 0, None, None), "fbc_hmat_partition")
    blocks = np.zeros((n.value, 5), dtype=np.int64)
    perm_p = np.zeros(len(xp) * L, dtype=np.int64)
    perm_i = np.zeros(len(xi) * L, dtype=np.int64)
    _check(lib.fbc_hmat_partition(xi.ctypes.data_as(i32), len(xi), xp.ctypes.data_as(i32), len(xp), L, c, gamma, b_min,
                                  ctypes.byref(n), blocks.ctypes.data_as(i64), n.value, perm_p.ctypes.data_as(i64),
                                  perm_i.ctypes.data_as(i64)), "fbc_hmat_partition")
    return blocks, perm_p, perm_i


def fbc_hmat_create(plan: int, eps: float, gamma: float, b_min: int, max_rank: int, scratch_bytes: int,
                    stream=None) -> int:
    h = _vp()
    opt = fbc_hmat_options(eps, gamma, b_min, max_rank, scratch_bytes)
    _check(load().fbc_hmat_create(plan, ctypes.byref(opt), _stream_handle(stream), ctypes.byref(h)), "fbc_hmat_create")
    return h.value


def fbc_hmat_apply(h: int, f_ptr: int, u_ptr: int, n_rhs: int, alpha: float, beta: float, flags: int, stream=None):
    _check(load().fbc_hmat_apply(h, f_ptr, u_ptr, n_rhs, alpha, beta, flags, _stream_handle(stream)), "fbc_hmat_apply")


def fbc_hmat_get_info(h: int) -> dict:
    info = fbc_hmat_info()
    _check(load().fbc_hmat_get_info(h, ctypes.byref(info)), "fbc_hmat_get_info")
    return info.as_dict()


def fbc_hmat_blocks(h: int, n_blocks: int) -> tuple[np.ndarray, np.ndarray]:
    blocks = np.zeros((n_blocks, 5), dtype=np.int64)
    ranks = np.zeros(n_blocks, dtype=np.int32)
    _check(load().fbc_hmat_blocks(h, blocks.ctypes.data_as(_P(ctypes.c_int64)), ranks.ctypes.data_as(_P(ctypes.c_int32)),
                                  n_blocks), "fbc_hmat_blocks")
    return blocks, ranks


def fbc_hmat_destroy(h: int):
    load().fbc_hmat_destroy(h)


def material_struct(material: dict) -> fbc_material:
    m = fbc_material()
    kind = material.get("kind", "isotropic")
    Q = np.asarray(material.get("Q", np.eye(3)), dtype=np.float64).reshape(9)
    for t in range(9):
        m.Q[t] = float(Q[t])
    if kind == "isotropic":
        m.kind = FBC_MATERIAL_ISOTROPIC
        m.mu, m.nu = float(material["mu"]), float(material["nu"])
    elif kind == "cubic":
        m.kind = FBC_MATERIAL_CUBIC
        m.C11, m.C12, m.C44 = float(material["C11"]), float(material["C12"]), float(material["C44"])
    else:
        raise ValueError(f"unknown material kind {kind!r}")
    return m


class Plan:
    """Owning handle of one ``fbc_plan`` (tables + workspace on the current device)."""

    def __init__(self, xy_i, xy_p, L: int, material: dict, c: float = 1.0, precision: str | int = "fp64",
                 rich_n: int | None = None, rich_N: int | None = None, quad: int | None = None, max_rhs: int = 1,
                 host_only: bool = False, tc_fast_accumulate: bool = False, self_terms: bool = False):
        self._h = None
        self._sur = None
        xy_i = np.ascontiguousarray(xy_i, dtype=np.int32)
        xy_p = np.ascontiguousarray(xy_p, dtype=np.int32)
        g = fbc_geometry(len(xy_i), len(xy_p), int(L), float(c), xy_i.ctypes.data_as(_P(ctypes.c_int32)),
                         xy_p.ctypes.data_as(_P(ctypes.c_int32)))
        o = fbc_default_options()
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if rich_n is not None:
            o.rich_n = rich_n
        if rich_N is not None:
            o.rich_N = rich_N
        if quad is not None:
            o.quad = quad
        o.max_rhs = int(max_rhs)
        o.flags = ((FBC_PLAN_HOST_ONLY if host_only else 0) | (FBC_PLAN_TC_FAST_ACCUMULATE if tc_fast_accumulate else 0)
                   | (FBC_PLAN_SELF_TERMS if self_terms else 0))
        self._h = fbc_plan_create(g, material_struct(material), o)
        self.n_i, self.n_p, self.L, self.K = len(xy_i), len(xy_p), int(L), int(L) // 2 + 1
        self.max_rhs = int(max_rhs)

    @property
    def handle(self) -> int:
        if self._h is None:
            raise FBCError(FBC_ERR_INVALID_ARG, "Plan", "plan is closed")
        return self._h

    def tabulate(self, stream=None):
        fbc_tabulate_kernel(self.handle, stream)

    def set_precision(self, precision: str | int):
        fbc_plan_set_precision(self.handle, PRECISIONS[precision] if isinstance(precision, str) else int(precision))

    def info(self) -> dict:
        return fbc_plan_info_get(self.handle).as_dict()

    def layout(self) -> dict:
        return fbc_plan_layout(self.handle)

    def mode_table(self, d) -> np.ndarray:
        return fbc_get_mode_table(self.handle, d, self.K)

    @staticmethod
    def flags(project: bool = True, zero_mean: bool = False) -> int:
        return (FBC_APPLY_PROJECT_NEUTRAL if project else 0) | (FBC_APPLY_ZERO_MEAN_U if zero_mean else 0)

    def apply(self, f, u, alpha: float = 1.0, beta: float = 0.0, project: bool = True, zero_mean: bool = False,
              stream=None):
        """u <- beta u + alpha G f on device tensors ``f [n_rhs][n_i][L][3]``, ``u [n_rhs][n_p][L][3]`` (float64)."""
        import torch

        n_rhs = f.shape[0]
        if f.dtype != torch.float64 or u.dtype != torch.float64 or not f.is_cuda or not u.is_cuda:
            raise TypeError("f and u must be float64 CUDA tensors")
        if tuple(f.shape) != (n_rhs, self.n_i, self.L, 3) or tuple(u.shape) != (n_rhs, self.n_p, self.L, 3):
            raise ValueError(f"shape mismatch: f {tuple(f.shape)}, u {tuple(u.shape)}")
        if not f.is_contiguous() or not u.is_contiguous():
            raise ValueError("f and u must be contiguous")
        if stream is None:
            stream = torch.cuda.current_stream(f.device)
        fbc_apply(self.handle, f.data_ptr(), u.data_ptr(), n_rhs, alpha, beta, self.flags(project, zero_mean), stream)
        return u

    def apply_relaxed(self, f_new, f_old, u, alpha, du_max: float = 0.0, project: bool = True,
                      zero_mean: bool = False, stream=None):
        """One relaxed FBC update on device tensors: u <- u - alpha G f_new with alpha from the residual-based
        relaxation (f_old may be None); ``alpha`` is a float64 CUDA tensor [n_rhs], updated in place."""
        import torch

        n_rhs = f_new.shape[0]
        for t, n in ((f_new, self.n_i), (u, self.n_p)) + (((f_old, self.n_i),) if f_old is not None else ()):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != (n_rhs, n, self.L, 3):
                raise ValueError("f_new, f_old and u must be contiguous float64 CUDA tensors of the plan's shapes")
        if alpha.dtype != torch.float64 or not alpha.is_cuda or tuple(alpha.shape) != (n_rhs,):
            raise ValueError("alpha must be a float64 CUDA tensor [n_rhs]")
        if stream is None:
            stream = torch.cuda.current_stream(f_new.device)
        fbc_apply_relaxed(self.handle, f_new.data_ptr(), None if f_old is None else f_old.data_ptr(), u.data_ptr(),
                          n_rhs, alpha.data_ptr(), du_max, self.flags(project, zero_mean), stream)
        return u

    def apply_host(self, f: np.ndarray, u: np.ndarray, alpha: float = 1.0, beta: float = 0.0, project: bool = True,
                   zero_mean: bool = False, stream=None):
        """Host-memory form: numpy (or pinned torch CPU) arrays in, ``u`` updated in place."""
        fp = f.data_ptr() if hasattr(f, "data_ptr") else f.ctypes.data
        up = u.data_ptr() if hasattr(u, "data_ptr") else u.ctypes.data
        n_rhs = f.shape[0]
        fbc_apply_host(self.handle, fp, up, n_rhs, alpha, beta, self.flags(project, zero_mean), stream)
        return u

    def set_wait_limit(self, polls: int = 0):
        """Bound of the tensor-core pipeline waits in polls (0: the default); for tests of the timeout path."""
        fbc_plan_set_wait_limit(self.handle, polls)

    def set_timing(self, enable: bool = True):
        fbc_plan_set_timing(self.handle, enable)

    def stage_times(self) -> list[float]:
        """[forward, contraction, inverse] milliseconds of the last timed apply."""
        return fbc_plan_stage_times(self.handle)

    def sync_status(self, stream=None):
        fbc_plan_sync_status(self.handle, stream)

    def lattice_near_field(self, K, r_cut: float, d_ref, n_zone: int = 1024):
        """Replace the table entries with |d| <= r_cut by the lattice Green function of the stencil K; the
        k = 0 mode joins the continuum one at the table difference d_ref (|d_ref| > r_cut)."""
        fbc_plan_lattice_near_field(self.handle, K, r_cut, d_ref, n_zone)

    def attach_surrogate(self, sur: "Surrogate | None", r_min: float = 8.0, release_tables: bool = False):
        """Serve modes k >= 1 at |d| >= r_min from ``sur`` (None detaches); see fbc_plan_attach_surrogate."""
        fbc_plan_attach_surrogate(self.handle, None if sur is None else sur.handle, r_min, release_tables)
        self._sur = sur  # keep the surrogate alive while attached

    def close(self):
        if self._h is not None:
            fbc_destroy(self._h)
            self._h = None
        self._sur = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """Owning handle of one ``fbc_surrogate`` (MLP 4 -> H -> H -> H -> 6 of the scaled mode table)."""

    def __init__(self, width: int = 128, seed: int = 0):
        self._h = None
        self._h = fbc_surrogate_create(width, seed)
        self.width = width

    @property
    def handle(self) -> int:
        if self._h is None:
            raise ValueError("surrogate is closed")
        return self._h

    @property
    def n_params(self) -> int:
        return fbc_surrogate_n_params(self.handle)

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        fbc_surrogate_params(self.handle, out, None)
        return out

    def set_params(self, p: np.ndarray):
        fbc_surrogate_params(self.handle, None, np.ascontiguousarray(p, dtype=np.float32))

    def forward(self, x, bf16_weights: bool = False):
        """y [n][6] = MLP(x [n][4]) on float32 CUDA tensors."""
        import torch

        if x.dtype != torch.float32 or not x.is_cuda or x.dim() != 2 or x.shape[1] != 4 or not x.is_contiguous():
            raise TypeError("x must be a contiguous float32 CUDA tensor [n][4]")
        y = torch.empty((x.shape[0], 6), dtype=torch.float32, device=x.device)
        fbc_surrogate_forward(self.handle, x.data_ptr(), y.data_ptr(), x.shape[0], bf16_weights,
                              torch.cuda.current_stream(x.device))
        return y

    def loss_grad(self, x, t) -> tuple[float, np.ndarray]:
        import torch

        for a, w in ((x, 4), (t, 6)):
            if a.dtype != torch.float32 or not a.is_cuda or a.dim() != 2 or a.shape[1] != w or not a.is_contiguous():
                raise TypeError("x [n][4] and t [n][6] must be contiguous float32 CUDA tensors")
        return fbc_surrogate_loss_grad(self.handle, x.data_ptr(), t.data_ptr(), x.shape[0],
                                       torch.cuda.current_stream(x.device))

    def train(self, plan: Plan, n_samples: int = 1 << 20, r_min: float = 8.0, epochs: int = 50, batch: int = 4096,
              lr: float = 2e-3, seed: int = 0) -> float:
        return fbc_surrogate_train(self.handle, plan.handle, n_samples, r_min, epochs, batch, lr, seed)

    def sync_status(self, stream=None):
        fbc_surrogate_sync_status(self.handle, stream)

    def table(self, plan: Plan, d, k) -> np.ndarray:
        return fbc_surrogate_eval_table(self.handle, plan.handle, d, k)

    def close(self):
        if self._h is not None:
            fbc_surrogate_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stencil:
    """Owning handle of one ``fbc_stencil``: the harmonic operator restricted to the interface rows."""

    def __init__(self, xy_i, sources: list, L: int, K):
        self._h = None
        self.n_i, self.L = len(xy_i), int(L)
        self.n_site = [len(np.asarray(x).reshape(-1, 2)) for x in sources]
        self._h = fbc_stencil_create(xy_i, sources, L, K)

    @property
    def handle(self) -> int:
        if self._h is None:
            raise ValueError("stencil is closed")
        return self._h

    def incompat_force(self, u_list: list, f=None, stream=None):
        """f_in [n_rhs][n_i][L][3] from the displacements ``u_list[s]`` [n_rhs][n_site[s]][L][3] (float64 CUDA
        tensors, one per source set, in the order given at construction)."""
        import torch

        if len(u_list) != len(self.n_site):
            raise ValueError("one displacement tensor per source set")
        n_rhs = u_list[0].shape[0]
        for u, n in zip(u_list, self.n_site):
            if u.dtype != torch.float64 or not u.is_cuda or not u.is_contiguous() or tuple(u.shape) != (n_rhs, n, self.L, 3):
                raise ValueError("u tensors must be contiguous float64 CUDA tensors [n_rhs][n_site][L][3]")
        if f is None:
            f = torch.empty((n_rhs, self.n_i, self.L, 3), dtype=torch.float64, device=u_list[0].device)
        elif f.dtype != torch.float64 or not f.is_cuda or not f.is_contiguous() or tuple(f.shape) != (n_rhs, self.n_i, self.L, 3):
            raise ValueError("f must be a contiguous float64 CUDA tensor [n_rhs][n_i][L][3]")
        if stream is None:
            stream = torch.cuda.current_stream(f.device)
        fbc_incompat_force(self.handle, [u.data_ptr() for u in u_list], f.data_ptr(), n_rhs, stream)
        return f

    def close(self):
        if self._h is not None:
            fbc_stencil_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owning handle of one ``fbc_batch`` over existing plans and device tensors."""

    def __init__(self, plans: list, f_list: list, u_list: list):
        import torch

        for f, u, p in zip(f_list, u_list, plans):
            if f.dtype != torch.float64 or u.dtype != torch.float64 or not f.is_cuda or not u.is_cuda:
                raise TypeError("f and u must be float64 CUDA tensors")
            if tuple(f.shape[1:]) != (p.n_i, p.L, 3) or tuple(u.shape[1:]) != (p.n_p, p.L, 3) or f.shape[0] != u.shape[0]:
                raise ValueError("shape mismatch between a plan and its buffers")
        self._plans = list(plans)
        self._keep = (list(f_list), list(u_list))
        self._h = fbc_batch_create([p.handle for p in plans], [f.data_ptr() for f in f_list],
                                   [u.data_ptr() for u in u_list], [int(f.shape[0]) for f in f_list])

    def apply(self, alpha: float = 1.0, beta: float = 0.0, project: bool = True, zero_mean: bool = False,
              graph: bool = True, stream=None):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream()
        flags = Plan.flags(project, zero_mean) | (0 if graph else FBC_APPLY_NO_GRAPH)
        fbc_batch_apply(self._h, alpha, beta, flags, stream)

    def autotune(self, stream=None) -> float:
        return fbc_batch_autotune(self._h, stream)

    def info(self) -> dict:
        return fbc_batch_info_get(self._h)

    def close(self):
        if self._h is not None:
            fbc_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HMatrix:
    """Owning handle of one ``fbc_hmat``: the H-matrix approximation of a plan's Green matrix
    (Sec. 3.2; App., the H-matrix construction).  Defaults are the paper's settings."""

    def __init__(self, plan: Plan, eps: float = 1e-5, gamma: float = 2.0, b_min: int = 20, max_rank: int = 0,
                 scratch_bytes: int = 0, stream=None):
        self._h = None
        self.n_i, self.n_p, self.L = plan.n_i, plan.n_p, plan.L
        self._h = fbc_hmat_create(plan.handle, eps, gamma, b_min, max_rank, scratch_bytes, stream)

    @property
    def handle(self) -> int:
        if self._h is None:
            raise ValueError("H-matrix is closed")
        return self._h

    def info(self) -> dict:
        return fbc_hmat_get_info(self.handle)

    def blocks(self) -> tuple[np.ndarray, np.ndarray]:
        """The partition (rows of (row start, row count, col start, col count, low rank)) and the ranks."""
        i = self.info()
        return fbc_hmat_blocks(self.handle, int(i["n_lowrank"] + i["n_dense"]))

    def apply(self, f, u, alpha: float = 1.0, beta: float = 0.0, project: bool = True, zero_mean: bool = False,
              stream=None):
        """u <- beta u + alpha G_H f on float64 CUDA tensors f [n_rhs][n_i][L][3], u [n_rhs][n_p][L][3]."""
        import torch

        n_rhs = f.shape[0]
        if f.dtype != torch.float64 or u.dtype != torch.float64 or not f.is_cuda or not u.is_cuda:
            raise TypeError("f and u must be float64 CUDA tensors")
        if tuple(f.shape) != (n_rhs, self.n_i, self.L, 3) or tuple(u.shape) != (n_rhs, self.n_p, self.L, 3):
            raise ValueError(f"shape mismatch: f {tuple(f.shape)}, u {tuple(u.shape)}")
        if not f.is_contiguous() or not u.is_contiguous():
            raise ValueError("f and u must be contiguous")
        if stream is None:
            stream = torch.cuda.current_stream(f.device)
        fbc_hmat_apply(self.handle, f.data_ptr(), u.data_ptr(), n_rhs, alpha, beta, Plan.flags(project, zero_mean),
                       stream)
        return u

    def close(self):
        if self._h is not None:
            fbc_hmat_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
