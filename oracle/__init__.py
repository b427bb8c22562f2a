"""Plain FP64 CPU oracle for the FBC Green's-function pad update.

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the product path never
does.  It shares no code with the CUDA library and never imports it.

The numerical core is ``fbc_oracle.c`` (built with ``build()``), wrapped here
with ``ctypes``.  Every function cites the passage of the paper it follows:

* ``green``            -- the continuum Green function, Sec. 3.1, Eq. 33
                          (Kelvin, or Barnett's line integral).
* ``richardson_weights``, ``periodic``
                        -- the regularised image sum and its Richardson
                          extrapolation, Sec. 3.1, Eqs. 32, 35, 36.
* ``kernel_table``     -- the periodic kernel on the line lattice (same
                          equations, evaluated at the centred repeat offset).
* ``project_neutral``  -- removal of the net interface force: the per-component
                          mean over all interface atoms (the reading of the
                          workloads' "zero net force per column set").
* ``pad_update``       -- the real-space update u = G f (Sec. 1, Eq. 1;
                          Sec. 3.2, Eqs. 37-38) with the relaxation/update
                          form u <- beta u + alpha G f (Sec. 2.3.2, Eq. 22,
                          Algorithm 1) and the optional zero mean (Eq. 23).
* ``mode_table``       -- plain DFT of the tabulated kernel along the line.
* ``relax_alpha``      -- the residual-based relaxation parameter (Sec. 2.3.3,
                          Algorithm 2) and ``relaxed_update``, the pad update of
                          Algorithm 1 that uses it.
* ``real_space_update``-- the real-space update with a given real-space kernel
                          table (the lattice Green function's, or a blend).
* ``mode_space_update``-- the update evaluated mode by mode with a given mode
                          table (a cross-check of the real-space form).
* ``harmonic``         -- the harmonic model: the incompatibility force
                          (Sec. 2.3.2, Eq. 21) and the lattice Green function
                          of a block stencil (App.), per mode and in real space.

Parity is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fbc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_RICH_N = 4
DEFAULT_RICH_NN = 6
DEFAULT_NQUAD = 96


def build(force: bool = False) -> str:
    """Compile ``fbc_oracle.c`` into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    cc = os.environ.get("CC", "cc")
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = [cc, "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Material(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("mu", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("C11", ctypes.c_double),
        ("C12", ctypes.c_double),
        ("C44", ctypes.c_double),
        ("Q", ctypes.c_double * 9),
        ("nquad", ctypes.c_int32),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            d, i32 = ctypes.c_double, ctypes.c_int32
            lib.orc_green.argtypes = [P(_Material), P(d), P(d)]
            lib.orc_periodic.argtypes = [P(_Material), d, ctypes.c_int, ctypes.c_int, P(d), P(d)]
            lib.orc_richardson_weights.argtypes = [ctypes.c_int, ctypes.c_int, P(d)]
            lib.orc_kernel_table.argtypes = [P(_Material), ctypes.c_int, d, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, P(i32), P(d), ctypes.c_int]
            lib.orc_apply_samples.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P(i32), ctypes.c_int,
                                              P(d), ctypes.c_int, P(d), ctypes.c_int, P(i32), P(i32), P(d),
                                              ctypes.c_int]
            lib.orc_mode_table.argtypes = [ctypes.c_int, ctypes.c_int, P(d), P(d), P(d), ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def n_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def material_struct(material: dict, nquad: int | None = None) -> _Material:
    """Build the C material record from a workload material dict."""
    m = _Material()
    kind = material.get("kind", "isotropic")
    Q = np.asarray(material.get("Q", np.eye(3)), dtype=np.float64).reshape(9)
    for t in range(9):
        m.Q[t] = float(Q[t])
    m.nquad = int(nquad if nquad is not None else material.get("nquad", DEFAULT_NQUAD))
    if kind == "isotropic":
        m.kind = 0
        m.mu = float(material["mu"])
        m.nu = float(material["nu"])
    elif kind == "cubic":
        m.kind = 1
        m.C11 = float(material["C11"])
        m.C12 = float(material["C12"])
        m.C44 = float(material["C44"])
    else:
        raise ValueError(f"unknown material kind {kind!r}")
    return m


def _check(st: int, what: str):
    if st != 0:
        raise ValueError(f"oracle {what} failed with status {st}")


def green(material: dict, r, nquad: int | None = None) -> np.ndarray:
    """Continuum Green function G(r) of the infinite medium (Sec. 3.1, Eq. 33)."""
    lib = _load()
    m = material_struct(material, nquad)
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(3)
    G = np.zeros(9)
    _check(lib.orc_green(ctypes.byref(m), _ptr(r, ctypes.c_double), _ptr(G, ctypes.c_double)), "green")
    return G.reshape(3, 3)


def richardson_weights(n: int, N: int) -> np.ndarray:
    """Weights of Eq. 36: w_i = (n+i)^N (-1)^(i+N) / (i! (N-i)!)."""
    lib = _load()
    w = np.zeros(N + 1)
    _check(lib.orc_richardson_weights(n, N, _ptr(w, ctypes.c_double)), "richardson_weights")
    return w


def periodic(material: dict, l3: float, r, n: int = DEFAULT_RICH_N, N: int = DEFAULT_RICH_NN,
             nquad: int | None = None) -> np.ndarray:
    """Richardson-extrapolated regularised image sum Q0 at r (Sec. 3.1, Eqs. 32, 35, 36)."""
    lib = _load()
    m = material_struct(material, nquad)
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(3)
    out = np.zeros(9)
    _check(lib.orc_periodic(ctypes.byref(m), float(l3), n, N, _ptr(r, ctypes.c_double),
                            _ptr(out, ctypes.c_double)), "periodic")
    return out.reshape(3, 3)


def kernel_table(material: dict, L: int, c: float, d, n: int = DEFAULT_RICH_N, N: int = DEFAULT_RICH_NN,
                 nquad: int | None = None, nthreads: int | None = None) -> np.ndarray:
    """Periodic kernel G~(d, s) for each in-plane difference d and s = 0..L-1.

    Returns ``float64 [nd][L][3][3]``.  Evaluated at the centred repeat offset
    s' in (-L/2, L/2]; the two representatives of s = L/2 are averaged.
    """
    lib = _load()
    m = material_struct(material, nquad)
    d = np.ascontiguousarray(d, dtype=np.int32).reshape(-1, 2)
    out = np.zeros((len(d), L, 9))
    _check(lib.orc_kernel_table(ctypes.byref(m), int(L), float(c), n, N, len(d), _ptr(d, ctypes.c_int32),
                                _ptr(out, ctypes.c_double), nthreads or n_threads()), "kernel_table")
    return out.reshape(len(d), L, 3, 3)


def mode_table(table: np.ndarray, nthreads: int | None = None) -> np.ndarray:
    """Plain DFT along the line: g^k(d) = sum_s G~(d, s) exp(-2 pi i k s / L), k = 0..L/2.

    Returns ``complex128 [nd][L/2+1][3][3]``.
    """
    lib = _load()
    nd, L = table.shape[0], table.shape[1]
    T = np.ascontiguousarray(table, dtype=np.float64).reshape(nd, L, 9)
    K = L // 2 + 1
    re = np.zeros((nd, K, 9))
    im = np.zeros((nd, K, 9))
    _check(lib.orc_mode_table(int(L), nd, _ptr(T, ctypes.c_double), _ptr(re, ctypes.c_double),
                              _ptr(im, ctypes.c_double), nthreads or n_threads()), "mode_table")
    return (re + 1j * im).reshape(nd, K, 3, 3)


def project_neutral(f: np.ndarray) -> np.ndarray:
    """Remove the net interface force: per right-hand side and component,
    subtract the mean over all N_I * L interface atoms.

    Any constant tensor added to the kernel then changes u by C * sum f = 0,
    which is why the regularisation of Eq. 32 (a constant shift) is harmless.
    """
    f = np.asarray(f, dtype=np.float64)
    out = np.empty_like(f)
    for r in range(f.shape[0]):
        for c in range(3):
            col = f[r, :, :, c]
            mean = float(np.sum(col, dtype=np.float64)) / col.size
            # second pass picks up the rounding of the first (corrected two-pass mean)
            mean += float(np.sum(col - mean)) / col.size
            out[r, :, :, c] = col - mean
    return out


def zero_mean(u: np.ndarray) -> np.ndarray:
    """Set the mean pad displacement to zero per component (Sec. 2.3.2, Eq. 23)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.empty_like(u)
    for r in range(u.shape[0]):
        for c in range(3):
            col = u[r, :, :, c]
            mean = float(np.sum(col)) / col.size
            mean += float(np.sum(col - mean)) / col.size
            out[r, :, :, c] = col - mean
    return out


def difference_index(xy_i: np.ndarray, xy_p_cols: np.ndarray):
    """Distinct in-plane differences d = x_a - x_b for the given pad columns.

    Returns ``(d_list int32 [nd][2], index int32 [n_cols][n_i])``.
    """
    xy_i = np.asarray(xy_i, dtype=np.int64)
    xy_p_cols = np.asarray(xy_p_cols, dtype=np.int64).reshape(-1, 2)
    D = xy_p_cols[:, None, :] - xy_i[None, :, :]
    flat = D.reshape(-1, 2)
    uniq, inv = np.unique(flat, axis=0, return_inverse=True)
    return (np.ascontiguousarray(uniq, dtype=np.int32),
            np.ascontiguousarray(inv.reshape(len(xy_p_cols), len(xy_i)), dtype=np.int32))


def real_space_sum(d_index: np.ndarray, table: np.ndarray, f: np.ndarray, samp_col, samp_p,
                   nthreads: int | None = None) -> np.ndarray:
    """u(a, p) = sum_{b, q} G~(x_a - x_b, (p - q) mod L) f(b, q)  (Eq. 1, Eqs. 37-38).

    ``d_index[col][b]`` selects the row of ``table`` (``[nd][L][3][3]``) for
    the pair (pad column ``col``, interface column ``b``); each sample is a
    ``(col, p)`` pair.  Returns ``[n_rhs][n_samp][3]``.  Neumaier-compensated.
    """
    lib = _load()
    d_index = np.ascontiguousarray(d_index, dtype=np.int32)
    nd, L = table.shape[0], table.shape[1]
    T = np.ascontiguousarray(table, dtype=np.float64).reshape(nd, L, 9)
    f = np.ascontiguousarray(f, dtype=np.float64)
    n_rhs, n_i = f.shape[0], f.shape[1]
    assert f.shape == (n_rhs, n_i, L, 3) and d_index.shape[1] == n_i
    samp_col = np.ascontiguousarray(samp_col, dtype=np.int32)
    samp_p = np.ascontiguousarray(samp_p, dtype=np.int32)
    ns = len(samp_col)
    u = np.zeros((n_rhs, ns, 3))
    _check(lib.orc_apply_samples(n_i, int(L), d_index.shape[0], _ptr(d_index, ctypes.c_int32), nd,
                                 _ptr(T, ctypes.c_double), n_rhs, _ptr(f, ctypes.c_double), ns,
                                 _ptr(samp_col, ctypes.c_int32), _ptr(samp_p, ctypes.c_int32),
                                 _ptr(u, ctypes.c_double), nthreads or n_threads()), "apply")
    return u


def pad_update(xy_i, xy_p, L: int, c: float, material: dict, f: np.ndarray, *, samples=None,
               alpha: float = 1.0, beta: float = 0.0, u0: np.ndarray | None = None, project: bool = True,
               zero_mean_u: bool = False, n: int = DEFAULT_RICH_N, N: int = DEFAULT_RICH_NN,
               nquad: int | None = None, nthreads: int | None = None, return_table: bool = False):
    """Real-space pad update  u <- beta u0 + alpha * G~ f  (Eqs. 1, 22, 37-38).

    ``f`` is ``[n_rhs][N_I][L][3]``.  With ``samples=None`` every pad atom is
    evaluated and the result is ``[n_rhs][N_P][L][3]``; otherwise ``samples``
    is an ``int [n_samp][2]`` array of ``(pad column a, repeat p)`` pairs and
    the result is ``[n_rhs][n_samp][3]``.
    """
    lib = _load()
    xy_i = np.asarray(xy_i, dtype=np.int32)
    xy_p = np.asarray(xy_p, dtype=np.int32)
    f = np.asarray(f, dtype=np.float64)
    n_rhs, n_i = f.shape[0], f.shape[1]
    assert f.shape == (n_rhs, len(xy_i), L, 3)
    fp = project_neutral(f) if project else f
    fp = np.ascontiguousarray(fp)
    if samples is None:
        cols = np.arange(len(xy_p), dtype=np.int32)
        samp_col = np.repeat(cols, L).astype(np.int32)
        samp_p = np.tile(np.arange(L, dtype=np.int32), len(xy_p))
        col_ids = cols
    else:
        samples = np.asarray(samples, dtype=np.int64).reshape(-1, 2)
        col_ids, samp_col = np.unique(samples[:, 0], return_inverse=True)
        samp_col = samp_col.astype(np.int32)
        samp_p = samples[:, 1].astype(np.int32)
    d_list, d_index = difference_index(xy_i, xy_p[col_ids])
    table = kernel_table(material, L, c, d_list, n=n, N=N, nquad=nquad, nthreads=nthreads)
    u = real_space_sum(d_index, table, fp, samp_col, samp_p, nthreads=nthreads)
    if samples is None:
        u = u.reshape(n_rhs, len(xy_p), L, 3)
    out = alpha * u
    if beta != 0.0:
        if u0 is None:
            raise ValueError("beta != 0 needs u0")
        if samples is None:
            out = out + beta * np.asarray(u0, dtype=np.float64)
        else:
            u0 = np.asarray(u0, dtype=np.float64)
            out = out + beta * u0[:, samples[:, 0], samples[:, 1], :]
    if zero_mean_u:
        if samples is not None:
            raise ValueError("the zero-mean step needs every pad atom")
        out = zero_mean(out)
    if return_table:
        return out, (d_list, table)
    return out


def relax_alpha(f_new, f_old, alpha_k, g, du_max: float = 0.0) -> np.ndarray:
    """Relaxation parameter of Algorithm 2 (Sec. 2.3.3), one per right-hand side.

    alpha = -alpha_k <f_old, f_new - f_old> / ||f_new - f_old||^2 over all interface
    atoms and components (alpha_k kept when the denominator is zero, or when f_old
    is None); alpha = 1 where that is negative; alpha = du_max / ||g||_inf where
    du_max > 0 and ||alpha g||_inf > du_max, with g = G f_new.
    """
    f_new = np.asarray(f_new, dtype=np.float64)
    alpha = np.array(alpha_k, dtype=np.float64).reshape(-1).copy()
    g = np.asarray(g, dtype=np.float64)
    for r in range(f_new.shape[0]):
        if f_old is not None:
            a = f_new[r].ravel()
            b = np.asarray(f_old[r], dtype=np.float64).ravel()
            diff = a - b
            den = float(np.dot(diff, diff))
            if den > 0.0:
                alpha[r] = -alpha[r] * float(np.dot(b, diff)) / den
            if alpha[r] < 0.0:
                alpha[r] = 1.0
        if du_max > 0.0:
            gmax = float(np.max(np.abs(g[r])))
            if gmax > 0.0 and alpha[r] * gmax > du_max:
                alpha[r] = du_max / gmax
    return alpha


def relaxed_update(xy_i, xy_p, L: int, c: float, material: dict, f_new, f_old, u0, alpha_k, du_max: float = 0.0,
                   project: bool = True, zero_mean_u: bool = False, nquad: int | None = None):
    """One pad update of Algorithm 1 with the relaxation of Algorithm 2:
    u = u0 - alpha G f_new (then the optional zero mean, Eq. 23).  Returns (u, alpha)."""
    g = pad_update(xy_i, xy_p, L, c, material, f_new, project=project, nquad=nquad)
    alpha = relax_alpha(f_new, f_old, alpha_k, g, du_max)
    u = np.asarray(u0, dtype=np.float64) - alpha[:, None, None, None] * g
    if zero_mean_u:
        u = zero_mean(u)
    return u, alpha


def real_space_update(xy_i, xy_p, L: int, f, table_of_d, project: bool = True) -> np.ndarray:
    """u(a, p) = sum_{b, q} G~(x_a - x_b, (p - q) mod L) f(b, q) at every pad atom (Eq. 1, Sec. 3.2,
    Eqs. 37-38) with a given real-space kernel: ``table_of_d(d_list int32 [nd][2])`` returns
    float64 [nd][L][3][3].  The double sum is the C real-space sum of ``real_space_sum``."""
    f = np.asarray(f, dtype=np.float64)
    fp = np.ascontiguousarray(project_neutral(f) if project else f)
    xy_p = np.asarray(xy_p, dtype=np.int32).reshape(-1, 2)
    d_list, d_index = difference_index(xy_i, xy_p)
    table = np.asarray(table_of_d(d_list), dtype=np.float64)
    n_p = len(xy_p)
    samp_col = np.repeat(np.arange(n_p, dtype=np.int32), L)
    samp_p = np.tile(np.arange(L, dtype=np.int32), n_p)
    u = real_space_sum(d_index, table, fp, samp_col, samp_p)
    return u.reshape(f.shape[0], n_p, L, 3)


def mode_space_update(xy_i, xy_p, L: int, f, gk_of_d, project: bool = True) -> np.ndarray:
    """u = G f evaluated mode by mode with a given mode table (the convolution theorem along the
    line, Sec. 3.2, Eqs. 37-38): F(b, k) = sum_q f(b, q) exp(-2 pi i k q / L) for k = 0 .. L/2,
    U(a, k) = sum_b g^k(x_a - x_b) F(b, k), u = the real inverse transform of U.  ``gk_of_d(d)``
    returns complex [L/2 + 1][3][3] for a difference d.  numpy's real FFT serves as the transform."""
    f = np.asarray(f, dtype=np.float64)
    if project:
        f = project_neutral(f)
    F = np.fft.rfft(f, axis=2)  # [R][n_i][K][3]
    R, n_p = f.shape[0], len(xy_p)
    U = np.zeros((R, n_p, L // 2 + 1, 3), dtype=np.complex128)
    for a in range(n_p):
        for b in range(len(xy_i)):
            g = gk_of_d((int(xy_p[a][0] - xy_i[b][0]), int(xy_p[a][1] - xy_i[b][1])))
            U[:, a] += np.einsum("kij,rkj->rki", g, F[:, b])
    return np.fft.irfft(U, n=L, axis=2)


def sys_info() -> dict:
    """Host description for the CPU baseline record."""
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("processor name"):
                    model = line.split(":", 1)[1].strip()
                    if low.startswith("model name"):
                        break
    except OSError:  # pragma: no cover
        pass
    return {"cores": n_threads(), "cpu": model, "machine": os.uname().machine, "python": sys.version.split()[0]}
