"""The FBC iteration converges in two steps when the atomistic model is the harmonic one and G is its
exact lattice Green function (Sec. 2.3.1, Remark 1).  Oracle-level pin of the harmonic pieces
together: the incompatibility force (Eq. 21), the lattice Green function (App.) in real space along
the line and the real-space update (Sec. 3.2), with the interface columns inside the pad as in the
paper (self-terms d = 0).

Set-up: the synthetic spring model on the line-periodic lattice (L = 4); atoms |x|^2 <= 9; the
interface Lambda^{i+} = continuum sites next to an atom, the pad = Lambda^{i+} and their continuum
neighbours; a force e_x cos(2 pi q / L) on the central atom (modes k = 1 and L - 1 only, so the
k = 0 constant of the Green function plays no part).  The atomistic problem is solved exactly
(dense linear solve); the pad is updated by u_p <- u_p - G f_in.
"""

import itertools

import numpy as np

from oracle import harmonic

L, N_ZONE = 4, 64


def chebyshev_neighbours(p):
    return [(p[0] + dx, p[1] + dy) for dx in (-1, 0, 1) for dy in (-1, 0, 1) if (dx, dy) != (0, 0)]


def fbc_geometry():
    box = [(x, y) for x in range(-8, 9) for y in range(-8, 9)]
    atoms = [p for p in box if p[0] ** 2 + p[1] ** 2 <= 9]
    A = set(atoms)
    ip = sorted({q for a in atoms for q in chebyshev_neighbours(a) if q not in A})
    IP = set(ip)
    ipp = sorted({q for a in ip for q in chebyshev_neighbours(a) if q not in A and q not in IP})
    return atoms, ip, ip + ipp


def atomistic_solve(Kb, atoms, pad, up, fext):
    """Force balance of the harmonic model at every atom, the pad displacements held fixed."""
    idx_a = {p: i for i, p in enumerate(atoms)}
    idx_p = {p: i for i, p in enumerate(pad)}
    n = len(atoms) * L * 3
    M = np.zeros((n, n))
    rhs = fext.reshape(-1).copy()
    for a in atoms:
        for q in range(L):
            row = (idx_a[a] * L + q) * 3
            for j, (nx, ny, nz) in enumerate(itertools.product((-1, 0, 1), repeat=3)):
                if not Kb[j].any():
                    continue
                b, qq = (a[0] + nx, a[1] + ny), (q + nz) % L
                if b in idx_a:
                    col = (idx_a[b] * L + qq) * 3
                    M[row:row + 3, col:col + 3] += Kb[j]
                else:
                    rhs[row:row + 3] -= Kb[j] @ up[idx_p[b], qq]
    return np.linalg.solve(M, rhs).reshape(len(atoms), L, 3)


def test_two_step_convergence(oracle_mod):
    K = harmonic.spring_blocks(1.0, 0.4, 1.0)
    Kb = np.asarray(K).reshape(27, 3, 3)
    atoms, ip, pad = fbc_geometry()
    x0 = (0, 0)
    fext = np.zeros((len(atoms), L, 3))
    fext[atoms.index(x0), :, 0] = np.cos(2 * np.pi * np.arange(L) / L)
    need = sorted({(p[0] - q[0], p[1] - q[1]) for p in pad + atoms for q in ip + [x0]})
    assert (0, 0) in need  # self-terms
    G = harmonic.lattice_kernel_table(K, L, need, N_ZONE)  # real space along the line
    Gd = {d: G[i] for i, d in enumerate(need)}

    def table(d_list):
        return np.stack([Gd[(int(x), int(y))] for x, y in d_list])

    exact = oracle_mod.real_space_update(np.array([x0]), np.array(atoms + pad), L, fext[None, [atoms.index(x0)]],
                                         table, project=False)[0]
    # cross-check: the mode-by-mode form of the same sum
    g = harmonic.lattice_mode_table(K, L, need, list(range(L // 2 + 1)), N_ZONE)
    gk = {d: g[i] for i, d in enumerate(need)}
    cross = oracle_mod.mode_space_update(np.array([x0]), np.array(atoms + pad), L,
                                         fext[None, [atoms.index(x0)]], lambda d: gk[d], project=False)[0]
    assert np.linalg.norm(cross - exact) <= 1e-13 * np.linalg.norm(exact)
    ua_star = exact[:len(atoms)]
    up = np.zeros((len(pad), L, 3))
    errs = []
    for _ in range(3):
        ua = atomistic_solve(Kb, atoms, pad, up, fext)
        errs.append(np.linalg.norm(ua - ua_star) / np.linalg.norm(ua_star))
        fin = harmonic.stencil_apply(ip, [(np.array(atoms), ua[None]), (np.array(pad), up[None])], L, K)
        up = up - oracle_mod.real_space_update(np.array(ip), np.array(pad), L, fin, table, project=False)[0]
    assert errs[0] > 1e-3  # the first atomistic solve, with the pad at rest, is not the solution
    assert errs[1] <= 1e-12 and errs[2] <= 1e-12, errs
