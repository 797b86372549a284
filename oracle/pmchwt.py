"""Multiple-domain PMCHWT system of the paper, FP64, dense (test
infrastructure only).

Follows Sec. 2.2-2.3 in the paper's notation:

* Calderon operator of one (test j, trial i) block at wavenumber k
  (App. A, Sec. 2.2):  A_k^{ji} = [[-K, V], [W, K']]  acting on
  [gamma_D; gamma_N] (paper order [phi; psi]);
* density map D_j = diag(I, rho_j/rho_0), tilde A = D_j^{-1} A D_j
  (eq. Form1_BCs, Form1_calderon_sys_int_ptot);
* block system (eq. Form2_matrix_format_p1/_p2):
  [A_hat]_{jj} = A^j_{k0} + tilde A^j_{kj},  [A_hat]_{ji} = A^{ji}_{k0},
  u_j = gamma^{j,+} p_tot,  b_j = gamma^{j,+} p_inc, Galerkin-tested with
  P1 functions (eq. Galerkin_disc_lhs/_rhs1);
* the column permutation of Sec. 2.3 (reading: the unknown blocks are
  swapped to [psi; phi] = [gamma_N; gamma_D] so that V and W sit on the
  diagonal; the rows, hence the right-hand side, are unchanged).

System order used everywhere: per domain j, unknowns [psi_j (nv_j); phi_j
(nv_j)] and rows [row1_j; row2_j], domains concatenated.
"""
from __future__ import annotations

import numpy as np

from . import galerkin


def offsets(scene):
    off = [0]
    for d in scene.domains:
        off.append(off[-1] + 2 * d.verts.shape[0])
    return off


def calderon_block(V, K, Kp, W):
    """Paper order [[-K, V], [W, K']] as a dense 2x2 block matrix."""
    return np.block([[-K, V], [W, Kp]])


def density_map(nv, ratio):
    return np.concatenate([np.ones(nv), np.full(nv, ratio)])


def assemble(scene, rules=None, return_blocks=False):
    """Dense A_hat in system order (permuted columns)."""
    n = offsets(scene)
    N = n[-1]
    A = np.zeros((N, N), dtype=np.complex128)
    blocks = {}
    for j, dj in enumerate(scene.domains):
        for i, di in enumerate(scene.domains):
            same = i == j
            ops0 = galerkin.operator_rows(dj.verts, dj.tris, di.verts, di.tris, same, scene.k0, None, rules)
            Bji = calderon_block(*ops0)
            if same:
                opsj = galerkin.operator_rows(dj.verts, dj.tris, dj.verts, dj.tris, True, dj.k, None, rules)
                Aj = calderon_block(*opsj)
                dmap = density_map(dj.verts.shape[0], dj.rho / scene.rho0)
                Bji = Bji + (Aj * dmap[None, :]) / dmap[:, None]  # D^-1 A D
                blocks[("int", j)] = opsj
            blocks[("ext", j, i)] = ops0
            A[n[j]:n[j + 1], n[i]:n[i + 1]] = permute_columns(Bji, di.verts.shape[0])
    return (A, blocks) if return_blocks else A


def permute_columns(B, nv):
    """Paper column order [phi; psi] -> system order [psi; phi]."""
    return np.concatenate([B[:, nv:], B[:, :nv]], axis=1)


def apply_rows(scene, x, rows_per_domain, rules=None):
    """Selected rows of A_hat x without forming A_hat (for large scenes).
    rows_per_domain[j]: test vertex indices of domain j; returns, per
    domain, (row1, row2) values at those vertices."""
    n = offsets(scene)
    out = []
    for j, dj in enumerate(scene.domains):
        rows = np.asarray(rows_per_domain[j])
        r1 = np.zeros(rows.size, dtype=np.complex128)
        r2 = np.zeros(rows.size, dtype=np.complex128)
        if rows.size == 0:
            out.append((r1, r2))
            continue
        for i, di in enumerate(scene.domains):
            nvi = di.verts.shape[0]
            psi = x[n[i]:n[i] + nvi]
            phi = x[n[i] + nvi:n[i + 1]]
            V, K, Kp, W = galerkin.operator_rows(dj.verts, dj.tris, di.verts, di.tris, i == j, scene.k0, rows, rules)
            r1 += V @ psi - K @ phi
            r2 += W @ phi + Kp @ psi
            if i == j:
                rj = dj.rho / scene.rho0
                V, K, Kp, W = galerkin.operator_rows(dj.verts, dj.tris, dj.verts, dj.tris, True, dj.k, rows, rules)
                r1 += rj * (V @ psi) - K @ phi
                r2 += (W @ phi) / rj + Kp @ psi
        out.append((r1, r2))
    return out


def mass_block(scene):
    """Block-diagonal P1 mass matrix in system order (dense)."""
    n = offsets(scene)
    M = np.zeros((n[-1], n[-1]))
    for j, d in enumerate(scene.domains):
        nv = d.verts.shape[0]
        Mj = galerkin.mass_matrix(d.verts, d.tris).toarray()
        M[n[j]:n[j] + nv, n[j]:n[j] + nv] = Mj
        M[n[j] + nv:n[j + 1], n[j] + nv:n[j + 1]] = Mj
    return M


# ---------------------------------------------------------------- incident field / RHS


def plane_wave(k0, direction, amp=1.0):
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)

    def f(x, n):
        p = amp * np.exp(1j * k0 * (x @ d))
        return p, 1j * k0 * (n @ d) * p
    return f


def rhs(scene, field):
    """b = [<gamma_D p_inc, phi_r>; <gamma_N p_inc, phi_r>] per domain, by
    the regular rule (eq. Galerkin_disc_rhs1)."""
    out = []
    for d in scene.domains:
        x, wa, phi = galerkin.quad_points(d.verts, d.tris)
        nrm, _ = galerkin.tri_geometry(d.verts, d.tris)
        nt, nq = x.shape[0], x.shape[1]
        p, dp = field(x.reshape(-1, 3), np.repeat(nrm, nq, axis=0))
        bD = galerkin.project(d.verts, d.tris, p.reshape(nt, nq))
        bN = galerkin.project(d.verts, d.tris, dp.reshape(nt, nq))
        out.append(np.concatenate([bD, bN]))
    return np.concatenate(out)


def solve(scene, field, rules=None):
    A = assemble(scene, rules)
    b = rhs(scene, field)
    return np.linalg.solve(A, b), A, b


def split_traces(scene, u):
    """Per domain (gamma_D p_tot, gamma_N^+ p_tot) at the vertices."""
    n = offsets(scene)
    out = []
    for j, d in enumerate(scene.domains):
        nv = d.verts.shape[0]
        out.append((u[n[j] + nv:n[j + 1]], u[n[j]:n[j] + nv]))
    return out
