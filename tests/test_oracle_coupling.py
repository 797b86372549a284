"""Pins of the oracle's multiple-domain coupling: the off-diagonal blocks
A^{ji}_{k0} of the PMCHWT system (Sec. 2.2 eqs. Form2_matrix_format_p1/_p2)
and the diagonal blocks of several domains, against results that do not come
from the oracle's own blocks.

* A point source G(x - x_s) with x_s inside sphere i is a radiating solution
  of the exterior problem.  On the other sphere j it is regular inside, so
  the interior Calderon identity gives A^{jj} gamma^j G = +1/2 gamma^j G,
  and the exterior identity over both surfaces, sum_i A^{ji} gamma^i G =
  -1/2 gamma^j G, then leaves A^{ji}_{k0} gamma^i G = -gamma^j G (App. A eqs.
  Cald_formula_int, Cald_formula_ext0): the off-diagonal block maps the
  closed-form Cauchy data on one sphere to minus those on the other.  A
  flipped sign, the target's normal in place of the source's, or a block
  placed at the wrong (row, column) position all fail it.
* Transparent inclusions (k_j = k0, rho_j = rho0): the total field is the
  incident wave, so the solution is u = gamma p_inc on every surface.
* The solved two-sphere field: its scattered part is radiating in Omega^0
  (exterior identity over both surfaces) and its interior traces satisfy
  each domain's interior identity (with the density map of eq. Form1_BCs).
  This one uses the oracle's blocks on both sides and is a consistency check
  of the solve; the point-source pin is the independent one.

All identities are tested in the Galerkin (mass-matrix) form and converge at
O(h^2).  Rows keep the paper's order [Dirichlet row; Neumann row] while the
unknowns are [psi; phi] (Sec. 2.3 column permutation), so a row block is
compared with M gamma_D and the next with M gamma_N.
"""
import numpy as np
import pytest

from oracle import galerkin, pmchwt
from synth import meshes, scenes

CENTRES = (np.array([-1.3, 0.0, 0.0]), np.array([1.2, 0.1, 0.0]))  # of scenes.two_sphere_scene
LEVELS = (1, 2, 3)


@pytest.fixture(scope="module")
def two_spheres():
    out = {}
    for L in LEVELS:
        s = scenes.two_sphere_scene(L)
        A, blocks = pmchwt.assemble(s, return_blocks=True)
        out[L] = (s, A, blocks)
    return out


def _normals(v, c):
    d = v - c
    return d / np.linalg.norm(d, axis=1)[:, None]


def _point_source(v, nrm, xs, k):
    """Closed-form Cauchy data of exp(ik|x - xs|)/(4 pi |x - xs|) at v."""
    d = v - xs
    r = np.linalg.norm(d, axis=1)
    g = np.exp(1j * k * r) / (4 * np.pi * r)
    return g, g * (1j * k - 1 / r) * np.einsum("ij,ij->i", d, nrm) / r


def _rows_vs(M, dirichlet, neumann):
    """Galerkin rows [M gamma_D; M gamma_N] of Cauchy data."""
    return np.concatenate([M @ dirichlet, M @ neumann])


def offdiag_point_source_errors(s, A):
    """Relative error of A^{ji} gamma^i G = -gamma^j G for both ordered pairs,
    with the source inside sphere i (A: the assembled system)."""
    n = pmchwt.offsets(s)
    errs = []
    for i, j in ((0, 1), (1, 0)):
        di, dj = s.domains[i], s.domains[j]
        xs = CENTRES[i] + np.array([0.2, -0.1, 0.3]) * (1.0 if i == 0 else 0.6)
        gD, gN = _point_source(di.verts, _normals(di.verts, CENTRES[i]), xs, s.k0)
        hD, hN = _point_source(dj.verts, _normals(dj.verts, CENTRES[j]), xs, s.k0)
        Mj = galerkin.mass_matrix(dj.verts, dj.tris)
        got = A[n[j]:n[j + 1], n[i]:n[i + 1]] @ np.concatenate([gN, gD])  # system order [psi; phi]
        ref = -_rows_vs(Mj, hD, hN)
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return np.array(errs)


def test_off_diagonal_blocks_reproduce_a_point_source(two_spheres):
    errs = {L: offdiag_point_source_errors(s, A) for L, (s, A, _) in two_spheres.items()}
    assert errs[3].max() < 0.03
    assert (errs[1] / errs[2]).min() > 2.8  # O(h^2); level 1 (42 vertices) is not yet asymptotic
    assert (errs[2] / errs[3]).min() > 3.3
    # planted mistakes fail the pin: flipped off-diagonal sign, blocks swapped
    s, A, _ = two_spheres[3]
    n = pmchwt.offsets(s)
    flipped = A.copy()
    flipped[n[0]:n[1], n[1]:n[2]] *= -1
    flipped[n[1]:n[2], n[0]:n[1]] *= -1
    assert offdiag_point_source_errors(s, flipped).min() > 1.5
    swapped = A.copy()  # the two spheres have equal vertex counts, so the blocks can trade places
    swapped[n[0]:n[1], n[1]:n[2]] = A[n[1]:n[2], n[0]:n[1]]
    swapped[n[1]:n[2], n[0]:n[1]] = A[n[0]:n[1], n[1]:n[2]]
    assert offdiag_point_source_errors(s, swapped).min() > 0.5


def _transparent_scene(level, k0=4.0):
    """Three disjoint spheres whose material equals the exterior medium."""
    s = scenes.Scene(name=f"transparent_L{level}", k0=complex(k0), rho0=1.0, plane_wave_dir=(0.3, 0.5, 0.8))
    for c, r in (((-1.3, 0.0, 0.0), 1.0), ((1.2, 0.1, 0.0), 0.8), ((0.0, 1.9, 0.4), 0.6)):
        v, t = meshes.icosphere(level, r, c)
        s.domains.append(scenes.Domain(f"s{len(s.domains)}", v, t, complex(k0), 1.0))
        s.meta.setdefault("spheres", []).append((np.array(c), r))
    return s


def test_transparent_inclusions_give_the_incident_traces():
    """k_j = k0 and rho_j = rho0 on three spheres: the dense solve converges
    to u = gamma p_inc (psi = d p_inc / dn, phi = p_inc) at O(h^2)."""
    errs = {}
    for L in (1, 2):
        s = _transparent_scene(L)
        dvec = np.asarray(s.plane_wave_dir) / np.linalg.norm(s.plane_wave_dir)
        u, A, b = pmchwt.solve(s, pmchwt.plane_wave(s.k0, dvec))
        num = den = 0.0
        n = pmchwt.offsets(s)
        for j, (d, (c, _)) in enumerate(zip(s.domains, s.meta["spheres"])):
            nv = d.verts.shape[0]
            p = np.exp(1j * s.k0 * (d.verts @ dvec))
            ex = np.concatenate([1j * s.k0 * (_normals(d.verts, c) @ dvec) * p, p])
            M = galerkin.mass_matrix(d.verts, d.tris)
            e = u[n[j]:n[j + 1]] - ex
            for part in (slice(0, nv), slice(nv, 2 * nv)):
                num += np.real(np.conj(e[part]) @ (M @ e[part]))
                den += np.real(np.conj(ex[part]) @ (M @ ex[part]))
        errs[L] = np.sqrt(num / den)
    assert errs[2] < 0.08
    assert errs[1] / errs[2] > 2.8


def _swap_halves(s, x):
    """Per domain [a; b] -> [b; a] (unknown order -> row order of its traces)."""
    n = pmchwt.offsets(s)
    out = np.empty_like(x)
    for j, d in enumerate(s.domains):
        nv = d.verts.shape[0]
        out[n[j]:n[j] + nv] = x[n[j] + nv:n[j + 1]]
        out[n[j] + nv:n[j + 1]] = x[n[j]:n[j] + nv]
    return out


def test_multi_domain_solve_consistency(two_spheres):
    """Two spheres of different materials: the dense solution satisfies the
    system; its scattered part u - gamma p_inc satisfies the exterior
    Calderon identity over both surfaces, A_k0 (u - gamma p_inc) =
    -1/2 M (u - gamma p_inc) with every (j, i) block at k0; and each domain's
    interior traces D_j u_j satisfy the interior identity of A_kj
    (eq. Form1_calderon_sys_int_ptot).  All three converge at O(h^2)."""
    res = {}
    for L in (2, 3):
        s, A, blocks = two_spheres[L]
        n = pmchwt.offsets(s)
        N = n[-1]
        dvec = np.asarray(s.plane_wave_dir) / np.linalg.norm(s.plane_wave_dir)
        b = pmchwt.rhs(s, pmchwt.plane_wave(s.k0, dvec))
        u = np.linalg.solve(A, b)
        assert np.linalg.norm(A @ u - b) / np.linalg.norm(b) < 1e-12
        inc, Ms = [], []
        A_ext = np.zeros((N, N), dtype=np.complex128)
        for j, d in enumerate(s.domains):
            p = np.exp(1j * s.k0 * (d.verts @ dvec))
            inc.append(np.concatenate([1j * s.k0 * (_normals(d.verts, CENTRES[j]) @ dvec) * p, p]))
            Ms.append(galerkin.mass_matrix(d.verts, d.tris))
            for i, di in enumerate(s.domains):
                A_ext[n[j]:n[j + 1], n[i]:n[i + 1]] = pmchwt.permute_columns(
                    pmchwt.calderon_block(*blocks[("ext", j, i)]), di.verts.shape[0])

        def mass(x):
            return np.concatenate([np.concatenate([M @ x[n[j]:n[j] + d.verts.shape[0]],
                                                   M @ x[n[j] + d.verts.shape[0]:n[j + 1]]])
                                   for j, (d, M) in enumerate(zip(s.domains, Ms))])
        sc = u - np.concatenate(inc)
        e_ext = np.linalg.norm(A_ext @ sc + 0.5 * mass(_swap_halves(s, sc))) / np.linalg.norm(mass(sc))
        e_int = []
        for j, d in enumerate(s.domains):
            nv = d.verts.shape[0]
            dm = pmchwt.density_map(nv, d.rho / s.rho0)
            At = pmchwt.permute_columns((pmchwt.calderon_block(*blocks[("int", j)]) * dm[None, :]) / dm[:, None], nv)
            uj = u[n[j]:n[j + 1]]
            ref = 0.5 * np.concatenate([Ms[j] @ uj[nv:], Ms[j] @ uj[:nv]])
            e_int.append(np.linalg.norm(At @ uj - ref) / np.linalg.norm(ref))
        res[L] = np.array([e_ext] + e_int)
    assert res[3].max() < 0.05
    assert (res[2] / res[3]).min() > 3.0
