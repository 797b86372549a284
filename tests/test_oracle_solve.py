"""Pins of the oracle's PMCHWT solve (Mie series), GMRES, the OSRC
preconditioner and the Rayleigh incident field."""
import os

import numpy as np
import pytest

from oracle import galerkin, gmres, mie, osrc, pmchwt, rayleigh
from synth import meshes, scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def _gold():
    out = {}
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            out[k] = float(v)
    return out


@pytest.fixture(scope="module")
def sphere_solves():
    out = {}
    for L in (1, 2, 3):
        s = scenes.sphere_scene(L)
        u, A, b = pmchwt.solve(s, pmchwt.plane_wave(s.k0, (0, 0, 1)))
        out[L] = (s, u, A, b)
    return out


def _mie_err(s, u):
    d = s.domains[0]
    uD, uN = pmchwt.split_traces(s, u)[0]
    pts = d.verts / np.linalg.norm(d.verts, axis=1)[:, None]
    eD, eN = mie.surface_traces(pts, 1.0, s.k0, d.k, s.rho0, d.rho)
    M = galerkin.mass_matrix(d.verts, d.tris)

    def rel(a, b):
        e = a - b
        return np.sqrt(np.real(np.conj(e) @ (M @ e)) / np.real(np.conj(b) @ (M @ b)))
    return rel(uD, eD), rel(uN, eN)


def test_mie_convergence(sphere_solves):
    """PMCHWT traces (eq. Form2_calderon_sys_simp3) against the Mie series:
    O(h^2), and below the paper's 3 % at level 3 (about 8 el/lambda)."""
    errs = {L: _mie_err(v[0], v[1]) for L, v in sphere_solves.items()}
    assert max(errs[3]) < _gold()["sphere_field_error_bound_6_el_per_lambda"]
    for L in (1, 2):
        assert errs[L][0] / errs[L + 1][0] > 3.0
        assert errs[L][1] / errs[L + 1][1] > 3.0


def test_mie_series_self_consistency():
    """The series satisfies both transmission conditions of eq. model."""
    a, k0, k1, r0, r1 = 1.0, 5.0, 5.25 + 0.1j, 1.0, 1.1
    n, an, cn = mie.coefficients(a, k0, k1, r0, r1)
    from scipy.special import spherical_jn, spherical_yn
    h = spherical_jn(n, k0 * a) + 1j * spherical_yn(n, k0 * a)
    dh = spherical_jn(n, k0 * a, True) + 1j * spherical_yn(n, k0 * a, True)
    ext = spherical_jn(n, k0 * a) + an * h
    intr = cn * spherical_jn(n, k1 * a)
    assert np.abs(ext - intr).max() < 1e-12
    dext = k0 / r0 * (spherical_jn(n, k0 * a, True) + an * dh)
    dint = k1 / r1 * cn * spherical_jn(n, k1 * a, True)
    assert np.abs(dext - dint).max() < 1e-12


def test_block_assembly_matches_paper_form(sphere_solves):
    """The diagonal block equals A_k0 + D^-1 A_k1 D with the columns
    swapped (Sec. 2.2-2.3)."""
    s, u, A, b = sphere_solves[2]
    d = s.domains[0]
    V0, K0, Kp0, W0 = galerkin.operators(d.verts, d.tris, s.k0)
    V1, K1, Kp1, W1 = galerkin.operators(d.verts, d.tris, d.k)
    r = d.rho / s.rho0
    ref = np.block([[V0 + r * V1, -(K0 + K1)], [Kp0 + Kp1, W0 + W1 / r]])
    assert np.abs(A - ref).max() < 1e-15 * np.abs(ref).max() * 10


def test_gmres_matches_dense_solve(sphere_solves):
    s, u, A, b = sphere_solves[2]
    x, it, hist = gmres.gmres(lambda v: A @ v, b, tol=1e-12, restart=100)
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-9
    x2, it2, _ = gmres.gmres(lambda v: A @ v, b, tol=1e-12, restart=30, maxiter=5000)
    assert np.linalg.norm(x2 - u) / np.linalg.norm(u) < 1e-9


def test_pade_sqrt_closed_form():
    """Rotated Pade approximant against sqrt(1+z): accurate on the real
    axis including z < -1 (evanescent part) where the rotation matters."""
    z = np.concatenate([np.linspace(-4, 4, 41) + 0.05j, np.linspace(-0.9, 3, 20)])
    for N, tol in ((4, 6e-2), (8, 2e-3), (16, 1e-6), (32, 1e-11)):
        err = np.abs(osrc.pade_sqrt(z, N, np.pi / 3) - np.sqrt(1 + z + 0j))
        assert err.max() < tol
    z = np.linspace(-0.5, 2.0, 11)
    assert np.abs(osrc.pade_sqrt(z, 16, np.pi / 3) - np.sqrt(1 + z)).max() < 1e-12


def test_osrc_dtn_on_sphere_harmonics():
    """Discrete DtN (strong form M^-1 C_weak) on spherical harmonics of
    degree n: symbol i k sqrt(1 - n(n+1)/(k_eps^2 a^2)) up to Pade and O(h^2)
    errors (Delta_Gamma Y_n = -n(n+1)/a^2 Y_n)."""
    v, t = meshes.icosphere(3)
    k = 5.0
    P = osrc.DomainOSRC(v, t, k, R_eps=0.5, n_pade=8)
    for n, f in ((1, v[:, 2]), (2, 3 * v[:, 2] ** 2 - 1)):
        y = P.minv(P.dtn_weak(f.astype(complex)))
        sym = 1j * k * osrc.pade_sqrt(-n * (n + 1) / P.keps ** 2, 8, np.pi / 3)
        closed = 1j * k * np.sqrt(1 - n * (n + 1) / P.keps ** 2)
        assert abs(sym - closed) / abs(closed) < 2e-3
        assert np.linalg.norm(y - sym * f) / np.linalg.norm(sym * f) < 2e-2


def _harmonics(v):
    z = v[:, 2] / np.linalg.norm(v, axis=1)
    return ((1, z), (2, 3 * z ** 2 - 1), (3, 5 * z ** 3 - 3 * z))


def ntd_symbol(n, P, n_pade=8, theta=np.pi / 3):
    """(i k)^-1 R(X) / (1 + X) on degree-n harmonics of the unit sphere,
    X = -n(n+1)/k_eps^2, R the rotated Pade square root: the NtD map of
    eq. OSRC_DtN_NtD_maps with the (1+X)^-1 sqrt(1+X) reading."""
    X = -n * (n + 1) / P.keps ** 2
    return osrc.pade_sqrt(X, n_pade, theta) / (1 + X) / (1j * P.k)


def dtn_symbol(n, P, n_pade=8, theta=np.pi / 3):
    return 1j * P.k * osrc.pade_sqrt(-n * (n + 1) / P.keps ** 2, n_pade, theta)


def _ntd_errors(ntd, L, k=5.0):
    v, t = meshes.icosphere(L)
    P = osrc.DomainOSRC(v, t, k, R_eps=0.5, n_pade=8)
    out = []
    for n, f in _harmonics(v):
        sym = ntd_symbol(n, P)
        y = ntd(P, f.astype(complex))
        out.append(np.linalg.norm(y - sym * f) / np.linalg.norm(sym * f))
    return np.array(out)


def test_osrc_ntd_on_sphere_harmonics():
    """Discrete NtD (strong form (ik)^-1 (M - S/k_eps^2)^-1 [C0 M u - ...]) on
    spherical harmonics of degree 1..3 against its symbol
    (ik)^-1 R(X)/(1+X), X = -n(n+1)/k_eps^2, converging at O(h^2); the
    symbol itself is within the Pade error of the closed form
    (ik)^-1 (1+X)^-1/2.  Planted mistakes fail: the (M - S/k_eps^2)^-1 dropped,
    or the sign of S/k_eps^2 flipped."""
    import scipy.sparse.linalg as spla
    errs = {L: _ntd_errors(lambda P, f: P.ntd_strong(f), L) for L in (2, 3, 4)}
    assert errs[4].max() < 3e-3
    for L in (2, 3):
        assert (errs[L] / errs[L + 1]).min() > 3.5
    v, t = meshes.icosphere(2)
    P = osrc.DomainOSRC(v, t, 5.0, R_eps=0.5, n_pade=8)
    for n in (1, 2, 3):
        closed = 1 / (1j * P.k * np.sqrt(1 - n * (n + 1) / P.keps ** 2))
        assert abs(ntd_symbol(n, P) - closed) / abs(closed) < 3e-3

    def dropped(P, f):
        return P.bracket(f) / (1j * P.k)

    def flipped(P, f):
        return spla.splu((P.M + P.S / P.keps ** 2).astype(complex).tocsc()).solve(P.bracket(f)) / (1j * P.k)
    assert _ntd_errors(dropped, 3).min() > 0.5
    assert _ntd_errors(flipped, 3).min() > 0.1


def test_osrc_composition_on_sphere_harmonics():
    """osrc.apply on Galerkin rows [M f; M g] of one sphere: the DtN acts on
    the V row and the NtD on the W row (eq. OSRC_prec_blocks with the column
    permutation of Sec. 2.3), giving [DtN_n f; NtD_n g] up to O(h^2); the
    roles swapped fail."""
    res = {}
    for L in (2, 3):
        s = scenes.sphere_scene(L, k0=5.0)
        d = s.domains[0]
        pre = osrc.build(s, R_eps=0.5, n_pade=8)
        P = pre[0]
        M = galerkin.mass_matrix(d.verts, d.tris)
        e, e_swapped = [], []
        for (n, f), (m, g) in zip(_harmonics(d.verts), _harmonics(d.verts)[::-1]):
            y = osrc.apply(s, pre, np.concatenate([M @ f, M @ g]).astype(complex))
            ref = np.concatenate([dtn_symbol(n, P) * f, ntd_symbol(m, P) * g])
            e.append(np.linalg.norm(y - ref) / np.linalg.norm(ref))
            swapped = np.concatenate([ntd_symbol(n, P) * f, dtn_symbol(m, P) * g])
            e_swapped.append(np.linalg.norm(y - swapped) / np.linalg.norm(swapped))
        res[L] = np.array(e)
        assert min(e_swapped) > 0.5
    assert res[3].max() < 0.01
    assert (res[2] / res[3]).min() > 3.0


def test_preconditioned_gmres_same_solution_fewer_iterations(sphere_solves):
    s, u, A, b = sphere_solves[3]
    pre = osrc.build(s, R_eps=0.1, n_pade=4)
    x0, it0, _ = gmres.gmres(lambda v: A @ v, b, tol=1e-8, restart=100)
    x1, it1, _ = gmres.gmres(lambda v: osrc.apply(s, pre, A @ v), osrc.apply(s, pre, b), tol=1e-8, restart=100)
    assert np.linalg.norm(x1 - u) / np.linalg.norm(u) < 1e-6
    assert it1 * 4 < it0


def test_rayleigh_piston_on_axis():
    """Baffled piston on its axis: |p| = 2 rho c u0 |sin(k (sqrt(z^2+a^2) - z)/2)|."""
    tr = {"centres": np.array([[0, 0, 0.0]]), "normals": np.array([[0, 0, 1.0]]), "radii": np.array([3e-3])}
    k0 = 2 * np.pi * 1e6 / 1500
    f = rayleigh.field(tr, [1.0], k0, 2 * np.pi * 1e6, 1000.0, n_r=24, n_t=16)
    z = np.array([0.005, 0.01, 0.05, 0.1])
    p, dp = f(np.stack([0 * z, 0 * z, z], 1), np.tile([0, 0, 1.0], (4, 1)))
    ex = 2 * 1000 * 1500 * np.abs(np.sin(k0 * (np.sqrt(z ** 2 + 3e-3 ** 2) - z) / 2))
    assert np.abs(np.abs(p) - ex).max() / ex.max() < 1e-10
    # d/dz of the on-axis closed form rho c (e^{ikz} - e^{ik sqrt(z^2+a^2)})
    a = 3e-3
    R1 = np.sqrt(z ** 2 + a ** 2)
    dex = 1000 * 1500 * (1j * k0 * np.exp(1j * k0 * z) - 1j * k0 * z / R1 * np.exp(1j * k0 * R1))
    assert np.abs(dp - dex).max() / np.abs(dex).max() < 1e-9
