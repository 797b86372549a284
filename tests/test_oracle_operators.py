"""Pins of the oracle's Galerkin operators on closed surfaces: symmetry,
sphere eigenvalues and the Calderon identities (App. A)."""
import numpy as np
import pytest

from oracle import galerkin, mie, pmchwt
from synth import meshes


@pytest.fixture(scope="module")
def sphere_ops():
    out = {}
    for L in (2, 3):
        v, t = meshes.icosphere(L)
        out[L] = (v, t, galerkin.operators(v, t, 2.0 + 0.3j), galerkin.mass_matrix(v, t).toarray())
    return out


def test_symmetries(sphere_ops):
    """Galerkin matrices with the same rule on both sides: V and W are
    complex symmetric, K' is the transpose of K (to quadrature round-off of
    the non-symmetric singular maps)."""
    v, t, (V, K, Kp, W), M = sphere_ops[2]
    s = np.abs(V).max()
    assert np.abs(V - V.T).max() < 1e-7 * s
    assert np.abs(W - W.T).max() < 1e-7 * np.abs(W).max()
    assert np.abs(Kp - K.T).max() < 1e-6 * np.abs(K).max()


def test_sphere_eigenvalues_converge(sphere_ops):
    """V, K, K', W applied to spherical harmonics of degree 1..3 against the
    closed-form eigenvalues (addition theorem); error O(h^2)."""
    errs = {}
    for L in (2, 3):
        v, t, (V, K, Kp, W), M = sphere_ops[L]
        e = []
        for n, f in ((1, v[:, 2]), (2, 3 * v[:, 2] ** 2 - 1), (3, 5 * v[:, 2] ** 3 - 3 * v[:, 2])):
            Vn, Kn, Wn = mie.sphere_eigenvalues(n, 2.0 + 0.3j, 1.0)
            for A, lam in ((V, Vn), (K, Kn), (Kp, Kn), (W, Wn)):
                y = np.linalg.solve(M, A @ f)
                e.append(np.linalg.norm(y - lam * f) / np.linalg.norm(lam * f))
        errs[L] = np.array(e)
    assert errs[3].max() < 0.04
    assert (errs[2] / errs[3]).min() > 2.8  # ~4x per halving of h


def test_calderon_identities(sphere_ops):
    """Interior (plane wave): A gamma u = +1/2 gamma u; exterior radiating
    (point source inside): A gamma u = -1/2 gamma u (eqs. Cald_formula_int,
    Cald_formula_ext0); and the projector property A^2 = I/4, all tested in
    the mass-matrix (strong) form and converging at O(h^2)."""
    res = {}
    k = 2.0 + 0.3j
    for L in (2, 3):
        v, t, (V, K, Kp, W), M = sphere_ops[L]
        nv = v / np.linalg.norm(v, axis=1)[:, None]
        A = pmchwt.calderon_block(V, K, Kp, W)
        Mb = np.kron(np.eye(2), M)
        d = np.array([0.3, 0.4, 0.866])
        d /= np.linalg.norm(d)
        uD = np.exp(1j * k * (v @ d))
        x_in = np.concatenate([uD, 1j * k * (nv @ d) * uD])
        xs = np.array([0.2, -0.1, 0.3])
        dd = v - xs
        r = np.linalg.norm(dd, axis=1)
        g = np.exp(1j * k * r) / (4 * np.pi * r)
        x_out = np.concatenate([g, g * (1j * k - 1 / r) * np.einsum("ij,ij->i", dd, nv) / r])
        P = np.linalg.solve(Mb, A)
        res[L] = (np.linalg.norm(A @ x_in - 0.5 * Mb @ x_in) / np.linalg.norm(Mb @ x_in),
                  np.linalg.norm(A @ x_out + 0.5 * Mb @ x_out) / np.linalg.norm(Mb @ x_out),
                  np.linalg.norm(P @ (P @ x_out) - 0.25 * x_out) / np.linalg.norm(x_out))
    assert max(res[3]) < 6e-3
    for a, b in zip(res[2], res[3]):
        assert a / b > 3.0


def test_laplace_gauss_identity_sphere():
    """k = 0: K_h 1 -> -1/2 M 1 on a closed surface (solid angle)."""
    v, t = meshes.icosphere(2)
    V, K, Kp, W = galerkin.operators(v, t, 0.0)
    M = galerkin.mass_matrix(v, t).toarray()
    e = np.abs(K.sum(1) + 0.5 * M.sum(1)).max() / np.abs(M.sum(1)).max()
    assert e < 2e-3
    assert np.abs(W.sum(1)).max() < 1e-12 * np.abs(W).max()
