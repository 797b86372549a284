"""Pins of the oracle's element-pair integrals (regular and Sauter-Schwab)
against brute force and exact identities of the potentials."""
import numpy as np
import pytest

from oracle import quadrature
from synth import meshes

import _brute

P = np.array([[0, 0, 0], [1.0, 0.1, 0], [0.3, 0.9, 0]])
CASES = {
    "identical": (P, [0, 1, 2], P, [0, 1, 2], 3),
    "edge_coplanar": (P, [0, 1, 2], np.array([[0, 0, 0], [0.8, -0.9, 0], [1.0, 0.1, 0]]), [0, 3, 1], 2),
    "edge_bent": (P, [0, 1, 2], np.array([[0, 0, 0], [0.7, -0.6, 0.5], [1.0, 0.1, 0]]), [0, 3, 1], 2),
    "vertex": (P, [0, 1, 2], np.array([[0.3, 0.9, 0], [-0.5, 1.2, 0.4], [-0.6, 0.4, -0.3]]), [2, 4, 5], 1),
}


@pytest.mark.parametrize("name", ["identical", "edge_bent", "vertex"])
def test_single_layer_and_hypersingular_vs_brute_force(orc, name):
    """V and W (Maue form) of touching pairs against a brute-force integral
    (Duffy-split inner integral, subdivided outer rule): independent of the
    Sauter-Schwab maps.  The brute force is accurate to ~1e-4 here."""
    PX, ix, PY, iy, rel = CASES[name]
    k = 3.0 + 0.5j
    M, r = orc.pair(PX, ix, PY, iy, True, k, orc.Rules(n_gauss=10))
    assert r == rel
    B = _brute.pair_matrices(PX, PY, k, levels=3, n_out=8, n_in=20)
    for o in (0, 3):
        assert np.abs(M[o] - B[o]).max() <= 2e-4 * np.abs(B[o]).max(), o


@pytest.mark.parametrize("name", ["identical", "edge_bent", "vertex"])
def test_sauter_schwab_converges_exponentially(orc, name):
    """A valid cover (previous file) that converges in n integrates the
    singular kernel correctly; at the default n = 6 it is within 1e-5."""
    PX, ix, PY, iy, rel = CASES[name]
    k = 3.0 + 0.5j
    ref, _ = orc.pair(PX, ix, PY, iy, True, k, orc.Rules(n_gauss=16))
    m6, _ = orc.pair(PX, ix, PY, iy, True, k, orc.Rules(n_gauss=6))
    m10, _ = orc.pair(PX, ix, PY, iy, True, k, orc.Rules(n_gauss=10))
    for o in range(4):
        s = max(np.abs(ref[o]).max(), 1e-300)
        assert np.abs(m10[o] - ref[o]).max() < 1e-9 * s + 1e-300
        assert np.abs(m6[o] - ref[o]).max() < 1e-5 * s + 1e-300


def test_regular_pair_vs_high_order(orc):
    """Far pair: the 6-point rule on both triangles against a converged
    high-order rule (error bound of a degree-4 rule at distance 4)."""
    PX = P
    PY = P + np.array([3.0, 2.0, 1.5])
    k = 2.0 + 0.2j
    lo, r = orc.pair(PX, [0, 1, 2], PY, [3, 4, 5], True, k)
    assert r == 0
    hi, _ = orc.pair(PX, [0, 1, 2], PY, [3, 4, 5], True, k, orc.Rules(quadrature.collapsed_gauss_rule(12)))
    for o in range(4):
        assert np.abs(lo[o] - hi[o]).max() < 1e-3 * np.abs(hi[o]).max()


def test_gauss_solid_angle_identity_octahedron(orc):
    """Laplace double layer on a closed polyhedron: the potential of a unit
    density is exactly -1/2 on every face, so K_h 1 = -1/2 M 1 (App. A jump
    relations with the outward normal).  Every touching pair of the
    octahedron uses the singular rules (edge and vertex cases); the one
    non-touching pair per face gets a converged high-order rule."""
    v, t = meshes.octahedron()
    rules = orc.Rules(quadrature.collapsed_gauss_rule(20), n_gauss=8)
    V, K, Kp, W = orc.operators(v, t, 0.0, rules)
    M = orc.mass_matrix(v, t).toarray()
    assert np.abs(K.sum(1) + 0.5 * M.sum(1)).max() < 1e-8
    assert np.abs(W.sum(1)).max() < 1e-14
    assert np.abs(Kp - K.T).max() < 1e-7


def test_gauss_identity_tetrahedron(orc):
    """Every pair of faces of a tetrahedron shares an edge: K_h 1 = -1/2 M 1
    exercises the edge case alone (sharp 70.5 degree dihedral angles)."""
    v, t = meshes.tetrahedron()
    V, K, Kp, W = orc.operators(v, t, 0.0, orc.Rules(n_gauss=12))
    M = orc.mass_matrix(v, t).toarray()
    assert np.abs(K.sum(1) + 0.5 * M.sum(1)).max() < 1e-8
