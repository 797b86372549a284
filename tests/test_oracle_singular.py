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


# A near pair: no common vertex, centroids 1.2 apart against a longest edge of
# about 1.06 (threshold: twice the longest edge of either triangle).
NEAR_Y = np.array([[1.25, 0.35, 0.15], [2.1, 0.2, -0.2], [1.6, 1.1, 0.3]])


def _regular_6x6(PX, PY, k):
    """The 6-point rule on both triangles, written out in numpy (V and K')."""
    l1, l2, w = quadrature.triangle_rule6()

    def pts(P):
        A = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
        x = P[0] + l1[:, None] * (P[1] - P[0]) + l2[:, None] * (P[2] - P[0])
        phi = np.stack([1 - l1 - l2, l1, l2], 1)
        n = np.cross(P[1] - P[0], P[2] - P[0])
        return x, phi, w * A, n / np.linalg.norm(n)
    x, px, wx, nx = pts(PX)
    y, py, wy, _ = pts(PY)
    d = x[:, None, :] - y[None, :, :]
    r = np.linalg.norm(d, axis=2)
    G = np.exp(1j * k * r) / (4 * np.pi * r)
    dGnx = G * (1j * k - 1 / r) / r * (d @ nx)
    V = np.einsum("a,b,ab,ai,bj->ij", wx, wy, G, px, py)
    Kp = np.einsum("a,b,ab,ai,bj->ij", wx, wy, dGnx, px, py)
    return V, Kp


def test_near_pair_rule(orc):
    """Near pairs (no common vertex, centroid distance under twice the longer
    longest edge) use the collapsed Gauss-Legendre rule on both triangles:
    detected as relation 4; against the independent brute-force integral to
    its accuracy; converged in n (6 vs 24 points per direction); and more
    accurate than the 6-point rule on the same pair."""
    k = 3.0 + 0.5j
    m6, rel = orc.pair(P, [0, 1, 2], NEAR_Y, [3, 4, 5], True, k)
    assert rel == 4
    far, rel_far = orc.pair(P, [0, 1, 2], NEAR_Y + np.array([2.5, 0.0, 0.0]), [3, 4, 5], True, k)
    assert rel_far == 0  # beyond twice the longest edge: the regular rule
    ref, _ = orc.pair(P, [0, 1, 2], NEAR_Y, [3, 4, 5], True, k, orc.Rules(n_gauss=24))
    B = _brute.pair_matrices(P, NEAR_Y, k, levels=3, n_out=8, n_in=20)
    for o in range(4):
        s = np.abs(ref[o]).max()
        assert np.abs(ref[o] - B[o]).max() <= 1e-4 * s, o
        assert np.abs(m6[o] - ref[o]).max() <= 1e-5 * s, o
    V6, Kp6 = _regular_6x6(P, NEAR_Y, k)
    e_reg = max(np.abs(V6 - ref[0]).max() / np.abs(ref[0]).max(), np.abs(Kp6 - ref[2]).max() / np.abs(ref[2]).max())
    e_near = max(np.abs(m6[0] - ref[0]).max() / np.abs(ref[0]).max(), np.abs(m6[2] - ref[2]).max() / np.abs(ref[2]).max())
    assert e_near * 30 < e_reg, (e_near, e_reg)
    # a cross-surface pair (different meshes) takes the same rule
    mx, relx = orc.pair(P, [0, 1, 2], NEAR_Y, [0, 1, 2], False, k)
    assert relx == 4 and max(np.abs(mx[o] - m6[o]).max() for o in range(4)) == 0.0
