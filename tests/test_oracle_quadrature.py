"""Pins of the oracle's quadrature rules against exact integrals."""
import math

import numpy as np
import pytest

from oracle import quadrature


def _exact_bary(i, j, k):
    # mean over the triangle of l1^i l2^j l3^k = 2 i! j! k! / (i+j+k+2)!
    return 2.0 * math.factorial(i) * math.factorial(j) * math.factorial(k) / math.factorial(i + j + k + 2)


def test_rule6_exact_to_degree_4():
    l1, l2, w = quadrature.triangle_rule6()
    assert l1.size == 6
    assert abs(w.sum() - 1.0) < 1e-15
    l0 = 1 - l1 - l2
    for i in range(5):
        for j in range(5 - i):
            for k in range(5 - i - j):
                q = np.sum(w * l0 ** i * l1 ** j * l2 ** k)
                assert abs(q - _exact_bary(i, j, k)) < 1e-15, (i, j, k)


def test_rule6_not_degree_5():
    # a degree-4 rule must fail on some degree-5 monomial (guards against a
    # degenerate table that happens to satisfy the invariant moments only)
    l1, l2, w = quadrature.triangle_rule6()
    l0 = 1 - l1 - l2
    errs = [abs(np.sum(w * l0 ** i * l1 ** (5 - i)) - _exact_bary(i, 5 - i, 0)) for i in range(6)]
    assert max(errs) > 1e-6


def test_rule6_points_inside_and_symmetric():
    l1, l2, w = quadrature.triangle_rule6()
    l0 = 1 - l1 - l2
    assert (l0 > 0).all() and (l1 > 0).all() and (l2 > 0).all()
    pts = sorted(tuple(sorted(p)) for p in zip(l0.round(14), l1.round(14), l2.round(14)))
    assert len(set(pts)) == 2  # two S3 orbits


def test_gauss_legendre01():
    g = quadrature.gauss_legendre01(6)
    for p in range(12):
        assert abs(np.sum(g[:, 1] * g[:, 0] ** p) - 1.0 / (p + 1)) < 1e-15


@pytest.mark.parametrize("rel", [1, 2, 3])
def test_sauter_schwab_maps_cover_product_of_triangles(orc, rel):
    """Each relation's maps, summed over regions with their Jacobians, must
    integrate any polynomial over {0<=s2<=s1<=1} x {0<=t2<=t1<=1} exactly:
    a measure-preserving cover of the 4-D domain (a dropped region, a wrong
    Jacobian power or a transposed coordinate fails this)."""
    S, T, W = orc.ss_points(rel, 8)

    def ex(a, b):
        return 1.0 / ((b + 1) * (a + b + 2))
    for (a, b, c, d) in [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (2, 1, 0, 1),
                         (1, 1, 1, 1), (0, 2, 2, 0), (3, 0, 1, 2), (2, 2, 2, 2), (0, 4, 0, 3)]:
        num = np.sum(W * S[:, 0] ** a * S[:, 1] ** b * T[:, 0] ** c * T[:, 1] ** d)
        assert abs(num - ex(a, b) * ex(c, d)) < 1e-13 * ex(a, b) * ex(c, d) * 10
    assert (S[:, 1] <= S[:, 0] + 1e-15).all() and (T[:, 1] <= T[:, 0] + 1e-15).all()
    assert (S >= 0).all() and (S <= 1).all() and (T >= 0).all() and (T <= 1).all()


def test_sauter_schwab_singular_sets(orc):
    """The singularity sits where each case needs it: as xi -> 0 (vertex,
    edge) or along s = t (identical) the two points coincide."""
    lib = orc.lib()
    import ctypes
    s = np.zeros(2)
    t = np.zeros(2)
    j = np.zeros(1)
    dp = ctypes.POINTER(ctypes.c_double)
    # vertex: xi -> 0 sends both points to the common vertex (0,0)
    for reg in range(2):
        lib.orc_ss_map(1, reg, 1e-9, 0.3, 0.6, 0.7, s.ctypes.data_as(dp), t.ctypes.data_as(dp), j.ctypes.data_as(dp))
        assert np.abs(s).max() < 1e-8 and np.abs(t).max() < 1e-8
    # edge: e1 -> 0 sends both to the same point of the common edge s2 = t2 = 0
    for reg in range(5):
        lib.orc_ss_map(2, reg, 0.7, 1e-10, 0.4, 0.6, s.ctypes.data_as(dp), t.ctypes.data_as(dp), j.ctypes.data_as(dp))
        assert abs(s[1]) < 1e-9 and abs(t[1]) < 1e-9 and abs(s[0] - t[0]) < 1e-9
    # identical: e1 -> 0 gives s = t
    for reg in range(6):
        lib.orc_ss_map(3, reg, 0.7, 1e-10, 0.4, 0.6, s.ctypes.data_as(dp), t.ctypes.data_as(dp), j.ctypes.data_as(dp))
        assert np.abs(s - t).max() < 1e-9
