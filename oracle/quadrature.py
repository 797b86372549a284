"""Quadrature rules for the oracle (test infrastructure only).

The paper leaves quadrature to its BEM library (Sec. 3, Bempp 3.3.4).  The
reading used here, and by the CUDA path as an independently derived table:

* regular pairs: the symmetric 6-point, degree-4 triangle rule, two orbits
  (a, a, 1-2a) and (b, b, 1-2b) with weights w1, w2.  Derived here from its
  moment equations: exactness on the S3-invariant polynomials 1, e2, e3, e2^2
  (e2, e3 elementary symmetric functions of the barycentrics), which spans
  the invariant polynomials of degree <= 4;
* singular pairs: n-point Gauss-Legendre on [0, 1] in each of the four
  Sauter-Schwab directions (numpy's Gauss-Legendre nodes, a library
  primitive).
"""
from __future__ import annotations

import numpy as np


def _moments(p):
    a, b, w1, w2 = p

    def e2(t):
        return 2 * t - 3 * t * t

    def e3(t):
        return t * t * (1 - 2 * t)

    # Exact integrals (mean over the triangle) of 1, e2, e3, e2^2:
    # int l1^i l2^j l3^k / |T| = 2 i! j! k! / (i+j+k+2)!
    return np.array([
        3 * w1 + 3 * w2 - 1.0,
        3 * w1 * e2(a) + 3 * w2 * e2(b) - 1.0 / 4.0,
        3 * w1 * e3(a) + 3 * w2 * e3(b) - 1.0 / 60.0,
        3 * w1 * e2(a) ** 2 + 3 * w2 * e2(b) ** 2 - 1.0 / 15.0,
    ])


def triangle_rule6():
    """Return (l1, l2, w) arrays of the 6-point degree-4 rule: points
    P0 + l1 (P1-P0) + l2 (P2-P0), weights summing to 1 (multiply by area)."""
    p = np.array([0.44, 0.09, 0.22, 0.11])
    for _ in range(60):
        f = _moments(p)
        J = np.empty((4, 4))
        for j in range(4):
            dp = np.zeros(4)
            dp[j] = 1e-7
            J[:, j] = (_moments(p + dp) - _moments(p - dp)) / 2e-7
        step = np.linalg.solve(J, f)
        p = p - step
        if np.max(np.abs(step)) < 1e-16:
            break
    a, b, w1, w2 = p
    bary = []
    for t, w in ((a, w1), (b, w2)):
        for perm in ((t, t, 1 - 2 * t), (t, 1 - 2 * t, t), (1 - 2 * t, t, t)):
            bary.append((perm[1], perm[2], w))
    r = np.array(bary)
    return r[:, 0].copy(), r[:, 1].copy(), r[:, 2].copy()


def rule_table(rule=None) -> np.ndarray:
    """(nq, 3) float64 table [l1, l2, w] in the layout the C oracle reads."""
    l1, l2, w = triangle_rule6() if rule is None else rule
    return np.ascontiguousarray(np.stack([l1, l2, w], axis=1), dtype=np.float64)


def gauss_legendre01(n: int) -> np.ndarray:
    """(n, 2) table [node, weight] of n-point Gauss-Legendre on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return np.ascontiguousarray(np.stack([0.5 * (x + 1.0), 0.5 * w], axis=1), dtype=np.float64)


def collapsed_gauss_rule(n: int):
    """A high-order triangle rule (for pins only): Gauss-Legendre n x n on the
    square mapped to the triangle by the Duffy collapse
    (u, v) -> (l1, l2) = (u (1 - v), u v), Jacobian u; weights sum to 1."""
    g = gauss_legendre01(n)
    l1, l2, w = [], [], []
    for u, wu in g:
        for v, wv in g:
            l1.append(u * (1 - v))
            l2.append(u * v)
            w.append(2.0 * wu * wv * u)
    return np.array(l1), np.array(l2), np.array(w)
