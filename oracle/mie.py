"""Analytic series for a penetrable sphere in a plane wave (test
infrastructure only).

Transmission problem of Sec. 2.1 (eq. model) for one sphere of radius a
centred at the origin, exterior (k0, rho0), interior (k1, rho1), incident
plane wave exp(i k0 z).  The paper validates against this series (Sec. 3.1,
ref. Anderson 1950).  With x0 = k0 a, x1 = k1 a and h_n the outgoing
spherical Hankel function h_n^(1) (time factor exp(-i w t), Sec. 2.1):

  p_inc  = sum_n i^n (2n+1) j_n(k0 r) P_n(cos t)
  p_s    = sum_n i^n (2n+1) a_n h_n(k0 r) P_n(cos t)
  p_1    = sum_n i^n (2n+1) c_n j_n(k1 r) P_n(cos t)

Continuity of p and of (1/rho) dp/dr at r = a gives

  a_n = [(k1/rho1) j_n(x0) j_n'(x1) - (k0/rho0) j_n'(x0) j_n(x1)]
        / [(k0/rho0) h_n'(x0) j_n(x1) - (k1/rho1) h_n(x0) j_n'(x1)].
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_legendre, spherical_jn, spherical_yn


def _h(n, z, derivative=False):
    return spherical_jn(n, z, derivative) + 1j * spherical_yn(n, z, derivative)


def n_terms(x: complex) -> int:
    ax = abs(x)
    return int(ax + 4.0 * ax ** (1.0 / 3.0) + 10)


def coefficients(a, k0, k1, rho0, rho1):
    x0, x1 = k0 * a, k1 * a
    N = n_terms(max(abs(x0), abs(x1)))
    n = np.arange(N + 1)
    j0, dj0 = spherical_jn(n, x0), spherical_jn(n, x0, True)
    j1, dj1 = spherical_jn(n, x1), spherical_jn(n, x1, True)
    h0, dh0 = _h(n, x0), _h(n, x0, True)
    num = (k1 / rho1) * j0 * dj1 - (k0 / rho0) * dj0 * j1
    den = (k0 / rho0) * dh0 * j1 - (k1 / rho1) * h0 * dj1
    an = num / den
    cn = (j0 + an * h0) / j1
    return n, an, cn


def surface_traces(points, a, k0, k1, rho0, rho1):
    """Exterior total-field traces (gamma_D p_tot, gamma_N^+ p_tot) at points
    on the sphere |x| = a (normal derivative along the outward radius)."""
    n, an, _ = coefficients(a, k0, k1, rho0, rho1)
    x0 = k0 * a
    ct = points[:, 2] / np.linalg.norm(points, axis=1)
    pref = (1j ** n) * (2 * n + 1)
    jD = spherical_jn(n, x0) + an * _h(n, x0)
    jN = k0 * (spherical_jn(n, x0, True) + an * _h(n, x0, True))
    P = np.stack([eval_legendre(m, ct) for m in n], axis=1)
    return P @ (pref * jD), P @ (pref * jN)


def total_field(points, a, k0, k1, rho0, rho1):
    """Total pressure at arbitrary points (exterior: the exact incident
    plane wave plus the scattered series, whose coefficients a_n decay past
    n ~ k0 a; interior: the transmitted series).  The incident wave is not
    summed as a series: at k0 r >> k0 a its series needs ~k0 r terms."""
    n, an, cn = coefficients(a, k0, k1, rho0, rho1)
    r = np.linalg.norm(points, axis=1)
    ct = np.where(r > 0, points[:, 2] / np.where(r > 0, r, 1), 1.0)
    pref = (1j ** n) * (2 * n + 1)
    P = np.stack([eval_legendre(m, ct) for m in n], axis=1)
    out = np.empty(points.shape[0], dtype=np.complex128)
    ext = r >= a
    if ext.any():
        re = r[ext][:, None]
        out[ext] = np.exp(1j * k0 * points[ext, 2]) + (P[ext] * pref * an * _h(n, k0 * re)).sum(1)
    if (~ext).any():
        ri = r[~ext][:, None]
        out[~ext] = (P[~ext] * pref * cn * spherical_jn(n, k1 * ri)).sum(1)
    return out


def sphere_eigenvalues(n, k, a):
    """Eigenvalues of V, K (= K') and W on the sphere for spherical harmonics
    of degree n (addition theorem for G, App. A definitions; W carries the
    leading minus of eq. HYP):
      V_n = i k a^2 j_n h_n,  K_n = (i k^2 a^2 / 2)(j_n h_n' + j_n' h_n),
      W_n = -i k^3 a^2 j_n' h_n'   (arguments k a)."""
    x = k * a
    j, dj = spherical_jn(n, x), spherical_jn(n, x, True)
    h, dh = _h(n, x), _h(n, x, True)
    V = 1j * k * a * a * j * h
    K = 0.5j * k * k * a * a * (j * dh + dj * h)
    W = -1j * k ** 3 * a * a * dj * dh
    return V, K, W
