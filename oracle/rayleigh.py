"""Incident field of a piston array by the Rayleigh integral (test
infrastructure only).

The paper defers the transducer field to its ref. elwin2015 (Sec. 3.2).
Reading used: each piston is a flat disc with unit normal velocity radiating
as if baffled, time factor exp(-i w t):

  p(x)      = -(i w rho0 / 2 pi) sum_m w_m int_{S_m} exp(i k0 R)/R dS,  R = |x - y|
  dp/dn (x) = -(i w rho0 / 2 pi) sum_m w_m int_{S_m} exp(i k0 R)(i k0 - 1/R)/R ((x-y).n)/R dS

Disc rule: n_r Gauss-Legendre radii on [0, a] (weight rho drho) times n_t
equally spaced angles theta_j = 2 pi (j + 1/2)/n_t.  In-plane axes of a
piston with normal n: e1 = normalise(z^ x n), or normalise(x^ x n) when
|n_z| > 0.9; e2 = n x e1.
"""
from __future__ import annotations

import numpy as np


def disc_rule(n_r: int = 4, n_t: int = 8):
    x, w = np.polynomial.legendre.leggauss(n_r)
    r = 0.5 * (x + 1.0)
    wr = 0.5 * w * r                      # int_0^1 f(r) r dr
    th = 2.0 * np.pi * (np.arange(n_t) + 0.5) / n_t
    wt = np.full(n_t, 2.0 * np.pi / n_t)
    R, T = np.meshgrid(r, th, indexing="ij")
    W = (wr[:, None] * wt[None, :])
    return R.ravel(), T.ravel(), W.ravel()


def piston_points(centres, normals, radii, n_r=4, n_t=8):
    r, th, w = disc_rule(n_r, n_t)
    pts, wts = [], []
    for c, n, a in zip(centres, normals, radii):
        ax = np.array([1.0, 0.0, 0.0]) if abs(n[2]) > 0.9 else np.array([0.0, 0.0, 1.0])
        e1 = np.cross(ax, n)
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(n, e1)
        p = c[None, :] + a * r[:, None] * (np.cos(th)[:, None] * e1[None, :] + np.sin(th)[:, None] * e2[None, :])
        pts.append(p)
        wts.append(w * a * a)
    return np.stack(pts), np.stack(wts)           # (n_elem, nq, 3), (n_elem, nq)


def field(tr: dict, weights, k0: complex, omega: float, rho0: float, n_r=4, n_t=8):
    """Returns f(x, n) -> (p, dp/dn) for piston weights `weights` (n_elem,)."""
    Y, WY = piston_points(tr["centres"], tr["normals"], tr["radii"], n_r, n_t)
    pref = -1j * omega * rho0 / (2.0 * np.pi)
    wts = np.asarray(weights)

    def f(x, nrm):
        p = np.zeros(x.shape[0], dtype=np.complex128)
        dp = np.zeros(x.shape[0], dtype=np.complex128)
        for m in range(Y.shape[0]):
            d = x[:, None, :] - Y[m][None, :, :]
            R = np.linalg.norm(d, axis=2)
            g = np.exp(1j * k0 * R) / R
            p += wts[m] * (g * WY[m][None, :]).sum(1)
            dn = np.einsum("pqd,pd->pq", d, nrm)
            dp += wts[m] * (g * (1j * k0 - 1.0 / R) * dn / R * WY[m][None, :]).sum(1)
        return pref * p, pref * dp
    return f
