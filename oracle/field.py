"""Off-surface field from the solved traces (test infrastructure only).

Representation formula of App. A (eq. rep_formula_gen) with the PMCHWT jump
potentials: in the exterior the scattered field is
  p_s(x) = DL_k0(gamma_D p_tot)(x) - SL_k0(gamma_N^+ p_tot)(x)
over all surfaces (the incident field is an entire solution and drops out),
and p_tot = p_inc + p_s; inside domain j
  p^j(x) = SL_kj((rho_j/rho_0) gamma_N^+ p_tot)(x) - DL_kj(gamma_D p_tot)(x)
over the surface of domain j (interior traces from eq. Form1_BCs).
SL psi(x) = int G psi, DL phi(x) = int dG/dn_y phi, G = exp(ikr)/(4 pi r).
Surface integrals by the regular rule with P1 interpolation of the traces.
"""
from __future__ import annotations

import numpy as np

from . import galerkin, pmchwt


def layer_potentials(v, t, k, dirichlet, neumann, points):
    """(SL neumann, DL dirichlet) at the points."""
    x, wa, phi = galerkin.quad_points(v, t)
    nrm, _ = galerkin.tri_geometry(v, t)
    nt, nq = x.shape[0], x.shape[1]
    y = x.reshape(-1, 3)
    w = wa.reshape(-1)
    ny = np.repeat(nrm, nq, axis=0)
    psi = (neumann[t] @ phi.T).reshape(-1)        # (nt, nq) interpolated
    ph = (dirichlet[t] @ phi.T).reshape(-1)
    sl = np.zeros(points.shape[0], dtype=np.complex128)
    dl = np.zeros(points.shape[0], dtype=np.complex128)
    for i0 in range(0, points.shape[0], 256):
        p = points[i0:i0 + 256]
        d = p[:, None, :] - y[None, :, :]              # x - y
        r = np.linalg.norm(d, axis=2)
        G = np.exp(1j * k * r) / (4 * np.pi * r)
        dGdny = G * (1j * k - 1 / r) * (-(d * ny[None]).sum(2)) / r   # (y - x).n_y / r
        sl[i0:i0 + 256] = (G * (w * psi)[None]).sum(1)
        dl[i0:i0 + 256] = (dGdny * (w * ph)[None]).sum(1)
    return sl, dl


def total_field(scene, u, points, domain_of_point, incident):
    """Total pressure at points; domain_of_point[i] = -1 (exterior) or j."""
    tr = pmchwt.split_traces(scene, u)
    out = np.zeros(points.shape[0], dtype=np.complex128)
    ext = domain_of_point < 0
    if ext.any():
        pe = points[ext]
        acc = np.zeros(pe.shape[0], dtype=np.complex128)
        for d, (D, N) in zip(scene.domains, tr):
            sl, dl = layer_potentials(d.verts, d.tris, scene.k0, D, N, pe)
            acc += dl - sl
        pinc, _ = incident(pe, np.zeros_like(pe))
        out[ext] = acc + pinc
    for j, (d, (D, N)) in enumerate(zip(scene.domains, tr)):
        m = domain_of_point == j
        if m.any():
            sl, dl = layer_potentials(d.verts, d.tris, d.k, D, (d.rho / scene.rho0) * N, points[m])
            out[m] = sl - dl
    return out
