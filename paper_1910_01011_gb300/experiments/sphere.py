"""The paper's single-sphere model problem (Sec. 3.1): a 1 cm diameter
penetrable sphere in water at 1 MHz, fat (Z_int/Z_ext = 0.86) or bone
(Z_int/Z_ext = 5.2), plane-wave incidence; GMRES iterations, time per
iteration and the l2 error of the total field on a 200 x 200 grid over
+-3R through the centre, at several mesh densities (elements per
wavelength, lambda = min(lambda_0, lambda_j)).

The paper reports, for 6 elements per wavelength, a field error below 3 %
and about 0.2 s per GMRES iteration on its 32-core workstation; Figs. 2-3
give the trends only as images.

Materials: water c = 1500 m/s, rho = 1000 kg/m^3; fat from Table 1
(rho 917, c 1412, 9.3 Np/m at 1 MHz); bone: the paper gives only the
impedance ratio 5.2, taken here as rho = 1900 kg/m^3, c = 4100 m/s with
Table 1's rib attenuation (47 Np/m at 1 MHz).  The mesh is a cube-sphere
(synthetic; the paper's meshes are not available).

This module runs the GPU solve and evaluates the total field on the grid;
the comparison with the analytic series lives with the tests
(tests/sphere_experiment.py), which may use the oracle's Mie routine.
"""
from __future__ import annotations

import math
import time

import numpy as np

MATERIALS = {"fat": (917.0, 1412.0, 9.3), "bone": (1900.0, 4100.0, 47.0)}


def build_scene(material: str, el_per_lambda: float, f: float = 1e6, radius: float = 5e-3):
    from synth import meshes, scenes
    rho, c, alpha = MATERIALS[material]
    k0 = scenes.wavenumber(f, 1500.0)
    kj = scenes.wavenumber(f, c, alpha, 1.0)
    lam = min(1500.0, c) / f
    h = lam / el_per_lambda
    # cube-sphere: a cube-face cell of side 2R/m maps to an arc of about
    # (pi/2) R / m, so the box spacing is scaled to give edges of about h
    v, t = meshes.rounded_box((radius, radius, radius), 2.0, h * 4.0 / math.pi)
    s = scenes.Scene(name=f"sphere_{material}_{el_per_lambda}", k0=k0, rho0=1000.0, plane_wave_dir=(0, 0, 1), freq=f)
    s.domains.append(scenes.Domain(material, v, t, kj, rho))
    s.meta["radius"] = radius
    s.meta["el_per_lambda_actual"] = lam / meshes.mesh_stats(v, t)["h_mean"]
    return s


def field_grid(radius: float, n: int = 200):
    g = np.linspace(-3 * radius, 3 * radius, n)
    X, Z = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), np.zeros(X.size), Z.ravel()], 1)
    r = np.linalg.norm(pts, axis=1)
    # points within 5 % of the radius of the surface are left out (regular rule)
    keep = np.abs(r - radius) > 0.05 * radius
    pts = pts[keep]
    return pts, np.where(np.linalg.norm(pts, axis=1) < radius, 0, -1).astype(np.int32)


def run(material: str, el_per_lambda: float, device: int = 0, tol: float = 1e-5, precision: int = 1,
        operator_mode: int = 1):
    """One point of the experiment: solve, then the total field on the grid.
    Returns the measurements plus `points`, `field` and the sphere's
    parameters (`radius`, `k0`, `kj`, `rho0`, `rho`) for the comparison."""
    from paper_1910_01011_gb300.api import Context
    s = build_scene(material, el_per_lambda)
    d = s.domains[0]
    R = s.meta["radius"]
    c = Context.from_scene(s, device=device, n_pade=4, r_eps=R / 10.0)
    c.set_plane_wave((0, 0, 1))
    t0 = time.perf_counter()
    rep = c.solve(precision=precision, tol=tol, restart=100, max_iter=3000, operator_mode=operator_mode)
    wall = time.perf_counter() - t0
    pts, dom = field_grid(R)
    got = c.field(pts, dom)
    c.close()
    return {"material": material, "el_per_lambda": el_per_lambda,
            "el_per_lambda_mean_edge": s.meta["el_per_lambda_actual"], "triangles": int(d.tris.shape[0]),
            "dofs": 2 * int(d.verts.shape[0]), "iterations": rep["iterations"], "refinements": rep["refinements"],
            "converged": rep["converged"], "solve_s": wall, "s_per_iteration": wall / max(1, rep["iterations"]),
            "z_ratio": d.rho * (2 * math.pi * s.freq / d.k.real) / (s.rho0 * 1500.0),
            "points": pts, "field": got, "radius": R, "k0": s.k0, "kj": d.k, "rho0": s.rho0, "rho": d.rho}
