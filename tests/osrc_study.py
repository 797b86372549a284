"""GMRES iteration counts of the PMCHWT system under OSRC preconditioner
variants, on the FP64 oracle (a study runner, not a test; no GPU).

The paper's OSRC block preconditioner (Sec. 2.3 eqs. OSRC_prec,
OSRC_prec_blocks, OSRC_DtN_NtD_maps) leaves several choices open; this
tabulates GMRES(100) iterations to relative residuals 1e-5 (the paper's
tolerance, Sec. 3) and 1e-8 for each reading, on
  * the paper's bone sphere (1 cm diameter, 1 MHz, impedance ratio 5.2) and
    its fat sphere, cube-sphere meshes at about 4 elements per wavelength,
  * the rib / fat / liver scene at 6 mm elements and the frequency that mesh
    resolves (k h ~ 1).
Variants: no preconditioner; the paper's reading (block wavenumber k0, damping
exponent +1/3, R_eps 1/10 of the largest domain diameter, theta = pi/3, left
composition); block wavenumber k_j; the printed exponent -1/3; R_eps x 1/10
and x 3; theta pi/4 and pi/2; right composition (GMRES on A P, x = P y);
N_pade 4 vs 8.

    python tests/osrc_study.py [sphere_bone sphere_fat rib_small] > table.md
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import galerkin, gmres, osrc, pmchwt, rayleigh  # noqa: E402
from synth import scenes  # noqa: E402


def sphere(material):
    from paper_1910_01011_gb300.experiments import sphere as ex  # scene construction only (synthetic input)
    return ex.build_scene(material, 4.0)


def rib_small():
    return scenes.rib_scene(h=6e-3, freq=0.1e6 * 2.65 / 6.0)


def incident(s):
    if s.transducer is not None:
        tr = s.transducer
        w = scenes.focusing_weights(tr, s.k0)
        return rayleigh.field(tr, w, s.k0, 2 * np.pi * s.freq, s.rho0)
    return pmchwt.plane_wave(s.k0, s.plane_wave_dir)


def default_r_eps(s):
    d = max(np.linalg.norm(np.ptp(dm.verts, axis=0)) for dm in s.domains)
    return 0.1 * d


def build_pre(s, r_eps, n_pade=8, theta=np.pi / 3, eps_exponent=1.0 / 3.0, block_k="k0"):
    return osrc.build(s, r_eps, n_pade, theta, eps_exponent, "exterior" if block_k == "k0" else "interior")


def iterations(A, b, pre, s, tol, side="left"):
    if pre is None:
        _, it, _ = gmres.gmres(lambda v: A @ v, b, tol=tol, restart=100, maxiter=4000)
    elif side == "left":
        _, it, _ = gmres.gmres(lambda v: osrc.apply(s, pre, A @ v), osrc.apply(s, pre, b), tol=tol, restart=100,
                               maxiter=4000)
    else:
        _, it, _ = gmres.gmres(lambda v: A @ osrc.apply(s, pre, v), b, tol=tol, restart=100, maxiter=4000)
    return it


def study(name):
    s = {"sphere_bone": lambda: sphere("bone"), "sphere_fat": lambda: sphere("fat"), "rib_small": rib_small}[name]()
    t0 = time.time()
    A = pmchwt.assemble(s)
    b = pmchwt.rhs(s, incident(s))
    t_asm = time.time() - t0
    r0 = default_r_eps(s)
    npd = 4 if name.startswith("sphere") else 8
    variants = [
        ("none", None, "left"),
        ("k0 (exterior)", dict(r_eps=r0, n_pade=npd), "left"),
        ("block k_j", dict(r_eps=r0, n_pade=npd, block_k="kj"), "left"),
        ("eps exponent -1/3", dict(r_eps=r0, n_pade=npd, eps_exponent=-1.0 / 3.0), "left"),
        ("R_eps x 1/10", dict(r_eps=0.1 * r0, n_pade=npd), "left"),
        ("R_eps x 3", dict(r_eps=3 * r0, n_pade=npd), "left"),
        ("theta pi/4", dict(r_eps=r0, n_pade=npd, theta=np.pi / 4), "left"),
        ("theta pi/2", dict(r_eps=r0, n_pade=npd, theta=np.pi / 2), "left"),
        ("right composition", dict(r_eps=r0, n_pade=npd), "right"),
        (f"N_pade {12 - npd}", dict(r_eps=r0, n_pade=12 - npd), "left"),
    ]
    rows = []
    for label, kw, side in variants:
        pre = None if kw is None else build_pre(s, **kw)
        its = [iterations(A, b, pre, s, tol, side) for tol in (1e-5, 1e-8)]
        rows.append((label, its))
        print(f"  {name}: {label}: {its}", file=sys.stderr, flush=True)
    return s, t_asm, r0, rows


def main():
    names = sys.argv[1:] or ["sphere_bone", "sphere_fat", "rib_small"]
    galerkin.build()
    for n in names:
        s, t_asm, r0, rows = study(n)
        print(f"\n### {n}: {s.n_triangles} triangles, N = {s.n_dofs}, R_eps default {r0:.3g} m "
              f"(assembly {t_asm:.0f} s)\n")
        print("| variant | its to 1e-5 | its to 1e-8 |\n|---|---:|---:|")
        for label, its in rows:
            print(f"| {label} | {its[0]} | {its[1]} |")
        sys.stdout.flush()


if __name__ == "__main__":
    main()
