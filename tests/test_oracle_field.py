"""Pins of the oracle's off-surface field (representation formula, App. A
eq. rep_formula_gen)."""
import numpy as np
import pytest

from oracle import field, mie, pmchwt
from synth import meshes, scenes


def test_green_identity_entire_and_radiating():
    """Traces of an entire solution (plane wave): DL - SL vanishes outside
    and reproduces the wave inside; traces of a radiating solution (point
    source inside): DL - SL reproduces it outside.  O(h^2) in the mesh."""
    errs = []
    for L in (2, 3):
        v, t = meshes.icosphere(L)
        nv = v / np.linalg.norm(v, axis=1)[:, None]
        k = 3.0 + 0.2j
        d = np.array([0.0, 0.6, 0.8])
        D = np.exp(1j * k * (v @ d))
        N = 1j * k * (nv @ d) * D
        out = np.array([[0, 0, 2.5], [1.5, 1.5, 0.3], [-2, 0.5, 1]])
        inn = np.array([[0.1, 0.2, -0.1], [0.3, -0.2, 0.1]])
        sl, dl = field.layer_potentials(v, t, k, D, N, out)
        e1 = np.abs(dl - sl).max()
        sl, dl = field.layer_potentials(v, t, k, D, N, inn)
        e2 = np.abs((sl - dl) - np.exp(1j * k * (inn @ d))).max()
        xs = np.array([0.2, -0.1, 0.3])
        dd = v - xs
        r = np.linalg.norm(dd, axis=1)
        Dp = np.exp(1j * k * r) / (4 * np.pi * r)
        Np = Dp * (1j * k - 1 / r) * np.einsum("ij,ij->i", dd, nv) / r
        sl, dl = field.layer_potentials(v, t, k, Dp, Np, out)
        rr = np.linalg.norm(out - xs, axis=1)
        ex = np.exp(1j * k * rr) / (4 * np.pi * rr)
        e3 = np.abs((dl - sl) - ex).max() / np.abs(ex).max()
        errs.append((e1, e2, e3))
    assert max(errs[1]) < 0.015
    for a, b in zip(errs[0], errs[1]):
        assert a / b > 3.0


@pytest.mark.slow
def test_total_field_against_mie():
    """The paper's check (Sec. 3.1): total field on a grid through the
    sphere centre over +-3R against the analytic series; O(h^2) away from the
    surface, below 3 % already at level 2."""
    res = {}
    for L in (2, 3):
        s = scenes.sphere_scene(L)
        u, _, _ = pmchwt.solve(s, pmchwt.plane_wave(s.k0, (0, 0, 1)))
        g = np.linspace(-3, 3, 21)
        X, Z = np.meshgrid(g, g)
        pts = np.stack([X.ravel(), 0 * X.ravel(), Z.ravel()], 1)
        r = np.linalg.norm(pts, axis=1)
        pts = pts[(r > 1.5) | (r < 0.5)]
        dom = np.where(np.linalg.norm(pts, axis=1) < 1, 0, -1)
        f = field.total_field(s, u, pts, dom, pmchwt.plane_wave(s.k0, (0, 0, 1)))
        ref = mie.total_field(pts, 1.0, s.k0, s.domains[0].k, s.rho0, s.domains[0].rho)
        res[L] = np.linalg.norm(f - ref) / np.linalg.norm(ref)
    assert res[2] < 0.03 and res[3] < 0.005
    assert res[2] / res[3] > 3.0


def test_mie_field_matches_surface_traces():
    """The field series and the surface-trace series agree on the sphere."""
    pts = scenes.meshes.icosphere(2)[0] * (1.0 + 1e-9)
    a, k0, k1 = 1.0, 5.0, 5.25
    D, _ = mie.surface_traces(pts, a, k0, k1, 1.0, 1.1)
    f = mie.total_field(pts, a, k0, k1, 1.0, 1.1)
    assert np.abs(f - D).max() < 1e-6
