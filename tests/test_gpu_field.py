"""Off-surface field (representation formula) on the GPU against the
oracle's evaluation from the same traces, and the paper's sphere check
(Sec. 3.1: total field on a 200 x 200 grid over +-3R through the centre,
error below 3 % at about 6 elements per wavelength) against the Mie series."""
import numpy as np
import pytest

from oracle import field, mie, pmchwt, rayleigh
from synth import scenes

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def grid(n=41, half=3.0, shell=(0.15,)):
    g = np.linspace(-half, half, n)
    X, Z = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), 0.05 + 0 * X.ravel(), Z.ravel()], 1)
    r = np.linalg.norm(pts, axis=1)
    keep = np.abs(r - 1.0) > shell[0]
    pts = pts[keep]
    return pts, np.where(np.linalg.norm(pts, axis=1) < 1.0, 0, -1).astype(np.int32)


def test_field_matches_oracle_same_traces():
    from paper_1910_01011_gb300 import api
    s = scenes.sphere_scene(2, k0=5.0, k1=5.25 + 0.1j)
    c = api.Context.from_scene(s)
    c.set_plane_wave((0, 0, 1))
    assert c.solve(precision=0, tol=1e-11)["converged"]
    D, N = c.traces(0)
    u = np.concatenate([N, D])
    pts, dom = grid(31)
    got = c.field(pts, dom)
    ref = field.total_field(s, u, pts, dom, pmchwt.plane_wave(s.k0, (0, 0, 1)))
    assert rel(got, ref) < 1e-5
    c.close()


def test_sphere_field_against_mie_paper_grid():
    """200 x 200 grid over +-3R (the paper's check), level-3 icosphere."""
    from paper_1910_01011_gb300 import api
    s = scenes.sphere_scene(3)
    c = api.Context.from_scene(s)
    c.set_plane_wave((0, 0, 1))
    c.solve(precision=1, tol=1e-9)
    pts, dom = grid(200, shell=(0.1,))
    got = c.field(pts, dom)
    d = s.domains[0]
    ref = mie.total_field(pts, 1.0, s.k0, d.k, s.rho0, d.rho)
    assert rel(got, ref) < 0.03
    c.close()


def test_field_with_transducer_incident():
    from paper_1910_01011_gb300 import api
    s = scenes.two_sphere_scene(1)
    tr = scenes.bowl_transducer(seed=3, n_elem=5, R=4.0, aperture=3.0, piston_radius=0.3, gap=0.05)
    c = api.Context.from_scene(s)
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], 2.6)
    W = scenes.focusing_weights(tr, s.k0)[None, :]
    c.set_excitations(W)
    assert c.solve(precision=0, tol=1e-11)["converged"]
    u = np.concatenate([np.concatenate([c.traces(j)[1], c.traces(j)[0]]) for j in range(2)])
    pts = np.array([[0.0, 0.0, 2.5], [0.0, 2.0, 0.0], [-1.3, 0.0, 0.2], [1.2, 0.1, 0.1], [3.0, -1.0, 0.5]])
    dom = np.array([-1, -1, 0, 1, -1], dtype=np.int32)
    got = c.field(pts, dom)
    inc = rayleigh.field(tr, W[0], s.k0, 2.0, 1.3)
    ref = field.total_field(s, u, pts, dom, inc)
    assert rel(got, ref) < 1e-5
    c.close()


def test_field_many_points_against_oracle_sample():
    """A 200 x 200 grid: enough points that each CTA takes a chunk of several
    source tiles; a seeded sample of the points against the oracle from the
    same traces."""
    from paper_1910_01011_gb300 import api
    s = scenes.sphere_scene(3, k0=5.0, k1=5.25 + 0.1j)
    c = api.Context.from_scene(s)
    c.set_plane_wave((0, 0, 1))
    assert c.solve(precision=0, tol=1e-11)["converged"]
    D, N = c.traces(0)
    u = np.concatenate([N, D])
    pts, dom = grid(200)
    got = c.field(pts, dom)
    pick = np.random.default_rng(11).choice(pts.shape[0], size=300, replace=False)
    ref = field.total_field(s, u, pts[pick], dom[pick], pmchwt.plane_wave(s.k0, (0, 0, 1)))
    assert rel(got[pick], ref) < 1e-5
    # the sampled points alone (one source tile per chunk) give the same values
    alone = c.field(pts[pick], dom[pick])
    assert rel(got[pick], alone) < 1e-6
    c.close()


def test_field_device_domain_ids_checked_by_the_kernels():
    """Domain ids in a device array are range-checked by the field kernels:
    an id beyond the domain count gives INVALID_ARG (and NaN at that point)
    instead of an out-of-range read, and the context stays usable."""
    import ctypes

    import torch

    from paper_1910_01011_gb300 import api
    s = scenes.sphere_scene(1)
    c = api.Context.from_scene(s)
    c.set_plane_wave((0, 0, 1))
    assert c.solve(precision=0, tol=1e-10)["converged"]
    pts, dom = grid(9)
    good = c.field(pts, dom)
    dom_bad = dom.copy()
    dom_bad[3] = 5  # one domain only
    dp = torch.from_numpy(pts).cuda()
    dd = torch.from_numpy(dom_bad).cuda()
    out = torch.zeros(pts.shape[0], dtype=torch.complex128, device="cuda")
    rc = c.lib.bem_field(c.h, 0, ctypes.c_void_p(dp.data_ptr()), ctypes.c_void_p(dd.data_ptr()), pts.shape[0],
                         ctypes.c_void_p(out.data_ptr()), 1)
    assert rc == -1  # BEM_ERR_INVALID_ARG
    o = out.cpu().numpy()
    assert np.isnan(o[3])
    keep = np.arange(pts.shape[0]) != 3
    assert rel(o[keep], good[keep]) < 1e-12
    again = c.field(pts, dom)  # the flag was cleared
    assert rel(again, good) < 1e-14
    c.close()
