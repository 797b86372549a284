"""Parity of the CUDA operator application with the FP64 oracle, through
the C ABI.  Bars (from the method's precision design): relative l2 <= 1e-11
on the FP64 path, <= 2e-5 on the FP32 far-field path."""
import numpy as np
import pytest

from oracle import galerkin, pmchwt
from synth import meshes, scenes

pytestmark = pytest.mark.gpu

TOL = {0: 1e-11, 1: 2e-5}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def api():
    from paper_1910_01011_gb300 import api, build
    build.build()
    return api


def ragged_scene():
    """Two domains with triangle counts that are not multiples of the tile
    size: a rounded box (ragged last tile) and an icosphere of level 1 (80
    triangles, 2.5 tiles)."""
    vb, tb = meshes.rounded_box((1.0, 0.7, 0.5), 4.0, 0.3, center=(-1.4, 0.0, 0.0))
    vs, ts = meshes.icosphere(1, 0.6, (1.1, 0.2, 0.1))
    s = scenes.Scene(name="ragged", k0=3.0 + 0.0j, rho0=1.0, plane_wave_dir=(0.3, 0.4, 0.866))
    s.domains.append(scenes.Domain("box", vb, tb, 3.7 + 0.2j, 1.4))
    s.domains.append(scenes.Domain("ball", vs, ts, 2.6, 0.7))
    return s


def ctx_for(api, s, **kw):
    return api.Context.from_scene(s, **kw)


@pytest.mark.parametrize("prec", [0, 1])
def test_block_operators_single_surface(api, prec):
    """Each Calderon block [[-K, V], [W, K']] on one surface (touching pairs
    through the Sauter-Schwab correction) against the oracle's dense matrices."""
    s = ragged_scene()
    c = ctx_for(api, s)
    rng = np.random.default_rng(1)
    for j, d in enumerate(s.domains):
        nv = d.verts.shape[0]
        for k in (s.k0, d.k, 0.5 + 0.0j):
            V, K, Kp, W = galerkin.operators(d.verts, d.tris, k)
            A = np.block([[-K, V], [W, Kp]])
            x = rng.standard_normal(2 * nv) + 1j * rng.standard_normal(2 * nv)
            y = c.apply_block(j, j, k, x, prec)
            assert rel(y, A @ x) < TOL[prec], (j, k)
            # each operator separately (psi = 0 or phi = 0)
            for part in (0, 1):
                xp = x.copy()
                xp[(1 - part) * nv:(2 - part) * nv] = 0
                assert rel(c.apply_block(j, j, k, xp, prec), A @ xp) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_block_operators_between_surfaces(api, prec):
    s = ragged_scene()
    c = ctx_for(api, s)
    d0, d1 = s.domains
    rng = np.random.default_rng(2)
    for (j, i) in ((0, 1), (1, 0)):
        dj, di = s.domains[j], s.domains[i]
        V, K, Kp, W = galerkin.operator_rows(dj.verts, dj.tris, di.verts, di.tris, False, s.k0)
        A = np.block([[-K, V], [W, Kp]])
        x = rng.standard_normal(2 * di.verts.shape[0]) + 1j * rng.standard_normal(2 * di.verts.shape[0])
        assert rel(c.apply_block(j, i, s.k0, x, prec), A @ x) < TOL[prec]


@pytest.mark.parametrize("name", ["sphere", "ragged", "shell"])
@pytest.mark.parametrize("prec", [0, 1])
def test_pmchwt_apply(api, name, prec):
    """The full multiple-domain system A_hat (Sec. 2.2-2.3) against the
    oracle's dense assembly."""
    s = {"sphere": lambda: scenes.sphere_scene(2), "ragged": ragged_scene, "shell": lambda: scenes.shell_scene(1)}[name]()
    A = pmchwt.assemble(s)
    c = ctx_for(api, s)
    assert c.n_dofs == A.shape[0]
    rng = np.random.default_rng(3)
    for _ in range(2):
        x = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
        assert rel(c.apply(x, precision=prec), A @ x) < TOL[prec]
    xs = scenes.smooth_trace_vector(s, 4)
    assert rel(c.apply(xs, precision=prec), A @ xs) < TOL[prec]


def test_pmchwt_apply_multi_rhs_and_device_pointers(api):
    import torch
    s = scenes.two_sphere_scene(1)
    A = pmchwt.assemble(s)
    c = ctx_for(api, s)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, A.shape[0])) + 1j * rng.standard_normal((3, A.shape[0]))
    Y = c.apply(X, precision=1)
    for r in range(3):
        assert rel(Y[r], A @ X[r]) < TOL[1]
    Xd = torch.from_numpy(X).cuda()
    Yd = c.apply(Xd, precision=0)
    torch.cuda.synchronize()
    Yh = Yd.cpu().numpy()
    for r in range(3):
        assert rel(Yh[r], A @ X[r]) < TOL[0]


@pytest.mark.parametrize("name", ["ragged", "shell", "phase"])
def test_multi_rhs_far_field_matches_oracle(api, name):
    """Several right-hand sides in one FP32 far-field launch (the Green's
    function and gradient factor of each pair shared by a group of four):
    every column against the oracle's dense A_hat (FP32 bar) and against the
    one-vector FP32 path (which differs only in the chunking of the source
    sums); group counts 2, 4, 5 (a short last group) and 9."""
    s = {"ragged": ragged_scene, "shell": lambda: scenes.shell_scene(1),
         "phase": lambda: scenes.sphere_scene(2, k0=60.0, k1=66.0 + 0.5j)}[name]()
    A = pmchwt.assemble(s)
    c = ctx_for(api, s)
    for R in (2, 4, 5, 9):
        X = np.stack([scenes.random_complex(A.shape[0], 40 + r) for r in range(R - 1)] +
                     [scenes.smooth_trace_vector(s, 3)])
        Y = c.apply(X, precision=1)
        for r in range(R):
            ref = A @ X[r]
            assert rel(Y[r], ref) < TOL[1], (R, r)
            assert rel(Y[r], c.apply(X[r], precision=1)) < 2e-6, (R, r)


@pytest.mark.parametrize("name", ["ragged", "shell", "phase"])
def test_multi_rhs_fp64_far_field_matches_oracle(api, name):
    """Several vectors in one FP64 far-field launch (kernel values of a pair
    shared by a group of four, one launch per slot and group): every column
    against the oracle's dense A_hat (FP64 bar) and against the one-vector
    FP64 path; group counts 2, 4, 5 (a short last group) and 9, on a
    complex interior wavenumber (the attenuated branch) and real ones."""
    s = {"ragged": ragged_scene, "shell": lambda: scenes.shell_scene(1),
         "phase": lambda: scenes.sphere_scene(2, k0=60.0, k1=66.0 + 0.5j)}[name]()
    A = pmchwt.assemble(s)
    c = ctx_for(api, s)
    for R in (2, 4, 5, 9):
        X = np.stack([scenes.random_complex(A.shape[0], 60 + r) for r in range(R - 1)] +
                     [scenes.smooth_trace_vector(s, 3)])
        Y = c.apply(X, precision=0)
        for r in range(R):
            assert rel(Y[r], A @ X[r]) < TOL[0], (R, r)
            assert rel(Y[r], c.apply(X[r], precision=0)) < 1e-13, (R, r)


@pytest.mark.parametrize("name", ["ragged", "shell", "phase"])
def test_fp64_double_float_far_field_matches_native(api, name):
    """The FP64 path's far field in double-float FP32 arithmetic (the default)
    against the same field in native FP64 arithmetic: one vector and five in
    one launch, on an attenuating interior wavenumber (3.7 + 0.2i, 66 + 0.5i)
    and phases k|x - y| up to ~130 rad; both within the FP64 bar of the
    oracle's dense A_hat."""
    s = {"ragged": ragged_scene, "shell": lambda: scenes.shell_scene(1),
         "phase": lambda: scenes.sphere_scene(2, k0=60.0, k1=66.0 + 0.5j)}[name]()
    A = pmchwt.assemble(s)
    cd = ctx_for(api, s)
    cn = ctx_for(api, s, fp64_far=1)
    X = np.stack([scenes.random_complex(A.shape[0], 80 + r) for r in range(4)] + [scenes.smooth_trace_vector(s, 2)])
    for x in (X[0], X[4]):
        yd, yn = cd.apply(x, precision=0), cn.apply(x, precision=0)
        assert rel(yd, yn) < 1e-12
        assert rel(yd, A @ x) < TOL[0]
    Yd, Yn = cd.apply(X, precision=0), cn.apply(X, precision=0)
    for r in range(X.shape[0]):
        assert rel(Yd[r], Yn[r]) < 1e-12, r


def test_fp64_double_float_far_field_large_phase(api):
    """Phases k|x - y| up to ~10,000 rad (unit sphere, k0 = 5,000): the
    double-float far field, near build and reduction stay at the FP64 bar
    against native FP64 and the oracle; a geometry whose phases may pass
    1e5 rad is refused (native FP64 remains available)."""
    from paper_1910_01011_gb300._lib import BemError
    s = scenes.sphere_scene(2, k0=5000.0, k1=5250.0)
    A = pmchwt.assemble(s)
    x = scenes.random_complex(A.shape[0], 12)
    yd = ctx_for(api, s).apply(x, precision=0)
    yn = ctx_for(api, s, fp64_far=1).apply(x, precision=0)
    assert rel(yd, yn) < 1e-10
    assert rel(yd, A @ x) < 1e-10
    far = scenes.sphere_scene(2, k0=1.0e6, k1=1.05e6)
    with pytest.raises(BemError):
        ctx_for(api, far).apply(scenes.random_complex(A.shape[0], 13), precision=0)


def test_large_phase_accuracy_fp32(api):
    """k|x-y| up to ~120 rad on a unit sphere: the FP32 path keeps the
    phase through the tile-local offsets (a plain FP32 distance would lose
    ~1e-5 rad per term)."""
    s = scenes.sphere_scene(2, k0=60.0, k1=66.0 + 0.5j)
    A = pmchwt.assemble(s)
    c = ctx_for(api, s)
    x = scenes.random_complex(A.shape[0], 7)
    assert rel(c.apply(x, precision=1), A @ x) < TOL[1]


def test_plane_wave_rhs(api):
    s = scenes.two_sphere_scene(1)
    b_ref = pmchwt.rhs(s, pmchwt.plane_wave(s.k0, s.plane_wave_dir))
    c = ctx_for(api, s)
    c.set_plane_wave(s.plane_wave_dir)
    assert rel(c.rhs(), b_ref) < 1e-13


def test_mesh_errors_are_reported(api):
    from paper_1910_01011_gb300._lib import BemError
    c = api.Context()
    v, t = meshes.icosphere(1)
    with pytest.raises(BemError) as e:
        c.add_domain(v, t[:-1], 1.0, 1.0)          # open surface
    assert e.value.code == -2
    with pytest.raises(BemError) as e:
        c.add_domain(v, t[:, [0, 2, 1]][np.r_[0:40]].tolist() + t[40:].tolist(), 1.0, 1.0)  # mixed orientation
    assert e.value.code == -2
    bad = t.copy()
    bad[0, 0] = 10 ** 6
    with pytest.raises(BemError):
        c.add_domain(v, bad, 1.0, 1.0)


def test_memory_budget_is_enforced(api):
    from paper_1910_01011_gb300._lib import BemError
    s = scenes.sphere_scene(2)
    c = ctx_for(api, s, hbm_budget_bytes=1 << 16)
    with pytest.raises(BemError) as e:
        c.apply(np.ones(c.n_dofs, dtype=complex))
    assert e.value.code == -3


@pytest.mark.parametrize("prec", [0, 1])
def test_autotuned_launch_shape_keeps_parity(api, prec):
    """The autotuner's chosen source-chunk length is one of the candidates and
    the operator it then applies still meets the precision's bar; a second
    context of the same size reuses the cached choice."""
    s = ragged_scene()
    A = pmchwt.assemble(s)
    c = ctx_for(api, s)
    t = c.autotune(prec)
    assert t["chunk_tiles"] in (0, 8, 16, 32, 64, 128, 256) and t["ms"] > 0
    x = scenes.random_complex(A.shape[0], 9)
    assert rel(c.apply(x, precision=prec), A @ x) < TOL[prec]
    c2 = ctx_for(api, s)
    assert c2.autotune(prec, timed=False)["chunk_tiles"] == t["chunk_tiles"]
    assert rel(c2.apply(x, precision=prec), A @ x) < TOL[prec]


def test_group_apply_matches_single_applies(api):
    """Several meshes in one far-field launch (bem_apply_group): each result
    matches that context's own FP32 application and the oracle; the replayed
    graph gives the same result again, and new vectors are captured anew."""
    import torch
    built = [scenes.sphere_scene(2), scenes.two_sphere_scene(1), scenes.shell_scene(1), ragged_scene(),
             scenes.sphere_scene(1)]
    ctxs = [ctx_for(api, s) for s in built]
    xs = [torch.from_numpy(scenes.random_complex(c.n_dofs, 30 + i)).cuda() for i, c in enumerate(ctxs)]
    ys = api.apply_group(ctxs, xs)
    torch.cuda.synchronize()
    first = [y.cpu().numpy() for y in ys]
    for c, s, x, y in zip(ctxs, built, xs, first):
        own = c.apply(x.cpu().numpy(), precision=1)
        assert rel(y, own) < 1e-6
        A = pmchwt.assemble(s)
        assert rel(y, A @ x.cpu().numpy()) < TOL[1]
    ys2 = api.apply_group(ctxs, xs, ys)      # same vectors: the captured graph is replayed
    torch.cuda.synchronize()
    for y, y0 in zip(ys2, first):
        assert np.array_equal(y.cpu().numpy(), y0)
    xs[2] = torch.from_numpy(scenes.random_complex(ctxs[2].n_dofs, 99)).cuda()   # a new vector: new capture
    ys3 = api.apply_group(ctxs, xs)
    torch.cuda.synchronize()
    assert rel(ys3[2].cpu().numpy(), ctxs[2].apply(xs[2].cpu().numpy(), precision=1)) < 1e-6
    assert np.array_equal(ys3[0].cpu().numpy(), first[0])
