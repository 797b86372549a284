"""Parity of the OSRC preconditioner, the transducer right-hand side and the
GPU solves (plain FP64 GMRES and FP32-inner GMRES with FP64 residual
refinement) with the FP64 oracle, through the C ABI.  Bars: solved traces
within 1e-6 (relative l2) of the oracle's dense solution; the preconditioner
to 1e-9 (its sparse solves run to a 1e-12 relative residual)."""
import numpy as np
import pytest

from oracle import gmres, mie, osrc, pmchwt, rayleigh
from synth import scenes

pytestmark = pytest.mark.gpu

R_EPS = 0.2


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def api():
    from paper_1910_01011_gb300 import api, build
    build.build()
    return api


def ctx_for(api, s, **kw):
    kw.setdefault("r_eps", R_EPS)
    return api.Context.from_scene(s, **kw)


@pytest.mark.parametrize("name,npade,solver", [("sphere", 4, 0), ("two", 8, 0), ("shell", 4, 0), ("two", 8, 2),
                                                ("shell", 4, 2), ("two", 8, 1), ("shell", 4, 1), ("two", 8, 3),
                                                ("shell", 4, 3), ("two", 8, 4), ("shell", 4, 4)])
def test_preconditioner_matches_oracle(api, name, npade, solver):
    """Every sparse solver: automatic, one CTA per system and domain, grid-wide
    kernels, one thread-block cluster per system and domain, one cluster per
    group of Pade shifts."""
    s = {"sphere": lambda: scenes.sphere_scene(2), "two": lambda: scenes.two_sphere_scene(1),
         "shell": lambda: scenes.shell_scene(1)}[name]()
    pre = osrc.build(s, R_eps=R_EPS, n_pade=npade)
    c = ctx_for(api, s, n_pade=npade, osrc_solver=solver)
    rng = np.random.default_rng(8)
    x = rng.standard_normal(c.n_dofs) + 1j * rng.standard_normal(c.n_dofs)
    assert rel(c.apply(x, op=api.PREC), osrc.apply(s, pre, x)) < 1e-9
    A = pmchwt.assemble(s)
    ref = osrc.apply(s, pre, A @ x)
    assert rel(c.apply(x, op=api.PREC_AHAT, precision=api.FP64), ref) < 1e-9
    assert rel(c.apply(x, op=api.PREC_AHAT, precision=api.FP32), ref) < 2e-5


@pytest.fixture(scope="module")
def sphere_ref():
    s = scenes.sphere_scene(3)
    u, A, b = pmchwt.solve(s, pmchwt.plane_wave(s.k0, (0, 0, 1)))
    return s, u, A, b


def _traces(c, s):
    out = []
    for j, d in enumerate(s.domains):
        D, Nn = c.traces(j)
        out.append(np.concatenate([Nn, D]))
    return np.concatenate(out)


@pytest.mark.parametrize("precision,precondition,flexible", [(0, 1, 1), (1, 1, 1), (0, 1, 0), (1, 1, 0), (0, 0, 1)])
def test_sphere_solve_matches_oracle(api, sphere_ref, precision, precondition, flexible):
    """Config-1 sphere (icosphere level 3, k0=5, k1=5.25, density ratio 1.1,
    plane wave +z): GPU traces within 1e-6 of the oracle's dense solve, with
    the preconditioner on the right of a flexible GMRES (loose sparse solves)
    or on the left (the paper's composition)."""
    s, u, A, b = sphere_ref
    c = ctx_for(api, s, n_pade=4)
    c.set_plane_wave((0, 0, 1))
    assert rel(c.rhs(), b) < 1e-13
    rep = c.solve(precision=precision, precondition=precondition, tol=1e-10, restart=100, max_iter=3000,
                  flexible=flexible)
    assert rep["converged"], rep
    ug = _traces(c, s)
    assert rel(ug, u) < 1e-6, rep
    if precondition:
        assert rep["iterations"] < 120, rep
    if precision == 1:
        assert rep["refinements"] >= 1


def test_solve_mie_accuracy(api, sphere_ref):
    """End to end on the GPU: traces of the mixed-precision solve against the
    Mie series (the paper's < 3 % at about 6-8 elements per wavelength)."""
    s, u, A, b = sphere_ref
    c = ctx_for(api, s)
    c.set_plane_wave((0, 0, 1))
    c.solve(precision=1, tol=1e-8)
    d = s.domains[0]
    D, Nn = c.traces(0)
    pts = d.verts / np.linalg.norm(d.verts, axis=1)[:, None]
    eD, eN = mie.surface_traces(pts, 1.0, s.k0, d.k, s.rho0, d.rho)
    assert rel(D, eD) < 0.03 and rel(Nn, eN) < 0.03


def test_multi_domain_mixed_solve(api):
    s = scenes.shell_scene(1)
    u, A, b = pmchwt.solve(s, pmchwt.plane_wave(s.k0, s.plane_wave_dir))
    c = ctx_for(api, s)
    c.set_plane_wave(s.plane_wave_dir)
    rep = c.solve(precision=1, tol=1e-10)
    assert rep["converged"]
    assert rel(_traces(c, s), u) < 1e-6


def small_transducer(n=6, seed=3):
    tr = scenes.bowl_transducer(seed=seed, n_elem=n, R=4.0, aperture=3.0, piston_radius=0.3, gap=0.05)
    return tr


def test_transducer_rhs_and_multi_rhs_solve(api):
    """Rayleigh pistons (one excitation per piston and one focused set) on the
    two-sphere scene: right-hand sides against the oracle, and each solve of
    the batch equal to the oracle's dense solve of that excitation."""
    s = scenes.two_sphere_scene(1)
    tr = small_transducer()
    k0 = s.k0
    omega, rho0 = 2.0, 1.3
    W = np.vstack([np.eye(tr["radii"].size), scenes.focusing_weights(tr, k0)[None, :]]).astype(complex)
    c = ctx_for(api, s)
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], omega * rho0)
    c.set_excitations(W)
    B = c.rhs(W.shape[0])
    A = pmchwt.assemble(s)
    for r in range(W.shape[0]):
        ref = pmchwt.rhs(s, rayleigh.field(tr, W[r], k0, omega, rho0))
        assert rel(B[r], ref) < 1e-12
    rep = c.solve(precision=1, tol=1e-10)
    assert rep["converged"]
    for r in (0, W.shape[0] - 1):
        u = np.linalg.solve(A, B[r])
        got = np.concatenate([np.concatenate([c.traces(j, r)[1], c.traces(j, r)[0]]) for j in range(2)])
        assert rel(got, u) < 1e-6


def test_transducer_rhs_excitation_groups(api):
    """Right-hand sides of 37 excitations (the piston kernel's groups of 16
    excitations: two full, one ragged) mixing unit, sparse, dense random-phase
    and all-zero weight rows, so that pistons skipped for a whole group and
    pistons shared by several excitations both occur: every row against the
    oracle's Rayleigh field (a zero row gives an exactly zero right-hand side)."""
    s = scenes.two_sphere_scene(1)
    tr = small_transducer()
    ne = tr["radii"].size
    rng = np.random.default_rng(17)
    W = np.exp(2j * np.pi * rng.random((37, ne)))
    W[:ne] = np.eye(ne)                       # group 0: unit excitations, then dense rows
    W[16:32] *= rng.random((16, ne)) < 0.4    # group 1: sparse rows (some pistons unused by all)
    W[16:32, 2] = 0.0
    W[20] = 0.0                               # an all-zero row
    omega, rho0 = 2.0, 1.3
    c = ctx_for(api, s)
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], omega * rho0)
    c.set_excitations(W)
    B = c.rhs(W.shape[0])
    for r in range(W.shape[0]):
        if not W[r].any():
            assert not B[r].any(), r
            continue
        ref = pmchwt.rhs(s, rayleigh.field(tr, W[r], s.k0, omega, rho0))
        assert rel(B[r], ref) < 1e-12, r


def test_automatic_operator_mode(api):
    """operator_mode 2 resolves to the assembled operators on a small scene
    (36 N^2 bytes far below 4 GiB): the same solution and memory estimate
    as operator_mode 1; an out-of-range mode is refused."""
    from paper_1910_01011_gb300._lib import BemError
    s = scenes.two_sphere_scene(1)
    tr = small_transducer()
    W = np.exp(2j * np.pi * np.random.default_rng(4).random((3, tr["radii"].size)))
    sols, reps = [], []
    for mode in (1, 2):
        c = ctx_for(api, s)
        c.set_transducer(tr["centres"], tr["normals"], tr["radii"], 2.6)
        c.set_excitations(W)
        reps.append(c.solve(precision=1, tol=1e-10, batch_rhs=3, operator_mode=mode))
        sols.append(np.stack([c.solution(r) for r in range(3)]))
        if mode == 2:
            assert c.estimate_solve_bytes(3, batch_rhs=3, operator_mode=2) == \
                c.estimate_solve_bytes(3, batch_rhs=3, operator_mode=1)
            with pytest.raises(BemError):
                c.solve(operator_mode=3)
        c.close()
    # the near-field corrections enter the assembled matrices through atomic
    # additions, so two contexts agree to rounding, not bit for bit
    assert abs(reps[0]["iterations"] - reps[1]["iterations"]) <= 3
    assert rel(sols[1].ravel(), sols[0].ravel()) < 1e-8


def test_recycled_solution_space(api):
    """bem_solve_opts.recycle: solved pairs (b, u) of earlier batched solves
    start later ones.  Six pistons: excitations in the span of earlier ones
    start converged (no iteration); once six independent excitations were
    solved, any excitation does; every solution meets the oracle's dense
    solve; a material change drops the space (iterations again)."""
    s = scenes.two_sphere_scene(1)
    tr = small_transducer()
    A = pmchwt.assemble(s)
    rng = np.random.default_rng(31)
    W1 = np.exp(2j * np.pi * rng.random((4, 6)))
    W2 = (rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))) @ W1  # in the span of W1
    W3 = np.exp(2j * np.pi * rng.random((4, 6)))
    W4 = np.exp(2j * np.pi * rng.random((2, 6)))
    c = ctx_for(api, s)
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], 2.6)
    kw = dict(precision=1, batch_rhs=4, block_gmres=1, recycle=16, operator_mode=1)

    def run(W, tol):
        c.set_excitations(W)
        rep = c.solve(tol=tol, **kw)
        assert rep["converged"], rep
        B = c.rhs(W.shape[0]).reshape(W.shape[0], -1)
        for r in range(W.shape[0]):
            assert rel(c.solution(r), np.linalg.solve(A, B[r])) < 1e-6, r
        return rep["iterations"]

    assert run(W1, 1e-10) > 0
    assert run(W2, 1e-8) == 0
    assert run(W3, 1e-10) > 0
    assert run(W4, 1e-8) == 0
    d = s.domains[0]
    c.set_material(0, d.k, d.rho)  # same values: the operator is rebuilt, the space dropped
    assert run(W4, 1e-8) > 0


def test_solve_reports_not_converged(api):
    s = scenes.sphere_scene(2)
    c = ctx_for(api, s)
    c.set_plane_wave((0, 0, 1))
    rep = c.solve(precision=0, precondition=0, tol=1e-12, max_iter=5, restart=5)
    assert not rep["converged"] and rep["iterations"] <= 5


@pytest.mark.parametrize("solver", [0, 1, 3, 4])
def test_batched_preconditioner_matches_single(api, solver):
    """The preconditioner applied to several right-hand sides in one batch
    equals the oracle's column by column."""
    s = scenes.two_sphere_scene(1)
    pre = osrc.build(s, R_eps=R_EPS, n_pade=8)
    c = ctx_for(api, s, n_pade=8, osrc_solver=solver)
    X = scenes.random_complex(c.n_dofs * 5, 21).reshape(5, c.n_dofs)
    Y = c.apply(X, op=api.PREC)
    for r in range(5):
        assert rel(Y[r], osrc.apply(s, pre, X[r])) < 1e-9


@pytest.mark.parametrize("precision,operator_mode,flexible,block", [(0, 0, 1, 0), (1, 0, 1, 0), (1, 1, 1, 0), (0, 1, 1, 0),
                                                                    (1, 0, 0, 0), (1, 1, 1, 1), (0, 1, 1, 1),
                                                                    (1, 0, 1, 1), (1, 0, 0, 1)])
def test_batched_solve_matches_oracle(api, precision, operator_mode, flexible, block):
    """Excitations solved in blocks of batch_rhs = 3 over 7 excitations (so
    one ragged block), either as independent GMRES runs in lockstep or by block
    GMRES (one Krylov space per block): every column within 1e-6 of the
    oracle's dense solve, as the one-at-a-time path."""
    s = scenes.two_sphere_scene(1)
    tr = small_transducer()
    W = np.vstack([np.eye(tr["radii"].size), scenes.focusing_weights(tr, s.k0)[None, :]]).astype(complex)
    c = ctx_for(api, s)
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], 2.6)
    c.set_excitations(W)
    B = c.rhs(W.shape[0])
    A = pmchwt.assemble(s)
    rep = c.solve(precision=precision, tol=1e-10, batch_rhs=3, operator_mode=operator_mode, flexible=flexible,
                  block_gmres=block)
    assert rep["converged"], rep
    for r in range(W.shape[0]):
        u = np.linalg.solve(A, B[r])
        got = np.concatenate([np.concatenate([c.traces(j, r)[1], c.traces(j, r)[0]]) for j in range(2)])
        assert rel(got, u) < 1e-6, r


@pytest.mark.parametrize("precision", [1, 0])
def test_block_gmres_dependent_excitations(api, precision):
    """Block GMRES on a block whose right-hand sides are dependent: nine
    excitations of a six-piston array (one repeated, one all zero) in one
    block.  The block of starting residuals has rank six, so the solve takes
    the lockstep path for it; every column still meets the oracle's dense
    solve (the zero excitation gives a zero solution)."""
    s = scenes.two_sphere_scene(1)
    tr = small_transducer()
    rng = np.random.default_rng(23)
    W = np.exp(2j * np.pi * rng.random((9, tr["radii"].size)))
    W[4] = W[1]
    W[6] = 0.0
    c = ctx_for(api, s)
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], 2.6)
    c.set_excitations(W)
    B = c.rhs(W.shape[0])
    A = pmchwt.assemble(s)
    rep = c.solve(precision=precision, tol=1e-10, batch_rhs=9, operator_mode=1, block_gmres=1)
    assert rep["converged"], rep
    for r in range(W.shape[0]):
        got = np.concatenate([np.concatenate([c.traces(j, r)[1], c.traces(j, r)[0]]) for j in range(2)])
        if r == 6:
            assert np.linalg.norm(got) < 1e-12
            continue
        assert rel(got, np.linalg.solve(A, B[r])) < 1e-6, r


def test_superposition_matches_direct_solves(api):
    """Excitation superposition: the solutions of arbitrary piston weights,
    formed from the per-piston basis by one GEMM, equal direct solves of those
    excitations and the oracle's dense solves (traces are linear in the
    weights)."""
    s = scenes.two_sphere_scene(1)
    tr = small_transducer()
    A = pmchwt.assemble(s)
    c = ctx_for(api, s)
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], 2.6)
    with pytest.raises(Exception):
        c.superpose(np.ones((1, tr["radii"].size)))       # no basis yet
    rep = c.solve_basis(precision=1, tol=1e-12, batch_rhs=6)
    assert rep["converged"], rep
    basis = np.stack([c.solution(m) for m in range(tr["radii"].size)])  # the unit-excitation solutions
    W = np.exp(2j * np.pi * np.random.default_rng(4).random((3, tr["radii"].size)))
    U = c.superpose(W)
    assert rel(U, W @ basis) < 1e-12  # the product itself, to FP64 accuracy
    c.set_excitations(W)
    B = c.rhs(3)
    assert c.solve(precision=1, tol=1e-10)["converged"]
    for r in range(3):
        assert rel(U[r], c.solution(r)) < 1e-6
        assert rel(U[r], np.linalg.solve(A, B[r])) < 1e-6
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], 2.6)  # a new transducer drops the basis
    with pytest.raises(Exception):
        c.superpose(W)


def test_superposition_512_element_array(api):
    """A 512-element array (the size of the full-matrix-capture arrays the
    paper's introduction cites): every piston solved alone in lockstep
    batches of 64 (bem_solve_basis), then two random-phase patterns formed
    from the basis by one product, against the oracle's dense solves."""
    s = scenes.sphere_scene(2)
    tr = scenes.bowl_transducer(seed=5, n_elem=512, R=4.0, aperture=6.0, piston_radius=0.06, gap=0.02)
    A = pmchwt.assemble(s)
    c = ctx_for(api, s)
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], 2.6)
    rep = c.solve_basis(precision=1, tol=1e-10, batch_rhs=64)
    assert rep["converged"], rep
    W = np.exp(2j * np.pi * np.random.default_rng(12).random((2, 512)))
    U = c.superpose(W)
    for r in range(2):
        b = pmchwt.rhs(s, rayleigh.field(tr, W[r], s.k0, 2.6, 1.0))
        assert rel(U[r], np.linalg.solve(A, b)) < 1e-6
    c.close()
