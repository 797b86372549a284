"""Parity on the anatomical stand-in scenes beyond the rib-scene rows of
test_gpu_fullsize.py.

* Kidney scene (kidney + hollow perinephric fat shell 1-8 mm off it, 1 MHz,
  61,996 triangles, k|x - y| up to ~545 rad): both Galerkin rows of sampled
  vertices of both domains, computed one at a time by the FP64 oracle, for
  the FP32 matrix-free path and the assembled split-BF16 path (bar 2e-5).
* Multi-domain solve, the form of the 256-RHS rib workload (one unit
  excitation per piston) on the rib / fat / liver scene at 6 mm elements
  (8,172 triangles, N = 8,200) at the frequency its mesh resolves (k h ~ 1):
  8 seeded pistons, each alone, solved by the oracle's dense LU and on the
  GPU by the mixed and the plain FP64 paths, each with the 8 excitations in
  lockstep and as one block GMRES (bar 1e-6 on the traces, eq.
  Galerkin_disc_lhs/_rhs1 with the Rayleigh incident field)."""
import numpy as np
import pytest

from oracle import pmchwt, rayleigh
from synth import scenes

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def kidney():
    s = scenes.kidney_scene()
    rng = np.random.default_rng(23)
    rows = [np.sort(rng.choice(d.verts.shape[0], size=6, replace=False)) for d in s.domains]
    x = scenes.smooth_trace_vector(s, 7) + 0.3 * scenes.random_complex(s.n_dofs, 8)
    ref = pmchwt.apply_rows(s, x, rows)
    return s, rows, x, ref


@pytest.mark.parametrize("prec,tol", [(1, 2e-5), (2, 2e-5)])
def test_kidney_scene_sampled_rows(kidney, prec, tol):
    from paper_1910_01011_gb300 import api
    s, rows, x, ref = kidney
    c = api.Context.from_scene(s)
    y = c.apply(x, precision=prec)
    off = pmchwt.offsets(s)
    errs = []
    for j, d in enumerate(s.domains):
        nv = d.verts.shape[0]
        got = np.concatenate([y[off[j] + rows[j]], y[off[j] + nv + rows[j]]])
        errs.append(rel(got, np.concatenate(ref[j])))
    print(prec, errs)
    assert max(errs) < tol
    c.close()


def test_kidney_scene_16_rhs_one_launch(kidney):
    """The kidney workload with 16 right-hand sides in one matrix-free FP32
    far-field launch: sampled rows of every column against the oracle."""
    from paper_1910_01011_gb300 import api
    s, rows, x, _ = kidney
    X = np.stack([x * np.exp(0.37j * r) + 0.2 * scenes.random_complex(s.n_dofs, 60 + r) for r in range(16)])
    c = api.Context.from_scene(s)
    Y = c.apply(X, precision=1)
    off = pmchwt.offsets(s)
    errs = []
    for r in (0, 7, 15):
        ref = pmchwt.apply_rows(s, X[r], rows)
        for j, d in enumerate(s.domains):
            nv = d.verts.shape[0]
            got = np.concatenate([Y[r][off[j] + rows[j]], Y[r][off[j] + nv + rows[j]]])
            errs.append(rel(got, np.concatenate(ref[j])))
    print(errs)
    assert max(errs) < 2e-5
    c.close()


RIB_SMALL_H = 6e-3
RIB_SMALL_FREQ = 0.1e6 * 2.65 / 6.0  # k h as for the 41k-triangle scene at 0.1 MHz


@pytest.fixture(scope="module")
def rib_small():
    """Oracle: dense A_hat (complex128), the 8 right-hand sides, dense LU."""
    s = scenes.rib_scene(h=RIB_SMALL_H, freq=RIB_SMALL_FREQ)
    tr = s.transducer
    n_elem = tr["radii"].size
    pistons = np.sort(np.random.default_rng(8).choice(n_elem, size=8, replace=False))
    A = pmchwt.assemble(s)
    omega = 2 * np.pi * s.freq
    # the field of a unit weight on piston m and zero elsewhere is that piston's field alone
    B = np.stack([pmchwt.rhs(s, rayleigh.field({k: tr[k][m:m + 1] for k in ("centres", "normals", "radii")}, [1.0],
                                                s.k0, omega, s.rho0)) for m in pistons], axis=1)
    U = np.linalg.solve(A, B)
    return s, pistons, B, U


@pytest.mark.parametrize("precision,batch,block", [(1, 8, 0), (0, 8, 0), (1, 8, 1), (0, 8, 1)])
def test_rib_scene_piston_solves_match_oracle(rib_small, precision, batch, block):
    from paper_1910_01011_gb300 import api
    s, pistons, B, U = rib_small
    tr = s.transducer
    n_elem = tr["radii"].size
    c = api.Context.from_scene(s, n_pade=8, r_eps=1e-4 * 1e6 / s.freq)
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], 2 * np.pi * s.freq * s.rho0)
    W = np.zeros((len(pistons), n_elem), dtype=np.complex128)
    W[np.arange(len(pistons)), pistons] = 1.0
    c.set_excitations(W)
    b = c.rhs(len(pistons))
    assert rel(b.reshape(len(pistons), -1).T, B) < 1e-12
    rep = c.solve(precision=precision, operator_mode=1, tol=1e-9, batch_rhs=batch, max_iter=20000, max_refine=20,
                  block_gmres=block)
    assert rep["converged"], rep
    errs = [rel(c.solution(r), U[:, r]) for r in range(len(pistons))]
    print(precision, rep, errs)
    assert max(errs) < 1e-6
    c.close()
