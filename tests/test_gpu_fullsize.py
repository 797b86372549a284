"""Full-size parity (the bench workload: rib / fat / liver scene, 41,292
triangles, 0.5 MHz) on outputs the FP64 oracle computes one row at a time:
both Galerkin rows of sampled vertices of every domain, for the FP32
matrix-free path (the configuration bench.py times) and the assembled
split-BF16 path."""
import numpy as np
import pytest

from oracle import pmchwt
from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rib():
    s = scenes.rib_scene()
    rng = np.random.default_rng(17)
    rows = [np.sort(rng.choice(d.verts.shape[0], size=6, replace=False)) for d in s.domains]
    x = scenes.smooth_trace_vector(s, 5) + 0.3 * scenes.random_complex(s.n_dofs, 6)
    ref = pmchwt.apply_rows(s, x, rows)
    return s, rows, x, ref


def _sampled(s, rows, y):
    off = pmchwt.offsets(s)
    out = []
    for j, d in enumerate(s.domains):
        nv = d.verts.shape[0]
        out.append(np.concatenate([y[off[j] + rows[j]], y[off[j] + nv + rows[j]]]))
    return out


def _errs(s, rows, y, ref):
    got = _sampled(s, rows, y)
    return [np.linalg.norm(g - np.concatenate(r)) / np.linalg.norm(np.concatenate(r)) for g, r in zip(got, ref)]


@pytest.mark.parametrize("prec,tol", [(1, 2e-5), (2, 2e-5)])
def test_rib_scene_sampled_rows(rib, prec, tol):
    from paper_1910_01011_gb300 import api
    s, rows, x, ref = rib
    c = api.Context.from_scene(s)
    y = c.apply(x, precision=prec)
    errs = _errs(s, rows, y, ref)
    print(prec, errs)
    assert max(errs) < tol
    c.close()
