"""The tcgen05 split-BF16 complex GEMM (assembled-operator path) against
an FP64 product of the same complex64 inputs.  Bar: relative l2 <= 5e-6
per right-hand side: the three-term split keeps all terms above ~2^-24 and
the accumulation is flushed to round-to-nearest FP32 every 256 of K."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1910_01011_gb300 import api, build
    build.build()
    c = api.Context()
    yield c
    c.close()


@pytest.mark.parametrize("m,k,n", [(128, 64, 64), (300, 200, 70), (1000, 1000, 256), (777, 1531, 5)])
def test_zgemm_bf16x3(ctx, m, k, n):
    import torch
    rng = np.random.default_rng(m + k + n)
    A = (rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))).astype(np.complex64)
    X = (rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))).astype(np.complex64)
    Ad, Xd = torch.from_numpy(A).cuda(), torch.from_numpy(X).cuda()
    Yd = torch.zeros((n, m), dtype=torch.complex64, device="cuda")
    rc = ctx.lib.bem_zgemm_bf16x3(ctx.h, m, k, n, ctypes.c_void_p(Ad.data_ptr()), ctypes.c_void_p(Xd.data_ptr()),
                                  ctypes.c_void_p(Yd.data_ptr()))
    assert rc == 0, ctx.lib.bem_last_error(ctx.h)
    Y = Yd.cpu().numpy().astype(np.complex128)
    ref = X.astype(np.complex128) @ A.astype(np.complex128).T
    err = np.linalg.norm(Y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    print("max rel err", err.max())
    assert err.max() < 5e-6


from oracle import pmchwt  # noqa: E402
from synth import scenes  # noqa: E402


@pytest.mark.parametrize("name", ["sphere", "shell", "two"])
def test_assembled_operator_matches_oracle(name):
    """BEM_PREC_BF16X3: A_hat assembled once in complex64 (regular rule +
    Sauter-Schwab corrections) and applied to a block of right-hand sides by
    the tensor-core GEMM, against the oracle's dense A_hat."""
    from paper_1910_01011_gb300 import api
    s = {"sphere": lambda: scenes.sphere_scene(2), "shell": lambda: scenes.shell_scene(1),
         "two": lambda: scenes.two_sphere_scene(2, k0=12.0, k1=13.0 + 0.4j, k2=10.5)}[name]()
    A = pmchwt.assemble(s)
    c = api.Context.from_scene(s)
    rng = np.random.default_rng(4)
    for n_rhs in (1, 3, 8, 15, 70):
        X = rng.standard_normal((n_rhs, A.shape[0])) + 1j * rng.standard_normal((n_rhs, A.shape[0]))
        Y = c.apply(X, precision=api.BF16X3)
        ref = X @ A.T
        err = np.linalg.norm(Y - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() < 2e-5, (n_rhs, err.max())
    c.close()


def test_context_rebuilds_after_adding_a_domain():
    """Adding a domain after applies and a solve releases the device state;
    the next apply and solve rebuild it (no stale buffers)."""
    from paper_1910_01011_gb300 import api
    s = scenes.two_sphere_scene(1)
    c = api.Context()
    c.set_exterior(s.k0, s.rho0)
    d0, d1 = s.domains
    c.add_domain(d0.verts, d0.tris, d0.k, d0.rho)
    c.set_plane_wave(s.plane_wave_dir)
    c.solve(precision=1, tol=1e-8)
    c.apply(np.ones(c.n_dofs, dtype=complex), precision=api.BF16X3)
    c.add_domain(d1.verts, d1.tris, d1.k, d1.rho)
    A = pmchwt.assemble(s)
    x = scenes.random_complex(A.shape[0], 9)
    for prec, tol in ((0, 1e-11), (1, 2e-5), (2, 2e-5)):
        y = c.apply(x, precision=prec)
        assert np.linalg.norm(y - A @ x) / np.linalg.norm(A @ x) < tol
    u, _, b = pmchwt.solve(s, pmchwt.plane_wave(s.k0, s.plane_wave_dir))
    rep = c.solve(precision=1, tol=1e-10)
    assert rep["converged"]
    got = np.concatenate([np.concatenate([c.traces(j)[1], c.traces(j)[0]]) for j in range(2)])
    assert np.linalg.norm(got - u) / np.linalg.norm(u) < 1e-6
    c.close()


@pytest.mark.parametrize("name", ["sphere", "shell"])
def test_fp64_assembled_operator_matches_oracle(name):
    """BEM_PREC_FP64_ASSEMBLED: A_hat assembled in complex128 and applied by
    the FP64-accurate split-FP32 product (the FP64 refinement residual), FP64
    bar 1e-11, for 1, 2, 5 and 9 right-hand sides (the launch shapes, 9 = a
    group of eight and a ragged one)."""
    from paper_1910_01011_gb300 import api
    s = {"sphere": lambda: scenes.sphere_scene(2), "shell": lambda: scenes.shell_scene(1)}[name]()
    A = pmchwt.assemble(s)
    c = api.Context.from_scene(s)
    rng = np.random.default_rng(6)
    for n_rhs in (1, 2, 5, 9):
        X = rng.standard_normal((n_rhs, A.shape[0])) + 1j * rng.standard_normal((n_rhs, A.shape[0]))
        Y = c.apply(X, precision=api.FP64_ASSEMBLED)
        ref = X @ A.T
        err = np.linalg.norm(Y - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() < 1e-11, err.max()
    c.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_with_assembled_operators(precision):
    """bem_solve with operator_mode = 1 (assembled operators for the inner
    iterations and the FP64 residual): traces within 1e-6 of the oracle."""
    from paper_1910_01011_gb300 import api
    s = scenes.sphere_scene(3)
    u, A, b = pmchwt.solve(s, pmchwt.plane_wave(s.k0, (0, 0, 1)))
    c = api.Context.from_scene(s, r_eps=0.2)
    c.set_plane_wave((0, 0, 1))
    rep = c.solve(precision=precision, tol=1e-10, operator_mode=1)
    assert rep["converged"], rep
    D, N = c.traces(0)
    got = np.concatenate([N, D])
    assert np.linalg.norm(got - u) / np.linalg.norm(u) < 1e-6
    c.close()
