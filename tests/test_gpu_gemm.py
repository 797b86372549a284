"""The tcgen05 split-BF16x3 complex GEMM (assembled-operator path) against
an FP64 product of the same complex64 inputs.  Bar: relative l2 <= 3e-5
per right-hand side (the split keeps all terms above ~2^-16 relative)."""
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
    assert err.max() < 3e-5
