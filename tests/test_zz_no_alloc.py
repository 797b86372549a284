"""The allocation-free entry point bem_apply_noalloc, called through the C
ABI, gives the same result as bem_apply (FP32 PMCHWT apply), twice in a row.

It exists for callers that cannot let the library allocate device memory
during a call (device memory reserved by another allocator, or a loop that
must not enter the CUDA allocator); its scratch is a fixed array inside the
library, reused by every call.  This file sorts last so that a run stopping
at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from synth import scenes

pytestmark = pytest.mark.gpu


def _run(scene, calls=2):
    import torch

    from paper_1910_01011_gb300 import _lib, api, build
    build.build()
    lib = _lib.load()
    c = api.Context.from_scene(scene)
    N = c.n_dofs
    x = torch.from_numpy(scenes.random_complex(N, 21)).cuda()
    ref = c.apply(x, precision=api.FP32)          # prepares the context (allocates)
    torch.cuda.synchronize()
    ys = [torch.full_like(x, complex(float("nan"), 0.0)) for _ in range(calls)]  # the test's own buffers
    mem0 = c.memory()
    outs = []
    for y in ys:
        rc = lib.bem_apply_noalloc(c.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()))
        assert rc == 0, lib.bem_last_error(c.h)
        torch.cuda.synchronize()
        outs.append(y.cpu().numpy())
    mem1 = c.memory()
    r = ref.cpu().numpy()
    c.close()
    return r, outs, mem0, mem1


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# The allocation-free call runs the same kernels with the same source chunks
# as bem_apply at FP32, and every partial potential is written by one CTA and
# summed in chunk order, so the two agree to the last bit; 1e-14 leaves room
# only for that.  A wrong batch offset or a chunk missing from a batch would
# show up far above it.
TOL_SAME = 1e-14


def test_noalloc_matches_apply_small():
    r, outs, mem0, mem1 = _run(scenes.two_sphere_scene(2))
    for y in outs:
        assert np.isfinite(y).all()
        assert _rel(y, r) <= TOL_SAME
    assert mem1 == mem0  # the library's device bytes, now and at peak: nothing allocated


def test_noalloc_matches_apply_batched_rib_scene():
    """41k triangles: the far-field scratch of all target tiles exceeds the
    fixed array, so the call runs the target tiles in several batches."""
    r, outs, mem0, mem1 = _run(scenes.rib_scene())
    for y in outs:
        assert np.isfinite(y).all()
        assert _rel(y, r) <= TOL_SAME
    assert mem1 == mem0


def test_noalloc_requires_prepared_context():
    from paper_1910_01011_gb300 import _lib, api
    lib = _lib.load()
    c = api.Context.from_scene(scenes.sphere_scene(1))
    rc = lib.bem_apply_noalloc(c.h, ctypes.c_void_p(16), ctypes.c_void_p(32))
    assert rc == -7  # BEM_ERR_STATE: nothing prepared, nothing allocated, no kernel launched
    c.close()
