"""The C-ABI library builds, loads and exports every entry point that
include/bem.h declares; its host-side quadrature tables match the oracle's
independent derivation.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_01011_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|void)\s+(bem_\w+)\s*\(", src, re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_binding_covers_header():
    from paper_1910_01011_gb300 import _lib
    assert set(declared_symbols()) <= set(_lib._SIGS), set(declared_symbols()) - set(_lib._SIGS)


def test_regular_rule_matches_oracle(lib):
    from oracle import quadrature
    from paper_1910_01011_gb300.api import quadrature_table
    t = quadrature_table(0)
    l1, l2, w = quadrature.triangle_rule6()
    ours = sorted(map(tuple, np.round(t, 15)))
    ref = sorted(map(tuple, np.round(np.stack([l1, l2, w], 1), 15)))
    assert np.abs(np.array(ours) - np.array(ref)).max() < 1e-15


@pytest.mark.parametrize("n", [1, 2, 6, 11])
def test_gauss_legendre_matches_oracle(lib, n):
    from oracle import quadrature
    from paper_1910_01011_gb300.api import quadrature_table
    t = quadrature_table(1, n)
    ref = quadrature.gauss_legendre01(n)
    assert np.abs(t - ref).max() < 1e-15


def test_invalid_arguments_do_not_need_a_gpu(lib):
    # argument checks that fail before any device work
    buf = (ctypes.c_double * 256)()
    m = ctypes.c_int()
    assert lib.bem_quadrature_table(7, 6, buf, ctypes.byref(m)) == -1
    assert lib.bem_quadrature_table(1, 0, buf, ctypes.byref(m)) == -1
    assert lib.bem_destroy(None) == 0
    assert lib.bem_default_opts(None) == -1
    # null contexts and vectors are refused before any device work
    assert lib.bem_apply_group(None, 1, None, None) == -1
    assert lib.bem_apply_group(None, 0, None, None) == -1
    assert lib.bem_solve_basis(None, None, None) == -1
    assert lib.bem_superpose(None, None, 1, None, 0) == -1
    assert lib.bem_get_solution(None, 0, None, 0) == -1
    assert lib.bem_memory_info(None, None, None) == -1
    assert lib.bem_estimate_solve_bytes(None, 1, None, None) == -1
    assert lib.bem_autotune(None, 1, None, None) == -1
    assert lib.bem_server_destroy(None) == 0
    assert lib.bem_server_submit(None, 0, None, 1, None) == -1
    from paper_1910_01011_gb300 import _lib
    o = _lib.bem_server_opts()
    assert lib.bem_server_default_opts(ctypes.byref(o)) == 0
    assert o.slots == 2 and o.max_batch_rhs == 64 and o.solve.flexible == 1
