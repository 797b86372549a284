"""ctypes front end of the FP64 C oracle (bem_oracle.c) plus plain numpy
surface geometry.  Test infrastructure only.

build() compiles bem_oracle.c with gcc (OpenMP) into oracle/_build/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import quadrature

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bem_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liborc.so")
_lib = None

REL_NONE, REL_VERTEX, REL_EDGE, REL_SAME, REL_NEAR = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        # no fused multiply-adds: the near-pair test must round exactly as written
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.orc_rows.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, ctypes.c_int, dp, ctypes.c_int, ip,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp,
                                  ctypes.c_int, dp, ip, ctypes.c_int, dp]
        _lib.orc_pair.argtypes = [dp, ip, dp, ip, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  dp, ctypes.c_int, dp, dp, ip]
        _lib.orc_ss_map.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, dp, dp, dp]
        _lib.orc_ss_nregions.argtypes = [ctypes.c_int]
        _lib.orc_rows_regular_evals.restype = ctypes.c_longlong
        _lib.orc_rows_regular_evals.argtypes = [ctypes.c_int, ip, ctypes.c_int, ip, ctypes.c_int]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class Rules:
    """Quadrature rules handed to the C oracle (defaults: the 6-point rule
    and 6 Gauss points per Sauter-Schwab direction)."""

    def __init__(self, regular=None, n_gauss: int = 6):
        self.qr = quadrature.rule_table(regular)
        self.gl = quadrature.gauss_legendre01(n_gauss)


DEFAULT_RULES = None


def default_rules() -> Rules:
    global DEFAULT_RULES
    if DEFAULT_RULES is None:
        DEFAULT_RULES = Rules()
    return DEFAULT_RULES


def operator_rows(vx, tx, vy, ty, same_surface: bool, k: complex, rows=None, rules: Rules | None = None):
    """Galerkin rows of (V, K, K', W) at wavenumber k between test surface
    (vx, tx) and trial surface (vy, ty).  rows: test vertex indices (None =
    all).  Returns 4 complex arrays of shape (len(rows), nvy)."""
    rules = rules or default_rules()
    vx = np.ascontiguousarray(vx, dtype=np.float64)
    vy = np.ascontiguousarray(vy, dtype=np.float64)
    tx = np.ascontiguousarray(tx, dtype=np.int32)
    ty = np.ascontiguousarray(ty, dtype=np.int32)
    nvx, nvy = vx.shape[0], vy.shape[0]
    if rows is None:
        rows = np.arange(nvx)
    rows = np.asarray(rows, dtype=np.int64)
    rowmap = np.full(nvx, -1, dtype=np.int32)
    rowmap[rows] = np.arange(rows.size, dtype=np.int32)
    out = np.zeros((4, rows.size, nvy), dtype=np.complex128)
    lib().orc_rows(nvx, _dp(vx), tx.shape[0], _ip(tx), nvy, _dp(vy), ty.shape[0], _ip(ty),
                   1 if same_surface else 0, float(np.real(k)), float(np.imag(k)),
                   rules.qr.shape[0], _dp(rules.qr), rules.gl.shape[0], _dp(rules.gl), _ip(rowmap),
                   rows.size, _dp(out.view(np.float64)))
    return out[0], out[1], out[2], out[3]


def operators(v, t, k, rules=None):
    """Dense Galerkin matrices (V, K, K', W) of one closed surface."""
    return operator_rows(v, t, v, t, True, k, None, rules)


def pair(vx3, ix, vy3, iy, same_surface, k, rules=None):
    rules = rules or default_rules()
    vx3 = np.ascontiguousarray(vx3, dtype=np.float64)
    vy3 = np.ascontiguousarray(vy3, dtype=np.float64)
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    out = np.zeros(36, dtype=np.complex128)
    rel = np.zeros(1, dtype=np.int32)
    lib().orc_pair(_dp(vx3), _ip(ix), _dp(vy3), _ip(iy), 1 if same_surface else 0, float(np.real(k)),
                   float(np.imag(k)), rules.qr.shape[0], _dp(rules.qr), rules.gl.shape[0], _dp(rules.gl),
                   _dp(out.view(np.float64)), _ip(rel))
    return out.reshape(4, 3, 3), int(rel[0])


def ss_points(rel: int, n_gauss: int):
    """All Sauter-Schwab points of one relation as arrays s (m,2), t (m,2)
    and weights (m,), exactly as the oracle integrates them."""
    gl = quadrature.gauss_legendre01(n_gauss)
    L = lib()
    nreg = L.orc_ss_nregions(rel)
    s = np.zeros(2)
    tt = np.zeros(2)
    jac = np.zeros(1)
    S, T, W = [], [], []
    for a in range(n_gauss):
        for b in range(n_gauss):
            for c in range(n_gauss):
                for e in range(n_gauss):
                    w = gl[a, 1] * gl[b, 1] * gl[c, 1] * gl[e, 1]
                    for reg in range(nreg):
                        L.orc_ss_map(rel, reg, gl[a, 0], gl[b, 0], gl[c, 0], gl[e, 0], _dp(s), _dp(tt), _dp(jac))
                        S.append(s.copy())
                        T.append(tt.copy())
                        W.append(w * jac[0])
    return np.array(S), np.array(T), np.array(W)


def regular_evals(tx, nty, rows, nvx, nq=6) -> int:
    tx = np.ascontiguousarray(tx, dtype=np.int32)
    rowmap = np.full(nvx, -1, dtype=np.int32)
    rowmap[np.asarray(rows)] = 0
    return int(lib().orc_rows_regular_evals(tx.shape[0], _ip(tx), int(nty), _ip(rowmap), nq))


# ---------------------------------------------------------------- geometry (numpy)


def tri_geometry(v, t):
    """Per-triangle unit normals (from the CCW order) and areas."""
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    cr = np.cross(b - a, c - a)
    ln = np.linalg.norm(cr, axis=1)
    return cr / ln[:, None], 0.5 * ln


def quad_points(v, t, rule=None):
    """Regular-rule points of every triangle: positions (nt, nq, 3), weights
    times area (nt, nq), P1 values (nq, 3)."""
    l1, l2, w = quadrature.triangle_rule6() if rule is None else rule
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    x = a[:, None, :] + l1[None, :, None] * (b - a)[:, None, :] + l2[None, :, None] * (c - a)[:, None, :]
    _, area = tri_geometry(v, t)
    phi = np.stack([1 - l1 - l2, l1, l2], axis=1)
    return x, area[:, None] * w[None, :], phi


def mass_matrix(v, t):
    """P1 mass matrix, exact: |T|/12 [[2,1,1],[1,2,1],[1,1,2]] per triangle."""
    import scipy.sparse as sp
    _, area = tri_geometry(v, t)
    loc = np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]], dtype=np.float64) / 12.0
    rows = np.repeat(t, 3, axis=1).ravel()
    cols = np.tile(t, (1, 3)).ravel()
    vals = (area[:, None, None] * loc[None]).ravel()
    n = v.shape[0]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def stiffness_matrix(v, t):
    """P1 surface stiffness int grad_G phi_i . grad_G phi_j, exact per
    triangle (constant gradients)."""
    import scipy.sparse as sp
    n, area = tri_geometry(v, t)
    P = [v[t[:, i]] for i in range(3)]
    grads = []
    for i in range(3):
        e = P[(i + 2) % 3] - P[(i + 1) % 3]
        grads.append(np.cross(n, e) / (2.0 * area[:, None]))
    loc = np.empty((t.shape[0], 3, 3))
    for i in range(3):
        for j in range(3):
            loc[:, i, j] = area * np.einsum("ij,ij->i", grads[i], grads[j])
    rows = np.repeat(t, 3, axis=1).ravel()
    cols = np.tile(t, (1, 3)).ravel()
    nv = v.shape[0]
    return sp.csr_matrix((loc.ravel(), (rows, cols)), shape=(nv, nv))


def project(v, t, f_at_points):
    """<f, phi_r> for every vertex r, with f given at the regular-rule points
    (nt, nq), integrated by the regular rule."""
    _, wa, phi = quad_points(v, t)
    loc = np.einsum("tq,tq,qa->ta", f_at_points, wa, phi)
    out = np.zeros(v.shape[0], dtype=np.result_type(loc.dtype, np.complex128))
    np.add.at(out, t.ravel(), loc.ravel())
    return out
