"""Seeded synthetic surface meshes (closed, oriented, triangle surfaces).

Input generation only: every function here returns vertex coordinates and
triangle index lists.  Nothing in this module evaluates any part of the
boundary element method (no normals used by the solver, no quadrature, no
kernels); both the CUDA library and the FP64 oracle receive these arrays as
plain inputs.

Conventions: vertices are float64 arrays of shape (nv, 3) in metres (or the
unit sphere's units); triangles are int32 arrays of shape (nt, 3), ordered
counter-clockwise when seen from outside the enclosed volume, so that the
right-hand normal points out of the domain (the normal convention of the
paper's traces, Sec. 2.1).
"""
from __future__ import annotations

import math

import numpy as np


def _signed_volume(v: np.ndarray, t: np.ndarray) -> float:
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def orient_outward(v: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Flip every triangle if the enclosed signed volume is negative."""
    if _signed_volume(v, t) < 0:
        t = t[:, [0, 2, 1]].copy()
    return t


def icosahedron():
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [[-1, g, 0], [1, g, 0], [-1, -g, 0], [1, -g, 0],
         [0, -1, g], [0, 1, g], [0, -1, -g], [0, 1, -g],
         [g, 0, -1], [g, 0, 1], [-g, 0, -1], [-g, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int32)
    return v, orient_outward(v, f)


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Recursive midpoint subdivision of the icosahedron, each new vertex
    projected onto the sphere.  Level L has 10*4^L+2 vertices and 20*4^L
    triangles (level 3: 642 / 1280)."""
    v, f = icosahedron()
    verts = [tuple(p) for p in v]
    faces = [tuple(x) for x in f]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key in cache:
                return cache[key]
            p = (np.array(verts[a]) + np.array(verts[b])) * 0.5
            p /= np.linalg.norm(p)
            verts.append(tuple(p))
            cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    v = np.array(verts, dtype=np.float64) * radius + np.asarray(center, dtype=np.float64)
    t = np.array(faces, dtype=np.int32)
    return v, orient_outward(v, t)


def tetrahedron(scale: float = 1.0):
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64) * scale
    t = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], dtype=np.int32)
    return v, orient_outward(v, t)


def octahedron(scale: float = 1.0):
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                 dtype=np.float64) * scale
    t = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                  [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], dtype=np.int32)
    return v, orient_outward(v, t)


def rounded_box(semi, p: float, h: float, center=(0.0, 0.0, 0.0), equiangular=None):
    """Closed surface |x/a|^p + |y/b|^p + |z/c|^p = 1 (a superellipsoid;
    p = 2 is an ellipsoid, large p a box with rounded edges).

    Built from a structured triangulation of the box [-a,a]x[-b,b]x[-c,c]
    with grid spacing about h, each lattice point projected radially onto
    the superellipsoid.  For p == 2 the grid is tangent-warped (equiangular
    cube map) to even out triangle sizes."""
    semi = np.asarray(semi, dtype=np.float64)
    m = [max(1, int(math.ceil(2.0 * s / h))) for s in semi]
    if equiangular is None:
        equiangular = abs(p - 2.0) < 1e-12
    key_to_idx: dict[tuple[int, int, int], int] = {}
    pts: list[tuple[int, int, int]] = []

    def vid(I: int, J: int, K: int) -> int:
        k = (I, J, K)
        if k not in key_to_idx:
            key_to_idx[k] = len(pts)
            pts.append(k)
        return key_to_idx[k]

    tris = []
    for ax in range(3):
        u, w = (ax + 1) % 3, (ax + 2) % 3  # e_u x e_w = e_ax
        for side in (0, 1):
            for i in range(m[u]):
                for j in range(m[w]):
                    def P(di, dj):
                        c = [0, 0, 0]
                        c[ax] = side * m[ax]
                        c[u] = i + di
                        c[w] = j + dj
                        return vid(*c)
                    p00, p10, p11, p01 = P(0, 0), P(1, 0), P(1, 1), P(0, 1)
                    if side == 1:
                        tris += [(p00, p10, p11), (p00, p11, p01)]
                    else:
                        tris += [(p00, p11, p10), (p00, p01, p11)]
    L = np.array(pts, dtype=np.float64)
    q = -1.0 + 2.0 * L / np.asarray(m, dtype=np.float64)
    if equiangular:
        q = np.tan(q * (math.pi / 4.0))
    x = q * semi
    nrm = (np.abs(x / semi) ** p).sum(axis=1) ** (1.0 / p)
    v = x / nrm[:, None] + np.asarray(center, dtype=np.float64)
    t = np.array(tris, dtype=np.int32)
    return v, orient_outward(v, t)


def capsule(semi, p: float, h: float, center=(0.0, 0.0, 0.0)):
    """Rounded capsule elongated along x: a superelliptic tube
    |y/b|^p + |z/c|^p = 1 over |x| <= a - b, closed by superelliptic end
    caps of length b.  Built from the structured box triangulation, each
    lattice point projected from the nearest point of the core segment
    [-(a-b), a-b] x {0} x {0}."""
    a, b, c = (float(s) for s in semi)
    m = [max(1, int(math.ceil(2.0 * s / h))) for s in (a, b, c)]
    v0, t = rounded_box((a, b, c), 2.0, h, equiangular=False)
    # rebuild the box lattice positions (rounded_box projected them): recover
    # the box point by scaling each vertex back onto the box surface
    q = v0 / np.array([a, b, c])
    q = q / np.abs(q).max(axis=1, keepdims=True)
    x = q * np.array([a, b, c])
    s = a - b
    o = np.zeros_like(x)
    o[:, 0] = np.clip(x[:, 0], -s, s)
    d = x - o
    semi_cap = np.array([b, b, c])
    tt = (np.abs(d / semi_cap) ** p).sum(axis=1) ** (-1.0 / p)
    v = o + tt[:, None] * d + np.asarray(center, dtype=np.float64)
    return v, orient_outward(v, t)


def flip(v: np.ndarray, t: np.ndarray):
    """Reverse orientation (normals point inward): used for the inner
    surface of a hollow shell domain."""
    return v, t[:, [0, 2, 1]].copy()


def merge(parts):
    """Concatenate several closed surfaces into one vertex/triangle list
    (one domain made of disjoint components)."""
    vs, ts, off = [], [], 0
    for v, t in parts:
        vs.append(v)
        ts.append(t + off)
        off += v.shape[0]
    return np.concatenate(vs, axis=0), np.concatenate(ts, axis=0).astype(np.int32)


def mesh_stats(v: np.ndarray, t: np.ndarray) -> dict:
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    e = np.concatenate([np.linalg.norm(b - a, axis=1), np.linalg.norm(c - b, axis=1),
                        np.linalg.norm(a - c, axis=1)])
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    return {"nv": int(v.shape[0]), "nt": int(t.shape[0]), "h_mean": float(e.mean()),
            "h_max": float(e.max()), "area": float(area.sum())}
