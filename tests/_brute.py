"""Brute-force element-pair integrals used to pin the oracle's singular
quadrature.  Independent of the oracle's Sauter-Schwab code: the inner
integral over the trial triangle is split into sub-triangles with apex at
the projection of the target point (Duffy collapse, which cancels the 1/r
singularity), the outer integral uses a high-order rule on a uniform
subdivision of the test triangle."""
import numpy as np


def gauss01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1), 0.5 * w


def tri_normal_area(P):
    c = np.cross(P[1] - P[0], P[2] - P[0])
    l = np.linalg.norm(c)
    return c / l, 0.5 * l


def bary(P, y):
    """Barycentric coordinates of points y (m,3) in the plane of P."""
    n, A = tri_normal_area(P)
    lam = []
    for i in range(3):
        a, b = P[(i + 1) % 3], P[(i + 2) % 3]
        lam.append(np.einsum("mi,i->m", np.cross(b - a, y - a), n) / (2 * A))
    return np.stack(lam, axis=1)


def inner(x, P, kern, n=24):
    """int_T kern(x, y, phi(y)) dy for one point x; kern returns (m, ...)
    values given y (m,3) and the three P1 values (m,3)."""
    nrm, _ = tri_normal_area(P)
    x0 = x - np.dot(x - P[0], nrm) * nrm
    u, wu = gauss01(n)
    U, V = np.meshgrid(u, u, indexing="ij")
    W = np.outer(wu, wu)
    total = 0
    for e in range(3):
        a, b = P[e], P[(e + 1) % 3]
        # signed sub-triangle (x0, a, b)
        sa = np.dot(np.cross(a - x0, b - x0), nrm)
        y = x0[None, None, :] + U[..., None] * ((a - x0)[None, None, :] + V[..., None] * (b - a)[None, None, :])
        y = y.reshape(-1, 3)
        jac = (U * sa).ravel()
        val = kern(y, bary(P, y))
        total = total + np.tensordot(W.ravel() * jac, val, axes=(0, 0))
    return total


def subdivide(P, levels):
    tris = [P]
    for _ in range(levels):
        nt = []
        for T in tris:
            a, b, c = T
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, c]), np.array([ab, bc, ca])]
        tris = nt
    return tris


def outer_points(P, levels=3, n=8):
    """Points and weights of a high-order rule on the subdivided triangle."""
    u, wu = gauss01(n)
    pts, wts = [], []
    for T in subdivide(P, levels):
        _, A = tri_normal_area(T)
        for i in range(n):
            for j in range(n):
                s, t = u[i], u[j]
                l1, l2 = s * (1 - t), s * t
                pts.append(T[0] + l1 * (T[1] - T[0]) + l2 * (T[2] - T[0]))
                wts.append(2 * A * wu[i] * wu[j] * s)
    return np.array(pts), np.array(wts)


def pair_matrices(PX, PY, k, levels=3, n_out=8, n_in=24):
    """Brute-force 3x3 (V, K, K', W) of one pair: same definitions as the
    oracle, P1 functions in each triangle's given vertex order."""
    nx, Ax = tri_normal_area(PX)
    ny, Ay = tri_normal_area(PY)

    def curls(P, n, A):
        return [np.cross(n, np.cross(n, P[(i + 2) % 3] - P[(i + 1) % 3])) / (2 * A) for i in range(3)]
    cx, cy = curls(PX, nx, Ax), curls(PY, ny, Ay)
    cc = np.array([[np.dot(cx[i], cy[j]) for j in range(3)] for i in range(3)])
    X, WX = outer_points(PX, levels, n_out)
    phx = bary(PX, X)
    out = np.zeros((4, 3, 3), dtype=np.complex128)
    for xi, wx, px in zip(X, WX, phx):
        def kern(y, py):
            d = xi[None, :] - y
            r = np.linalg.norm(d, axis=1)
            G = np.exp(1j * k * r) / (4 * np.pi * r)
            dGr = G * (1j * k - 1 / r) / r
            dny = dGr * (-(d @ ny))
            dnx = dGr * (d @ nx)
            v = np.empty((y.shape[0], 4, 3), dtype=np.complex128)
            v[:, 0] = G[:, None] * py
            v[:, 1] = dny[:, None] * py
            v[:, 2] = dnx[:, None] * py
            v[:, 3] = G[:, None] * py  # phi_j weight; curl and k^2 parts combined below
            Gs = G
            return np.concatenate([v.reshape(-1, 12), Gs[:, None]], axis=1)
        I = inner(xi, PY, kern, n_in)
        Iv = I[:12].reshape(4, 3)
        Ig = I[12]
        for i in range(3):
            out[0, i] += wx * px[i] * Iv[0]
            out[1, i] += wx * px[i] * Iv[1]
            out[2, i] += wx * px[i] * Iv[2]
            out[3, i] += wx * (cc[i] * Ig - k * k * np.dot(nx, ny) * px[i] * Iv[3])
    return out
