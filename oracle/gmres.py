"""Restarted GMRES, FP64, numpy (test infrastructure only).

Textbook GMRES(m) (Saad & Schultz 1986): Arnoldi with modified
Gram-Schmidt, Givens rotations on the Hessenberg matrix, zero initial
guess, stopping on the relative residual ||r|| / ||b|| of the system it is
given (the paper's solver: SciPy GMRES, restart 100, Sec. 3).
"""
from __future__ import annotations

import numpy as np


def gmres(apply, b, tol=1e-8, restart=100, maxiter=2000, x0=None):
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else x0.astype(np.complex128).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, 0, [0.0]
    hist = []
    it = 0
    while it < maxiter:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol:
            break
        Q = np.zeros((n, restart + 1), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        Q[:, 0] = r / beta
        j_end = 0
        for j in range(restart):
            w = apply(Q[:, j])
            for i in range(j + 1):
                H[i, j] = np.vdot(Q[:, i], w)
                w = w - H[i, j] * Q[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                Q[:, j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[j] = a / den if den else 1.0
            sn[j] = c / den if den else 0.0
            H[j, j] = den
            H[j + 1, j] = 0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or it >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        x = x + Q[:, :j_end] @ y
        if hist[-1] <= tol:
            break
    return x, it, hist
