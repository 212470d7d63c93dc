"""Oracle: outer Krylov solvers (FP64, CPU).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package.

The paper wraps the RSD preconditioner in GMRES on K u = f, zero initial guess,
stopping on the relative 2-norm of the residual (Sec. 3 and Sec. 4).  For the SPD
systems with an exact (linear, symmetric) preconditioner, preconditioned CG is the
Krylov method used here; a flexible, right-preconditioned GMRES(m) covers the
nonsymmetric or nonlinear (finite gamma) preconditioners.
"""
from __future__ import annotations

import numpy as np


def pcg(A, b: np.ndarray, M, tol: float, maxit: int = 500):
    """Hestenes-Stiefel PCG from x0 = 0.  Stops when ||r_k|| / ||b|| <= tol on the
    recursively updated residual.  Returns (x, iterations, history of ||r_k||/||b||)."""
    x = np.zeros_like(b, dtype=np.float64)
    r = b.astype(np.float64).copy()
    bnorm = np.linalg.norm(b)
    hist = [1.0]
    if bnorm == 0.0:
        return x, 0, hist
    z = M(r)
    p = z.copy()
    rz = r @ z
    k = 0
    for k in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        hist.append(np.linalg.norm(r) / bnorm)
        if hist[-1] <= tol:
            break
        z = M(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, k, hist


def fgmres(A, b: np.ndarray, M, tol: float, restart: int = 30, maxit: int = 1000):
    """Right-preconditioned flexible GMRES(restart) from x0 = 0, modified Gram-Schmidt.
    Stops when the least-squares residual estimate ||r_k|| / ||b|| <= tol.
    Returns (x, total iterations, history)."""
    n = len(b)
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    hist = [1.0]
    if bnorm == 0.0:
        return x, 0, hist
    it = 0
    while it < maxit:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol:
            break
        V = np.zeros((n, restart + 1))
        Z = np.zeros((n, restart))
        H = np.zeros((restart + 1, restart))
        V[:, 0] = r / beta
        g = np.zeros(restart + 1)
        g[0] = beta
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        j_last = 0
        for j in range(restart):
            Z[:, j] = M(V[:, j])
            w = A @ Z[:, j]
            for i in range(j + 1):
                H[i, j] = V[:, i] @ w
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):                      # apply earlier Givens rotations
                tmp = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = tmp
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_last = j
            hist.append(abs(g[j + 1]) / bnorm)
            if hist[-1] <= tol or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_last + 1, :j_last + 1]), g[:j_last + 1])
        x = x + Z[:, :j_last + 1] @ y
        if hist[-1] <= tol:
            break
    return x, it, hist
