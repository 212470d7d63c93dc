"""Oracle: adjoint solve and per-element coefficient gradient (FP64, CPU).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package.

The paper's solver handles K u = f with K from the FEM discretisation of Sec. 4.  For
-div(kappa grad u) with kappa constant per element, K is linear in kappa:
    K(kappa) = sum_e kappa_e K_e,    K_e = h * Khat restricted to the interior nodes of e,
so for a loss L(u) with u = K(kappa)^-1 b the adjoint method gives
    K^T lam = dL/du,    dL/dkappa_e = -lam_e^T K_e u_e,    dL/db = lam,
and with kappa = exp(m), dL/dm_e = kappa_e dL/dkappa_e.  K is symmetric, so the adjoint
system is a solve with the same matrix.  Everything here is the definition written out,
with a direct sparse solve standing in for the preconditioned Krylov solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem


def element_values(n: int, v: np.ndarray) -> np.ndarray:
    """(n_elem, 8) nodal values of an interior-node vector v on every element, local
    node a = ax + 2 ay + 4 az; Dirichlet boundary nodes contribute 0."""
    m, ne = n - 2, n - 1
    e = np.arange(ne ** 3)
    ex, ey, ez = e % ne, (e // ne) % ne, e // (ne * ne)
    out = np.zeros((ne ** 3, 8))
    for a in range(8):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        x, y, z = ex + ax, ey + ay, ez + az
        inside = (x >= 1) & (x <= m) & (y >= 1) & (y <= m) & (z >= 1) & (z <= m)
        out[inside, a] = v[fem.interior_id(n, x[inside], y[inside], z[inside])]
    return out


def coef_grad(n: int, u: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """dL/dkappa_e = -lam_e^T (h Khat) u_e for every element (the derivative of the
    bilinear form lam^T K(kappa) u in kappa_e, with the sign of the adjoint identity)."""
    h = 1.0 / (n - 1)
    Kref = fem.reference_stiffness()
    ue, le = element_values(n, u), element_values(n, lam)
    return -h * np.einsum("ea,ab,eb->e", le, Kref, ue)


def loss_and_grad(n: int, m: np.ndarray, b: np.ndarray, u_obs: np.ndarray) -> dict:
    """L = 1/2 |u - u_obs|^2 with u = K(exp(m))^-1 b; returns u, lam, L, dL/dm, dL/db."""
    kappa = np.exp(m)
    A = fem.assemble(n, kappa).tocsc()
    lu = spla.splu(A)
    u = lu.solve(b)
    r = u - u_obs
    lam = lu.solve(r)                      # K^T = K
    dkappa = coef_grad(n, u, lam)
    return dict(u=u, lam=lam, loss=0.5 * float(r @ r), dkappa=dkappa, dm=kappa * dkappa, db=lam)


def loss(n: int, m: np.ndarray, b: np.ndarray, u_obs: np.ndarray) -> float:
    A = fem.assemble(n, np.exp(m)).tocsc()
    r = spla.spsolve(A, b) - u_obs
    return 0.5 * float(r @ r)
