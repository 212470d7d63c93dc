"""Oracle: the paper's own 2-D setting (Sec. 2 and Sec. 4), for pinning against Table 1.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package.

A long, thin strip of P true sub-domains, each meshed by an N x N node grid of
unit-square bilinear elements, joined along the length; homogeneous Dirichlet data
on all sides (Sec. 4).  The strip has P*(N-1)+1 by N nodes, so
(P*(N-1) - 1)*(N - 2) unknowns.  The binary tree of Sec. 2 halves the strip along
its length; every internal node's interface is the column of nodes on its mid line.
Node (x, y) with 1 <= x <= P*(N-1)-1, 1 <= y <= N-2 has id (x-1) + (X-1)*(y-1),
X = P*(N-1).  Element size is 1 (the Laplacian stiffness of a square bilinear
element does not depend on its size).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

GAUSS2 = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))


def reference_stiffness_2d() -> np.ndarray:
    """4x4 int_{[0,1]^2} grad(phi_a).grad(phi_b), local node a = ax + 2*ay, 2x2 Gauss."""
    K = np.zeros((4, 4))
    for gx in GAUSS2:
        for gy in GAUSS2:
            G = []
            for a in range(4):
                ax, ay = a & 1, (a >> 1) & 1
                lx = gx if ax else 1 - gx
                ly = gy if ay else 1 - gy
                G.append([(1 if ax else -1) * ly, lx * (1 if ay else -1)])
            G = np.array(G)
            K += 0.25 * G @ G.T
    return K


def strip_poisson(N: int, P: int) -> tuple[sp.csr_matrix, np.ndarray]:
    """Stiffness of -Laplace(u) on the strip and the (x, y) coords of its unknowns."""
    X, Y = P * (N - 1), N - 1                  # elements along / across
    nx, ny = X - 1, Y - 1                      # interior nodes along / across
    Kref = reference_stiffness_2d()
    rows, cols, vals = [], [], []
    ex, ey = np.meshgrid(np.arange(X), np.arange(Y), indexing="ij")
    ex, ey = ex.ravel(), ey.ravel()
    for a in range(4):
        xa, ya = ex + (a & 1), ey + ((a >> 1) & 1)
        ia = (xa >= 1) & (xa <= nx) & (ya >= 1) & (ya <= ny)
        for b in range(4):
            xb, yb = ex + (b & 1), ey + ((b >> 1) & 1)
            ib = (xb >= 1) & (xb <= nx) & (yb >= 1) & (yb <= ny)
            k = ia & ib
            rows.append((xa[k] - 1) + nx * (ya[k] - 1))
            cols.append((xb[k] - 1) + nx * (yb[k] - 1))
            vals.append(np.full(k.sum(), Kref[a, b]))
    n = nx * ny
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    ids = np.arange(n)
    coords = np.stack([ids % nx + 1, ids // nx + 1], axis=1)
    return A, coords


def binary_parent(height: int) -> np.ndarray:
    n_nodes = 2 ** (height + 1) - 1
    parent = np.full(n_nodes, -1, dtype=np.int64)
    for t in range(1, n_nodes):
        parent[t] = (t - 1) // 2
    return parent


def binary_owner(N: int, P: int, coords: np.ndarray) -> np.ndarray:
    """Owner of each unknown: the first tree node whose mid line holds it, else the leaf."""
    height = int(np.log2(P))
    x = coords[:, 0]
    lo = np.zeros(len(x), dtype=np.int64)
    hi = np.full(len(x), P * (N - 1), dtype=np.int64)
    node = np.zeros(len(x), dtype=np.int64)
    owner = np.full(len(x), -1, dtype=np.int64)
    for level in range(height + 1):
        open_ = owner < 0
        if level == height:
            owner[open_] = node[open_]
            break
        mid = lo + (hi - lo) // 2
        hit = open_ & (x == mid)
        owner[hit] = node[hit]
        go = open_ & ~hit
        right = x > mid
        node = np.where(go, 2 * node + 1 + right, node)
        lo = np.where(go & right, mid, lo)
        hi = np.where(go & ~right, mid, hi)
    return owner


def reference_mass_2d() -> np.ndarray:
    """4x4 int_{[0,1]^2} phi_a phi_b (consistent bilinear mass), 2x2 Gauss."""
    M = np.zeros((4, 4))
    for gx in GAUSS2:
        for gy in GAUSS2:
            phi = np.array([(gx if a & 1 else 1 - gx) * (gy if (a >> 1) & 1 else 1 - gy) for a in range(4)])
            M += 0.25 * np.outer(phi, phi)
    return M


def reference_stiffness_aniso(ax: float, ay: float) -> np.ndarray:
    """4x4 int_{[0,1]^2} ax phi_a,x phi_b,x + ay phi_a,y phi_b,y, 2x2 Gauss (size-free in 2-D)."""
    K = np.zeros((4, 4))
    for gx in GAUSS2:
        for gy in GAUSS2:
            G = []
            for a in range(4):
                bx, by = a & 1, (a >> 1) & 1
                lx = gx if bx else 1 - gx
                ly = gy if by else 1 - gy
                G.append([(1 if bx else -1) * ly, lx * (1 if by else -1)])
            G = np.array(G)
            K += 0.25 * (ax * np.outer(G[:, 0], G[:, 0]) + ay * np.outer(G[:, 1], G[:, 1]))
    return K


def strip_system(N: int, P: int, c: float) -> tuple[sp.csr_matrix, np.ndarray]:
    """The paper's two-variable systems (Sec. 4, Eqs. 4.2 and 4.3) on the strip:
        -u_xx/100 - u_yy + c v = f,   -c u - v_xx - v_yy/100 = g,
    c = 1/100 (Eq. 4.2) or 100 (Eq. 4.3).  Bilinear elements; every true sub-domain is a
    unit square of N x N nodes, so h = 1/(N-1): the stiffness of a square element does not
    depend on h in 2-D, the consistent mass scales with h^2.  DOF 2 * node + component
    (u = 0, v = 1), node ids as in strip_poisson; homogeneous Dirichlet on both variables.
    The zero-order coupling is skew (+c M, -c M), so K is nonsymmetric with the symmetric
    part blockdiag(K_u, K_v), which is positive definite."""
    X, Y = P * (N - 1), N - 1
    nx, ny = X - 1, Y - 1
    h = 1.0 / (N - 1)
    Ku = reference_stiffness_aniso(0.01, 1.0)
    Kv = reference_stiffness_aniso(1.0, 0.01)
    M = h * h * reference_mass_2d()
    ex, ey = np.meshgrid(np.arange(X), np.arange(Y), indexing="ij")
    ex, ey = ex.ravel(), ey.ravel()
    rows, cols, vals = [], [], []
    blocks = ((0, 0, Ku), (1, 1, Kv), (0, 1, c * M), (1, 0, -c * M))
    for a in range(4):
        xa, ya = ex + (a & 1), ey + ((a >> 1) & 1)
        ia = (xa >= 1) & (xa <= nx) & (ya >= 1) & (ya <= ny)
        for b in range(4):
            xb, yb = ex + (b & 1), ey + ((b >> 1) & 1)
            ib = (xb >= 1) & (xb <= nx) & (yb >= 1) & (yb <= ny)
            k = ia & ib
            na = (xa[k] - 1) + nx * (ya[k] - 1)
            nb = (xb[k] - 1) + nx * (yb[k] - 1)
            for ca, cb, E in blocks:
                rows.append(2 * na + ca)
                cols.append(2 * nb + cb)
                vals.append(np.full(k.sum(), E[a, b]))
    n = 2 * nx * ny
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    ids = np.arange(nx * ny)
    coords = np.stack([ids % nx + 1, ids // nx + 1], axis=1)
    return A, coords
