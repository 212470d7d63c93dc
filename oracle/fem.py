"""Oracle: trilinear hexahedral FEM on a structured cube grid (FP64, CPU).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package;
only tests/, the smoke check and the bench's CPU-baseline leg use it.

The paper discretises with bilinear elements on regular grids with homogeneous
Dirichlet data on every side (Sec. 4); the 3-D generalisation uses trilinear
hexahedra on an n x n x n node grid of the unit cube, h = 1/(n-1).  Boundary
nodes are eliminated (their rows and columns are dropped, not penalised).

Numbering: node (x, y, z), 0 <= x, y, z <= n-1; interior nodes get the natural
id (x-1) + m*((y-1) + m*(z-1)) with m = n-2.  Element (ex, ey, ez) has id
ex + (n-1)*(ey + (n-1)*ez); its local node a = ax + 2*ay + 4*az sits at
(ex+ax, ey+ay, ez+az).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

GAUSS2 = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))   # on [0, 1], weights 1/2


def _corner_bits(a: int) -> tuple[int, int, int]:
    return a & 1, (a >> 1) & 1, (a >> 2) & 1


def _grad_phi(a: int, xi: np.ndarray) -> np.ndarray:
    """Gradient of the trilinear shape function of local node a on the unit cube."""
    bits = _corner_bits(a)
    lin = [xi[d] if bits[d] else 1.0 - xi[d] for d in range(3)]
    dlin = [1.0 if bits[d] else -1.0 for d in range(3)]
    return np.array([dlin[0] * lin[1] * lin[2],
                     lin[0] * dlin[1] * lin[2],
                     lin[0] * lin[1] * dlin[2]])


def reference_stiffness() -> np.ndarray:
    """8x8 matrix int_{[0,1]^3} grad(phi_a) . grad(phi_b), by 2x2x2 Gauss quadrature
    (exact: the integrand has degree <= 2 in each coordinate)."""
    K = np.zeros((8, 8))
    for gx in GAUSS2:
        for gy in GAUSS2:
            for gz in GAUSS2:
                xi = np.array([gx, gy, gz])
                G = np.stack([_grad_phi(a, xi) for a in range(8)])
                K += 0.125 * (G @ G.T)
    return K


def reference_mass() -> np.ndarray:
    """8x8 consistent mass matrix on the unit cube, by 2x2x2 Gauss quadrature."""
    M = np.zeros((8, 8))
    for gx in GAUSS2:
        for gy in GAUSS2:
            for gz in GAUSS2:
                xi = (gx, gy, gz)
                phi = np.array([np.prod([xi[d] if b else 1.0 - xi[d]
                                         for d, b in enumerate(_corner_bits(a))])
                                for a in range(8)])
                M += 0.125 * np.outer(phi, phi)
    return M


def interior_id(n: int, x, y, z):
    m = n - 2
    return (x - 1) + m * ((y - 1) + m * (z - 1))


def interior_coords(n: int) -> np.ndarray:
    """(n_dof, 3) array of (x, y, z) node coordinates of the interior nodes, in id order."""
    m = n - 2
    ids = np.arange(m ** 3)
    return np.stack([ids % m + 1, (ids // m) % m + 1, ids // (m * m) + 1], axis=1)


def assemble(n: int, kappa: np.ndarray, chunk: int = 1 << 18) -> sp.csr_matrix:
    """Global stiffness of -div(kappa grad u) with kappa constant per element,
    assembled element by element (K_e = kappa_e * h * Khat) and restricted to the
    interior nodes.  Returns CSR with sorted column indices, duplicates summed."""
    h = 1.0 / (n - 1)
    m = n - 2
    ne = n - 1
    Kref = reference_stiffness()
    A = sp.csr_matrix((m ** 3, m ** 3))
    for e0 in range(0, ne ** 3, chunk):
        e = np.arange(e0, min(e0 + chunk, ne ** 3))
        ex, ey, ez = e % ne, (e // ne) % ne, e // (ne * ne)
        rows, cols, vals = [], [], []
        for a in range(8):
            ax, ay, az = _corner_bits(a)
            xa, ya, za = ex + ax, ey + ay, ez + az
            ia = (xa >= 1) & (xa <= m) & (ya >= 1) & (ya <= m) & (za >= 1) & (za <= m)
            for b in range(8):
                bx, by, bz = _corner_bits(b)
                xb, yb, zb = ex + bx, ey + by, ez + bz
                ib = (xb >= 1) & (xb <= m) & (yb >= 1) & (yb <= m) & (zb >= 1) & (zb <= m)
                keep = ia & ib
                rows.append(interior_id(n, xa[keep], ya[keep], za[keep]))
                cols.append(interior_id(n, xb[keep], yb[keep], zb[keep]))
                vals.append(kappa[e[keep]] * h * Kref[a, b])
        part = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(m ** 3, m ** 3)).tocsr()
        A = A + part
    A = A.tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def assemble_row(n: int, kappa: np.ndarray, node: int) -> dict[int, float]:
    """One row of the global matrix, by looping over the (up to) 8 elements that
    contain interior node `node`; used to spot-check rows of large problems."""
    h = 1.0 / (n - 1)
    m = n - 2
    ne = n - 1
    Kref = reference_stiffness()
    x, y, z = node % m + 1, (node // m) % m + 1, node // (m * m) + 1
    row: dict[int, float] = {}
    for ez in (z - 1, z):
        for ey in (y - 1, y):
            for ex in (x - 1, x):
                e = ex + ne * (ey + ne * ez)
                a = (x - ex) + 2 * (y - ey) + 4 * (z - ez)
                for b in range(8):
                    bx, by, bz = _corner_bits(b)
                    xb, yb, zb = ex + bx, ey + by, ez + bz
                    if 1 <= xb <= m and 1 <= yb <= m and 1 <= zb <= m:
                        j = int(interior_id(n, xb, yb, zb))
                        row[j] = row.get(j, 0.0) + kappa[e] * h * Kref[a, b]
    return row


def load_vector(n: int, f_nodal: np.ndarray) -> np.ndarray:
    """Lumped-mass load: b_i = h^3 f_i at each interior node (each interior node
    carries a lumped mass of exactly h^3 from its 8 surrounding elements)."""
    h = 1.0 / (n - 1)
    return h ** 3 * np.asarray(f_nodal, dtype=np.float64)
