"""Oracle: 3-D linear elasticity with trilinear hexahedra on a structured cube grid (FP64).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package.

The paper's Problem 4 (Sec. 4, Eq. 4.4) is a 2-D Navier-Lame system; its printed sign is
garbled, and the reading used here is the SPD form -div sigma(u) = f with
sigma = lambda tr(eps) I + 2 mu eps, eps = (grad u + grad u^T) / 2, extended to 3-D
(three DOFs per node).  Young's modulus E and Poisson's ratio nu give
lambda = E nu / ((1 + nu)(1 - 2 nu)), mu = E / (2 (1 + nu)).

Numbering: DOF = 3 * node + component, node = the interior node's natural id of fem.py.
The element matrix is B^T D B integrated by 2 x 2 x 2 Gauss points on the unit cube
(Voigt order xx, yy, zz, yz, xz, xy with engineering shear strains); on a cube of side
h it scales by E_e * h.  Boundary nodes are eliminated (homogeneous Dirichlet on every
component).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fem import GAUSS2, _corner_bits, _grad_phi, interior_id


def lame(E: float, nu: float) -> tuple[float, float]:
    return E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


def material_matrix(E: float, nu: float) -> np.ndarray:
    """6 x 6 isotropic elasticity matrix in Voigt notation (engineering shears)."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] = lam + 2.0 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    return D


def strain_matrix(xi: np.ndarray) -> np.ndarray:
    """6 x 24 strain-displacement matrix B at a point of the unit cube (column 3a + c is
    local node a, component c)."""
    B = np.zeros((6, 24))
    for a in range(8):
        gx, gy, gz = _grad_phi(a, xi)
        c = 3 * a
        B[0, c] = gx
        B[1, c + 1] = gy
        B[2, c + 2] = gz
        B[3, c + 1], B[3, c + 2] = gz, gy          # gamma_yz
        B[4, c], B[4, c + 2] = gz, gx              # gamma_xz
        B[5, c], B[5, c + 1] = gy, gx              # gamma_xy
    return B


def reference_stiffness(nu: float) -> np.ndarray:
    """24 x 24 element stiffness on the unit cube for E = 1 (2 x 2 x 2 Gauss, exact for
    the trilinear integrand)."""
    D = material_matrix(1.0, nu)
    K = np.zeros((24, 24))
    for gx in GAUSS2:
        for gy in GAUSS2:
            for gz in GAUSS2:
                B = strain_matrix(np.array([gx, gy, gz]))
                K += 0.125 * (B.T @ D @ B)
    return K


def rigid_body_modes(coords: np.ndarray) -> np.ndarray:
    """(3k, 6) displacement fields of the rigid motions at k points: three translations
    and three infinitesimal rotations (omega x x)."""
    k = coords.shape[0]
    R = np.zeros((3 * k, 6))
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    for c in range(3):
        R[c::3, c] = 1.0
    R[0::3, 3], R[1::3, 3] = -y, x                  # rotation about z
    R[1::3, 4], R[2::3, 4] = -z, y                  # rotation about x
    R[2::3, 5], R[0::3, 5] = -x, z                  # rotation about y
    return R


def leaf_of_element(n: int, depth: int) -> np.ndarray:
    """Leaf (0 .. 8^depth - 1, breadth-first order among the leaves) of each element: an
    element spans [e, e + 1] per coordinate and lies in the lower child of a box
    [lo, hi] when e < mid = lo + (hi - lo) // 2 (the octree of partition.py)."""
    ne = n - 1
    e = np.arange(ne ** 3)
    ec = np.stack([e % ne, (e // ne) % ne, e // (ne * ne)], axis=1)
    lo = np.zeros_like(ec)
    hi = np.full_like(ec, n - 1)
    node = np.zeros(len(e), dtype=np.int64)
    for _ in range(depth):
        mid = lo + (hi - lo) // 2
        upper = ec >= mid
        node = 8 * node + 1 + upper[:, 0] * 1 + upper[:, 1] * 2 + upper[:, 2] * 4
        lo = np.where(upper, mid, lo)
        hi = np.where(upper, hi, mid)
    first_leaf = (8 ** depth - 1) // 7
    return node - first_leaf


def assemble(n: int, E_elem: np.ndarray, nu: float, full: bool = False) -> sp.csr_matrix:
    """Global stiffness, element by element (K_e = E_e h Khat(nu)).  full=False: restricted
    to the interior nodes' DOFs (Dirichlet elimination, DOF 3 * interior id + c);
    full=True: every node of the grid, DOF 3 * (x + n (y + n z)) + c (for the patch test)."""
    h = 1.0 / (n - 1)
    m = n - 2
    ne = n - 1
    Kref = reference_stiffness(nu)
    e = np.arange(ne ** 3)
    ex, ey, ez = e % ne, (e // ne) % ne, e // (ne * ne)
    rows, cols, vals = [], [], []
    for a in range(8):
        ax, ay, az = _corner_bits(a)
        xa, ya, za = ex + ax, ey + ay, ez + az
        for b in range(8):
            bx, by, bz = _corner_bits(b)
            xb, yb, zb = ex + bx, ey + by, ez + bz
            if full:
                keep = np.ones(len(e), dtype=bool)
                ia = xa + n * (ya + n * za)
                ib = xb + n * (yb + n * zb)
            else:
                keep = ((xa >= 1) & (xa <= m) & (ya >= 1) & (ya <= m) & (za >= 1) & (za <= m) &
                        (xb >= 1) & (xb <= m) & (yb >= 1) & (yb <= m) & (zb >= 1) & (zb <= m))
                ia = interior_id(n, xa, ya, za)
                ib = interior_id(n, xb, yb, zb)
            for c in range(3):
                for d in range(3):
                    rows.append(3 * ia[keep] + c)
                    cols.append(3 * ib[keep] + d)
                    vals.append(E_elem[e[keep]] * h * Kref[3 * a + c, 3 * b + d])
    nd = 3 * (n ** 3 if full else m ** 3)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nd, nd)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def load_vector(n: int, f_nodal: np.ndarray) -> np.ndarray:
    """Lumped load b = h^3 f per DOF (f given per interior node and component, DOF order)."""
    h = 1.0 / (n - 1)
    return h ** 3 * np.asarray(f_nodal, dtype=np.float64)


def dof_owner(node_owner: np.ndarray) -> np.ndarray:
    """Owner tree node of each DOF: the owner of its node (three DOFs per node)."""
    return np.repeat(np.asarray(node_owner), 3)
