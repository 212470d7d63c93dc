"""Oracle: Algorithm 2 (RSD) with the V-hat truncation of Sec. 3.2 (FP64, CPU).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package.

Algorithm 2 at a node t with children c (octree reading: 8 children instead of L, R):
  1. v <- RSD on each child subtree (recursion; leaves solve K_ll u = f exactly),
  2. g = f_I - sum_{l in V-hat_t} K_{I l} v_l,
  3. u_I ~= S~^-1 g, S~ applied by Algorithm 1 (S-MatVec),
  4. w_l = K_{l I} u_I, z_l = K_ll^-1 w_l, u_l = v_l - z_l for l in V-hat_t,
  5. every other DOF of the subtree keeps the value the recursion returned.
Readings (3-D): V-hat_t = the leaves inside the subtree of t that are coupled to
I_t (in 2-D it is the single true sub-domain beside the interface); step 2 uses only
those leaves' values (lower interfaces are not subtracted); Algorithm 1's two
partial products K_II^(L-hat) x + K_II^(R-hat) x sum to K_II x.  Hence
    S~_t = K_{I I} - sum_{l in V-hat_t} K_{I l} K_ll^-1 K_{l I},
which equals the principal block S_Gamma[I_t, I_t] of the Schur complement of K onto
all interface DOFs (S_Gamma = K_GG - K_GW K_WW^-1 K_WG, W = union of leaf interiors).
gamma = 0 means S~ u_I = g is solved exactly (dense); gamma > 0 runs gamma GMRES
iterations (x0 = 0, no restart, modified Gram-Schmidt, no inner preconditioner).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .partition import Symbolic


class PaperRSD:
    def __init__(self, A: sp.csr_matrix, sym: Symbolic, gamma: int = 0):
        self.A = A.tocsr()
        self.sym = sym
        self.gamma = gamma
        self.leaves = sym.leaves()
        self.leaf_lu = {l: spla.splu(self.A[sym.I[l]][:, sym.I[l]].tocsc()) for l in self.leaves}
        # V-hat_t and the couplings K_{I_t, l}
        self.vhat: dict[int, list[int]] = {}
        self.K_Il: dict[tuple[int, int], sp.csr_matrix] = {}
        self.K_lI: dict[tuple[int, int], sp.csr_matrix] = {}
        for t in range(sym.n_nodes):
            if not sym.children[t]:
                continue
            I = sym.I[t]
            hits = []
            for l in self.leaves:
                if self._in_subtree(l, t):
                    blk = self.A[I][:, sym.I[l]]
                    if blk.nnz:
                        hits.append(l)
                        self.K_Il[(t, l)] = blk.tocsr()
                        self.K_lI[(t, l)] = self.A[sym.I[l]][:, I].tocsr()   # K_lI (K may be nonsymmetric)
            self.vhat[t] = hits
        self.S_dense: dict[int, np.ndarray] = {}
        if gamma == 0:
            for t in self.vhat:
                self.S_dense[t] = self.s_tilde(t)

    def _in_subtree(self, d: int, t: int) -> bool:
        while d >= 0:
            if d == t:
                return True
            d = self.sym.parent[d]
        return False

    # Algorithm 1: y = S~ x on interface I_t
    def s_matvec(self, t: int, x: np.ndarray) -> np.ndarray:
        I = self.sym.I[t]
        y = self.A[I][:, I] @ x
        for l in self.vhat[t]:
            w = self.leaf_lu[l].solve(self.K_lI[(t, l)] @ x)
            y -= self.K_Il[(t, l)] @ w
        return y

    def s_tilde(self, t: int) -> np.ndarray:
        I = self.sym.I[t]
        S = self.A[I][:, I].toarray()
        for l in self.vhat[t]:
            S -= self.K_Il[(t, l)].toarray() @ self.leaf_lu[l].solve(self.K_lI[(t, l)].toarray())
        return S

    def _interface_solve(self, t: int, g: np.ndarray) -> np.ndarray:
        if self.gamma == 0:
            return np.linalg.solve(self.S_dense[t], g)
        return gmres_fixed(lambda x: self.s_matvec(t, x), g, self.gamma)

    # Algorithm 2, literal recursion over the tree
    def apply_recursive(self, f: np.ndarray) -> np.ndarray:
        u = np.zeros_like(f, dtype=np.float64)
        self._rsd(0, f, u)
        return u

    def _rsd(self, t: int, f: np.ndarray, u: np.ndarray) -> None:
        sym = self.sym
        if not sym.children[t]:
            u[sym.I[t]] = self.leaf_lu[t].solve(f[sym.I[t]])
            return
        for c in sym.children[t]:
            self._rsd(c, f, u)
        self._interface_step(t, f, u)

    def _interface_step(self, t: int, f: np.ndarray, u: np.ndarray) -> None:
        sym = self.sym
        I = sym.I[t]
        g = f[I].astype(np.float64).copy()
        for l in self.vhat[t]:
            g -= self.K_Il[(t, l)] @ u[sym.I[l]]
        uI = self._interface_solve(t, g)
        u[I] = uI
        for l in self.vhat[t]:
            u[sym.I[l]] -= self.leaf_lu[l].solve(self.K_lI[(t, l)] @ uI)

    # the same computation flattened into level-wise sweeps (bottom-up)
    def apply_levelwise(self, f: np.ndarray) -> np.ndarray:
        sym = self.sym
        u = np.zeros_like(f, dtype=np.float64)
        for l in self.leaves:
            u[sym.I[l]] = self.leaf_lu[l].solve(f[sym.I[l]])
        for d in range(int(sym.depth.max()) - 1, -1, -1):
            for t in range(sym.n_nodes):
                if sym.depth[t] == d and sym.children[t]:
                    self._interface_step(t, f, u)
        return u

    def operator(self, n: int) -> np.ndarray:
        return np.stack([self.apply_recursive(e) for e in np.eye(n)], axis=1)


def schur_gamma(A: sp.csr_matrix, sym: Symbolic) -> tuple[np.ndarray, np.ndarray]:
    """S_Gamma = K_GG - K_GW K_WW^-1 K_WG over all interface DOFs G (dense, small n)."""
    leaves = set(sym.leaves())
    W = np.sort(np.concatenate([sym.I[l] for l in leaves]))
    G = np.sort(np.concatenate([sym.I[t] for t in range(sym.n_nodes) if t not in leaves]))
    A = A.tocsc()
    KWW = A[W][:, W].tocsc()
    KWG = A[W][:, G].toarray()
    S = A[G][:, G].toarray() - KWG.T @ spla.splu(KWW).solve(KWG)
    return S, G


def gmres_fixed(matvec, b: np.ndarray, iters: int) -> np.ndarray:
    """`iters` GMRES steps from x0 = 0 (no restart, modified Gram-Schmidt); returns
    the least-squares iterate after the last step (or earlier on exact breakdown)."""
    n = len(b)
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros(n)
    m = min(iters, n)
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = b / beta
    k_used = m
    for j in range(m):
        w = matvec(V[:, j])
        for i in range(j + 1):
            H[i, j] = V[:, i] @ w
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-14 * beta:
            k_used = j + 1
            break
        V[:, j + 1] = w / H[j + 1, j]
    e1 = np.zeros(k_used + 1)
    e1[0] = beta
    y, *_ = np.linalg.lstsq(H[:k_used + 1, :k_used], e1, rcond=None)
    return V[:, :k_used] @ y
