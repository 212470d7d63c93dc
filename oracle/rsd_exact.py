"""Oracle: exact recursive Schur decomposition (FP64, CPU, dense per tree node).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package.

Sec. 3.1 eliminates the two sub-domains L, R and leaves the interface system
S u_I = g with S = K_II - K_IL K_LL^-1 K_LI - K_IR K_RR^-1 K_RI (Eq. 3.2), then
recovers u_L, u_R by back-substitution (Eq. 3.3).  Sec. 3.2 applies the same step
at every level of the tree, recursing into the pseudo sub-domains.  This module is
that recursion carried out exactly (sub-domain and interface solves exact, no V-hat
truncation), which is the gamma -> infinity, V-hat = V limit of Algorithm 2; the
preconditioner it yields is K^-1 itself.

Per tree node t (postorder), with I = I_t and B = B_t (the ancestor DOFs coupled to
the subtree of t):
    F_t        = K restricted to the rows/columns of I (against I and B)
                 + sum over children c of U_c placed at the parent positions ea[c]
    F_t[I, I]  is the interface Schur complement S_t of Eq. 3.2 (children eliminated)
    L_t L_t^T  = F_t[I, I]                         (dense Cholesky)
    X_t        = F_t[B, I] L_t^-T
    U_t        = F_t[B, B] - X_t X_t^T             (what t contributes to ancestors)
Apply z = K^-1 r: the forward pass computes g of Eq. 3.2 level by level
(y_t = L_t^-1 (r_I + children's contributions), contribution_t = (...)_B - X_t y_t);
the backward pass is Eq. 3.3 (x_I = L_t^-T (y_t - X_t^T x_B)).  ExactFactorLU is the
same recursion for a nonsymmetric K (LU without pivoting per front).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .partition import Symbolic


class ExactFactor:
    def __init__(self, A: sp.csr_matrix, sym: Symbolic):
        self.sym = sym
        self.L: list[np.ndarray | None] = [None] * sym.n_nodes     # s x s lower
        self.X: list[np.ndarray | None] = [None] * sym.n_nodes     # b x s
        self.S: list[np.ndarray | None] = [None] * sym.n_nodes     # s x s (Eq. 3.2 at t)
        self.U: list[np.ndarray | None] = [None] * sym.n_nodes     # b x b
        A = A.tocsr()
        for t in sym.post:
            I, Bt = sym.I[t], sym.B[t]
            s, b = len(I), len(Bt)
            F = np.zeros((s + b, s + b))
            front = sym.front[t]
            if s:
                rows = A[I][:, front].toarray()              # (s, s+b): K[I, I u B]
                F[:s, :] = rows
                F[s:, :s] = rows[:, s:].T                    # K[B, I] = K[I, B]^T (K symmetric)
            for c in sym.children[t]:
                pos = sym.ea[c]
                F[np.ix_(pos, pos)] += self.U[c]
                self.U[c] = None                              # consumed by the parent
            self.S[t] = F[:s, :s].copy()
            L = np.linalg.cholesky(F[:s, :s]) if s else np.zeros((0, 0))
            X = sla.solve_triangular(L, F[s:, :s].T, lower=True).T if s and b else np.zeros((b, s))
            self.L[t], self.X[t] = L, X
            self.U[t] = F[s:, s:] - X @ X.T

    def apply(self, r: np.ndarray) -> np.ndarray:
        sym = self.sym
        y: list[np.ndarray | None] = [None] * sym.n_nodes
        contrib: list[np.ndarray | None] = [None] * sym.n_nodes
        for t in sym.post:
            s, b = sym.s(t), sym.b(t)
            v = np.zeros(s + b)
            v[:s] = r[sym.I[t]]
            for c in sym.children[t]:
                np.add.at(v, sym.ea[c], contrib[c])
            y[t] = sla.solve_triangular(self.L[t], v[:s], lower=True) if s else v[:0]
            contrib[t] = v[s:] - self.X[t] @ y[t]
        z = np.zeros_like(r, dtype=np.float64)
        for t in reversed(sym.post):
            s = sym.s(t)
            if not s:
                continue
            xB = z[sym.B[t]]
            z[sym.I[t]] = sla.solve_triangular(self.L[t], y[t] - self.X[t].T @ xB, lower=True, trans="T")
        return z

    def operator(self, n: int) -> np.ndarray:
        """The preconditioner as an explicit dense matrix (columns = apply(e_j)); tiny n only."""
        return np.stack([self.apply(e) for e in np.eye(n)], axis=1)


def schur_direct(A: sp.csr_matrix, sym: Symbolic, t: int) -> np.ndarray:
    """Eq. 3.2 written out for node t with its children as the sub-domains:
    S = K_II - sum_c K_{I,V_c} K_{V_c V_c}^-1 K_{V_c,I}, V_c = all DOFs of the subtree of c.
    (The children's subtrees are mutually uncoupled by Eq. 3.1, so their blocks are
    eliminated independently.)  Sparse direct solves; small problems only."""
    A = A.tocsc()
    I = sym.I[t]
    S = A[I][:, I].toarray()
    for c in sym.children[t]:
        V = np.sort(np.concatenate([sym.I[d] for d in subtree(sym, c)]))
        KVV = A[V][:, V].tocsc()
        KVI = A[V][:, I].toarray()
        S -= KVI.T @ spla.splu(KVV).solve(KVI)
    return S


def subtree(sym: Symbolic, t: int) -> list[int]:
    out, stack = [], [t]
    while stack:
        u = stack.pop()
        out.append(u)
        stack.extend(sym.children[u])
    return out


def dense_solve(A: sp.csr_matrix, b: np.ndarray) -> np.ndarray:
    """Reference solve by dense partial-pivot LU (LAPACK gesv); n up to ~20k."""
    return np.linalg.solve(A.toarray(), b)


def lu_nopivot(F: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Doolittle LU without row exchanges, F = L U with L unit lower, U upper (column by
    column elimination as in Sec. 3's Gaussian elimination of a sub-domain block).
    Raises ZeroDivisionError on an exactly zero pivot."""
    n = F.shape[0]
    A = F.astype(np.float64).copy()
    for k in range(n):
        if A[k, k] == 0.0:
            raise ZeroDivisionError(f"zero pivot at {k}")
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    L = np.tril(A, -1) + np.eye(n)
    U = np.triu(A)
    return L, U


class ExactFactorLU:
    """The exact recursion for a nonsymmetric K with a structurally symmetric pattern
    (the two-variable systems of Sec. 4, Eqs. 4.2-4.3).  Per tree node t (postorder):
        F_t        = K[I u B, I u B] entries owned by t + sum_c U_c at ea[c]
        F_t[I, I]  = L_t U_t                        (no pivoting)
        X_t        = F_t[B, I] U_t^-1,  Y_t = L_t^-1 F_t[I, B]
        U_t'       = F_t[B, B] - X_t Y_t            (t's contribution to its ancestors)
    apply: forward y_t = L_t^-1 (r_I + children), contribution v_B - X_t y_t; backward
    x_I = U_t^-1 (y_t - Y_t x_B) (Eqs. 3.2-3.3 with the two off-diagonal blocks distinct)."""

    def __init__(self, A: sp.csr_matrix, sym: Symbolic):
        self.sym = sym
        n_nodes = sym.n_nodes
        self.L: list = [None] * n_nodes
        self.Uf: list = [None] * n_nodes
        self.X: list = [None] * n_nodes
        self.Y: list = [None] * n_nodes
        self.S: list = [None] * n_nodes
        self.U: list = [None] * n_nodes
        A = A.tocsr()
        for t in sym.post:
            I, Bt = sym.I[t], sym.B[t]
            s, b = len(I), len(Bt)
            F = np.zeros((s + b, s + b))
            front = sym.front[t]
            if s:
                F[:s, :] = A[I][:, front].toarray()           # K[I, I u B]
                F[s:, :s] = A[Bt][:, I].toarray()            # K[B, I]
            for c in sym.children[t]:
                pos = sym.ea[c]
                F[np.ix_(pos, pos)] += self.U[c]
                self.U[c] = None
            self.S[t] = F[:s, :s].copy()
            L, U = lu_nopivot(F[:s, :s]) if s else (np.zeros((0, 0)), np.zeros((0, 0)))
            X = sla.solve_triangular(U, F[s:, :s].T, lower=False, trans="T").T if s and b else np.zeros((b, s))
            Y = sla.solve_triangular(L, F[:s, s:], lower=True, unit_diagonal=True) if s and b else np.zeros((s, b))
            self.L[t], self.Uf[t], self.X[t], self.Y[t] = L, U, X, Y
            self.U[t] = F[s:, s:] - X @ Y

    def apply(self, r: np.ndarray) -> np.ndarray:
        sym = self.sym
        y: list = [None] * sym.n_nodes
        contrib: list = [None] * sym.n_nodes
        for t in sym.post:
            s, b = sym.s(t), sym.b(t)
            v = np.zeros(s + b)
            v[:s] = r[sym.I[t]]
            for c in sym.children[t]:
                np.add.at(v, sym.ea[c], contrib[c])
            y[t] = sla.solve_triangular(self.L[t], v[:s], lower=True, unit_diagonal=True) if s else v[:0]
            contrib[t] = v[s:] - self.X[t] @ y[t]
        z = np.zeros_like(r, dtype=np.float64)
        for t in reversed(sym.post):
            if not sym.s(t):
                continue
            z[sym.I[t]] = sla.solve_triangular(self.Uf[t], y[t] - self.Y[t] @ z[sym.B[t]], lower=False)
        return z


def schur_direct_general(A: sp.csr_matrix, sym: Symbolic, t: int) -> np.ndarray:
    """Eq. 3.2 for a nonsymmetric K: S = K_II - sum_c K_{I,V_c} K_{V_c V_c}^-1 K_{V_c,I}."""
    A = A.tocsc()
    I = sym.I[t]
    S = A[I][:, I].toarray()
    for c in sym.children[t]:
        V = np.sort(np.concatenate([sym.I[d] for d in subtree(sym, c)]))
        S -= A[I][:, V].toarray() @ spla.splu(A[V][:, V].tocsc()).solve(A[V][:, I].toarray())
    return S
