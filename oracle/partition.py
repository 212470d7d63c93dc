"""Oracle: hierarchical domain decomposition and interface index sets (CPU, integer).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package.

Sec. 2 builds a binary tree by halving a long, thin domain; its conclusions name
octrees as the 3-D extension.  Reading used here (octree generalisation):
  * every internal box [lo, hi]^3 (node coordinates, boundary layers included)
    splits at mid_d = lo_d + (hi_d - lo_d) // 2 in all three dimensions into 8
    children, child index cx + 2*cy + 4*cz;
  * an interior node belongs to the first box on the walk down from the root whose
    mid-planes contain it (the union of the three planes is that box's interface I);
    otherwise it descends into the child with c_d = (x_d > mid_d); nodes that reach a
    leaf box belong to that leaf (the "true" sub-domains of Sec. 2);
  * tree ids are breadth-first: root 0, children of t are 8t+1 .. 8t+8.
Sec. 3.1's block structure (Eq. 3.1, K_LR = 0) is the validity condition: every
nonzero K_ij must couple DOFs whose owners are ancestor-related.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def octree_parent(depth: int) -> np.ndarray:
    """Parent array of the complete octree of the given depth (BFS ids, parent[0] = -1)."""
    n_nodes = (8 ** (depth + 1) - 1) // 7
    parent = np.full(n_nodes, -1, dtype=np.int64)
    for t in range(1, n_nodes):
        parent[t] = (t - 1) // 8
    return parent


def octree_owner(n: int, depth: int, coords: np.ndarray) -> np.ndarray:
    """Owner tree node of each interior node (coords: (k, 3) node coordinates)."""
    k = coords.shape[0]
    lo = np.zeros((k, 3), dtype=np.int64)
    hi = np.full((k, 3), n - 1, dtype=np.int64)
    node = np.zeros(k, dtype=np.int64)
    owner = np.full(k, -1, dtype=np.int64)
    for level in range(depth + 1):
        open_ = owner < 0
        if level == depth:
            owner[open_] = node[open_]
            break
        mid = lo + (hi - lo) // 2
        on_plane = open_ & np.any(coords == mid, axis=1)
        owner[on_plane] = node[on_plane]
        go = open_ & ~on_plane
        upper = coords > mid                                  # (k, 3) bool
        child = upper[:, 0] * 1 + upper[:, 1] * 2 + upper[:, 2] * 4
        node = np.where(go, 8 * node + 1 + child, node)
        lo = np.where(go[:, None] & upper, mid, lo)
        hi = np.where(go[:, None] & ~upper, mid, hi)
    return owner


def children_of(parent: np.ndarray) -> list[list[int]]:
    ch: list[list[int]] = [[] for _ in range(len(parent))]
    for t in range(len(parent)):
        if parent[t] >= 0:
            ch[parent[t]].append(t)
    return ch


def depth_of(parent: np.ndarray) -> np.ndarray:
    d = np.zeros(len(parent), dtype=np.int64)
    for t in range(len(parent)):                    # BFS ids: parent[t] < t
        if parent[t] >= 0:
            d[t] = d[parent[t]] + 1
    return d


def postorder(parent: np.ndarray) -> list[int]:
    ch = children_of(parent)
    out: list[int] = []
    stack = [(0, False)]
    while stack:
        t, done = stack.pop()
        if done:
            out.append(t)
            continue
        stack.append((t, True))
        for c in reversed(ch[t]):
            stack.append((c, False))
    return out


def is_ancestor_or_self(parent: np.ndarray, a: int, b: int) -> bool:
    while b >= 0:
        if b == a:
            return True
        b = parent[b]
    return False


def check_structure(A: sp.csr_matrix, owner: np.ndarray, parent: np.ndarray) -> bool:
    """Eq. 3.1: no nonzero couples two DOFs whose owners are not ancestor-related
    (in particular no leaf-leaf coupling)."""
    coo = A.tocoo()
    pairs = set(zip(owner[coo.row].tolist(), owner[coo.col].tolist()))
    for a, b in pairs:
        if not (is_ancestor_or_self(parent, a, b) or is_ancestor_or_self(parent, b, a)):
            return False
    return True


class Symbolic:
    """Per tree node t: I[t] (DOFs owned by t, ascending), B[t] (DOFs outside the
    subtree of t that are coupled to it, ascending; all owned by proper ancestors),
    front[t] = I[t] ++ B[t], and for every non-root t the extend-add map ea[t]
    (positions of B[t] inside front[parent[t]])."""

    def __init__(self, A: sp.csr_matrix, owner: np.ndarray, parent: np.ndarray):
        self.parent = np.asarray(parent)
        self.owner = np.asarray(owner)
        self.n_nodes = len(parent)
        self.children = children_of(self.parent)
        self.depth = depth_of(self.parent)
        self.post = postorder(self.parent)
        n = A.shape[0]
        order = np.argsort(self.owner, kind="stable")
        counts = np.bincount(self.owner, minlength=self.n_nodes)
        starts = np.concatenate([[0], np.cumsum(counts)])
        self.I = [order[starts[t]:starts[t + 1]] for t in range(self.n_nodes)]
        self.B: list[np.ndarray] = [np.zeros(0, dtype=np.int64)] * self.n_nodes
        for t in self.post:
            rows = self.I[t]
            nbrs = A[rows].indices if len(rows) else np.zeros(0, dtype=np.int64)
            cand = np.unique(np.concatenate([nbrs] + [self.B[c] for c in self.children[t]]))
            keep = np.array([self._proper_ancestor(int(self.owner[j]), t) for j in cand], dtype=bool)
            self.B[t] = cand[keep].astype(np.int64) if len(cand) else cand.astype(np.int64)
        self.front = [np.concatenate([self.I[t], self.B[t]]) for t in range(self.n_nodes)]
        self.ea: list[np.ndarray | None] = [None] * self.n_nodes
        for t in range(self.n_nodes):
            p = self.parent[t]
            if p < 0:
                continue
            pos = np.empty(len(self.B[t]), dtype=np.int64)
            for k, j in enumerate(self.B[t]):
                i_hit = np.searchsorted(self.I[p], j)
                if i_hit < len(self.I[p]) and self.I[p][i_hit] == j:
                    pos[k] = i_hit
                else:
                    b_hit = np.searchsorted(self.B[p], j)
                    assert b_hit < len(self.B[p]) and self.B[p][b_hit] == j, "B_c not inside front(parent)"
                    pos[k] = len(self.I[p]) + b_hit
            self.ea[t] = pos
        assert sum(len(i) for i in self.I) == n

    def _proper_ancestor(self, a: int, t: int) -> bool:
        b = self.parent[t]
        while b >= 0:
            if b == a:
                return True
            b = self.parent[b]
        return False

    def s(self, t: int) -> int:
        return len(self.I[t])

    def b(self, t: int) -> int:
        return len(self.B[t])

    def leaves(self) -> list[int]:
        return [t for t in range(self.n_nodes) if not self.children[t]]


def separator_count(m: int) -> int:
    """Nodes on the three mid-planes of a box with m interior nodes per side (m odd):
    m^3 - (m-1)^3 = 3m^2 - 3m + 1."""
    return 3 * m * m - 3 * m + 1
