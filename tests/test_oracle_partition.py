"""Pins for the oracle's decomposition and interface sets (CPU only)."""
import numpy as np
import pytest

import synth
from oracle import fem, fem2d, partition


def _setup(n, depth, kappa=None):
    kappa = np.ones((n - 1) ** 3) if kappa is None else kappa
    A = fem.assemble(n, kappa)
    owner = partition.octree_owner(n, depth, fem.interior_coords(n))
    parent = partition.octree_parent(depth)
    return A, owner, parent


def _boxes(n, depth):
    """Box [lo, hi]^3 of every tree node, from the geometric split rule."""
    boxes = {0: (np.zeros(3, int), np.full(3, n - 1))}
    for t in range(len(partition.octree_parent(depth))):
        if 8 * t + 1 >= len(partition.octree_parent(depth)):
            continue
        lo, hi = boxes[t]
        mid = lo + (hi - lo) // 2
        for c in range(8):
            up = np.array([(c >> d) & 1 for d in range(3)], bool)
            boxes[8 * t + 1 + c] = (np.where(up, mid, lo), np.where(up, hi, mid))
    return boxes


def test_separator_closed_form_counts_full_size_diffusion129():
    # 129^3 nodes, depth 3: 48007 + 8*11719 + 64*2791 + 512*3375 = 2,048,383
    n, depth = 129, 3
    owner = partition.octree_owner(n, depth, fem.interior_coords(n))
    counts = np.bincount(owner, minlength=585)
    assert counts[0] == partition.separator_count(127) == 48007
    assert np.all(counts[1:9] == partition.separator_count(63)) and counts[1] == 11719
    assert np.all(counts[9:73] == partition.separator_count(31)) and counts[9] == 2791
    assert np.all(counts[73:] == 15 ** 3)
    assert counts.sum() == 2_048_383 == 127 ** 3


def test_elasticity_and_adjoint_sizes():
    owner = partition.octree_owner(65, 2, fem.interior_coords(65))
    assert np.bincount(owner).sum() == 250_047
    assert np.bincount(owner)[0] == partition.separator_count(63)
    assert 3 * 95 ** 3 == 2_572_125


def test_poisson13_sizes():
    A, owner, parent = _setup(13, 1)
    sym = partition.Symbolic(A, owner, parent)
    assert sym.s(0) == 331 and sym.b(0) == 0
    assert all(sym.s(t) == 125 and sym.b(t) == 91 for t in range(1, 9))


@pytest.mark.parametrize("n,depth", [(13, 1), (17, 2), (20, 2), (11, 2)])
def test_interfaces_equal_box_surfaces(n, depth):
    """B_t must be exactly the non-Dirichlet nodes on the closed surface of box t,
    and I_t the nodes on its mid-planes (internal) or inside it (leaf)."""
    A, owner, parent = _setup(n, depth)
    sym = partition.Symbolic(A, owner, parent)
    coords = fem.interior_coords(n)
    for t, (lo, hi) in _boxes(n, depth).items():
        inside = np.all((coords >= lo) & (coords <= hi), axis=1)
        strict = np.all((coords > lo) & (coords < hi), axis=1)
        surface = np.nonzero(inside & ~strict)[0]
        assert np.array_equal(sym.B[t], surface), t
        if sym.children[t]:
            mid = lo + (hi - lo) // 2
            mine = strict & np.any(coords == mid, axis=1)
        else:
            mine = strict
        # nodes strictly inside the box and on its planes, minus those owned by
        # an ancestor plane (never: they are strictly inside)
        assert np.array_equal(sym.I[t], np.nonzero(mine)[0]), t


@pytest.mark.parametrize("n,depth", [(13, 1), (17, 2)])
def test_interface_equals_neighbours_of_subtree(n, depth):
    """Non-recursive definition: B_t = adj(subtree(t)) minus subtree(t)."""
    A, owner, parent = _setup(n, depth)
    sym = partition.Symbolic(A, owner, parent)
    from oracle.rsd_exact import subtree
    for t in range(sym.n_nodes):
        V = np.concatenate([sym.I[d] for d in subtree(sym, t)])
        adj = np.unique(A[V].indices)
        assert np.array_equal(sym.B[t], np.setdiff1d(adj, V)), t


def test_extend_add_maps_point_at_same_dofs():
    A, owner, parent = _setup(17, 2)
    sym = partition.Symbolic(A, owner, parent)
    for t in range(1, sym.n_nodes):
        assert np.array_equal(sym.front[parent[t]][sym.ea[t]], sym.B[t])


def test_structure_check_accepts_and_rejects():
    A, owner, parent = _setup(13, 1)
    assert partition.check_structure(A, owner, parent)
    # plant a coupling between two different leaves: Eq. 3.1 forbids it
    i = int(np.nonzero(owner == 1)[0][0])
    j = int(np.nonzero(owner == 8)[0][0])
    B = A.tolil()
    B[i, j] = B[j, i] = -1.0
    assert not partition.check_structure(B.tocsr(), owner, parent)


def test_uneven_batched_depths():
    sizes = synth.batched_sizes(256, 4)
    assert sizes.min() >= 17 and sizes.max() <= 65
    assert synth.batched_depth(17) == 1 and synth.batched_depth(32) == 1
    assert synth.batched_depth(33) == 2


def test_binary_strip_partition():
    N, P = 9, 4
    A, coords = fem2d.strip_poisson(N, P)
    owner = fem2d.binary_owner(N, P, coords)
    parent = fem2d.binary_parent(2)
    assert partition.check_structure(A, owner, parent)
    counts = np.bincount(owner, minlength=7)
    assert np.all(counts[:3] == N - 2)                # interface columns
    assert np.all(counts[3:] == (N - 2) ** 2)         # leaf interiors
