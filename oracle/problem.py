"""Oracle: assemble a synthetic workload into (K, f, owner, parent) on the CPU.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package.
"""
from __future__ import annotations

import time

import numpy as np

from . import fem, partition
from .krylov import pcg
from .rsd_exact import ExactFactor


def build(work: dict):
    """work: a dict from synth (n, depth, kappa, f).  Returns (A, b, owner, parent)."""
    n, depth = work["n"], work["depth"]
    A = fem.assemble(n, work["kappa"])
    b = fem.load_vector(n, work["f"])
    owner = partition.octree_owner(n, depth, fem.interior_coords(n))
    parent = partition.octree_parent(depth)
    return A, b, owner, parent


def solve_timed(work: dict, tol: float = 1e-8) -> dict:
    """Setup (symbolic + exact factorisation) and PCG solve, timed on this host.
    Problem assembly is input preparation and is not timed."""
    A, b, owner, parent = build(work)
    t0 = time.perf_counter()
    sym = partition.Symbolic(A, owner, parent)
    fac = ExactFactor(A, sym)
    t1 = time.perf_counter()
    x, it, hist = pcg(A, b, fac.apply, tol)
    t2 = time.perf_counter()
    res = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    return dict(n_dof=A.shape[0], t_setup=t1 - t0, t_solve=t2 - t1, iters=it, relres=res, x=x)
