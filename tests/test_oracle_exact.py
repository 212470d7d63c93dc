"""Pins for the oracle's exact recursive Schur decomposition (CPU only)."""
import numpy as np
import pytest

import synth
from oracle import fem, partition, problem
from oracle.krylov import pcg
from oracle.rsd_exact import ExactFactor, dense_solve, schur_direct


def _case(n, depth, lognormal=False, seed=21):
    kappa = np.exp(synth.normal(seed, (n - 1) ** 3)) if lognormal else np.ones((n - 1) ** 3)
    A = fem.assemble(n, kappa)
    owner = partition.octree_owner(n, depth, fem.interior_coords(n))
    parent = partition.octree_parent(depth)
    sym = partition.Symbolic(A, owner, parent)
    return A, sym


CASES = [(13, 1, False), (11, 2, True), (14, 2, False), (9, 1, True)]


@pytest.mark.parametrize("n,depth,logn", CASES)
def test_apply_equals_dense_lu_solve(n, depth, logn):
    A, sym = _case(n, depth, logn)
    fac = ExactFactor(A, sym)
    r = synth.uniform(99, A.shape[0])
    z = fac.apply(r)
    zr = dense_solve(A, r)
    assert np.abs(z - zr).max() <= 1e-12 * np.abs(zr).max()


@pytest.mark.parametrize("n,depth,logn", CASES[:3])
def test_interface_schur_matches_eq_3_2(n, depth, logn):
    A, sym = _case(n, depth, logn)
    fac = ExactFactor(A, sym)
    for t in range(sym.n_nodes):
        if sym.children[t]:
            S = schur_direct(A, sym, t)
            assert np.abs(S - fac.S[t]).max() <= 1e-12 * np.abs(S).max(), t


def test_root_schur_is_inverse_block_and_spd():
    A, sym = _case(11, 2, True)
    fac = ExactFactor(A, sym)
    I = sym.I[0]
    Kinv = np.linalg.inv(A.toarray())
    S = fac.S[0]
    assert np.allclose(S, S.T, atol=1e-13 * np.abs(S).max())
    assert np.linalg.eigvalsh(S).min() > 0
    assert np.abs(np.linalg.inv(S) - Kinv[np.ix_(I, I)]).max() <= 1e-10 * np.abs(Kinv).max()


def test_operator_is_k_inverse():
    A, sym = _case(9, 2, True)
    fac = ExactFactor(A, sym)
    M = fac.operator(A.shape[0])
    assert np.abs(M @ A.toarray() - np.eye(A.shape[0])).max() < 1e-11


def test_pcg_converges_in_one_iteration_poisson13():
    w = synth.make("poisson13")
    A, b, owner, parent = problem.build(w)
    sym = partition.Symbolic(A, owner, parent)
    fac = ExactFactor(A, sym)
    x, it, hist = pcg(A, b, fac.apply, 1e-10)
    assert it == 1
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) < 1e-12


def test_leaf_update_is_negative_schur_term():
    """A leaf's contribution to its ancestors is -K_BI K_II^-1 K_IB (Eq. 3.2's subtracted term)."""
    A, sym = _case(11, 1, True)
    fac = ExactFactor(A, sym)
    # U_t is consumed by the parent; recompute one leaf by hand
    t = 3
    I, B = sym.I[t], sym.B[t]
    KII = A[I][:, I].toarray()
    KIB = A[I][:, B].toarray()
    Uref = -KIB.T @ np.linalg.solve(KII, KIB)
    L, X = fac.L[t], fac.X[t]
    assert np.abs((-X @ X.T) - Uref).max() <= 1e-12 * np.abs(Uref).max()
    assert np.abs(L @ L.T - KII).max() <= 1e-13 * np.abs(KII).max()


@pytest.mark.parametrize("n,depth,logn", CASES)
def test_factor_rows_bounded_by_sqrt_diagonal(n, depth, logn):
    """Every row of a front's factor [L_t; X_t] has 2-norm at most sqrt(K_ii), i the row's
    DOF.  For L_t the squared row norm is the diagonal entry of the interface Schur
    complement S_t (Eq. 3.2); for X_t it is at most -U_t[i, i], and K_BB + U_t is the Schur
    complement left on B_t after the subtree is eliminated.  A Schur complement of an SPD
    matrix is SPD with diagonal at most K's, so both are bounded by K_ii.  The GPU path
    scales each factor row by a power of two chosen from sqrt(K_ii) before storing it in
    FP16, which relies on this bound."""
    A, sym = _case(n, depth, logn)
    fac = ExactFactor(A, sym)
    d = A.diagonal()
    checked = 0
    for t in range(sym.n_nodes):
        I, Bt = np.asarray(sym.I[t]), np.asarray(sym.B[t])
        if fac.L[t].size:
            rn = np.linalg.norm(fac.L[t], axis=1)
            assert np.all(rn <= np.sqrt(d[I]) * (1 + 1e-12)), t
            assert np.allclose(rn ** 2, np.diag(fac.S[t]), rtol=1e-10)
            checked += len(I)
        if fac.X[t].size:
            assert np.all(np.linalg.norm(fac.X[t], axis=1) <= np.sqrt(d[Bt]) * (1 + 1e-12)), t
            checked += len(Bt)
    assert checked > A.shape[0]
