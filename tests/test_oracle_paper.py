"""Pins for the oracle's Algorithm 2 (paper mode) and the Krylov solvers (CPU only)."""
import os

import numpy as np
import pytest

import synth
from oracle import fem, fem2d, partition
from oracle.krylov import fgmres, pcg
from oracle.rsd_exact import ExactFactor
from oracle.rsd_paper import PaperRSD, gmres_fixed, schur_gamma

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _case(n, depth, seed=31):
    kappa = np.exp(synth.normal(seed, (n - 1) ** 3))
    A = fem.assemble(n, kappa)
    owner = partition.octree_owner(n, depth, fem.interior_coords(n))
    sym = partition.Symbolic(A, owner, partition.octree_parent(depth))
    return A, sym


def test_depth_one_paper_equals_exact():
    # with leaf children, V-hat = V and S~ = S: Algorithm 2 is the exact solve
    A, sym = _case(11, 1)
    r = synth.uniform(7, A.shape[0])
    z_exact = ExactFactor(A, sym).apply(r)
    z_paper = PaperRSD(A, sym, 0).apply_recursive(r)
    assert np.abs(z_paper - z_exact).max() <= 1e-12 * np.abs(z_exact).max()


def test_recursive_equals_levelwise_depth2():
    A, sym = _case(14, 2)
    R = PaperRSD(A, sym, 0)
    M1 = R.operator(A.shape[0])
    M2 = np.stack([R.apply_levelwise(e) for e in np.eye(A.shape[0])], axis=1)
    assert np.abs(M1 - M2).max() <= 1e-13 * np.abs(M1).max()


def test_s_tilde_is_principal_block_of_s_gamma():
    A, sym = _case(14, 2)
    R = PaperRSD(A, sym, 0)
    SG, G = schur_gamma(A, sym)
    for t in R.vhat:
        pos = np.searchsorted(G, sym.I[t])
        assert np.abs(R.s_tilde(t) - SG[np.ix_(pos, pos)]).max() <= 1e-12 * np.abs(SG).max(), t


def test_depth2_paper_mode_is_not_exact_but_converges():
    A, sym = _case(14, 2)
    R = PaperRSD(A, sym, 0)
    r = synth.uniform(8, A.shape[0])
    z = R.apply_recursive(r)
    zx = np.linalg.solve(A.toarray(), r)
    assert np.abs(z - zx).max() > 1e-6 * np.abs(zx).max()       # truncation is an approximation
    x, it, _ = fgmres(A, r, R.apply_recursive, 1e-10)
    assert np.linalg.norm(r - A @ x) <= 1e-9 * np.linalg.norm(r)
    assert it < 40


def test_gmres_fixed_exact_after_n_steps():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((12, 12)) + 12 * np.eye(12)
    b = rng.standard_normal(12)
    assert np.allclose(gmres_fixed(lambda v: M @ v, b, 12), np.linalg.solve(M, b), atol=1e-10)
    # one step = the minimiser of ||b - a M b|| over scalars a
    x1 = gmres_fixed(lambda v: M @ v, b, 1)
    Mb = M @ b
    assert np.allclose(x1, (Mb @ b) / (Mb @ Mb) * b, atol=1e-12)


def test_pcg_textbook_properties():
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    A = Q @ np.diag(np.repeat([1.0, 3.0, 10.0], 10)) @ Q.T      # 3 distinct eigenvalues
    b = rng.standard_normal(30)
    x, it, _ = pcg(A, b, lambda r: r, 1e-10)
    assert it <= 3 and np.allclose(x, np.linalg.solve(A, b), atol=1e-9)
    Ms = rng.standard_normal((30, 30)) + 10 * np.eye(30)
    x, it, _ = fgmres(Ms, b, lambda r: r, 1e-12, restart=8)
    assert np.allclose(x, np.linalg.solve(Ms, b), atol=1e-9)


def test_fgmres_with_a_preconditioner_that_changes_every_step():
    """The flexible variant keeps z_j = M_j(v_j) per step: with a preconditioner that
    differs from call to call, n steps still reach the exact solution, and at every step
    the iterate minimises ||b - A x|| over span{z_0 .. z_k} (checked by an independent
    least-squares solve on the same z's)."""
    rng = np.random.default_rng(5)
    n = 12
    A = rng.standard_normal((n, n)) + 8 * np.eye(n)
    b = rng.standard_normal(n)
    P = [np.linalg.inv(A + rng.standard_normal((n, n))), np.diag(1.0 / np.diag(A)), np.eye(n)]
    calls = []

    def M(v):
        z = P[len(calls) % 3] @ v
        calls.append(z)
        return z

    x, it, _ = fgmres(A, b, M, 1e-13, restart=n)
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-10)
    for k in (1, 3, 5):
        calls.clear()
        xk, itk, _ = fgmres(A, b, M, 1e-30, restart=k, maxit=k)
        assert itk == k
        Zk = np.stack(calls[:k], axis=1)
        y, *_ = np.linalg.lstsq(A @ Zk, b, rcond=None)
        assert np.allclose(xk, Zk @ y, atol=1e-10), k


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_poisson_iterations.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", _table1())
def test_table1_outer_iterations_2d_strip(row):
    """Algorithm 2 with gamma inner GMRES steps reproduces the paper's Table 1
    (Problem 1) outer iteration counts to within 30 percent."""
    N, P, *betas = row
    A, coords = fem2d.strip_poisson(N, P)
    owner = fem2d.binary_owner(N, P, coords)
    sym = partition.Symbolic(A, owner, fem2d.binary_parent(int(np.log2(P))))
    f = A @ synth.uniform(11, A.shape[0])             # random exact solution, f = K u*
    for gamma, beta in zip((2, 4, 8), betas):
        R = PaperRSD(A, sym, gamma)
        x, it, _ = fgmres(A, f, R.apply_recursive, 1e-12, restart=30)
        assert np.linalg.norm(f - A @ x) <= 1e-11 * np.linalg.norm(f)
        assert abs(it - beta) <= max(1, round(0.3 * beta)), (N, P, gamma, it, beta)
