"""Pins for the oracle's nonsymmetric path (CPU only): the paper's two-variable systems
(Sec. 4, Eqs. 4.2 and 4.3) on the 2-D strip, the exact recursion with LU fronts (Eqs.
3.2-3.3 without the symmetry of K), and Algorithm 2 against the paper's Tables 4 and 7."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import fem2d, partition
from oracle.krylov import fgmres
from oracle.rsd_exact import ExactFactor, ExactFactorLU, lu_nopivot, schur_direct_general
from oracle.rsd_paper import PaperRSD

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _strip(N, P, c):
    A, coords = fem2d.strip_system(N, P, c)
    owner = np.repeat(fem2d.binary_owner(N, P, coords), 2)
    parent = fem2d.binary_parent(int(np.log2(P)))
    return A, owner, parent


def test_element_matrices_closed_form():
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    M1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    # local node a = ax + 2 ay  ->  kron order (y, x)
    assert np.allclose(fem2d.reference_mass_2d(), np.kron(M1, M1), atol=1e-15)
    assert np.allclose(fem2d.reference_stiffness_aniso(0.01, 1.0), 0.01 * np.kron(M1, K1) + np.kron(K1, M1), atol=1e-15)
    assert np.allclose(fem2d.reference_stiffness_aniso(1.0, 1.0), fem2d.reference_stiffness_2d(), atol=1e-15)


@pytest.mark.parametrize("c", [0.01, 100.0])
def test_system_has_skew_coupling_and_positive_definite_symmetric_part(c):
    N, P = 9, 4
    A, owner, parent = _strip(N, P, c)
    D = A.toarray()
    sym_part, skew = 0.5 * (D + D.T), 0.5 * (D - D.T)
    assert np.linalg.eigvalsh(sym_part).min() > 0
    # the skew part is the zero-order coupling: u rows against v columns, c h^2 M
    h = 1.0 / (N - 1)
    assert np.allclose(skew[0::2, 0::2], 0) and np.allclose(skew[1::2, 1::2], 0)
    assert np.allclose(D[0::2, 1::2], -D[1::2, 0::2].T)     # +c M against -c M
    # an interior node's coupling row is c h^2 times the assembled bilinear mass row:
    # 4/9 on the diagonal (four elements), 2/9 to the edge neighbours, 1/36 diagonally
    row = D[0::2, 1::2][3]
    assert np.isclose(np.abs(row).max(), c * h * h * 4 / 9)
    assert np.isclose(np.sort(np.abs(row[row != 0]))[0], c * h * h / 36)
    assert partition.check_structure(A, owner, parent)       # Eq. 3.1


def test_lu_nopivot_factors():
    rng = np.random.default_rng(4)
    F = rng.standard_normal((30, 30)) + 30 * np.eye(30)
    L, U = lu_nopivot(F)
    assert np.allclose(np.tril(L), L) and np.allclose(np.diag(L), 1) and np.allclose(np.triu(U), U)
    assert np.abs(L @ U - F).max() <= 1e-12 * np.abs(F).max()


@pytest.mark.parametrize("c", [0.01, 100.0])
@pytest.mark.parametrize("N,P", [(9, 4), (9, 8)])
def test_exact_lu_recursion_is_the_inverse(c, N, P):
    A, owner, parent = _strip(N, P, c)
    sym = partition.Symbolic(A, owner, parent)
    fac = ExactFactorLU(A, sym)
    r = synth.uniform(21, A.shape[0])
    z = fac.apply(r)
    zx = np.linalg.solve(A.toarray(), r)
    assert np.abs(z - zx).max() <= 1e-11 * np.abs(zx).max()
    for t in range(sym.n_nodes):
        if sym.children[t]:
            S = schur_direct_general(A, sym, t)
            assert np.abs(fac.S[t] - S).max() <= 1e-11 * np.abs(S).max(), t
        Lt, Ut = fac.L[t], fac.Uf[t]
        assert np.abs(Lt @ Ut - fac.S[t]).max() <= 1e-12 * max(np.abs(fac.S[t]).max(), 1e-300)
    x, it, _ = fgmres(A, r, fac.apply, 1e-10)
    assert it == 1


def test_exact_lu_recursion_equals_cholesky_one_on_spd_input():
    A, owner, parent = _strip(9, 4, 0.0)                       # c = 0: SPD (two decoupled fields)
    sym = partition.Symbolic(A, owner, parent)
    lu, ch = ExactFactorLU(A, sym), ExactFactor(A, sym)
    r = synth.uniform(22, A.shape[0])
    assert np.abs(lu.apply(r) - ch.apply(r)).max() <= 1e-12 * np.abs(ch.apply(r)).max()
    for t in range(sym.n_nodes):
        assert np.allclose(np.diag(lu.Uf[t]), np.diag(ch.L[t]) ** 2, rtol=1e-12)


def _tables():
    rows = []
    with open(os.path.join(GOLDEN, "table4_7_system_iterations.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                rows.append((float(v[0]), int(v[1]), int(v[2]), [int(x) for x in v[3:]]))
    return rows


@pytest.mark.parametrize("row", [r for r in _tables() if r[2] == 8])
def test_tables_4_and_7_outer_iterations(row):
    """Algorithm 2 with gamma inner GMRES iterations on Eqs. 4.2 / 4.3 reproduces the
    paper's outer iteration counts to within 20 percent (P = 8 columns)."""
    c, N, P, betas = row
    A, owner, parent = _strip(N, P, c)
    sym = partition.Symbolic(A, owner, parent)
    f = A @ synth.uniform(11, A.shape[0])
    for gamma, beta in zip((2, 4, 8), betas):
        x, it, _ = fgmres(A, f, PaperRSD(A, sym, gamma).apply_recursive, 1e-12, restart=30, maxit=2000)
        assert np.linalg.norm(f - A @ x) <= 1e-11 * np.linalg.norm(f)
        assert abs(it - beta) <= max(1, round(0.2 * beta)), (c, N, P, gamma, it, beta)


def test_paper_mode_depth_one_is_exact_on_the_nonsymmetric_system():
    A, owner, parent = _strip(9, 2, 100.0)                     # two leaves: V-hat = V
    sym = partition.Symbolic(A, owner, parent)
    r = synth.uniform(23, A.shape[0])
    z = PaperRSD(A, sym, 0).apply_recursive(r)
    assert np.abs(z - spla.spsolve(A.tocsc(), r)).max() <= 1e-11 * np.abs(z).max()
