"""Pins for the oracle's FEM discretisation (CPU only)."""
import numpy as np
import pytest

import synth
from oracle import fem, fem2d


def _tensor_q1():
    # closed form: Khat = K1 x M1 x M1 + M1 x K1 x M1 + M1 x M1 x K1 (unit interval 1-D matrices),
    # index a = ax + 2 ay + 4 az  ->  kron order (z, y, x)
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    M1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    k = np.kron
    return k(M1, k(M1, K1)) + k(M1, k(K1, M1)) + k(K1, k(M1, M1)), k(M1, k(M1, M1))


def test_reference_element_matches_tensor_product():
    K, M = _tensor_q1()
    assert np.allclose(fem.reference_stiffness(), K, atol=1e-14)
    assert np.allclose(fem.reference_mass(), M, atol=1e-15)


def test_reference_element_kernel_is_constants():
    K = fem.reference_stiffness()
    w = np.linalg.eigvalsh(K)
    assert abs(w[0]) < 1e-14 and w[1] > 1e-3          # rank 7, constants only in the null space
    assert np.allclose(K @ np.ones(8), 0.0, atol=1e-14)


def test_interior_row_is_q1_27_point_stencil():
    n = 9
    h = 1.0 / (n - 1)
    A = fem.assemble(n, np.ones((n - 1) ** 3))
    c = fem.interior_id(n, 4, 4, 4)
    row = A[c].toarray().ravel()
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                j = fem.interior_id(n, 4 + dx, 4 + dy, 4 + dz)
                k = abs(dx) + abs(dy) + abs(dz)
                expect = {0: 8 / 3, 1: 0.0, 2: -1 / 6, 3: -1 / 12}[k] * h
                assert row[j] == pytest.approx(expect, abs=1e-15)
    assert abs(row.sum()) < 1e-15                      # zero row sum away from the boundary
    assert np.count_nonzero(np.abs(row) > 1e-15) == 1 + 12 + 8


def test_assembly_symmetric_and_row_assembly_agrees():
    n = 8
    kappa = np.exp(synth.normal(5, (n - 1) ** 3))
    A = fem.assemble(n, kappa, chunk=50)               # several chunks
    assert abs(A - A.T).max() < 1e-15
    for node in (0, 17, 100, A.shape[0] - 1):
        row = fem.assemble_row(n, kappa, node)
        dense = A[node].toarray().ravel()
        for j, v in row.items():
            assert dense[j] == pytest.approx(v, rel=1e-14)
        assert len(row) == A[node].nnz
    w = np.linalg.eigvalsh(A.toarray())
    assert w[0] > 0


def test_variable_kappa_scales_elements():
    # doubling kappa in every element doubles the matrix
    n = 7
    kap = np.exp(synth.normal(3, (n - 1) ** 3))
    assert abs(fem.assemble(n, 2 * kap) - 2 * fem.assemble(n, kap)).max() < 1e-14


def test_lumped_load_equals_mass_row_sums():
    M = fem.reference_mass()
    assert M.sum() == pytest.approx(1.0, abs=1e-14)
    assert np.allclose(M.sum(axis=1), 1 / 8, atol=1e-15)
    n = 5
    assert np.allclose(fem.load_vector(n, np.ones(27)), (1 / 4) ** 3)


def test_manufactured_solution_second_order():
    # u = sin(pi x) sin(pi y) sin(pi z), -Laplace u = 3 pi^2 u; nodal max error ~ h^2
    import scipy.sparse.linalg as spla
    errs = []
    for n in (9, 17, 33):
        xyz = fem.interior_coords(n) / (n - 1)
        u = np.prod(np.sin(np.pi * xyz), axis=1)
        A = fem.assemble(n, np.ones((n - 1) ** 3))
        b = fem.load_vector(n, 3 * np.pi ** 2 * u)
        uh = spla.spsolve(A.tocsc(), b)
        errs.append(np.abs(uh - u).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs


def test_2d_reference_element():
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    M1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    K = np.kron(M1, K1) + np.kron(K1, M1)
    assert np.allclose(fem2d.reference_stiffness_2d(), K, atol=1e-15)


def test_2d_strip_size_matches_formula():
    for N, P in ((17, 8), (9, 4)):
        A, _ = fem2d.strip_poisson(N, P)
        assert A.shape[0] == (P * (N - 1) - 1) * (N - 2)
