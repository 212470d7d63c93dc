"""Pins for the oracle's 3-D elasticity discretisation (the SPD Navier-Lame reading of
Eq. 4.4, three DOFs per node) and its octree partition (CPU only)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import fem, fem_elastic as fe, partition
from oracle.krylov import pcg
from oracle.rsd_exact import ExactFactor

CORNERS = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=float)


@pytest.mark.parametrize("nu", [0.0, 0.3, 0.45])
def test_element_kernel_is_the_six_rigid_body_modes(nu):
    K = fe.reference_stiffness(nu)
    assert np.abs(K - K.T).max() <= 1e-15
    R = fe.rigid_body_modes(CORNERS)
    assert np.abs(K @ R).max() <= 1e-14 * np.abs(K).max()
    w = np.linalg.eigvalsh(K)
    assert np.all(np.abs(w[:6]) <= 1e-13 * w[-1])              # exactly six zero modes
    assert w[6] > 1e-3 * w[-1]


@pytest.mark.parametrize("nu", [0.0, 0.3])
def test_element_entries_closed_form(nu):
    # node 0, components x, x and x, y: int (lam+2mu) phx^2 + mu (phy^2 + phz^2) = (lam + 4 mu)/9
    # and int (lam + mu) phx phy = (lam + mu)/12 on the unit cube
    lam, mu = fe.lame(1.0, nu)
    K = fe.reference_stiffness(nu)
    assert K[0, 0] == pytest.approx((lam + 4 * mu) / 9, abs=1e-15)
    assert K[0, 1] == pytest.approx((lam + mu) / 12, abs=1e-15)
    if nu == 0.0:
        assert K[0, 0] == pytest.approx(2.0 / 9.0, abs=1e-15)


def test_linear_patch_test():
    """A linear displacement field gives zero residual at every interior node of the
    unconstrained assembly with uniform E (constant strain is reproduced exactly)."""
    n, nu = 6, 0.3
    h = 1.0 / (n - 1)
    K = fe.assemble(n, np.full((n - 1) ** 3, 2.5), nu, full=True)
    rng = np.random.default_rng(3)
    Aff, c = rng.standard_normal((3, 3)), rng.standard_normal(3)
    g = np.arange(n ** 3)
    x = np.stack([g % n, (g // n) % n, g // (n * n)], axis=1) * h
    u = (x @ Aff.T + c).reshape(-1)
    r = K @ u
    inner = np.all((x > 0.5 * h) & (x < 1 - 0.5 * h), axis=1)
    assert np.abs(r.reshape(-1, 3)[inner]).max() <= 1e-12 * np.abs(K).max() * np.abs(u).max()
    assert np.abs(r.reshape(-1, 3)[~inner]).max() > 1e-6          # boundary rows carry the traction


def test_dirichlet_assembly_is_the_full_one_restricted():
    n, nu = 6, 0.3
    E = 10.0 ** synth.uniform(5, (n - 1) ** 3, 0.0, 3.0)
    Kf = fe.assemble(n, E, nu, full=True).toarray()
    Kd = fe.assemble(n, E, nu).toarray()
    ic = fem.interior_coords(n)
    gid = ic[:, 0] + n * (ic[:, 1] + n * ic[:, 2])
    dof = (3 * gid[:, None] + np.arange(3)[None, :]).reshape(-1)
    assert np.abs(Kd - Kf[np.ix_(dof, dof)]).max() <= 1e-12 * np.abs(Kf).max()
    assert np.linalg.eigvalsh(Kd).min() > 0                        # SPD after elimination


def _mms_error(n, nu=0.3):
    h = 1.0 / (n - 1)
    lam, mu = fe.lame(1.0, nu)
    e = np.array([1.0, 2.0, -1.0])
    xs = fem.interior_coords(n) * h
    s, c = np.sin(np.pi * xs), np.cos(np.pi * xs)
    phi = s[:, 0] * s[:, 1] * s[:, 2]
    H = np.empty((len(xs), 3, 3))                                  # Hessian of phi
    for i in range(3):
        for j in range(3):
            if i == j:
                H[:, i, j] = -np.pi ** 2 * phi
            else:
                k = 3 - i - j
                H[:, i, j] = np.pi ** 2 * c[:, i] * c[:, j] * s[:, k]
    f = mu * 3 * np.pi ** 2 * phi[:, None] * e[None, :] - (lam + mu) * (H @ e)
    K = fe.assemble(n, np.ones((n - 1) ** 3), nu)
    u = spla.spsolve(K.tocsc(), fe.load_vector(n, f.reshape(-1)))
    return np.abs(u - (phi[:, None] * e[None, :]).reshape(-1)).max()


def test_manufactured_solution_converges_at_second_order():
    e1, e2 = _mms_error(9), _mms_error(17)
    assert e2 < e1 and e1 / e2 > 3.5, (e1, e2)


def test_leaf_of_element_matches_the_octree_ownership():
    """Every node owned by a leaf (not on a separator) is surrounded by 8 elements of that
    same leaf, so E constant per leaf is constant over each leaf interior."""
    n, depth = 23, 2
    leaf = fe.leaf_of_element(n, depth)
    ic = fem.interior_coords(n)
    own = partition.octree_owner(n, depth, ic)
    first = (8 ** depth - 1) // 7
    ne = n - 1
    for k in np.flatnonzero(own >= first)[::7]:
        x, y, z = ic[k]
        els = [ex + ne * (ey + ne * ez) for ez in (z - 1, z) for ey in (y - 1, y) for ex in (x - 1, x)]
        assert np.all(leaf[els] == own[k] - first)
    assert leaf.min() == 0 and leaf.max() == 8 ** depth - 1


def test_elasticity97_dof_count_and_root_separator():
    n, depth = 97, 4
    own = partition.octree_owner(n, depth, fem.interior_coords(n))
    dof_own = fe.dof_owner(own)
    assert len(dof_own) == 2_572_125 == 3 * 95 ** 3
    assert np.count_nonzero(dof_own == 0) == 80_373 == 3 * partition.separator_count(95)


def test_small_elastic_problem_exact_rsd_is_one_iteration():
    n, depth, nu = 9, 1, 0.3
    E_leaf = synth.elasticity_moduli(8 ** depth, 9)
    E = E_leaf[fe.leaf_of_element(n, depth)]
    K = fe.assemble(n, E, nu)
    owner = fe.dof_owner(partition.octree_owner(n, depth, fem.interior_coords(n)))
    parent = partition.octree_parent(depth)
    assert partition.check_structure(K, owner, parent)             # Eq. 3.1 holds
    sym = partition.Symbolic(K, owner, parent)
    b = fe.load_vector(n, synth.uniform(10, K.shape[0]))
    x, it, _ = pcg(K, b, ExactFactor(K, sym).apply, 1e-10)
    assert it == 1
    assert np.linalg.norm(b - K @ x) <= 1e-10 * np.linalg.norm(b)
