"""3-D linear elasticity (three DOFs per node; the SPD Navier-Lame reading of Eq. 4.4) on
the GPU against the oracle: assembly and ownership, FP64 factors and application (Eqs.
3.2-3.3 at every node), one-iteration PCG, and the mixed forms to an FP64-checked 1e-8."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import fem, fem_elastic as fe, partition
from oracle.krylov import pcg
from oracle.rsd_exact import ExactFactor

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NU = 0.3


@pytest.fixture(scope="module")
def rsd():
    from paper_1210_6266_gb300 import build
    build.build()
    import paper_1210_6266_gb300 as m
    return m


_ORACLE = {}


def _case(n, depth, seed=131):
    key = (n, depth, seed)
    if key not in _ORACLE:
        E_leaf = synth.elasticity_moduli(8 ** depth, seed)
        f = synth.uniform(seed + 1, 3 * (n - 2) ** 3)
        K = fe.assemble(n, E_leaf[fe.leaf_of_element(n, depth)], NU)
        b = fe.load_vector(n, f)
        owner = fe.dof_owner(partition.octree_owner(n, depth, fem.interior_coords(n)))
        parent = partition.octree_parent(depth)
        sym = partition.Symbolic(K, owner, parent)
        _ORACLE[key] = (E_leaf, f, K, b, owner, parent, sym, ExactFactor(K, sym))
    return _ORACLE[key]


def _setup(rsd, prob, prec, root=None, **kw):
    return rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                         prec_leaf=prec, prec_mid=prec, prec_root=prec if root is None else root, **kw)


CASES = [(7, 1), (9, 1), (11, 2), (13, 2)]


@pytest.mark.parametrize("n,depth", CASES)
def test_elastic_assembly_and_ownership(rsd, n, depth):
    E_leaf, f, K, b, owner, parent, sym, _ = _case(n, depth)
    prob = rsd.grid_problem_elastic(n, depth, E_leaf, NU, f)
    assert np.array_equal(prob["rowptr"].cpu().numpy(), K.indptr)
    assert np.array_equal(prob["col"].cpu().numpy(), K.indices)
    val = prob["val"].cpu().numpy()
    assert np.abs(val - K.data).max() <= 1e-13 * np.abs(K.data).max()
    assert np.abs(prob["b"].cpu().numpy() - b).max() <= 1e-15 * np.abs(b).max()
    assert np.array_equal(prob["dof_node"].cpu().numpy(), owner)
    assert np.array_equal(prob["parent"], parent)


@pytest.mark.parametrize("n,depth", CASES)
def test_elastic_fp64_factors_apply_and_one_iteration(rsd, n, depth):
    E_leaf, f, K, b, owner, parent, sym, fac = _case(n, depth)
    prob = rsd.grid_problem_elastic(n, depth, E_leaf, NU, f)
    h = _setup(rsd, prob, rsd.RSD_PREC_FP64)
    for t in range(sym.n_nodes):
        assert h.front_dims(t)[:2] == (sym.s(t), sym.b(t))
        F = h.front_factor(t)
        ref = np.vstack([fac.L[t], fac.X[t]])
        assert np.abs(F - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1e-300), t
    r = synth.uniform(133, K.shape[0])
    z = h.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    zr = fac.apply(r)
    assert np.abs(z - zr).max() <= 1e-10 * np.abs(zr).max()
    u, st = h.solve(prob["b"], tol=1e-10)
    assert st["iterations"] == 1 and st["relres"] <= 1e-10
    x, it, _ = pcg(K, b, fac.apply, 1e-10)
    assert np.abs(u.cpu().numpy() - x).max() <= 1e-10 * np.abs(x).max()
    h.close()


@pytest.mark.parametrize("prec", ["TF32", "FP16"])
@pytest.mark.parametrize("n,depth", [(17, 2), (21, 2)])
def test_elastic_mixed_forms_reach_fp64_residual(rsd, prec, n, depth):
    E_leaf, f, K, b, owner, parent, sym, fac = _case(n, depth)
    prob = rsd.grid_problem_elastic(n, depth, E_leaf, NU, f)
    h = _setup(rsd, prob, getattr(rsd, "RSD_PREC_" + prec))
    u, st = h.solve(prob["b"], tol=1e-8)
    assert st["relres"] <= 1e-8 and st["iterations"] <= 40, st
    x = spla.spsolve(K.tocsc(), b)
    assert np.abs(u.cpu().numpy() - x).max() <= 1e-6 * np.abs(x).max()
    h.close()
