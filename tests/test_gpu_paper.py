"""Paper mode (Algorithm 2 with the V-hat truncation, dense S~ per interface) on the GPU
against the oracle's level-wise Algorithm 2."""
import numpy as np
import pytest

import synth
from oracle import fem, partition
from oracle.krylov import pcg
from oracle.rsd_exact import ExactFactor
from oracle.rsd_paper import PaperRSD

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsd():
    from paper_1210_6266_gb300 import build
    build.build()
    import paper_1210_6266_gb300 as m
    return m


def _case(n, depth, seed=91):
    kappa = np.exp(synth.normal(seed, (n - 1) ** 3))
    f = synth.uniform(seed + 1, (n - 2) ** 3)
    A = fem.assemble(n, kappa)
    sym = partition.Symbolic(A, partition.octree_owner(n, depth, fem.interior_coords(n)),
                             partition.octree_parent(depth))
    return kappa, f, A, sym


def _setup(rsd, prob, prec):
    return rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                         prec_leaf=prec, prec_mid=prec, prec_root=prec, mode=rsd.RSD_MODE_PAPER)


@pytest.mark.parametrize("n,depth", [(14, 2), (17, 2), (20, 2), (11, 1)])
def test_paper_fp64_interfaces_and_apply_match_oracle(rsd, n, depth):
    kappa, f, A, sym = _case(n, depth)
    R = PaperRSD(A, sym, 0)
    prob = rsd.grid_problem(n, depth, kappa, f)
    h = _setup(rsd, prob, rsd.RSD_PREC_FP64)
    for t in R.vhat:                                      # interface fronts: chol(S~_t)
        s, b, _ = h.front_dims(t)
        assert b == 0 and s == sym.s(t)
        L = np.linalg.cholesky(R.S_dense[t])
        F = h.front_factor(t)
        assert np.abs(F - L).max() <= 1e-10 * np.abs(L).max(), t
    r = torch.as_tensor(synth.uniform(93, A.shape[0]), device="cuda")
    z = h.apply(r).cpu().numpy()
    zr = R.apply_levelwise(r.cpu().numpy())
    assert np.abs(z - zr).max() <= 1e-10 * np.abs(zr).max()
    h.check()


def test_paper_depth_one_equals_exact(rsd):
    kappa, f, A, sym = _case(11, 1)
    prob = rsd.grid_problem(11, 1, kappa, f)
    hp = _setup(rsd, prob, rsd.RSD_PREC_FP64)
    he = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                       prec_leaf=rsd.RSD_PREC_FP64, prec_mid=rsd.RSD_PREC_FP64, prec_root=rsd.RSD_PREC_FP64)
    r = prob["b"]
    zp, ze = hp.apply(r), he.apply(r)
    assert (zp - ze).abs().max().item() <= 1e-10 * ze.abs().max().item()


@pytest.mark.parametrize("prec", ["FP64", "TF32"])
def test_paper_pcg_converges(rsd, prec):
    n, depth = 20, 2
    kappa, f, A, sym = _case(n, depth)
    prob = rsd.grid_problem(n, depth, kappa, f)
    h = _setup(rsd, prob, getattr(rsd, "RSD_PREC_" + prec))
    u, st = h.solve(prob["b"], tol=1e-8)
    b = fem.load_vector(n, f)
    assert np.linalg.norm(b - A @ u.cpu().numpy()) <= 1e-8 * np.linalg.norm(b)
    if prec == "FP64":
        R = PaperRSD(A, sym, 0)
        _, it, _ = pcg(A, b, R.apply_levelwise, 1e-8)
        assert abs(st["iterations"] - it) <= 1, (st["iterations"], it)
