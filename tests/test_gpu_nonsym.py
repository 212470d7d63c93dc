"""Nonsymmetric systems on the GPU (the paper's Eqs. 4.2 and 4.3 on the 2-D strip): LU
fronts without pivoting, the substitution sweeps on [L; X] and [U^T; Y^T], FGMRES; and
paper mode with gamma inner GMRES iterations on the same systems, against the oracle."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import fem2d, partition
from oracle.krylov import fgmres
from oracle.rsd_exact import ExactFactorLU
from oracle.rsd_paper import PaperRSD

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def rsd():
    from paper_1210_6266_gb300 import build
    build.build()
    import paper_1210_6266_gb300 as m
    return m


def _strip(N, P, c):
    A, coords = fem2d.strip_system(N, P, c)
    owner = np.repeat(fem2d.binary_owner(N, P, coords), 2)
    parent = fem2d.binary_parent(int(np.log2(P)))
    return A, owner, parent


def _setup(rsd, A, owner, parent, prec, **kw):
    return rsd.RSD.setup(torch.as_tensor(A.indptr.astype(np.int64)), torch.as_tensor(A.indices.astype(np.int32)),
                         torch.as_tensor(A.data.astype(np.float64)), torch.as_tensor(owner.astype(np.int32)),
                         parent.astype(np.int32), prec_leaf=prec, prec_mid=prec, prec_root=prec, nonsymmetric=True, **kw)


@pytest.mark.parametrize("c", [0.01, 100.0])
@pytest.mark.parametrize("N,P", [(9, 4), (17, 8), (33, 4)])
def test_lu_fronts_apply_and_one_iteration_match_oracle(rsd, c, N, P):
    A, owner, parent = _strip(N, P, c)
    sym = partition.Symbolic(A, owner, parent)
    fac = ExactFactorLU(A, sym)
    h = _setup(rsd, A, owner, parent, rsd.RSD_PREC_FP64)
    for t in range(sym.n_nodes):
        Lg, Ug = h.front_factor(t), h.front_factor_upper(t)
        refL = np.vstack([fac.L[t], fac.X[t]])
        refU = np.vstack([fac.Uf[t].T, fac.Y[t].T])
        assert np.abs(Lg - refL).max() <= 1e-10 * max(np.abs(refL).max(), 1e-300), t
        assert np.abs(Ug - refU).max() <= 1e-10 * max(np.abs(refU).max(), 1e-300), t
    r = synth.uniform(151, A.shape[0])
    z = h.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    zr = fac.apply(r)
    assert np.abs(z - zr).max() <= 1e-10 * np.abs(zr).max()
    f = torch.as_tensor(A @ synth.uniform(152, A.shape[0]), device="cuda")
    u, st = h.solve(f, tol=1e-10)
    assert st["iterations"] == 1 and st["relres"] <= 1e-10, st
    h.close()


@pytest.mark.parametrize("c", [0.01, 100.0])
def test_lu_fp32_fronts_reach_fp64_residual(rsd, c):
    N, P = 33, 8
    A, owner, parent = _strip(N, P, c)
    f = A @ synth.uniform(153, A.shape[0])
    h = _setup(rsd, A, owner, parent, rsd.RSD_PREC_FP32)
    u, st = h.solve(torch.as_tensor(f, device="cuda"), tol=1e-10)
    assert st["relres"] <= 1e-10 and st["iterations"] <= 6, st
    x = spla.spsolve(A.tocsc(), f)
    assert np.abs(u.cpu().numpy() - x).max() <= 1e-8 * np.abs(x).max()
    h.close()


@pytest.mark.parametrize("c", [0.01, 100.0])
@pytest.mark.parametrize("gamma", [2, 8])
def test_paper_gamma_on_nonsymmetric_systems_matches_oracle(rsd, c, gamma):
    N, P = 17, 8
    A, owner, parent = _strip(N, P, c)
    sym = partition.Symbolic(A, owner, parent)
    R = PaperRSD(A, sym, gamma)
    h = _setup(rsd, A, owner, parent, rsd.RSD_PREC_FP64, mode=rsd.RSD_MODE_PAPER, gamma=gamma, maxit=1000)
    r = synth.uniform(154, A.shape[0])
    z = h.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    zr = R.apply_recursive(r)
    assert np.abs(z - zr).max() <= 1e-10 * np.abs(zr).max()
    f = A @ synth.uniform(11, A.shape[0])
    _, it_ref, _ = fgmres(A, f, R.apply_recursive, 1e-12, restart=30, maxit=2000)
    u, st = h.solve(torch.as_tensor(f, device="cuda"), tol=1e-12)
    assert np.linalg.norm(f - A @ u.cpu().numpy()) <= 1e-11 * np.linalg.norm(f)
    assert abs(st["iterations"] - it_ref) <= 1, (st["iterations"], it_ref)
    h.close()


def _tables():
    rows = []
    with open(os.path.join(GOLDEN, "table4_7_system_iterations.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                rows.append((float(v[0]), int(v[1]), int(v[2]), [int(x) for x in v[3:]]))
    return rows


@pytest.mark.parametrize("row", _tables())
def test_paper_gamma_gpu_reproduces_tables_4_and_7(rsd, row):
    """The GPU's outer FGMRES iteration counts on Eqs. 4.2 / 4.3 within 20 % of the
    paper's Tables 4 and 7 (P = 8 and P = 128 columns; FP64 leaf factors)."""
    c, N, P, betas = row
    A, owner, parent = _strip(N, P, c)
    f = torch.as_tensor(A @ synth.uniform(11, A.shape[0]), device="cuda")
    for gamma, beta in zip((2, 4, 8), betas):
        h = _setup(rsd, A, owner, parent, rsd.RSD_PREC_FP64, mode=rsd.RSD_MODE_PAPER, gamma=gamma, maxit=2000)
        u, st = h.solve(f, tol=1e-12)
        assert st["relres"] <= 1e-11
        assert abs(st["iterations"] - beta) <= max(1, round(0.2 * beta)), (c, N, P, gamma, st["iterations"], beta)
        h.close()


def test_nonsymmetric_options_are_checked(rsd):
    A, owner, parent = _strip(9, 4, 0.01)
    with pytest.raises(rsd.RSDError):
        _setup(rsd, A, owner, parent, rsd.RSD_PREC_TF32)
    with pytest.raises(rsd.RSDError):
        _setup(rsd, A, owner, parent, rsd.RSD_PREC_FP64, krylov=rsd.RSD_KRYLOV_PCG)
    with pytest.raises(rsd.RSDError):
        _setup(rsd, A, owner, parent, rsd.RSD_PREC_FP64, mode=rsd.RSD_MODE_PAPER, gamma=0)
