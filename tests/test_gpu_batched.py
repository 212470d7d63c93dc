"""Batched form: several independent problems of uneven size and depth in one hierarchy,
every tree level of every problem in the same kernel launches.  Each problem's part of
the result must match that problem's oracle."""
import numpy as np
import pytest

import synth
from oracle import fem, partition
from oracle.rsd_exact import ExactFactor

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [(9, 1), (13, 1), (17, 2), (11, 2), (20, 2), (14, 1)]


@pytest.fixture(scope="module")
def rsd():
    from paper_1210_6266_gb300 import build
    build.build()
    import paper_1210_6266_gb300 as m
    return m


@pytest.fixture(scope="module")
def batch(rsd):
    probs, oracles = [], []
    for i, (n, depth) in enumerate(SIZES):
        kappa = np.exp(synth.normal(60 + i, (n - 1) ** 3))
        f = synth.uniform(70 + i, (n - 2) ** 3)
        probs.append(rsd.grid_problem(n, depth, kappa, f))
        A = fem.assemble(n, kappa)
        owner = partition.octree_owner(n, depth, fem.interior_coords(n))
        sym = partition.Symbolic(A, owner, partition.octree_parent(depth))
        oracles.append((A, fem.load_vector(n, f), ExactFactor(A, sym)))
    return probs, oracles


def _split(x, probs):
    out, off = [], 0
    for p in probs:
        out.append(x[off:off + p["n_dof"]])
        off += p["n_dof"]
    return out


def test_batched_fp64_apply_matches_each_problem(rsd, batch):
    probs, oracles = batch
    h = rsd.RSD.setup_batched(probs, prec_leaf=rsd.RSD_PREC_FP64, prec_mid=rsd.RSD_PREC_FP64,
                              prec_root=rsd.RSD_PREC_FP64)
    r = torch.as_tensor(synth.uniform(80, h.n), device="cuda")
    z = h.apply(r).cpu().numpy()
    for zp, rp, (A, b, fac) in zip(_split(z, probs), _split(r.cpu().numpy(), probs), oracles):
        zr = fac.apply(rp)
        assert np.abs(zp - zr).max() <= 1e-10 * np.abs(zr).max()
    h.check()


def test_batched_tf32_solve_reaches_fp64_residual_per_problem(rsd, batch):
    probs, oracles = batch
    h = rsd.RSD.setup_batched(probs, prec_leaf=rsd.RSD_PREC_TF32, prec_mid=rsd.RSD_PREC_TF32,
                              prec_root=rsd.RSD_PREC_TF32)
    b = torch.cat([p["b"] for p in probs])
    u, st = h.solve(b, tol=1e-10)
    for up, (A, bp, fac) in zip(_split(u.cpu().numpy(), probs), oracles):
        assert np.linalg.norm(bp - A @ up) <= 1e-8 * np.linalg.norm(bp)


def test_batched_handle_reports_each_front(rsd, batch):
    probs, _ = batch
    h = rsd.RSD.setup_batched(probs, prec_leaf=rsd.RSD_PREC_FP64, prec_mid=rsd.RSD_PREC_FP64)
    inf = h.info()
    assert inf["n"] == sum(p["n_dof"] for p in probs)
    assert inf["n_nodes"] == 1 + sum(len(p["parent"]) for p in probs)
    assert h.front_dims(0)[:2] == (0, 0)                # the empty super-root


def test_batched_tf32_factors_track_fp32_on_uneven_fronts(rsd, batch):
    """The problem roots form one level of fronts of uneven size (331 to 919 interface
    DOFs), factored with the look-ahead schedule in tensor cores: every front must match the
    FP32 CUDA-core factorisation of the same hierarchy to TF32 rounding."""
    probs, _ = batch
    h32 = rsd.RSD.setup_batched(probs, prec_leaf=rsd.RSD_PREC_FP32, prec_mid=rsd.RSD_PREC_FP32,
                                prec_root=rsd.RSD_PREC_FP32)
    htf = rsd.RSD.setup_batched(probs, prec_leaf=rsd.RSD_PREC_TF32, prec_mid=rsd.RSD_PREC_TF32,
                                prec_root=rsd.RSD_PREC_TF32)
    n_nodes = h32.info()["n_nodes"]
    big = 0
    for t in range(1, n_nodes):
        s, b, _ = h32.front_dims(t)
        if s == 0:
            continue
        big += s > 512
        a, c = h32.front_factor(t), htf.front_factor(t)
        scale = np.abs(a).max()
        assert np.abs(a - c).max() <= 5e-3 * scale, (t, np.abs(a - c).max() / scale)
    assert big >= 1                                     # some fronts span several 512-wide panels
    b = torch.cat([p["b"] for p in probs])
    _, st = htf.solve(b, tol=1e-8)
    assert st["iterations"] <= 10, st                   # TF32 factors keep PCG short
