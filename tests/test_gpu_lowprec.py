"""16-bit tensor-core operands for the long Schur-complement updates (RSD_PREC_FP16 and
RSD_PREC_BF16): factor parity against the FP32 CUDA-core factors, FP64-checked solves,
the FP16 copy's exactness, and the breakdown promotion of a BF16 front (Sec. 3.2 allows
an approximate leaf solver; a failed low-precision pivot is redone one precision up)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import fem, partition

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsd():
    from paper_1210_6266_gb300 import build
    build.build()
    import paper_1210_6266_gb300 as m
    return m


def _prob(rsd, n, depth, seed=111):
    kappa = np.exp(synth.normal(seed, (n - 1) ** 3))
    f = synth.uniform(seed + 1, (n - 2) ** 3)
    return rsd.grid_problem(n, depth, kappa, f), kappa, f


def _setup(rsd, prob, prec, root=None, **kw):
    return rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                         prec_leaf=prec, prec_mid=prec, prec_root=prec if root is None else root, **kw)


# (n, depth): one-panel fronts; a 3-panel root on the look-ahead path (26, 1 and 41, 1);
# 64 leaves of 2-3 panels on the bulk path (41, 2)
@pytest.mark.parametrize("n,depth", [(17, 2), (26, 1), (41, 1), (41, 2)])
@pytest.mark.parametrize("prec,tol", [("FP16", 5e-3), ("BF16", 4e-2)])
def test_16bit_operand_factors_track_fp32(rsd, n, depth, prec, tol):
    prob, _, _ = _prob(rsd, n, depth)
    h32 = _setup(rsd, prob, rsd.RSD_PREC_FP32)
    h16 = _setup(rsd, prob, getattr(rsd, "RSD_PREC_" + prec))
    assert h16.info()["promoted"] == 0
    for t in range(len(prob["parent"])):
        a, b = h32.front_factor(t), h16.front_factor(t)
        scale = np.abs(a).max()
        assert np.abs(a - b).max() <= tol * scale, (t, np.abs(a - b).max() / scale)
    u, st = h16.solve(prob["b"], tol=1e-8)
    assert st["relres"] <= 1e-8, st
    h32.close()
    h16.close()


@pytest.mark.parametrize("n,depth", [(41, 1), (41, 2)])
def test_fp16_operands_match_tf32_iterations(rsd, n, depth):
    """FP16 operands hold the TF32 factor entries exactly (row-scaled copy), so the FP16
    form needs the TF32 form's PCG iterations (one more at most)."""
    prob, _, _ = _prob(rsd, n, depth)
    its = {}
    for prec in ("TF32", "FP16"):
        h = _setup(rsd, prob, getattr(rsd, "RSD_PREC_" + prec))
        u, st = h.solve(prob["b"], tol=1e-10)
        assert st["relres"] <= 1e-10
        its[prec] = st["iterations"]
        h.close()
    assert its["FP16"] <= its["TF32"] + 1, its


@pytest.mark.parametrize("n,depth", [(41, 1), (41, 2)])
def test_fp16_level_copy_written_by_panels_holds_the_factor(rsd, n, depth):
    """An FP16 level writes its operand copy panel by panel; it is the copy the sweeps
    read, so it must equal the factor exactly wherever the scaled entry is an FP16
    normal (entries >= 2^-27 sqrt(K_ii)) and within 2^-38 sqrt(K_ii) elsewhere."""
    prob, kappa, f = _prob(rsd, n, depth)
    A = fem.assemble(n, kappa)
    h = _setup(rsd, prob, rsd.RSD_PREC_FP16)
    sq = np.sqrt(A.diagonal())
    for t in range(len(prob["parent"])):
        s, bb, _ = h.front_dims(t)
        P, Q = h.front_factor(t), h.front_factor16(t)
        bound = np.repeat(sq[h.front_dofs(t)][:, None], s, axis=1)
        rows, cols = np.arange(s + bb)[:, None], np.arange(s)[None, :]
        read = (rows >= s) | (cols // 128 < rows // 128)
        big = read & (np.abs(P) >= 2.0**-27 * bound)
        assert np.array_equal(Q[big], P[big]), t
        assert np.all(np.abs(Q - P)[read] <= 2.0**-38 * bound[read]), t
    h.close()


def _breakdown_matrix():
    """SPD K on a three-node tree (root 0, leaves 1 and 2).  Leaf 1 (1100 DOFs, three
    512-wide panels) is the identity except for the 2 x 2 block on DOFs 0 and 1050,
    [[1, a], [a, a^2 + eps]] with a = 1 - 2^-11 (exact in TF32 and FP16, rounded to 1 in
    BF16) and eps = 1e-4: its pivot on DOF 1050 is eps, but with a BF16 copy of
    L[1050, 0] = a the update of the third panel subtracts 1 and the pivot goes negative."""
    a, eps = 1.0 - 2.0**-11, 1e-4
    n1, n2, n0 = 1100, 10, 4
    n = n1 + n2 + n0
    K = sp.lil_matrix((n, n))
    for i in range(n1):
        K[i, i] = 1.0
    K[0, 1050] = K[1050, 0] = a
    K[1050, 1050] = a * a + eps
    for i in range(n1, n1 + n2):
        K[i, i] = 2.0
    for i in range(n1 + n2, n):
        K[i, i] = 4.0
    r0 = n1 + n2
    K[n1 - 1, r0] = K[r0, n1 - 1] = -0.1
    K[n1 + n2 - 1, r0 + 1] = K[r0 + 1, n1 + n2 - 1] = -0.1
    K = K.tocsr()
    K.sort_indices()
    owner = np.array([1] * n1 + [2] * n2 + [0] * n0, dtype=np.int32)
    parent = np.array([-1, 0, 0], dtype=np.int32)
    return K, owner, parent


def test_bf16_breakdown_is_promoted_and_the_solve_succeeds(rsd):
    K, owner, parent = _breakdown_matrix()
    assert np.linalg.eigvalsh(K.toarray()).min() > 0            # SPD
    rowptr = torch.as_tensor(K.indptr.astype(np.int64))
    col = torch.as_tensor(K.indices.astype(np.int32))
    val = torch.as_tensor(K.data.astype(np.float64))
    own = torch.as_tensor(owner)
    b = synth.uniform(121, K.shape[0])
    x_ref = spla.spsolve(K.tocsc(), b)
    bd = torch.as_tensor(b, device="cuda")
    for prec, promoted in (("TF32", 0), ("FP16", 0), ("BF16", 1)):
        p = getattr(rsd, "RSD_PREC_" + prec)
        h = rsd.RSD.setup(rowptr, col, val, own, parent, prec_leaf=p, prec_mid=p, prec_root=p)
        info = h.info()
        assert info["promoted"] == promoted, (prec, info)
        assert info["notspd_node"] == -1
        u, st = h.solve(bd, tol=1e-10)
        assert st["relres"] <= 1e-10, (prec, st)
        assert np.abs(u.cpu().numpy() - x_ref).max() <= 1e-8 * np.abs(x_ref).max()
        h.close()
