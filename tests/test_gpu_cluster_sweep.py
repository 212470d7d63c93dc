"""The root level's sweeps on clusters of CTAs (Eqs. 3.2-3.3 applied at a front without B
rows, the chain of its diagonal blocks handed on through distributed shared memory).

Reference: the block recursion of the sweeps in FP64 with exactly the factor data the
kernels read, taken back from the device -- the FP16 copy off the diagonal blocks
(rsd_front_factor16) and the stored inverted diagonal blocks (rsd_front_dinv) -- over the
oracle's interface sets and extend-add maps: upward, y_k = Dinv_k (v_k - sum_{j<k} L_kj y_j)
and the contribution v_B - X y (Eq. 3.2); downward, x_k = Dinv_k^T (t_k - sum_{r>k} L_rk^T x_r)
with t = y - X^T x_B (Eq. 3.3).  So the check isolates the substitution sweeps from the
factorisation.  The cases cover one partial cluster (5 blocks), two clusters with a
partial last block, and five clusters whose last one holds 3 blocks."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import partition

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsd():
    from paper_1210_6266_gb300 import build
    build.build()
    import paper_1210_6266_gb300 as m
    return m


def _problem(rsd, n, depth, seed=171):
    kappa = np.exp(synth.normal(seed, (n - 1) ** 3))
    f = synth.uniform(seed + 1, (n - 2) ** 3)
    prob = rsd.grid_problem(n, depth, kappa, f)
    nd = prob["n_dof"]
    A = sp.csr_matrix((prob["val"].cpu().numpy(), prob["col"].cpu().numpy(), prob["rowptr"].cpu().numpy()), shape=(nd, nd))
    sym = partition.Symbolic(A, prob["dof_node"].cpu().numpy(), np.asarray(prob["parent"]))
    return prob, sym


def _block_apply(h, sym, r):
    F = [h.front_factor16(t) for t in range(sym.n_nodes)]
    D = [h.front_dinv(t) for t in range(sym.n_nodes)]
    y, contrib = [None] * sym.n_nodes, [None] * sym.n_nodes
    for t in sym.post:
        s, b = sym.s(t), sym.b(t)
        v = np.zeros(s + b)
        v[:s] = r[sym.I[t]]
        for c in sym.children[t]:
            np.add.at(v, sym.ea[c], contrib[c])
        yt = np.zeros(s)
        for k in range((s + 127) // 128):
            lo, hi = 128 * k, min(s, 128 * k + 128)
            yt[lo:hi] = D[t][k][: hi - lo, : hi - lo] @ (v[lo:hi] - F[t][lo:hi, :lo] @ yt[:lo])
        y[t], contrib[t] = yt, v[s:] - F[t][s:, :] @ yt
    z = np.zeros(len(r))
    for t in reversed(sym.post):
        s = sym.s(t)
        if not s:
            continue
        tt = y[t] - F[t][s:, :].T @ z[sym.B[t]]
        xt = np.zeros(s)
        for k in reversed(range((s + 127) // 128)):
            lo, hi = 128 * k, min(s, 128 * k + 128)
            xt[lo:hi] = D[t][k][: hi - lo, : hi - lo].T @ (tt[lo:hi] - F[t][hi:s, lo:hi].T @ xt[hi:s])
        z[sym.I[t]] = xt
    return z


@pytest.mark.parametrize("prec", ["TF32", "FP16"])
@pytest.mark.parametrize("n,depth", [(17, 2), (26, 1), (41, 1)])
def test_cluster_sweeps_match_the_recursion_with_the_same_factors(rsd, n, depth, prec):
    prob, sym = _problem(rsd, n, depth)
    p = getattr(rsd, "RSD_PREC_" + prec)
    h = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                      prec_leaf=p, prec_mid=p, prec_root=p)
    s0, b0, _ = h.front_dims(0)
    assert b0 == 0 and s0 == sym.s(0)
    for seed in (181, 182):
        r = synth.uniform(seed, prob["n_dof"])
        z = h.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
        zr = _block_apply(h, sym, r)
        err = np.abs(z - zr).max() / np.abs(zr).max()
        assert err <= 1e-5, (seed, err)
    # fixed-order accumulation: the same input gives the same bits
    rt = torch.as_tensor(synth.uniform(183, prob["n_dof"]), device="cuda")
    assert torch.equal(h.apply(rt), h.apply(rt))
    h.close()


def test_cluster_sweeps_reach_the_fp64_residual_at_a_long_root(rsd):
    """A 4447-DOF root (35 diagonal blocks, five clusters): FP64 PCG to 1e-10."""
    prob, sym = _problem(rsd, 41, 1, seed=191)
    h = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                      prec_leaf=rsd.RSD_PREC_FP16, prec_mid=rsd.RSD_PREC_FP16, prec_root=rsd.RSD_PREC_FP16)
    u, st = h.solve(prob["b"], tol=1e-10)
    assert st["relres"] <= 1e-10 and st["iterations"] <= 12, st
    h.close()


def test_cluster_sweeps_on_a_level_of_many_roots(rsd):
    """Batched problems: their roots form one level of fronts without B rows, each front's
    first block solved by a cluster's first CTA with no earlier step.  Repeated applies give
    the same bits (no race between a CTA's own shared-memory writes and reads) and the FP64
    solve reaches its residual on every problem."""
    sizes = [(13, 1), (17, 1), (15, 1), (19, 1), (14, 1)]
    probs = []
    for q, (n, depth) in enumerate(sizes):
        kappa = np.exp(synth.normal(201 + q, (n - 1) ** 3))
        probs.append(rsd.grid_problem(n, depth, kappa, synth.uniform(211 + q, (n - 2) ** 3)))
    h = rsd.RSD.setup_batched(probs, prec_leaf=rsd.RSD_PREC_FP16, prec_mid=rsd.RSD_PREC_FP16,
                              prec_root=rsd.RSD_PREC_FP16)
    n = sum(p["n_dof"] for p in probs)
    rt = torch.as_tensor(synth.uniform(221, n), device="cuda")
    z0 = h.apply(rt)
    for _ in range(3):
        assert torch.equal(h.apply(rt), z0)
    b = torch.cat([p["b"] for p in probs])
    u, st = h.solve(b, tol=1e-10)
    assert st["relres"] <= 1e-10, st
    h.close()
