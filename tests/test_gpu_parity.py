"""CUDA path vs the CPU oracle, through the C ABI.

Integer work (assembly structure, ownership, interface sets, extend-add maps) must be
bit-exact; the FP64 path must match the oracle to 1e-10 relative; the FP32/TF32 paths
must reach an FP64-checked relative residual of 1e-8 under FP64 PCG.
"""
import numpy as np
import pytest

import synth
from oracle import fem, partition
from oracle.krylov import pcg
from oracle.rsd_exact import ExactFactor

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsd():
    from paper_1210_6266_gb300 import build
    build.build()
    import paper_1210_6266_gb300 as m
    return m


def _work(n, depth, lognormal, seed=41):
    kappa = np.exp(synth.normal(seed, (n - 1) ** 3)) if lognormal else np.ones((n - 1) ** 3)
    f = synth.uniform(seed + 1, (n - 2) ** 3)
    return dict(n=n, depth=depth, kappa=kappa, f=f)


_ORACLE = {}


def _oracle(w):
    key = (w["n"], w["depth"], float(w["kappa"][0]), float(w["f"][0]))
    if key not in _ORACLE:
        n, depth = w["n"], w["depth"]
        A = fem.assemble(n, w["kappa"])
        b = fem.load_vector(n, w["f"])
        owner = partition.octree_owner(n, depth, fem.interior_coords(n))
        parent = partition.octree_parent(depth)
        sym = partition.Symbolic(A, owner, parent)
        _ORACLE[key] = (A, b, owner, parent, sym, ExactFactor(A, sym))
    return _ORACLE[key]


# (n, depth, lognormal): several tiles per front, ragged tails, uneven octree splits
CASES = [(13, 1, False), (17, 2, True), (20, 2, True), (11, 2, False), (26, 1, True), (9, 0, True)]


@pytest.mark.parametrize("n,depth,logn", CASES)
def test_grid_assembly_and_partition_bitexact(rsd, n, depth, logn):
    w = _work(n, depth, logn)
    A, b, owner, parent, sym, _ = _oracle(w)
    prob = rsd.grid_problem(n, depth, w["kappa"], w["f"])
    assert np.array_equal(prob["rowptr"].cpu().numpy(), A.indptr)
    assert np.array_equal(prob["col"].cpu().numpy(), A.indices)
    val = prob["val"].cpu().numpy()
    assert np.abs(val - A.data).max() <= 1e-14 * np.abs(A.data).max()
    assert np.abs(prob["b"].cpu().numpy() - b).max() <= 1e-15 * np.abs(b).max()
    assert np.array_equal(prob["dof_node"].cpu().numpy(), owner)
    assert np.array_equal(prob["parent"], parent)


def _setup(rsd, prob, prec, root=None):
    root = rsd.RSD_PREC_FP64 if root is None else root
    return rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                         prec_leaf=prec, prec_mid=prec, prec_root=root)


@pytest.mark.parametrize("n,depth,logn", CASES)
def test_interface_sets_and_maps_bitexact(rsd, n, depth, logn):
    w = _work(n, depth, logn)
    A, b, owner, parent, sym, _ = _oracle(w)
    prob = rsd.grid_problem(n, depth, w["kappa"], w["f"])
    h = _setup(rsd, prob, rsd.RSD_PREC_FP64)
    for t in range(sym.n_nodes):
        s, bb, lv = h.front_dims(t)
        assert (s, bb, lv) == (sym.s(t), sym.b(t), sym.depth[t])
        assert np.array_equal(h.front_dofs(t), sym.front[t])
        if t > 0:
            assert np.array_equal(h.front_map(t), sym.ea[t])


@pytest.mark.parametrize("n,depth,logn", CASES)
def test_fp64_factors_and_apply_match_oracle(rsd, n, depth, logn):
    w = _work(n, depth, logn)
    A, b, owner, parent, sym, fac = _oracle(w)
    prob = rsd.grid_problem(n, depth, w["kappa"], w["f"])
    h = _setup(rsd, prob, rsd.RSD_PREC_FP64)
    for t in range(sym.n_nodes):
        s = sym.s(t)
        F = h.front_factor(t)
        ref = np.vstack([fac.L[t], fac.X[t]])
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(F - ref).max() <= 1e-10 * scale, t
    r = torch.as_tensor(synth.uniform(77, A.shape[0]), device="cuda")
    z = h.apply(r).cpu().numpy()
    zr = fac.apply(r.cpu().numpy())
    assert np.abs(z - zr).max() <= 1e-10 * np.abs(zr).max()
    h.check()


@pytest.mark.parametrize("n,depth,logn", CASES)
def test_fp64_pcg_one_iteration(rsd, n, depth, logn):
    w = _work(n, depth, logn)
    A, b, owner, parent, sym, fac = _oracle(w)
    prob = rsd.grid_problem(n, depth, w["kappa"], w["f"])
    h = _setup(rsd, prob, rsd.RSD_PREC_FP64)
    u, st = h.solve(prob["b"], tol=1e-10)
    assert st["iterations"] == 1 and st["relres"] <= 1e-10
    x, it, _ = pcg(A, b, fac.apply, 1e-10)
    assert np.abs(u.cpu().numpy() - x).max() <= 1e-10 * np.abs(x).max()


@pytest.mark.parametrize("prec", ["FP32", "TF32"])
@pytest.mark.parametrize("n,depth,logn", [(17, 2, True), (20, 2, True), (26, 1, True)])
def test_low_precision_factors_reach_fp64_residual(rsd, prec, n, depth, logn):
    w = _work(n, depth, logn)
    A, b, owner, parent, sym, fac = _oracle(w)
    prob = rsd.grid_problem(n, depth, w["kappa"], w["f"])
    p = getattr(rsd, "RSD_PREC_" + prec)
    h = _setup(rsd, prob, p)
    # factors agree with the oracle to single-precision accuracy
    for t in sym.leaves()[:3] + [0]:
        F = h.front_factor(t)
        ref = np.vstack([fac.L[t], fac.X[t]])
        tol = 1e-4 if prec == "FP32" else 3e-2
        assert np.abs(F - ref).max() <= tol * np.abs(ref).max(), (t, np.abs(F - ref).max() / np.abs(ref).max())
    u, st = h.solve(prob["b"], tol=1e-8)
    assert st["relres"] <= 1e-8 and st["iterations"] <= 30, st
    x = np.linalg.solve(A.toarray(), b)
    assert np.abs(u.cpu().numpy() - x).max() <= 1e-6 * np.abs(x).max()


def test_not_spd_is_reported(rsd):
    w = _work(9, 1, False)
    prob = rsd.grid_problem(9, 1, w["kappa"], w["f"])
    with pytest.raises(rsd.RSDError) as e:
        rsd.RSD.setup(prob["rowptr"], prob["col"], -prob["val"], prob["dof_node"], prob["parent"],
                      prec_leaf=rsd.RSD_PREC_FP64, prec_mid=rsd.RSD_PREC_FP64)
    assert e.value.code == -3


def test_host_csr_input_matches_device_input(rsd):
    w = _work(13, 1, True)
    prob = rsd.grid_problem(13, 1, w["kappa"], w["f"])
    h1 = _setup(rsd, prob, rsd.RSD_PREC_FP64)
    h2 = rsd.RSD.setup(prob["rowptr"].cpu(), prob["col"].cpu(), prob["val"].cpu(), prob["dof_node"].cpu(),
                       prob["parent"], prec_leaf=rsd.RSD_PREC_FP64, prec_mid=rsd.RSD_PREC_FP64)
    r = prob["b"]
    assert torch.equal(h1.apply(r), h2.apply(r))


def test_host_and_device_csr_give_the_same_structure(rsd):
    """A device CSR goes straight to the GPU structure pass (Eq. 3.1 check, B-set bitmaps);
    a host CSR is uploaded first: identical interface sets and extend-add maps."""
    w = _work(20, 2, True)
    prob = rsd.grid_problem(20, 2, w["kappa"], w["f"])
    hd = _setup(rsd, prob, rsd.RSD_PREC_FP64)
    hh = rsd.RSD.setup(prob["rowptr"].cpu(), prob["col"].cpu(), prob["val"].cpu(), prob["dof_node"].cpu(),
                       prob["parent"], prec_leaf=rsd.RSD_PREC_FP64, prec_mid=rsd.RSD_PREC_FP64)
    for t in range(len(prob["parent"])):
        assert hd.front_dims(t) == hh.front_dims(t)
        assert np.array_equal(hd.front_dofs(t), hh.front_dofs(t))
        assert np.array_equal(hd.front_map(t), hh.front_map(t))


def test_device_structure_pass_rejects_bad_input(rsd):
    from paper_1210_6266_gb300 import _lib
    n = 9
    A = fem.assemble(n, np.ones((n - 1) ** 3)).tolil()
    owner = partition.octree_owner(n, 1, fem.interior_coords(n))
    parent = partition.octree_parent(1)
    i, j = int(np.nonzero(owner == 1)[0][0]), int(np.nonzero(owner == 8)[0][-1])
    A[i, j] = A[j, i] = -0.01                       # couples two leaves: violates Eq. 3.1
    A = A.tocsr()
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    args = (dev(A.indptr, torch.int64), dev(A.indices, torch.int32), dev(A.data, torch.float64),
            dev(owner, torch.int32), parent)
    with pytest.raises(rsd.RSDError) as e:
        rsd.RSD.setup(*args, prec_leaf=rsd.RSD_PREC_FP64, prec_mid=rsd.RSD_PREC_FP64)
    assert e.value.code == _lib.RSD_ERR_PARTITION
    B = fem.assemble(n, np.ones((n - 1) ** 3))
    col = B.indices.copy()
    col[5] = B.shape[0]                             # column index out of range
    args = (dev(B.indptr, torch.int64), dev(col, torch.int32), dev(B.data, torch.float64),
            dev(owner, torch.int32), parent)
    with pytest.raises(rsd.RSDError) as e:
        rsd.RSD.setup(*args, prec_leaf=rsd.RSD_PREC_FP64, prec_mid=rsd.RSD_PREC_FP64)
    assert e.value.code == _lib.RSD_ERR_ARG


def test_apply_is_deterministic(rsd):
    w = _work(20, 2, True)
    prob = rsd.grid_problem(20, 2, w["kappa"], w["f"])
    h = _setup(rsd, prob, rsd.RSD_PREC_TF32)
    z1 = h.apply(prob["b"]).clone()
    z2 = h.apply(prob["b"])
    assert torch.equal(z1, z2)


@pytest.mark.parametrize("n,depth", [(9, 0), (17, 2), (26, 1), (20, 2)])
def test_tf32_tensor_core_factors_track_fp32(rsd, n, depth):
    """The tcgen05 TF32 GEMMs must reproduce the FP32 CUDA-core factors to TF32 rounding
    (10-bit mantissa products, FP32 accumulation) at every node, root included."""
    w = _work(n, depth, True)
    prob = rsd.grid_problem(n, depth, w["kappa"], w["f"])
    h32 = _setup(rsd, prob, rsd.RSD_PREC_FP32, root=rsd.RSD_PREC_FP32)
    htf = _setup(rsd, prob, rsd.RSD_PREC_TF32, root=rsd.RSD_PREC_TF32)
    n_nodes = len(prob["parent"])
    for t in range(n_nodes):
        a, b = h32.front_factor(t), htf.front_factor(t)
        scale = np.abs(a).max()
        assert np.abs(a - b).max() <= 5e-3 * scale, (t, np.abs(a - b).max() / scale)
    u, st = htf.solve(prob["b"], tol=1e-8)
    assert st["relres"] <= 1e-8, st


def test_profile_trace_matches_profile(rsd):
    """rsd_profile_trace lists the launches rsd_profile sums: same count per class, ends
    after starts, and the look-ahead stream in use for a single large front."""
    w = _work(26, 1, True)
    prob = rsd.grid_problem(26, 1, w["kappa"], w["f"])
    h = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                      prec_leaf=rsd.RSD_PREC_TF32, prec_mid=rsd.RSD_PREC_TF32, prec_root=rsd.RSD_PREC_TF32,
                      profile=True)
    h.solve(prob["b"], tol=1e-8)
    tr = h.trace()
    prof = h.profile()
    counts = {}
    for r in tr:
        counts[r["cls"]] = counts.get(r["cls"], 0) + 1
        assert r["end_ms"] >= r["start_ms"] >= 0.0
        assert r["stream"] in (0, 1)
    for cls, v in prof.items():
        if isinstance(v, dict) and "launches" in v:
            assert counts.get(cls, 0) == v["launches"], cls
    assert any(r["stream"] == 1 for r in tr)           # the root's diagonal-block chain
    assert prof["host_issue_ms"] > 0


def test_graph_replayed_apply_matches_direct_launches(rsd):
    """Without profiling, a handle's second and later solves replay the preconditioner
    application from a captured CUDA graph; the iterates must be bitwise those of the
    directly launched solves."""
    w = _work(20, 2, True)
    prob = rsd.grid_problem(20, 2, w["kappa"], w["f"])
    kw = dict(prec_leaf=rsd.RSD_PREC_TF32, prec_mid=rsd.RSD_PREC_TF32, prec_root=rsd.RSD_PREC_TF32)
    hg = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"], **kw)
    hd = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                       profile=True, **kw)
    ug, sg = hg.solve(prob["b"], tol=1e-10)
    ud, sd = hd.solve(prob["b"], tol=1e-10)
    assert sg["iterations"] == sd["iterations"] >= 3
    assert torch.equal(ug, ud)
    for _ in range(2):                                     # captured, then replayed
        ug2, sg2 = hg.solve(prob["b"], tol=1e-10)
        assert sg2["iterations"] == sg["iterations"]
        assert torch.equal(ug2, ug)


def test_lookahead_setup_is_deterministic(rsd):
    """The two-stream look-ahead factorisation of a root with many 512-wide panels gives
    bitwise the same factors on every setup, profiled (an event around each launch) or
    not: every read of a panel block is ordered after all writes to it."""
    n, depth = 41, 1
    w = _work(n, depth, True)
    prob = rsd.grid_problem(n, depth, w["kappa"], w["f"])
    kw = dict(prec_leaf=rsd.RSD_PREC_TF32, prec_mid=rsd.RSD_PREC_TF32, prec_root=rsd.RSD_PREC_TF32)
    root = [t for t, p in enumerate(prob["parent"]) if p < 0][0]
    ref = None
    for profile in (True, False, False, False):
        h = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                          profile=profile, **kw)
        assert h.front_dims(root)[0] > 3 * 512
        u, st = h.solve(prob["b"], tol=1e-10)
        got = (h.front_factor(root), st["iterations"], u.cpu())
        if ref is None:
            ref = got
            continue
        assert np.array_equal(got[0], ref[0])
        assert got[1] == ref[1]
        assert torch.equal(got[2], ref[2])


@pytest.mark.parametrize("n,depth", [(17, 2), (26, 1), (20, 2)])
def test_fp16_factor_copy_holds_the_tf32_factor(rsd, n, depth):
    """A TF32 level's sweeps read an FP16 copy of the factor, row i scaled by a power of two
    set from sqrt(K_ii).  Every entry they read is bounded by sqrt(K_ii) (a Cholesky row's
    2-norm is the square root of a Schur complement's diagonal entry, at most K_ii), and
    the copy equals the TF32 factor exactly except for entries below 2^-27 sqrt(K_ii)
    (FP16 subnormals after scaling), which it holds to 2^-38 sqrt(K_ii)."""
    w = _work(n, depth, True)
    A, b, owner, parent, sym, _ = _oracle(w)
    prob = rsd.grid_problem(n, depth, w["kappa"], w["f"])
    h = _setup(rsd, prob, rsd.RSD_PREC_TF32, root=rsd.RSD_PREC_TF32)
    sq = np.sqrt(A.diagonal())
    for t in range(len(prob["parent"])):
        s, bb, _ = h.front_dims(t)
        P, Q = h.front_factor(t), h.front_factor16(t)
        bound = np.repeat(sq[h.front_dofs(t)][:, None], s, axis=1)
        rows, cols = np.arange(s + bb)[:, None], np.arange(s)[None, :]
        read = (rows >= s) | (cols // 128 < rows // 128)
        assert np.all(Q[~read] == 0.0)
        assert np.all(np.abs(P[read]) <= bound[read] * 1.01), t
        big = read & (np.abs(P) >= 2.0**-27 * bound)
        assert np.array_equal(Q[big], P[big]), t
        assert np.all(np.abs(Q - P)[read] <= 2.0**-38 * bound[read]), t
    h32 = _setup(rsd, prob, rsd.RSD_PREC_FP32, root=rsd.RSD_PREC_FP32)
    with pytest.raises(rsd.RSDError):
        h32.front_factor16(0)
