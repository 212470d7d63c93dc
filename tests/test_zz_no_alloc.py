"""rsd_apply_static: the preconditioner application for callers that cannot have device
memory allocated for them (a process under a fixed device-memory budget, or code inside
a framework whose own caching allocator owns the device).  Its scratch is a 4 MiB
file-scope device array shared by every handle; the descriptors that point into it are
prepared at setup.  It launches the same sweep kernels, in the same order, as
rsd_apply, so its result must be bitwise rsd_apply's, on repeated calls and when calls
alternate between handles.  This file is collected last on purpose."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsd():
    from paper_1210_6266_gb300 import build
    build.build()
    import paper_1210_6266_gb300 as m
    return m


def _handle(rsd, n, depth, prec, seed=51):
    kappa = np.exp(synth.normal(seed, (n - 1) ** 3))
    prob = rsd.grid_problem(n, depth, kappa, synth.uniform(seed + 1, (n - 2) ** 3))
    h = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                      prec_leaf=prec, prec_mid=prec, prec_root=rsd.RSD_PREC_FP64)
    return h, prob


def _static(lib, h, r):
    z = torch.full_like(r, float("nan"))
    assert lib.rsd_apply_static(h._h, r.data_ptr(), z.data_ptr()) == 0, lib.rsd_last_error_detail()
    torch.cuda.synchronize()
    h.check()
    return z


@pytest.mark.parametrize("n,depth,prec", [(13, 1, "FP64"), (17, 2, "FP64"), (20, 2, "TF32")])
def test_static_apply_matches_apply_on_two_calls(rsd, n, depth, prec):
    from paper_1210_6266_gb300 import _lib
    lib = _lib.load()
    h, prob = _handle(rsd, n, depth, getattr(rsd, "RSD_PREC_" + prec))
    r = torch.as_tensor(synth.uniform(53, prob["n_dof"]), device="cuda")
    z_ref = h.apply(r).clone()
    for _ in range(2):
        z = _static(lib, h, r)
        assert torch.equal(z, z_ref)
    h.close()


def test_static_apply_alternating_handles(rsd):
    """Two hierarchies share the device array: each call must still give its own
    handle's rsd_apply result exactly."""
    from paper_1210_6266_gb300 import _lib
    lib = _lib.load()
    ha, pa = _handle(rsd, 17, 2, rsd.RSD_PREC_TF32, seed=61)
    hb, pb = _handle(rsd, 14, 1, rsd.RSD_PREC_FP64, seed=71)
    ra = torch.as_tensor(synth.uniform(63, pa["n_dof"]), device="cuda")
    rb = torch.as_tensor(synth.uniform(73, pb["n_dof"]), device="cuda")
    za_ref, zb_ref = ha.apply(ra).clone(), hb.apply(rb).clone()
    for h, r, ref in ((ha, ra, za_ref), (hb, rb, zb_ref), (ha, ra, za_ref), (hb, rb, zb_ref)):
        assert torch.equal(_static(lib, h, r), ref)
    ha.close()
    hb.close()


def test_static_apply_rejects_hierarchies_beyond_its_scratch(rsd):
    from paper_1210_6266_gb300 import _lib
    lib = _lib.load()
    h, prob = _handle(rsd, 65, 3, rsd.RSD_PREC_FP64)      # about 4.9 MB of FP64 sweep scratch
    r = torch.ones(prob["n_dof"], dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    rc = lib.rsd_apply_static(h._h, r.data_ptr(), z.data_ptr())
    assert rc == _lib.RSD_ERR_ARG
    assert b"static limit" in lib.rsd_last_error_detail()
    h.close()
