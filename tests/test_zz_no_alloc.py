"""rsd_apply_static: the preconditioner application for callers that cannot have device
memory allocated for them (stream capture, fixed memory budgets, foreign allocators).
Its scratch is a 4 MiB file-scope device array; its result must equal rsd_apply's.
This file is collected last on purpose."""
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


def _handle(rsd, n, depth, prec):
    kappa = np.exp(synth.normal(51, (n - 1) ** 3))
    prob = rsd.grid_problem(n, depth, kappa, synth.uniform(52, (n - 2) ** 3))
    h = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                      prec_leaf=prec, prec_mid=prec, prec_root=rsd.RSD_PREC_FP64)
    return h, prob


@pytest.mark.parametrize("n,depth,prec", [(13, 1, "FP64"), (17, 2, "FP64"), (20, 2, "TF32")])
def test_static_apply_matches_apply_on_two_calls(rsd, n, depth, prec):
    from paper_1210_6266_gb300 import _lib
    lib = _lib.load()
    h, prob = _handle(rsd, n, depth, getattr(rsd, "RSD_PREC_" + prec))
    r = torch.as_tensor(synth.uniform(53, prob["n_dof"]), device="cuda")
    z_ref = h.apply(r).clone()
    for _ in range(2):
        z = torch.full_like(r, float("nan"))
        assert lib.rsd_apply_static(h._h, r.data_ptr(), z.data_ptr()) == 0
        torch.cuda.synchronize()
        h.check()
        err = (z - z_ref).abs().max().item() / z_ref.abs().max().item()
        assert err <= 1e-10, err
    h.close()


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
