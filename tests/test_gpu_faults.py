"""Failure detection without a GPU fault: the bounded waits of the substitution sweeps.

A work item of an upward sweep is dropped on the host (rsd_inject_drop_sweep_item), so
the items that consume its result wait on a progress counter that nothing raises.  With
a short per-handle wait bound the waits give up, the kernels finish, the call completes
and rsd_check reports RSD_ERR_TIMEOUT; the CUDA context stays usable for a new handle."""
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


def _setup(rsd, prob, prec, wait_cycles=0):
    return rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                         prec_leaf=prec, prec_mid=prec, prec_root=rsd.RSD_PREC_FP64, wait_cycles=wait_cycles)


@pytest.mark.parametrize("prec,level", [("FP64", 2), ("TF32", 1)])
def test_dropped_sweep_item_times_out_and_is_reported(rsd, prec, level):
    from paper_1210_6266_gb300 import _lib
    lib = _lib.load()
    n = 17
    prob = rsd.grid_problem(n, 2, np.exp(synth.normal(81, (n - 1) ** 3)), synth.uniform(82, (n - 2) ** 3))
    r = torch.as_tensor(synth.uniform(83, prob["n_dof"]), device="cuda")
    p = getattr(rsd, "RSD_PREC_" + prec)
    h = _setup(rsd, prob, p, wait_cycles=100_000)          # ~50 us at 2 GHz
    z_ref = h.apply(r).clone()
    h.check()
    assert lib.rsd_inject_drop_sweep_item(h._h, 99) == _lib.RSD_ERR_ARG
    assert lib.rsd_inject_drop_sweep_item(h._h, level) == 0
    z = torch.empty_like(r)
    assert lib.rsd_apply(h._h, r.data_ptr(), z.data_ptr()) == 0
    torch.cuda.synchronize()                               # the kernels finished
    assert lib.rsd_check(h._h) == _lib.RSD_ERR_TIMEOUT
    h.close()
    # the context is still usable: a new handle gives the same application as before
    h2 = _setup(rsd, prob, p)
    z2 = h2.apply(r)
    h2.check()
    assert torch.equal(z2, z_ref)
    h2.close()
