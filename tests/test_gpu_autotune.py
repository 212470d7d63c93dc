"""The tile autotuner: rsd_autotune times the tensor-core GEMM configurations per size
bucket and writes a table; a setup that reads it (tune_cache) picks tile widths and split-K
counts from it and must give the same factors as the built-in rules up to the TF32 /
FP16 rounding of a different summation order, and a converged solve."""
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


@pytest.fixture(scope="module")
def table(rsd, tmp_path_factory):
    path = str(tmp_path_factory.mktemp("tune") / "tune.json")
    secs = rsd.autotune(path)
    assert secs > 0
    return path


def test_autotune_writes_every_bucket(rsd, table):
    assert rsd.tune_entries(table) == 2 * 5 * 4
    text = open(table).read()
    assert '"entries"' in text and '"bn": 256' in text


@pytest.mark.parametrize("prec", ["TF32", "FP16"])
@pytest.mark.parametrize("n,depth", [(41, 1), (41, 2)])
def test_tuned_setup_matches_the_rules(rsd, table, prec, n, depth):
    kappa = np.exp(synth.normal(141, (n - 1) ** 3))
    prob = rsd.grid_problem(n, depth, kappa, synth.uniform(142, (n - 2) ** 3))
    p = getattr(rsd, "RSD_PREC_" + prec)
    kw = dict(prec_leaf=p, prec_mid=p, prec_root=p)
    h0 = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"], **kw)
    h1 = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                       tune_cache=table, **kw)
    for t in range(len(prob["parent"])):
        a, b = h0.front_factor(t), h1.front_factor(t)
        assert np.abs(a - b).max() <= 5e-3 * np.abs(a).max(), t
    u, st = h1.solve(prob["b"], tol=1e-8)
    assert st["relres"] <= 1e-8
    h0.close()
    h1.close()
