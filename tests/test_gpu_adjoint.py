"""Adjoint gradient on the GPU vs the oracle and vs central differences.

Workload: -div(exp(m) grad u) = f with m a per-element Gaussian random field, loss
L = 1/2 |u - u_obs|^2, u_obs the solution for a second field; dL/dm and dL/db through
the differentiable solve (forward rsd_solve, backward rsd_solve_adjoint + the
per-element gradient kernel).  Tolerance: 1e-5 relative against central differences
(solves to 1e-12), as the gradient target states; against the oracle's direct-solve
gradient the FP64 path must agree to 1e-9 and the TF32 path to 1e-7 (both solves stop
at a 1e-12 residual, and the gradient is bilinear in u and lam).
"""
import numpy as np
import pytest

import synth
from oracle import adjoint, fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsd():
    from paper_1210_6266_gb300 import build
    build.build()
    import paper_1210_6266_gb300 as m
    return m


def _problem(n, m_seed=6, f_seed=7, m2_seed=8):
    nd = (n - 2) ** 3
    m = synth.gaussian_field(n, m_seed)
    b = fem.load_vector(n, synth.uniform(f_seed, nd))
    m2 = synth.gaussian_field(n, m2_seed)
    return m, b, m2


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n", [5, 17, 33])
def test_exp_and_coef_grad_kernels_match_oracle(rsd, n):
    nd, ne = (n - 2) ** 3, (n - 1) ** 3
    m = synth.gaussian_field(n, 21) if n > 5 else synth.normal(21, ne)
    u, lam = synth.normal(22, nd), synth.normal(23, nd)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    kappa = rsd.grid_exp(n, dev(m))
    assert np.allclose(kappa.cpu().numpy(), np.exp(m), rtol=1e-15, atol=0)
    dk, dm = rsd.coef_grad(n, dev(u), dev(lam), kappa)
    ref = adjoint.coef_grad(n, u, lam)
    scale = np.abs(ref).max()
    assert np.abs(dk.cpu().numpy() - ref).max() <= 1e-13 * scale
    assert np.abs(dm.cpu().numpy() - np.exp(m) * ref).max() <= 1e-13 * np.abs(np.exp(m) * ref).max()
    dk_only, none = rsd.coef_grad(n, dev(u), dev(lam))
    assert none is None and torch.equal(dk_only, dk)


def _gpu_grad(rsd, n, depth, m, b, u_obs, precs, tol=1e-12):
    mt = torch.tensor(m, dtype=torch.float64, device="cuda", requires_grad=True)
    bt = torch.tensor(b, dtype=torch.float64, device="cuda", requires_grad=True)
    u = rsd.diffusion_solve(mt, bt, n, depth, tol=tol, precs=precs)
    L = 0.5 * ((u - torch.tensor(u_obs, device="cuda")) ** 2).sum()
    L.backward()
    return float(L.detach()), u.detach().cpu().numpy(), mt.grad.cpu().numpy(), bt.grad.cpu().numpy()


def _gpu_loss(rsd, n, depth, m, b, u_obs, precs, tol=1e-12):
    with torch.no_grad():
        mt = torch.tensor(m, dtype=torch.float64, device="cuda")
        bt = torch.tensor(b, dtype=torch.float64, device="cuda")
        u = rsd.diffusion_solve(mt, bt, n, depth, tol=tol, precs=precs).cpu().numpy()
    return 0.5 * float((u - u_obs) @ (u - u_obs))


FP64 = "fp64"
TF32 = "tf32"


def _precs(rsd, form):
    if form == FP64:
        return (rsd.RSD_PREC_FP64,) * 3
    return (rsd.RSD_PREC_TF32, rsd.RSD_PREC_TF32, rsd.RSD_PREC_FP64)


@pytest.mark.parametrize("form", [FP64, TF32])
def test_gradient_matches_oracle_and_central_differences(rsd, form):
    n, depth = 17, 2
    m, b, m2 = _problem(n)
    u_obs = adjoint.loss_and_grad(n, m2, b, np.zeros_like(b))["u"]
    ref = adjoint.loss_and_grad(n, m, b, u_obs)
    precs = _precs(rsd, form)
    L, u, dm, db = _gpu_grad(rsd, n, depth, m, b, u_obs, precs)
    tol_ref = 1e-9 if form == FP64 else 1e-7
    assert L == pytest.approx(ref["loss"], rel=tol_ref)
    assert _rel(u, ref["u"]) < tol_ref
    assert _rel(dm, ref["dm"]) < tol_ref
    assert _rel(db, ref["db"]) < tol_ref
    # central differences through the GPU solve: 8 random directions, 16 single elements
    # (those with the largest |dL/dm_e|, where the difference quotient is well above the
    # solve's own error)
    eps = 1e-5
    ne = (n - 1) ** 3
    for k in range(8):
        d = synth.normal(300 + k, ne)
        fd = (_gpu_loss(rsd, n, depth, m + eps * d, b, u_obs, precs)
              - _gpu_loss(rsd, n, depth, m - eps * d, b, u_obs, precs)) / (2 * eps)
        assert dm @ d == pytest.approx(fd, rel=1e-5)
    for e in np.argsort(-np.abs(dm))[:16]:
        d = np.zeros(ne)
        d[e] = 1.0
        fd = (_gpu_loss(rsd, n, depth, m + eps * d, b, u_obs, precs)
              - _gpu_loss(rsd, n, depth, m - eps * d, b, u_obs, precs)) / (2 * eps)
        assert dm[e] == pytest.approx(fd, rel=1e-5)
    db_dir = synth.normal(400, b.size) * np.abs(b).max()
    epsb = 1e-3
    fd = (_gpu_loss(rsd, n, depth, m, b + epsb * db_dir, u_obs, precs)
          - _gpu_loss(rsd, n, depth, m, b - epsb * db_dir, u_obs, precs)) / (2 * epsb)
    assert db @ db_dir == pytest.approx(fd, rel=1e-5)


@pytest.mark.parametrize("form", [FP64, TF32])
def test_gradient_full_size_65(rsd, form):
    """The 65^3 gradient workload (depth 2, 64 leaves) through properties that hold at any
    size: the forward and adjoint residuals, Euler's identity for the kappa-linear K, and
    central differences along two random directions."""
    n, depth = 65, 2
    m, b, m2 = _problem(n)
    precs = _precs(rsd, form)
    with torch.no_grad():
        u_obs = rsd.diffusion_solve(torch.tensor(m2, device="cuda"), torch.tensor(b, device="cuda"),
                                    n, depth, tol=1e-12, precs=precs).cpu().numpy()
    mt = torch.tensor(m, dtype=torch.float64, device="cuda", requires_grad=True)
    bt = torch.tensor(b, dtype=torch.float64, device="cuda", requires_grad=True)
    u = rsd.diffusion_solve(mt, bt, n, depth, tol=1e-12, precs=precs)
    L = 0.5 * ((u - torch.tensor(u_obs, device="cuda")) ** 2).sum()
    L.backward()
    u = u.detach().cpu().numpy()
    dm, lam = mt.grad.cpu().numpy(), bt.grad.cpu().numpy()
    kappa = np.exp(m)
    A = fem.assemble(n, kappa)
    r = u - u_obs
    assert np.linalg.norm(A @ u - b) <= 1e-11 * np.linalg.norm(b)
    assert np.linalg.norm(A @ lam - r) <= 1e-11 * np.linalg.norm(r)
    assert dm.sum() == pytest.approx(-(lam @ (A @ u)), rel=1e-10)      # Euler's identity in kappa
    eps = 1e-5
    for k in range(2):
        d = synth.normal(500 + k, m.size)
        fd = (_gpu_loss(rsd, n, depth, m + eps * d, b, u_obs, precs)
              - _gpu_loss(rsd, n, depth, m - eps * d, b, u_obs, precs)) / (2 * eps)
        assert dm @ d == pytest.approx(fd, rel=1e-5)
