"""Pins for the oracle's adjoint gradient (CPU only): a closed form on the one-node
mesh, the derivative of a linear map equals the map at the unit direction, Euler's
identity for a function homogeneous of degree 1, and central finite differences."""
import numpy as np
import pytest

import synth
from oracle import adjoint, fem


def test_single_interior_node_closed_form():
    # n = 3: one interior node at the centre, corner a = 7 - (index of the element among 8);
    # K11 = h/3 sum_e kappa_e (the unit-cube trilinear stiffness has diagonal 1/3), u = b/K11,
    # L = (u - u0)^2 / 2, dL/dkappa_e = -(u - u0) u h / (3 K11).
    n, h = 3, 0.5
    kappa = np.array([1.0, 2.0, 0.5, 3.0, 1.5, 0.25, 4.0, 1.0])
    m = np.log(kappa)
    b, u0 = np.array([0.7]), np.array([-0.2])
    K11 = h / 3 * kappa.sum()
    u = b[0] / K11
    g = adjoint.loss_and_grad(n, m, b, u0)
    assert g["u"][0] == pytest.approx(u, rel=1e-14)
    expect = -(u - u0[0]) * u * h / (3 * K11)
    assert np.allclose(g["dkappa"], expect, rtol=1e-13, atol=0)
    assert np.allclose(g["dm"], kappa * expect, rtol=1e-13, atol=0)
    assert g["db"][0] == pytest.approx((u - u0[0]) / K11, rel=1e-14)


def test_gradient_is_the_bilinear_form_at_unit_coefficients():
    # K is linear in kappa, so -d(lam^T K u)/dkappa_e = -lam^T K(unit_e) u, with K(unit_e)
    # assembled by the (independently pinned) element-scatter assembly.
    n = 6
    nd = (n - 2) ** 3
    u, lam = synth.normal(11, nd), synth.normal(12, nd)
    g = adjoint.coef_grad(n, u, lam)
    ne = (n - 1) ** 3
    for e in (0, 1, 7, 31, 62, ne - 1):
        unit = np.zeros(ne)
        unit[e] = 1.0
        assert g[e] == pytest.approx(-(lam @ (fem.assemble(n, unit) @ u)), rel=1e-12, abs=1e-15)


def test_euler_identity():
    # lam^T K(kappa) u is homogeneous of degree 1 in kappa: sum_e kappa_e dkappa_e = -lam^T K u.
    n = 9
    nd, ne = (n - 2) ** 3, (n - 1) ** 3
    kappa = np.exp(synth.normal(13, ne))
    u, lam = synth.normal(14, nd), synth.normal(15, nd)
    g = adjoint.coef_grad(n, u, lam)
    A = fem.assemble(n, kappa)
    assert kappa @ g == pytest.approx(-(lam @ (A @ u)), rel=1e-12)


def test_central_differences_in_m_and_b():
    n = 7
    nd, ne = (n - 2) ** 3, (n - 1) ** 3
    m = synth.gaussian_field(n, 6)
    b = fem.load_vector(n, synth.uniform(7, nd))
    u_obs = adjoint.loss_and_grad(n, synth.gaussian_field(n, 8), b, np.zeros(nd))["u"]
    g = adjoint.loss_and_grad(n, m, b, u_obs)
    eps = 1e-5
    for k in range(4):
        d = synth.normal(100 + k, ne)
        fd = (adjoint.loss(n, m + eps * d, b, u_obs) - adjoint.loss(n, m - eps * d, b, u_obs)) / (2 * eps)
        assert g["dm"] @ d == pytest.approx(fd, rel=1e-6)
    for e in (0, 40, ne - 1):
        d = np.zeros(ne)
        d[e] = 1.0
        fd = (adjoint.loss(n, m + eps * d, b, u_obs) - adjoint.loss(n, m - eps * d, b, u_obs)) / (2 * eps)
        assert g["dm"][e] == pytest.approx(fd, rel=1e-5, abs=1e-12 * abs(g["loss"]))
    db = synth.normal(200, nd) * np.abs(b).max()
    epsb = 1e-3
    fd = (adjoint.loss(n, m, b + epsb * db, u_obs) - adjoint.loss(n, m, b - epsb * db, u_obs)) / (2 * epsb)
    assert g["db"] @ db == pytest.approx(fd, rel=1e-8)       # L is quadratic in b: exact up to rounding
