"""Pins of the oracle's nested-box boundary fill, forces and rotation curve."""
import numpy as np
import pytest

from tests.analytic import boundary_mask, node_coords


def test_boundary_fill_reproduces_trilinear_parent(ora):
    n, Lp, c = 16, 3200.0, (100.0, -50.0, 25.0)
    X, Y, Z = node_coords(n, Lp, c)
    field = lambda x, y, z: 2.0 + 0.01 * x - 0.02 * y + 0.005 * z + 1e-6 * x * y * z - 3e-5 * x * z
    up = field(X, Y, Z)
    u = np.zeros((n + 1) ** 3)
    ora.boundary_fill(n, Lp, c, up, Lp / 2, c, u)
    x, y, z = node_coords(n, Lp / 2, c)
    bnd = boundary_mask(n)
    assert np.max(np.abs(u[bnd] - field(x, y, z)[bnd])) < 1e-12
    assert np.all(u[~bnd] == 0.0)


def test_forces_exact_for_quadratic_potential(ora):
    n, L0, nb, c = 16, 16000.0, 3, (0.0, 0.0, 0.0)
    quad = lambda x, y, z: 1e-4 * x * x + 3e-5 * y * y - 2e-5 * z * z + 1e-5 * x * y + 0.2 * z
    grad = lambda x, y, z: (2e-4 * x + 1e-5 * y, 6e-5 * y + 1e-5 * x, -4e-5 * z + 0.2)
    phis = [quad(*node_coords(n, L0 / 2 ** b, c)) for b in range(nb)]
    rng = np.random.default_rng(1)
    q = (rng.random((3, 500)) - 0.5) * 0.8 * L0
    gx, gy, gz, missed = ora.forces(n, L0, c, phis, *q)
    assert missed == 0
    wx, wy, wz = grad(*q)
    assert np.max(np.abs(gx + wx)) < 1e-10 and np.max(np.abs(gy + wy)) < 1e-10 and np.max(np.abs(gz + wz)) < 1e-10
    # a point outside every interior cell gets no force
    gx, gy, gz, missed = ora.forces(n, L0, c, phis, [0.49 * L0], [0.0], [0.0])
    assert missed == 1 and gx[0] == 0.0


def test_rotation_curve_of_harmonic_potential(ora):
    # Phi = Omega^2 R^2 / 2 gives v_c = Omega R exactly (Eq. 4)
    n, L0, nb, c = 32, 64000.0, 3, (0.0, 0.0, 0.0)
    om = 0.01
    phis = [0.5 * om * om * (x * x + y * y) + 1e-6 * z * z
            for x, y, z in (node_coords(n, L0 / 2 ** b, c) for b in range(nb))]
    r, vc = ora.rotation_curve(n, L0, c, phis, 40, 20000.0, 64)
    assert np.allclose(r, (np.arange(40) + 0.5) * 500.0)
    assert np.max(np.abs(vc - om * r)) < 1e-9 * np.max(vc)


def test_chi2_definition(ora):
    # Section 3.5: chi^2/n; zero for a perfect fit, 1 when every point is off by one sigma
    v_obs = np.array([100.0, 120.0, 130.0, 135.0])
    sigma = 0.03 * v_obs
    vc = np.stack([v_obs, v_obs + sigma, v_obs - 2.0 * sigma])
    got = ora.chi2(vc, v_obs, sigma)
    assert got[0] == 0.0
    assert got[1] == pytest.approx(1.0, rel=1e-14)
    assert got[2] == pytest.approx(4.0, rel=1e-14)


def test_algebraic_curve_of_harmonic_potential(ora):
    # Eq. 3 on Phi_N = Omega^2 R^2 / 2: |g_N| = Omega^2 R in the plane, so
    # v_c^2 = R nu(Omega^2 R / a0) Omega^2 R exactly (the gradient is exact on a quadratic)
    n, L0, nb, c, a0 = 32, 64000.0, 3, (0.0, 0.0, 0.0), 3.6
    om = 0.01
    phis = [0.5 * om * om * (x * x + y * y) + 1e-6 * z * z
            for x, y, z in (node_coords(n, L0 / 2 ** b, c) for b in range(nb))]
    r, vc = ora.rotation_curve_algebraic(n, L0, c, phis, 40, 20000.0, 64, a0=a0)
    g = om * om * r
    nu = 0.5 + 0.5 * np.sqrt(1.0 + 4.0 * a0 / g)
    np.testing.assert_allclose(vc, np.sqrt(r * nu * g), rtol=1e-9)
    # a0 -> 0 is Newtonian: the plain rotation curve
    _, vN = ora.rotation_curve_algebraic(n, L0, c, phis, 40, 20000.0, 64, a0=0.0)
    np.testing.assert_allclose(vN, om * r, rtol=1e-9)


def test_sigma_z_of_vertical_harmonic_potential(ora):
    # Section 5.6: sigma_z^2 = -dPhi/dz rho/(d rho/dz); for Phi = k^2 z^2 / 2 and a
    # sech^2(z/h) layer at height z: sigma_z^2 = k^2 z h / (2 tanh(z/h))
    n, L0, nb, c = 32, 64000.0, 3, (0.0, 0.0, 0.0)
    k2 = 2e-3
    phis = [0.5 * k2 * z * z + 3e-5 * (x * x + y * y)
            for x, y, z in (node_coords(n, L0 / 2 ** b, c) for b in range(nb))]
    for z_eval, h in ((300.0, 300.0), (450.0, 600.0)):
        r, sg = ora.sigma_z(n, L0, c, phis, 30, 15000.0, z_eval, h, 64)
        want = np.sqrt(k2 * z_eval * h / (2.0 * np.tanh(z_eval / h)))
        np.testing.assert_allclose(sg, want, rtol=1e-9)
