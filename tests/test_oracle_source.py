"""Pins of the oracle's QUMOND source (Section 2 step 3, Eq. 2)."""
import numpy as np
import pytest
import sympy

from tests.analytic import boundary_mask, laplacian7, node_coords

A0 = 3.6


def test_linear_potential_has_zero_source(ora):
    n, L = 16, 1600.0
    x, y, z = node_coords(n, L)
    phi = 3.0 * x - 1.5 * y + 0.7 * z + 100.0
    src = ora.source(n, L / n, A0, phi)
    # constant gradient: every face carries the same nu, fluxes cancel pairwise
    assert np.max(np.abs(src)) < 1e-12 * 3.0 / (L / n)


def test_zero_a0_is_the_plain_laplacian(ora):
    rng = np.random.default_rng(2)
    n = 12
    phi = rng.standard_normal((n + 1) ** 3)
    src = ora.source(n, 2.0, 0.0, phi)
    lap = laplacian7(phi, n, 2.0)
    assert np.max(np.abs(src - lap)) < 1e-13 * np.max(np.abs(lap))
    assert np.all(src[boundary_mask(n)] == 0.0)


def _plummer_source():
    r, GM, b, a0 = sympy.symbols("r GM b a0", positive=True)
    dphi = GM * r / (r ** 2 + b ** 2) ** sympy.Rational(3, 2)  # dPhi_N/dr
    nu = sympy.Rational(1, 2) + sympy.Rational(1, 2) * sympy.sqrt(1 + 4 * a0 / dphi)
    s = sympy.diff(r ** 2 * nu * dphi, r) / r ** 2
    return sympy.lambdify((r, GM, b, a0), s, "numpy")


def test_spherical_source_second_order(ora):
    # Plummer potential Phi_N = -GM/sqrt(r^2+b^2): the exact QUMOND source is
    # r^-2 d/dr [r^2 nu(Phi_N'/a0) Phi_N'] (computed symbolically here)
    exact = _plummer_source()
    GM, b, L = 4.3e-3 * 1e10, 2000.0, 32000.0
    errs = []
    for n in (32, 64):
        x, y, z = node_coords(n, L)
        r = np.sqrt(x * x + y * y + z * z)
        phi = -GM / np.sqrt(r * r + b * b)
        src = ora.source(n, L / n, A0, phi)
        sel = (~boundary_mask(n)) & (r > 1500.0) & (r < 9000.0)
        want = exact(r[sel], GM, b, A0)
        errs.append(np.max(np.abs(src[sel] - want)) / np.max(np.abs(want)))
    assert errs[1] < 0.01
    assert 3.0 < errs[0] / errs[1] < 5.0
