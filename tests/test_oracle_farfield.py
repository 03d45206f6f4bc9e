"""Pins of the oracle's far-field boundary values (ora_far_field), the
outermost box's boundary from the mass inside it:

* a single mass at the box centre: Phi_N = -G M / r exactly and Phi = the
  closed-form point-mass QUMOND potential F(r) (tests/analytic.py, the
  Kuzmin potential with a = 0);
* a cluster of node masses: the expansion equals the truncated Legendre
  series of its definition, summed directly over the masses with scipy's
  Legendre polynomials (a library routine), to rounding, for every degree;
  and the exact potential (direct sum of -G m/|x - x_k|) within the
  truncation error, which falls with the degree as (d/r)^(lmax+1);
* the centre of mass is the expansion point: the dipole term vanishes;
* zero mass gives zero.
"""
import numpy as np
import pytest
from scipy.special import eval_legendre

from tests import analytic as an

G, A0 = 4.30e-3, 3.6


def boundary(n):
    return an.boundary_mask(n)


def test_point_mass_at_centre(ora):
    n, L = 16, 16000.0
    rho = np.zeros((n + 1) ** 3)
    h = L / n
    M = 3e10
    c = n // 2
    rho[c + (n + 1) * (c + (n + 1) * c)] = M / h ** 3
    phiN, phi, Mtot = ora.far_field(n, L, (0.0, 0.0, 0.0), rho, G=G, a0=A0, lmax=8)
    assert Mtot == pytest.approx(M, rel=1e-15)
    x, y, z = an.node_coords(n, L)
    b = boundary(n)
    r = np.sqrt(x * x + y * y + z * z)
    np.testing.assert_allclose(phiN[b], -G * M / r[b], rtol=1e-13)
    np.testing.assert_allclose(phi[b], an.kuzmin_phi_mond(x[b], y[b], z[b], M, 0.0, G, A0), rtol=1e-12)
    assert np.all(phiN[~b] == 0.0) and np.all(phi[~b] == 0.0)


def _cluster(n, L, seed, shift=(0, 0, 0)):
    """A few node masses within a small cube near the centre (node indices shifted by `shift`)."""
    rng = np.random.default_rng(seed)
    rho = np.zeros((n + 1) ** 3)
    c = n // 2
    idx = []
    for _ in range(12):
        i, j, k = (c + rng.integers(-2, 3, 3) + np.array(shift))
        idx.append((i, j, k))
        rho[i + (n + 1) * (j + (n + 1) * k)] += rng.random() * 1e7
    return rho


def _legendre_direct(n, L, rho, lmax):
    """The truncated series of the definition, summed mass by mass."""
    h = L / n
    x, y, z = an.node_coords(n, L)
    m = rho * h ** 3
    sel = m != 0.0
    M = m.sum()
    com = np.array([(m * x).sum(), (m * y).sum(), (m * z).sum()]) / M
    src = np.stack([x[sel], y[sel], z[sel]], axis=1) - com
    ms = m[sel]
    b = boundary(n)
    obs = np.stack([x[b], y[b], z[b]], axis=1) - com
    r = np.linalg.norm(obs, axis=1)
    rs = np.linalg.norm(src, axis=1)
    cosg = (obs @ src.T) / np.outer(r, rs)
    series = np.zeros(len(r))
    exact = -G * np.sum(ms[None, :] / np.linalg.norm(obs[:, None, :] - src[None, :, :], axis=2), axis=1)
    for l in range(lmax + 1):
        series += np.sum(ms[None, :] * (rs[None, :] ** l) * eval_legendre(l, cosg), axis=1) / r ** (l + 1)
    return -G * series, exact, r, np.max(rs)


@pytest.mark.parametrize("lmax", [0, 1, 2, 5, 8])
def test_cluster_equals_truncated_legendre_series(ora, lmax):
    n, L = 16, 16000.0
    rho = _cluster(n, L, seed=3)
    phiN, _, _ = ora.far_field(n, L, (0.0, 0.0, 0.0), rho, G=G, a0=A0, lmax=lmax)
    want, _, _, _ = _legendre_direct(n, L, rho, lmax)
    b = boundary(n)
    np.testing.assert_allclose(phiN[b], want, rtol=1e-12)


def test_cluster_converges_to_the_exact_potential(ora):
    n, L = 16, 16000.0
    rho = _cluster(n, L, seed=4)
    b = boundary(n)
    errs = []
    for lmax in (2, 4, 8):
        phiN, _, _ = ora.far_field(n, L, (0.0, 0.0, 0.0), rho, G=G, a0=A0, lmax=lmax)
        _, exact, r, dmax = _legendre_direct(n, L, rho, lmax)
        err = np.abs(phiN[b] - exact) / np.abs(exact)
        # remainder of the Legendre series: <= (d/r)^(lmax+1) / (1 - d/r) per mass
        q = dmax / r
        assert np.all(err <= q ** (lmax + 1) / (1.0 - q) + 1e-14)
        errs.append(err.max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4  # (d/r)^9 with d/r <= 0.44 here


def test_expansion_point_is_the_centre_of_mass(ora):
    # about the centre of mass the dipole moment vanishes: degree 1 adds nothing to degree 0, while the
    # quadrupole term (degree 2) does change the values
    n, L = 32, 32000.0
    rho = _cluster(n, L, seed=5, shift=(3, -2, 1))
    b = boundary(n)
    p0, _, _ = ora.far_field(n, L, (0.0, 0.0, 0.0), rho, G=G, a0=A0, lmax=0)
    p1, _, _ = ora.far_field(n, L, (0.0, 0.0, 0.0), rho, G=G, a0=A0, lmax=1)
    p2, _, _ = ora.far_field(n, L, (0.0, 0.0, 0.0), rho, G=G, a0=A0, lmax=2)
    assert np.max(np.abs(p1[b] - p0[b]) / np.abs(p0[b])) < 1e-13
    assert np.max(np.abs(p2[b] - p0[b]) / np.abs(p0[b])) > 1e-6


def test_zero_mass(ora):
    n = 8
    phiN, phi, M = ora.far_field(n, 100.0, (0.0, 0.0, 0.0), np.zeros((n + 1) ** 3))
    assert M == 0.0 and np.all(phiN == 0.0) and np.all(phi == 0.0)
