"""Pins of the oracle's fixed-point CIC deposit (Section 2, step 1)."""
import numpy as np
import pytest

from tests.analytic import node_coords

SHIFT = 24


def dep(ora, n, L, x, y, z, m, center=(0.0, 0.0, 0.0)):
    q, kept = ora.cic_deposit(n, L, center, SHIFT, np.atleast_1d(x), np.atleast_1d(y), np.atleast_1d(z),
                              np.atleast_1d(m))
    return q, kept


def test_particle_on_a_node_deposits_only_there(ora):
    n, L = 8, 800.0  # h = 100
    q, kept = dep(ora, n, L, -300.0, 100.0, 0.0, 1000.0)
    assert kept == 1
    nz = np.flatnonzero(q)
    assert nz.tolist() == [1 + 9 * (5 + 9 * 4)]  # node (1, 5, 4)
    assert q[nz[0]] == 1000 * 2 ** SHIFT


def test_cell_centre_gives_eight_equal_shares(ora):
    n, L = 8, 800.0
    q, _ = dep(ora, n, L, -350.0, 150.0, 50.0, 8.0)
    nz = np.flatnonzero(q)
    assert len(nz) == 8
    assert np.all(q[nz] == 2 ** SHIFT)  # 8 Msun / 8 corners


def test_hand_computed_weights(ora):
    # offset inside cell (2,3,4) is (0.25, 0.5, 0.75); mass 64 Msun
    n, L = 8, 800.0
    h = 100.0
    x, y, z = -400.0 + 2.25 * h, -400.0 + 3.5 * h, -400.0 + 4.75 * h
    q, _ = dep(ora, n, L, x, y, z, 64.0)
    Q = q.reshape(9, 9, 9)
    wx, wy, wz = [0.75, 0.25], [0.5, 0.5], [0.25, 0.75]
    for c in range(2):
        for b in range(2):
            for a in range(2):
                want = 64.0 * wx[a] * wy[b] * wz[c] * 2 ** SHIFT
                assert Q[4 + c, 3 + b, 2 + a] == want
    assert Q.sum() == 64 * 2 ** SHIFT


def test_half_open_box_and_nan(ora):
    n, L = 4, 400.0
    q, kept = dep(ora, n, L, [200.0, -200.0, np.nan, 0.0], [0.0, 0.0, 0.0, 200.0], [0.0] * 4, [1.0] * 4)
    # x = +L/2 is outside (half open), x = -L/2 inside, NaN dropped, y = +L/2 outside
    assert kept == 1
    assert q.sum() == 2 ** SHIFT


def test_mass_and_first_moment_conservation(ora):
    rng = np.random.default_rng(5)
    n, L = 16, 1600.0
    npart = 5000
    x, y, z = (rng.random((3, npart)) - 0.5) * 1500.0
    m = rng.random(npart) * 3.0 + 0.5
    q, kept = dep(ora, n, L, x, y, z, m)
    assert kept == npart
    total = float(q.sum())
    want = float(np.sum(m)) * 2 ** SHIFT
    assert abs(total - want) <= 4.0 * npart  # at most 1/2 per corner from rounding
    # CIC preserves the first moment exactly (up to the same rounding)
    xs, ys, zs = node_coords(n, L)
    for coord, pos in ((xs, x), (ys, y), (zs, z)):
        mom = float(np.sum(q.astype(np.float64) * coord))
        want_m = float(np.sum(m * pos)) * 2 ** SHIFT
        assert abs(mom - want_m) <= 4.0 * npart * L + 1e-9 * abs(want_m)


def test_order_independence(ora):
    rng = np.random.default_rng(9)
    n, L = 16, 1600.0
    x, y, z = (rng.random((3, 2000)) - 0.5) * 1600.0
    m = rng.random(2000)
    q1, _ = dep(ora, n, L, x, y, z, m)
    perm = rng.permutation(2000)
    q2, _ = dep(ora, n, L, x[perm], y[perm], z[perm], m[perm])
    assert np.array_equal(q1, q2)


def test_empty_particle_set(ora):
    q, kept = dep(ora, 8, 100.0, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    assert kept == 0 and not q.any()


def test_rho_scaling(ora):
    n, L = 8, 800.0
    q, _ = dep(ora, n, L, -300.0, 100.0, 0.0, 1000.0)
    rho = ora.rho_from_fixed(n, L, SHIFT, q)
    assert rho.max() == pytest.approx(1000.0 / 100.0 ** 3, rel=1e-15)
