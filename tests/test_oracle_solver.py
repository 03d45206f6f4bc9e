"""Pins of the oracle's multigrid solver (Section 2, steps 2 and 4)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from tests.analytic import boundary_mask, laplacian7, node_coords


def dirichlet_direct(n, h, f, bc):
    """Solve the 7-point Dirichlet problem with a sparse direct solver."""
    m = n - 1
    e = np.ones(m)
    T = sp.diags([e[:-1], -2 * e, e[:-1]], [-1, 0, 1])
    I = sp.identity(m)
    A = (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)) / (h * h)
    F = f.reshape(n + 1, n + 1, n + 1)[1:-1, 1:-1, 1:-1].ravel().copy()
    # move the boundary values to the right-hand side
    U0 = np.where(boundary_mask(n), bc, 0.0)
    F -= laplacian7(U0, n, h).reshape(n + 1, n + 1, n + 1)[1:-1, 1:-1, 1:-1].ravel()
    sol = spla.spsolve(A.tocsc(), F)
    out = U0.copy().reshape(n + 1, n + 1, n + 1)
    out[1:-1, 1:-1, 1:-1] = sol.reshape(m, m, m)
    return out.ravel()


def test_coarsest_grid_special_case(ora):
    # Section 2: on the 3x3x3 grid with zero boundary values the centre
    # potential is proportional to the centre density: u = -h^2 f / 6.
    u = np.zeros(27)
    f = np.zeros(27)
    f[13] = 2.5
    ora.coarsest(3.0, u, f)
    assert u[13] == pytest.approx(-9.0 * 2.5 / 6.0, rel=1e-15)
    u2 = np.zeros(27)
    ora.fmg(2, 3.0, u2, f, 6, 2, 2)
    assert u2[13] == pytest.approx(-9.0 * 2.5 / 6.0, rel=1e-15)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_matches_direct_sparse_solve(ora, n):
    rng = np.random.default_rng(n)
    h = 3.0
    f = rng.standard_normal((n + 1) ** 3)
    bc = rng.standard_normal((n + 1) ** 3) * 10.0
    u = np.where(boundary_mask(n), bc, 0.0)
    made, hist = ora.solve(n, h, u, f, tol=1e-13, max_vcycles=60)
    assert made >= 0
    want = dirichlet_direct(n, h, f, bc)
    assert np.max(np.abs(u - want)) <= 1e-11 * np.max(np.abs(want))


def test_quadratic_is_exact(ora):
    # the 7-point stencil is exact for quadratics, so the discrete solution is
    # the quadratic itself
    n, L = 32, 320.0
    h = L / n
    x, y, z = node_coords(n, L, (5.0, -3.0, 2.0))
    q = 0.3 * x * x - 0.1 * y * y + 0.05 * z * z + 0.02 * x * y - 0.07 * y * z + 0.4 * x - 2.0
    f = np.full_like(q, 2.0 * (0.3 - 0.1 + 0.05))
    u = np.where(boundary_mask(n), q, 0.0)
    made, _ = ora.solve(n, h, u, f, tol=1e-13, max_vcycles=60)
    assert made >= 0
    assert np.max(np.abs(u - q)) <= 1e-10 * np.max(np.abs(q))


def gaussian_problem(n, L=2.0, s=0.25):
    x, y, z = node_coords(n, L)
    r2 = x * x + y * y + z * z
    g = np.exp(-r2 / (2 * s * s))
    lap = g * (r2 / s ** 4 - 3.0 / s ** 2)
    return g, lap


def test_gaussian_second_order(ora):
    errs = []
    for n in (16, 32, 64):
        g, lap = gaussian_problem(n)
        u = np.where(boundary_mask(n), g, 0.0)
        ora.solve(n, 2.0 / n, u, lap, tol=1e-12, max_vcycles=60)
        errs.append(np.max(np.abs(u - g)))
    assert 3.5 < errs[0] / errs[1] < 4.5
    assert 3.7 < errs[1] / errs[2] < 4.3


def test_fmg_reaches_discretisation_error(ora):
    # the defining property of full multigrid: a fixed number of V-cycles per
    # level leaves an algebraic error bounded by a constant (independent of h)
    # times the discretisation error
    for n in (32, 64):
        g, lap = gaussian_problem(n)
        u_ex = np.where(boundary_mask(n), g, 0.0)
        ora.solve(n, 2.0 / n, u_ex, lap, tol=1e-13, max_vcycles=60)
        disc = np.max(np.abs(u_ex - g))
        u1 = np.where(boundary_mask(n), g, 0.0)
        ora.fmg(n, 2.0 / n, u1, lap, 1, 2, 2)
        assert np.max(np.abs(u1 - g)) < disc  # total error within the discretisation error
        u2 = np.where(boundary_mask(n), g, 0.0)
        ora.fmg(n, 2.0 / n, u2, lap, 2, 2, 2)
        assert np.max(np.abs(u2 - u_ex)) < 0.15 * disc


def test_vcycle_convergence_factor(ora):
    rng = np.random.default_rng(3)
    n = 32
    f = rng.standard_normal((n + 1) ** 3)
    u = np.zeros_like(f)
    hist = []
    for _ in range(6):
        ora.vcycle(n, 1.0, u, f, 2, 2)
        r = ora.residual(n, 1.0, u, f)
        hist.append(np.linalg.norm(r))
    factors = np.array(hist[1:]) / np.array(hist[:-1])
    assert np.all(factors < 0.15), factors


def test_rbgs_zeroes_black_residual(ora):
    # after a sweep the black nodes (updated last) satisfy their equation
    rng = np.random.default_rng(4)
    n = 8
    f = rng.standard_normal((n + 1) ** 3)
    u = rng.standard_normal((n + 1) ** 3)
    ora.relax_rbgs(n, 0.5, u, f)
    r = ora.residual(n, 0.5, u, f).reshape(n + 1, n + 1, n + 1)
    k, j, i = np.meshgrid(*(np.arange(n + 1),) * 3, indexing="ij")
    interior = (i > 0) & (i < n) & (j > 0) & (j < n) & (k > 0) & (k < n)
    black = interior & ((i + j + k) % 2 == 1)
    red = interior & ((i + j + k) % 2 == 0)
    assert np.max(np.abs(r[black])) < 1e-12 * np.max(np.abs(r[red]))


def test_restriction_prolongation_adjoint_and_exactness(ora):
    rng = np.random.default_rng(6)
    nc = 8
    nf = 2 * nc
    a = rng.standard_normal((nf + 1) ** 3) * (~boundary_mask(nf))
    b = rng.standard_normal((nc + 1) ** 3) * (~boundary_mask(nc))
    Ra = ora.restrict_fw(nf, a)
    Pb = np.zeros((nf + 1) ** 3)
    ora.prolong(nc, b, Pb, False)
    # full weighting is 1/8 of the transpose of trilinear prolongation
    assert np.dot(Ra, b) == pytest.approx(np.dot(a, Pb) / 8.0, rel=1e-12)
    # prolongation reproduces trilinear functions; restriction reproduces linear ones
    X, Y, Z = node_coords(nc, 2.0)
    tri = 1.0 + 0.5 * X - 0.3 * Y + 0.2 * Z + 0.1 * X * Y * Z - 0.4 * X * Z
    P = np.zeros((nf + 1) ** 3)
    ora.prolong(nc, tri, P, False)
    Xf, Yf, Zf = node_coords(nf, 2.0)
    trif = 1.0 + 0.5 * Xf - 0.3 * Yf + 0.2 * Zf + 0.1 * Xf * Yf * Zf - 0.4 * Xf * Zf
    inner = ~boundary_mask(nf)
    assert np.max(np.abs(P[inner] - trif[inner])) < 1e-14
    lin_f = 2.0 + Xf - 3.0 * Yf + 0.5 * Zf
    lin_c = 2.0 + X - 3.0 * Y + 0.5 * Z
    R = ora.restrict_fw(nf, lin_f)
    innc = ~boundary_mask(nc)
    assert np.max(np.abs(R[innc] - lin_c[innc])) < 1e-14


def test_paper_mode_six_vcycles_converged(ora):
    # Section 3.2: six V-cycles per level leave the rotation speed within 0.1%
    # of the 99-V-cycle result; fewer cycles are further away.
    import synth
    p = synth.two_component_disk(40000, seed=11, rmax=0.45 * 64000.0, zmax=0.45 * 64000.0)
    n, L0, nb = 32, 64000.0, 2
    curves = {}
    for nc in (1, 6, 99):
        boxes = ora.pipeline(p, n, L0, nb, ncycle=nc)
        _, vc = ora.rotation_curve(n, L0, (0.0, 0.0, 0.0), [b.phi for b in boxes], 20, 12000.0)
        curves[nc] = vc
    err6 = np.max(np.abs(curves[6] / curves[99] - 1.0))
    err1 = np.max(np.abs(curves[1] / curves[99] - 1.0))
    assert err6 < 1e-3
    assert err1 > err6
