"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
* deposit: bit-exact int64 grid, bit-exact FP64 density;
* FP64 solves at a fixed number of V-cycles: 1e-11 of max|u| (same iterates,
  only the rounding order differs);
* FP32-smoothing + FP64-refinement solves to rel. residual 1e-10: 1e-6 of
  max|Phi| (the stated bound of the path), v_c 1e-5;
* source: 1e-6 of max|src| (FP32 nu and fluxes from FP64 differences);
* forces, rotation curve, boundary fill from identical inputs: 1e-12.
"""
import numpy as np
import pytest
import torch

import synth
from tests import analytic as an
from tests.gpu_helpers import G, A0, gpu_pipeline, rel_max, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import paper_1201_3185_gb300 as q
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return q


def solve_given(q, n, L, f, bc, *, stats=True, **params):
    """Solve L u = f on one box with the caller's boundary values (C ABI)."""
    ctx = q.Context(n=n, nboxes=1, L0=L, bc_mode=q.QUMOND_BC_GIVEN, **params)
    u = to_dev(np.where(an.boundary_mask(n), bc, 0.0))
    st = None
    err = None
    try:
        st = ctx.qumond_solve_mond(0, to_dev(f), None, u, stats=stats)
    except q.NotConverged as e:
        err = e
    torch.cuda.synchronize()
    out = u.cpu().numpy()
    ctx.close()
    return out, st, err


# --- step 1: deposit ---------------------------------------------------------------
@pytest.mark.parametrize("n,L", [(8, 800.0), (64, 40000.0), (256, 120000.0)])
def test_deposit_bit_exact(q, ora, n, L):
    rng = np.random.default_rng(n)
    npart = 300_000
    x, y, z = (rng.random((3, npart)) - 0.5) * 1.05 * L  # some outside
    m = rng.random(npart) * 1e5
    h = L / n
    # edge cases: exactly on nodes, on the upper face, at the lower corner, NaN
    x[:5] = [-0.5 * L, 0.5 * L, -0.5 * L + 3 * h, np.nan, 0.0]
    y[:5] = [-0.5 * L, 0.0, -0.5 * L + 2 * h, 0.0, 0.5 * L - 1e-9 * h]
    z[:5] = [-0.5 * L, 0.0, 0.0, 0.0, 0.0]
    want, kept = ora.cic_deposit(n, L, (0.0, 0.0, 0.0), 24, x, y, z, m)
    ctx = q.Context(n=n, nboxes=1, L0=L)
    qf = torch.empty((n + 1) ** 3, dtype=torch.int64, device="cuda")
    rho = torch.empty((n + 1) ** 3, dtype=torch.float64, device="cuda")
    ctx.qumond_deposit(0, to_dev(x), to_dev(y), to_dev(z), to_dev(m), qf, rho)
    torch.cuda.synchronize()
    assert np.array_equal(qf.cpu().numpy(), want)
    assert np.array_equal(rho.cpu().numpy(), ora.rho_from_fixed(n, L, 24, want))
    ctx.close()


def test_deposit_empty_and_outside(q):
    n, L = 16, 1600.0
    ctx = q.Context(n=n, nboxes=1, L0=L)
    qf = torch.full(((n + 1) ** 3,), 7, dtype=torch.int64, device="cuda")
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    ctx.qumond_deposit(0, e, e, e, e, qf)
    assert int(qf.abs().sum()) == 0
    far = to_dev(np.full(10, 1e6))
    ctx.qumond_deposit(0, far, far, far, far, qf)
    assert int(qf.abs().sum()) == 0
    ctx.close()


# --- steps 2 and 4: the solver -------------------------------------------------------
@pytest.mark.parametrize("n", [2, 4, 16, 32, 64, 128])
def test_fp64_paper_mode_matches_oracle_fmg(q, ora, n):
    # six V-cycles per FMG level, no tolerance (Section 3.2's default)
    rng = np.random.default_rng(100 + n)
    L = 1000.0
    f = rng.standard_normal((n + 1) ** 3)
    bc = rng.standard_normal((n + 1) ** 3) * 50.0
    got, _, _ = solve_given(q, n, L, f, bc, precision=q.QUMOND_PREC_FP64, rel_tol=0.0)
    want = np.where(an.boundary_mask(n), bc, 0.0)
    ora.fmg(n, L / n, want, f, 6, 2, 2)
    assert rel_max(got, want) < 1e-11


@pytest.mark.parametrize("n,ncycle,npre,npost", [(64, 1, 1, 1), (64, 2, 2, 2), (128, 3, 1, 2)])
def test_fp64_fmg_variants_match_oracle(q, ora, n, ncycle, npre, npost):
    x, y, z = an.node_coords(n, 2.0)
    f = np.exp(-(x * x + 2 * y * y + 3 * z * z) / 0.1) * 100.0
    bc = 1.0 + x - 0.5 * y + z * z
    got, _, _ = solve_given(q, n, 2.0, f, bc, precision=q.QUMOND_PREC_FP64, ncycle=ncycle, npre=npre, npost=npost)
    want = np.where(an.boundary_mask(n), bc, 0.0)
    ora.fmg(n, 2.0 / n, want, f, ncycle, npre, npost)
    assert rel_max(got, want) < 1e-11


@pytest.mark.parametrize("n", [8, 64])
def test_fp64_extra_vcycles_match_oracle(q, ora, n):
    # the same number of V-cycles after FMG on both sides (tolerance never met)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((n + 1) ** 3)
    bc = rng.standard_normal((n + 1) ** 3)
    got, _, err = solve_given(q, n, 10.0, f, bc, precision=q.QUMOND_PREC_FP64, ncycle=1, rel_tol=1e-300,
                              max_vcycles=3, dc_vcycles=1)
    assert err is not None and err.status == 3  # NOT_CONVERGED, best iterate kept
    want = np.where(an.boundary_mask(n), bc, 0.0)
    made, _ = ora.solve(n, 10.0 / n, want, f, ncycle=1, tol=1e-300, max_vcycles=3)
    assert made == -1
    assert rel_max(got, want) < 1e-11


@pytest.mark.parametrize("n,prec", [(n, p) for n in (16, 64, 128) for p in (0, 1, 2)] + [(256, 1), (256, 2)])
def test_tolerance_mode_matches_oracle(q, ora, n, prec):
    # n = 256 runs the TMA-staged half-sweeps on the finest level and (prec 2)
    # the TMA-staged fixed-point update + residual
    x, y, z = an.node_coords(n, 4000.0)
    f = np.exp(-(x * x + y * y + 4 * z * z) / 2e5) * 0.05
    bc = -1000.0 / np.sqrt(x * x + y * y + z * z + 1e6)
    got, st, _ = solve_given(q, n, 4000.0, f, bc, precision=prec, rel_tol=1e-10, max_vcycles=40)
    assert st.converged and st.rel_residual <= 1e-10
    want = np.where(an.boundary_mask(n), bc, 0.0)
    ora.solve(n, 4000.0 / n, want, f, tol=1e-12, max_vcycles=60)
    assert rel_max(got, want) < (1e-9 if prec == 0 else 1e-6)
    # the reported residual is the true one
    r = ora.residual(n, 4000.0 / n, got, f)
    rel = np.sqrt(ora.interior_sumsq(n, r) / ora.interior_sumsq(n, f))
    # within 1% plus the FP64 floor: the fixed-point mode reports the exact
    # residual of its integer iterate; the oracle recomputes it in FP64 from
    # the FP64-rounded output.  Rounding the output (<= 2^-53 |u| per node)
    # moves the 7-point residual by <= 12 2^-53 |u| / h^2, and the FP64
    # evaluation of the stencil (7 roundings of sums of size up to 12 |u|)
    # adds <= 84 2^-53 |u| / h^2 per node; with |u| ~ 2.6e3 and h^2 ~ 244 at
    # n = 256 that floor (~1e-11 relative) is as large as the residual itself
    h2 = (4000.0 / n) ** 2
    inner = ~an.boundary_mask(n)
    floor = 96.0 * 2.0 ** -53 * np.sqrt(np.sum((got[inner] / h2) ** 2) / ora.interior_sumsq(n, f))
    assert abs(rel - st.rel_residual) <= 1e-2 * st.rel_residual + floor + 1e-14


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_vcycles_per_correction_step(q, ora, prec):
    # several V-cycles on the correction equation per defect-correction step
    # (dc_vcycles): the same tolerance is met with the same accuracy against
    # the oracle, the reported V-cycles are whole steps, and in FP64 (where a
    # V-cycle on the correction from zero is a V-cycle on u) the iterates are
    # those of as many plain V-cycles
    n = 64
    x, y, z = an.node_coords(n, 4000.0)
    f = np.exp(-(x * x + y * y + 4 * z * z) / 2e5) * 0.05
    bc = -1000.0 / np.sqrt(x * x + y * y + z * z + 1e6)
    want = np.where(an.boundary_mask(n), bc, 0.0)
    ora.solve(n, 4000.0 / n, want, f, tol=1e-12, max_vcycles=60)
    counts = {}
    for dc in (1, 2, 3, 4):
        got, st, _ = solve_given(q, n, 4000.0, f, bc, precision=prec, rel_tol=1e-10, max_vcycles=40, dc_vcycles=dc)
        assert st.converged and st.rel_residual <= 1e-10
        assert st.vcycles % dc == 0
        assert rel_max(got, want) < (1e-9 if prec == 0 else 1e-6)
        counts[dc] = st.vcycles
    # a step of dc V-cycles reduces the residual at least as much as dc steps of one
    assert all(counts[dc] <= counts[1] + dc - 1 for dc in counts)
    if prec == 0:
        rng = np.random.default_rng(8)
        fr = rng.standard_normal((n + 1) ** 3)
        br = rng.standard_normal((n + 1) ** 3)
        a, _, ea = solve_given(q, n, 10.0, fr, br, precision=0, ncycle=1, rel_tol=1e-300, max_vcycles=4, dc_vcycles=2)
        b, _, eb = solve_given(q, n, 10.0, fr, br, precision=0, ncycle=1, rel_tol=1e-300, max_vcycles=4, dc_vcycles=1)
        assert ea is not None and eb is not None  # the cap is reached: NOT_CONVERGED, best iterate kept
        assert rel_max(a, b) < 1e-11


def test_coarsest_grid_special_case(q):
    # Section 2: with zero boundary values the 3^3 centre potential is -h^2 f/6
    f = np.zeros(27)
    f[13] = 3.0
    got, _, _ = solve_given(q, 2, 8.0, f, np.zeros(27), precision=q.QUMOND_PREC_FP64)
    assert got[13] == pytest.approx(-16.0 * 3.0 / 6.0, rel=1e-15)


@pytest.mark.parametrize("prec", [1, 2])
def test_warm_start_from_solution_needs_no_vcycle(q, ora, prec):
    n = 32
    x, y, z = an.node_coords(n, 2.0)
    f = np.cos(3 * x) * np.sin(2 * y) * z
    bc = x * y
    want = np.where(an.boundary_mask(n), bc, 0.0)
    ora.solve(n, 2.0 / n, want, f, tol=1e-13, max_vcycles=60)
    # warm start: pass the converged solution's interior as the initial guess
    ctx = q.Context(n=n, nboxes=1, L0=2.0, bc_mode=q.QUMOND_BC_GIVEN, warm_start=1, rel_tol=1e-10,
                    max_vcycles=10, precision=prec)
    u = to_dev(want.copy())
    st = ctx.qumond_solve_mond(0, to_dev(f), None, u, stats=True)
    assert st.vcycles == 0 and st.rel_residual_fmg < 1e-10
    ctx.close()


# --- step 3: source --------------------------------------------------------------
def test_source_matches_oracle(q, ora):
    p = synth.two_component_disk(200_000, seed=4, rmax=27000.0, zmax=27000.0)
    n, L0 = 64, 60000.0
    boxes = ora.pipeline(p, n, L0, 1, tol=1e-11, max_vcycles=50)
    phiN = boxes[0].phiN
    ctx = q.Context(n=n, nboxes=1, L0=L0)
    src = torch.empty_like(to_dev(phiN))
    ctx.qumond_source(0, to_dev(phiN), src)
    got = src.cpu().numpy()
    assert rel_max(got, boxes[0].src) < 1e-6
    assert np.all(got[an.boundary_mask(n)] == 0.0)
    ctx.close()


def test_source_linear_and_plain_laplacian(q):
    n, L = 32, 3200.0
    x, y, z = an.node_coords(n, L)
    phi = 3.0 * x - 1.5 * y + 0.7 * z
    ctx = q.Context(n=n, nboxes=1, L0=L)
    src = torch.empty((n + 1) ** 3, dtype=torch.float64, device="cuda")
    ctx.qumond_source(0, to_dev(phi), src)
    assert float(src.abs().max()) < 1e-5 * 3.0 / (L / n)
    ctx.close()
    rng = np.random.default_rng(1)
    phi = rng.standard_normal((n + 1) ** 3)
    ctx = q.Context(n=n, nboxes=1, L0=L, a0=0.0)
    ctx.qumond_source(0, to_dev(phi), src)
    lap = an.laplacian7(phi, n, L / n)
    assert rel_max(src.cpu().numpy(), lap) < 1e-6
    ctx.close()


# --- nested boxes, forces and rotation curve -------------------------------------
@pytest.mark.parametrize("ratio", [2, 4])
def test_boundary_fill_matches_oracle(q, ora, ratio):
    n, L0 = 32, 32000.0
    rng = np.random.default_rng(ratio)
    parent = rng.standard_normal((n + 1) ** 3)
    ctx = q.Context(n=n, nboxes=2, L0=L0, box_ratio=ratio, precision=q.QUMOND_PREC_FP64)
    u = torch.zeros((n + 1) ** 3, dtype=torch.float64, device="cuda")
    ctx.qumond_solve_mond(1, to_dev(np.zeros((n + 1) ** 3)), to_dev(parent), u)
    got = u.cpu().numpy()
    want = np.zeros((n + 1) ** 3)
    ora.boundary_fill(n, L0, (0.0, 0.0, 0.0), parent, L0 / ratio, (0.0, 0.0, 0.0), want)
    bnd = an.boundary_mask(n)
    assert np.max(np.abs(got[bnd] - want[bnd])) < 1e-12
    ctx.close()


def test_forces_and_rotation_curve_match_oracle(q, ora):
    n, L0, nb = 64, 120000.0, 3
    p = synth.two_component_disk(100_000, seed=8, rmax=54000.0, zmax=54000.0)
    boxes = ora.pipeline(p, n, L0, nb, tol=1e-10, max_vcycles=40)
    phis = [b.phi for b in boxes]
    ctx = q.Context(n=n, nboxes=nb, L0=L0)
    dphis = [to_dev(a) for a in phis]
    qx, qy, qz = (to_dev(a) for a in (p.x, p.y, p.z))
    g = [torch.empty_like(qx) for _ in range(3)]
    ctx.qumond_forces(dphis, qx, qy, qz, *g)
    want = ora.forces(n, L0, (0.0, 0.0, 0.0), phis, p.x, p.y, p.z)
    scale = max(np.max(np.abs(w)) for w in want[:3])
    for a, b in zip(g, want[:3]):
        assert np.max(np.abs(a.cpu().numpy() - b)) < 1e-12 * scale
    r = torch.empty(50, dtype=torch.float64, device="cuda")
    vc = torch.empty(50, dtype=torch.float64, device="cuda")
    ctx.qumond_rotation_curve(dphis, 50, 30000.0, 64, r, vc)
    r_w, vc_w = ora.rotation_curve(n, L0, (0.0, 0.0, 0.0), phis, 50, 30000.0, 64)
    assert np.allclose(r.cpu().numpy(), r_w, rtol=0, atol=1e-9)
    assert np.max(np.abs(vc.cpu().numpy() / vc_w - 1.0)) < 1e-12
    ctx.close()


# --- the whole path --------------------------------------------------------------
def _compare_pipelines(gpu, boxes, n, L0, nbins, rmax, phi_tol, vc_tol, ratio=2, phiN_tol=None):
    phiN_tol = phi_tol if phiN_tol is None else phiN_tol
    for b, bx in enumerate(boxes):
        assert np.array_equal(gpu["rho_fixed"][b], bx.rho_fixed), "box %d deposit" % b
        assert rel_max(gpu["phiN"][b], bx.phiN) < phiN_tol, "box %d Phi_N" % b
        assert rel_max(gpu["phi"][b], bx.phi) < phi_tol, "box %d Phi" % b
    _, vc_w = __import__("oracle").rotation_curve(n, L0, (0.0, 0.0, 0.0), [b.phi for b in boxes], nbins, rmax,
                                                  ratio=ratio)
    assert np.max(np.abs(gpu["vc"] / vc_w - 1.0)) < vc_tol


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_kuzmin_check_config(q, ora, prec):
    # Kuzmin disk, M = 1e10, a = 2 kpc, 2e5 particles at z = 0; a 64^3 grid on
    # 40 kpc inside a 64^3 boundary box of 160 kpc; tolerance 1e-10; 50 bins
    M, a = 1e10, 2000.0
    p = synth.kuzmin_disk(200_000, M, a, seed=1)
    n, L0, nb, ratio = 64, 160000.0, 2, 4
    bcn = lambda x, y, z: an.kuzmin_phiN(x, y, z, M, a, G)
    bcm = lambda x, y, z: an.kuzmin_phi_mond(x, y, z, M, a, G, A0)
    gpu = gpu_pipeline(p, n, L0, nb, nbins=50, rmax=20000.0, box_ratio=ratio, rel_tol=1e-10, max_vcycles=40,
                       precision=prec, bc_newton=bcn, bc_mond=bcm)
    boxes = ora.pipeline(p, n, L0, nb, tol=1e-12, max_vcycles=60, bc_newton=bcn, bc_mond=bcm, ratio=ratio)
    _compare_pipelines(gpu, boxes, n, L0, 50, 20000.0, 1e-6, 1e-5, ratio=ratio)
    for st in gpu["newton_stats"] + gpu["mond_stats"]:
        assert st.converged and st.rel_residual <= 1e-10


def test_paper_mode_pipeline_fp64(q, ora):
    # the paper's defaults (6 V-cycles per level, zero outer boundary), 3 boxes
    p = synth.two_component_disk(100_000, seed=2, rmax=54000.0, zmax=54000.0)
    n, L0, nb = 64, 120000.0, 3
    gpu = gpu_pipeline(p, n, L0, nb, nbins=40, rmax=20000.0, precision=q.QUMOND_PREC_FP64, rel_tol=0.0)
    boxes = ora.pipeline(p, n, L0, nb)
    # Phi_N: identical iterates (FP64 FMG); Phi also carries the FP32 nu of the source
    _compare_pipelines(gpu, boxes, n, L0, 40, 20000.0, 1e-6, 1e-5, phiN_tol=1e-11)


def test_deterministic(q):
    p = synth.two_component_disk(50_000, seed=3, rmax=54000.0, zmax=54000.0)
    a = gpu_pipeline(p, 64, 120000.0, 2, rel_tol=1e-10, max_vcycles=40)
    b = gpu_pipeline(p, 64, 120000.0, 2, rel_tol=1e-10, max_vcycles=40)
    for key in ("phiN", "phi"):
        for x, y in zip(a[key], b[key]):
            assert np.array_equal(x, y)
    assert np.array_equal(a["vc"], b["vc"])


@pytest.mark.parametrize("prec", [1, 2])
def test_graph_and_one_by_one_launches_agree(q, prec):
    # each solve as one CUDA graph (device-side tolerance loop) or as kernels
    # launched one by one with host-side residual checks: the same kernels in
    # the same order, so the same bits
    p = synth.two_component_disk(50_000, seed=5, rmax=54000.0, zmax=54000.0)
    a = gpu_pipeline(p, 64, 120000.0, 3, rel_tol=1e-10, max_vcycles=40, use_graphs=1, precision=prec)
    b = gpu_pipeline(p, 64, 120000.0, 3, rel_tol=1e-10, max_vcycles=40, use_graphs=0, precision=prec)
    for key in ("phiN", "phi"):
        for x, y in zip(a[key], b[key]):
            assert np.array_equal(x, y)
    assert [s.vcycles for s in a["newton_stats"]] == [s.vcycles for s in b["newton_stats"]]
    assert np.array_equal(a["vc"], b["vc"])


@pytest.mark.parametrize("prec_name,graphs,form", [("MIXED_FIXED", 1, 1), ("MIXED_FIXED", 0, 1), ("FP64", 1, 1),
                                                    ("MIXED_FIXED", 1, 2), ("MIXED_FIXED", 0, 2), ("FP64", 1, 2),
                                                    ("MIXED", 1, 2)])
def test_cooperative_small_level_vcycle_gives_the_same_bits(q, prec_name, graphs, form):
    # the V-cycle on the levels n <= 64 below the finest as one cooperative
    # kernel with grid barriers (form 1) or one thread-block cluster with the
    # cluster's barrier (form 2), or one launch per step: the same node
    # arithmetic, so the same bits (n = 128: levels 64 and 32 above the coarse grid)
    prec = getattr(q, "QUMOND_PREC_" + prec_name)
    p = synth.two_component_disk(50_000, seed=12, rmax=54000.0, zmax=54000.0)
    a = gpu_pipeline(p, 128, 120000.0, 2, rel_tol=1e-10, max_vcycles=40, precision=prec, use_graphs=graphs,
                     persistent_vcycle=form)
    b = gpu_pipeline(p, 128, 120000.0, 2, rel_tol=1e-10, max_vcycles=40, precision=prec, use_graphs=graphs,
                     persistent_vcycle=0)
    for key in ("phiN", "phi"):
        for x, y in zip(a[key], b[key]):
            assert np.array_equal(x, y)
    assert [s.vcycles for s in a["mond_stats"]] == [s.vcycles for s in b["mond_stats"]]


@pytest.mark.parametrize("prec_name,graphs,cluster", [("MIXED_FIXED", 1, 0), ("MIXED_FIXED", 0, 8), ("MIXED", 1, 4),
                                                       ("MIXED_FIXED", 1, 16), ("MIXED", 0, 16)])
def test_shared_memory_small_vcycle_gives_the_same_bits(q, prec_name, graphs, cluster):
    # the level n = 32 and the levels under it in the distributed shared
    # memory of one thread-block cluster (form 3, 4 / 8 / 16 CTAs) or one
    # launch per step: the same node arithmetic, so the same bits; n = 64
    # (level 32 right under the finest) and n = 128 (level 64 between them)
    prec = getattr(q, "QUMOND_PREC_" + prec_name)
    p = synth.two_component_disk(50_000, seed=13, rmax=54000.0, zmax=54000.0)
    for n in (64, 128):
        kw = dict(rel_tol=1e-10, max_vcycles=40, precision=prec, use_graphs=graphs)
        a = gpu_pipeline(p, n, 120000.0, 2, persistent_vcycle=3, small_cluster=cluster, **kw)
        b = gpu_pipeline(p, n, 120000.0, 2, persistent_vcycle=0, **kw)
        for key in ("phiN", "phi"):
            for x, y in zip(a[key], b[key]):
                assert np.array_equal(x, y), (n, key)
        assert [s.vcycles for s in a["mond_stats"]] == [s.vcycles for s in b["mond_stats"]]


def test_shared_memory_small_vcycle_is_the_form_that_runs(q):
    # with form 3 every V-cycle below the finest level reaches the cluster
    # kernel (class vcycle_small_levels) and the coarse-grid kernel runs only
    # for FMG; form 3 on an FP64 context, or with the finest level at n = 32,
    # is the per-step form
    p = synth.two_component_disk(20_000, seed=14, rmax=54000.0, zmax=54000.0)
    x, y, z, m = (to_dev(a) for a in (p.x, p.y, p.z, p.m))
    for n, prec, expect in ((128, q.QUMOND_PREC_MIXED_FIXED, True), (64, q.QUMOND_PREC_MIXED, True),
                            (32, q.QUMOND_PREC_MIXED_FIXED, False), (128, q.QUMOND_PREC_FP64, False)):
        ctx = q.Context(n=n, nboxes=1, L0=120000.0, rel_tol=1e-10, max_vcycles=40, precision=prec,
                        use_graphs=0, persistent_vcycle=3)
        pipe = q.Pipeline(ctx)
        ctx.qumond_trace_read(reset=True)
        res = pipe.run(x, y, z, m, nbins=10, rmax=20000.0, stats=True)
        torch.cuda.synchronize()
        st, _, _ = ctx.qumond_trace_read()
        vc = res.newton_stats[0].vcycles + res.mond_stats[0].vcycles
        if expect:
            # FMG: ncycle V-cycles on each level above the coarse grid reach level 32 once each
            levels_above = n.bit_length() - 1 - 4
            assert st["vcycle_small_levels"].launches == vc + 2 * levels_above * ctx.params.ncycle, n
            assert st["coarse_solver"].launches == 2
        else:
            assert st["vcycle_small_levels"].launches == 0
        pipe.close()
        ctx.close()


def test_concurrent_chains_give_the_same_bits(q):
    # the QUMOND chain on its own context and stream, concurrent with the
    # Newtonian chain: the same kernels in the same order within each chain
    p = synth.two_component_disk(50_000, seed=9, rmax=54000.0, zmax=54000.0)
    kw = dict(n=64, nboxes=3, L0=120000.0, rel_tol=1e-10, max_vcycles=40, precision=q.QUMOND_PREC_MIXED_FIXED)
    x, y, z, m = (to_dev(a) for a in (p.x, p.y, p.z, p.m))
    c1 = q.Context(**kw)
    seq = q.Pipeline(c1)
    a = seq.run(x, y, z, m, nbins=30, rmax=20000.0, stats=True)
    ca, cb = q.Context(**kw), q.Context(**kw)
    con = q.Pipeline(ca, ctx_mond=cb)
    for _ in range(2):  # second pass relaunches the cached graphs
        b = con.run(x, y, z, m, nbins=30, rmax=20000.0, stats=True)
    torch.cuda.synchronize()
    for u, v in zip(seq.phiN + seq.phi, con.phiN + con.phi):
        assert torch.equal(u, v)
    assert torch.equal(a.vc, b.vc)
    assert [s.vcycles for s in a.mond_stats] == [s.vcycles for s in b.mond_stats]
    con.close()
    for c in (c1, ca, cb):
        c.close()


def test_graph_paper_mode_and_relaunch(q, ora):
    # paper mode (no residual checks) as a graph, launched twice on the same arrays
    p = synth.two_component_disk(50_000, seed=6, rmax=54000.0, zmax=54000.0)
    n, L0 = 32, 120000.0
    ctx = q.Context(n=n, nboxes=1, L0=L0, precision=q.QUMOND_PREC_FP64, rel_tol=0.0)
    pipe = q.Pipeline(ctx)
    x, y, z, m = (to_dev(a) for a in (p.x, p.y, p.z, p.m))
    for _ in range(2):
        pipe.potentials(x, y, z, m)
    torch.cuda.synchronize()
    boxes = ora.pipeline(p, n, L0, 1)
    assert rel_max(pipe.phiN[0].cpu().numpy(), boxes[0].phiN) < 1e-11
    ctx.close()


def test_invalid_arguments_rejected(q):
    with pytest.raises(q.QumondError):
        q.Context(n=48, nboxes=1, L0=1.0)
    with pytest.raises(q.QumondError):
        q.Context(n=64, nboxes=1, L0=1.0, npre=0)
    ctx = q.Context(n=8, nboxes=2, L0=100.0)
    # a host pointer handed to the C ABI is refused before any launch
    host = np.zeros(9 ** 3)
    st = q.qumond._lib.qumond_source(ctx._ptr, 0, host.ctypes.data_as(q.qumond._P),
                                     host.ctypes.data_as(q.qumond._P), None)
    assert st == q.qumond.QUMOND_ERR_INVALID_ARG
    dev = torch.zeros(9 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QumondError):  # box 1 without its parent
        ctx.qumond_solve_newton(1, dev, None, torch.zeros_like(dev))
    with pytest.raises(q.QumondError):  # box out of range
        ctx.qumond_source(2, dev, torch.zeros_like(dev))
    ctx.close()


@pytest.mark.parametrize("bc", ["zero", "multipole"])
def test_pipelined_evaluations_give_the_same_bits(q, bc):
    # run_many overlaps the Newtonian chain of evaluation i+1 with the QUMOND
    # chain, forces and curve of evaluation i, and run_lanes spreads the
    # evaluations over concurrent pipelines; every evaluation must give the
    # bits of a lone run()
    gals = [synth.two_component_disk(40_000, seed=40 + s, rmax=54000.0, zmax=54000.0) for s in range(2)]
    kw = dict(n=64, nboxes=3, L0=120000.0, rel_tol=1e-10, max_vcycles=40, precision=q.QUMOND_PREC_MIXED_FIXED,
              bc_mode=q.QUMOND_BC_MULTIPOLE if bc == "multipole" else q.QUMOND_BC_ZERO)
    dev = [tuple(to_dev(getattr(g, a)) for a in "xyzm") for g in gals]
    want = []
    for d in dev:
        ca, cb = q.Context(**kw), q.Context(**kw)
        pipe = q.Pipeline(ca, ctx_mond=cb)
        g = tuple(torch.empty_like(d[0]) for _ in range(3))
        r = pipe.run(*d, nbins=30, rmax=20000.0, forces=g)
        torch.cuda.synchronize()
        want.append((r.vc.clone(), [t.clone() for t in g], [t.clone() for t in pipe.phi]))
        pipe.close()
        ca.close()
        cb.close()
    ca, cb = q.Context(**kw), q.Context(**kw)
    pipe = q.Pipeline(ca, ctx_mond=cb)
    order = [0, 1, 1, 0, 1]
    inputs = [dev[k] for k in order]
    forces = [tuple(torch.empty_like(dev[k][0]) for _ in range(3)) for k in order]
    for _ in range(2):  # the second pass relaunches the cached graphs
        res = pipe.run_many(inputs, nbins=30, rmax=20000.0, forces=forces)
    torch.cuda.synchronize()
    for i, k in enumerate(order):
        assert torch.equal(res[i].vc, want[k][0]), i
        for a, b in zip(forces[i], want[k][1]):
            assert torch.equal(a, b), i
    for a, b in zip(pipe.phi, want[order[-1]][2]):  # the potentials of the last evaluation
        assert torch.equal(a, b)
    # the same evaluations over two lanes (two pipelines running concurrently), each evaluation's particles
    # copied in on another stream that its first kernel waits for
    cc, cd = q.Context(**kw), q.Context(**kw)
    pipe2 = q.Pipeline(cc, ctx_mond=cd)
    copies = [tuple(torch.empty_like(t) for t in dev[k]) for k in order]
    forces2 = [tuple(torch.empty_like(dev[k][0]) for _ in range(3)) for k in order]
    side = torch.cuda.Stream()
    for _ in range(2):
        ready = []
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for c, k in zip(copies, order):
                for a, b in zip(c, dev[k]):
                    a.copy_(b, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(side)
                ready.append(ev)
        res2 = q.run_lanes([pipe, pipe2], copies, nbins=30, rmax=20000.0, forces=forces2, ready=ready)
    torch.cuda.synchronize()
    for i, k in enumerate(order):
        assert res2[i].done is not None
        assert torch.equal(res2[i].vc, want[k][0]), i
        for a, b in zip(forces2[i], want[k][1]):
            assert torch.equal(a, b), i
    pipe2.close()
    cc.close()
    cd.close()
    pipe.close()
    ca.close()
    cb.close()
