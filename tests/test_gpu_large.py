"""The large-grid workload at full size: 512^3 intervals (513^3 nodes), 4 nested
boxes of 240/120/60/30 kpc, 2e7 particles (two disks + Hernquist bulge), in the
configuration `bench.py --workload large` times.

The oracle cannot solve four 513^3 boxes in test time, so each step is checked
on the GPU's own inputs, with checks that hold at any size:
* deposit: bit-exact against the oracle for every box;
* solves: the oracle's residual of the GPU's final potential meets the tolerance;
* source: the oracle's source of the GPU's Phi_N, 1e-6 of max;
* nested boundaries: the oracle's interpolation of the GPU's parent potential;
* rotation curve and forces at sampled particles: the oracle's, from the GPU's potentials.
"""
import numpy as np
import pytest
import torch

import synth
from tests.gpu_helpers import rel_max, to_dev
from tests.analytic import boundary_mask

pytestmark = pytest.mark.gpu

N, NB, L0, NP = 512, 4, 240000.0, 20_000_000


@pytest.fixture(scope="module")
def run():
    import paper_1201_3185_gb300 as q
    p = synth.large_galaxy(NP, seed=1, rmax=0.45 * L0)
    ctx = q.Context(n=N, nboxes=NB, L0=L0, rel_tol=1e-10, max_vcycles=40, ncycle=1,
                    precision=q.QUMOND_PREC_MIXED_FIXED)
    pipe = q.Pipeline(ctx)
    x, y, z, m = (to_dev(a) for a in (p.x, p.y, p.z, p.m))
    out = {"rho_fixed": [], "rho": [], "src": [], "stats": []}
    for b in range(NB):
        ctx.qumond_deposit(b, x, y, z, m, pipe.rho_fixed, pipe.rho)
        out["rho_fixed"].append(pipe.rho_fixed.cpu().numpy())
        out["rho"].append(pipe.rho.cpu().numpy())
        out["stats"].append(ctx.qumond_solve_newton(b, pipe.rho, pipe.phiN[b - 1] if b else None, pipe.phiN[b],
                                                   stats=True))
        ctx.qumond_source(b, pipe.phiN[b], pipe.src)
        out["src"].append(pipe.src.cpu().numpy())
        out["stats"].append(ctx.qumond_solve_mond(b, pipe.src, pipe.phi[b - 1] if b else None, pipe.phi[b],
                                                 stats=True))
    r = torch.empty(50, dtype=torch.float64, device="cuda")
    vc = torch.empty(50, dtype=torch.float64, device="cuda")
    ctx.qumond_rotation_curve(pipe.phi, 50, 30000.0, 64, r, vc)
    sel = np.random.default_rng(0).choice(NP, 20000, replace=False)
    qx, qy, qz = (to_dev(a[sel]) for a in (p.x, p.y, p.z))
    g = [torch.empty_like(qx) for _ in range(3)]
    ctx.qumond_forces(pipe.phi, qx, qy, qz, *g)
    torch.cuda.synchronize()
    out.update(p=p, sel=sel, phiN=[t.cpu().numpy() for t in pipe.phiN], phi=[t.cpu().numpy() for t in pipe.phi],
               vc=vc.cpu().numpy(), g=[t.cpu().numpy() for t in g])
    ctx.close()
    return out


def test_large_deposit_bit_exact(run, ora):
    p = run["p"]
    for b in range(NB):
        q, _ = ora.cic_deposit(N, L0 / 2 ** b, (0.0, 0.0, 0.0), 24, p.x, p.y, p.z, p.m)
        assert np.array_equal(run["rho_fixed"][b], q)


def test_large_solves_meet_tolerance(run, ora):
    assert all(s.converged and s.rel_residual <= 1e-10 for s in run["stats"])
    for b in (0, NB - 1):
        h = L0 / 2 ** b / N
        f = 4.0 * np.pi * 4.30e-3 * run["rho"][b]
        r = ora.residual(N, h, run["phiN"][b], f)
        assert np.sqrt(ora.interior_sumsq(N, r) / ora.interior_sumsq(N, f)) <= 1.05e-10
        r = ora.residual(N, h, run["phi"][b], run["src"][b])
        assert np.sqrt(ora.interior_sumsq(N, r) / ora.interior_sumsq(N, run["src"][b])) <= 1.05e-10


def test_large_source_and_boundaries(run, ora):
    for b in (0, NB - 1):
        want = ora.source(N, L0 / 2 ** b / N, 3.6, run["phiN"][b])
        assert rel_max(run["src"][b], want) < 1e-6
    bnd = boundary_mask(N)
    for b in range(1, NB):
        for key in ("phiN", "phi"):
            want = np.zeros((N + 1) ** 3)
            ora.boundary_fill(N, L0 / 2 ** (b - 1), (0.0, 0.0, 0.0), run[key][b - 1], L0 / 2 ** b, (0.0, 0.0, 0.0), want)
            assert np.max(np.abs(run[key][b][bnd] - want[bnd])) <= 1e-12 * np.max(np.abs(want[bnd]))


def test_large_rotation_curve_and_forces(run, ora):
    _, vc = ora.rotation_curve(N, L0, (0.0, 0.0, 0.0), run["phi"], 50, 30000.0, 64)
    assert np.max(np.abs(run["vc"] / vc - 1.0)) < 1e-12
    p, sel = run["p"], run["sel"]
    want = ora.forces(N, L0, (0.0, 0.0, 0.0), run["phi"], p.x[sel], p.y[sel], p.z[sel])
    scale = max(np.max(np.abs(w)) for w in want[:3])
    for a, w in zip(run["g"], want[:3]):
        assert np.max(np.abs(a - w)) < 1e-12 * scale
