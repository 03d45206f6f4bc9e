"""Fit sweep (Section 3.5) on the GPU: the chi^2 kernel, whole sweeps against
the oracle set by set, independence of the worker count, and the full-size
sweep (64 parameter sets, 129^3 x 2 boxes, 5e5 particles each) against the
oracle-made target curve.

Tolerances: v_c 1e-5 relative (the path's stated bound).  chi^2 from curves
that each carry that bound: with d_i = (v_i - v_obs,i)/sigma_i and
|dv_i| <= 1e-5 |v_i|, |d chi^2| <= (1/n) sum (2 |d_i| e_i + e_i^2) with
e_i = 1e-5 |v_i| / sigma_i; the tests allow twice that.  The chi^2 kernel on
identical inputs: 1e-13 relative (summation order only).
"""
import json
import os

import numpy as np
import pytest
import torch

import synth
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sweep_target_two_disk_129cube.json")
VC_TOL = 1e-5


@pytest.fixture(scope="module")
def q():
    import paper_1201_3185_gb300 as q
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return q


def chi2_bound(vc_ref, v_obs, sigma):
    d = (vc_ref - v_obs) / sigma
    e = VC_TOL * np.abs(vc_ref) / sigma
    return 2.0 * np.mean(2.0 * np.abs(d) * e + e * e, axis=-1)


@pytest.mark.parametrize("nsets,nbins", [(1, 1), (3, 32), (70, 45), (129, 100)])
def test_chi2_kernel(q, ora, nsets, nbins):
    rng = np.random.default_rng(nsets * 1000 + nbins)
    v_obs = 100.0 + 50.0 * rng.random(nbins)
    sigma = 0.03 * v_obs * (0.5 + rng.random(nbins))
    vc = v_obs * (1.0 + 0.05 * rng.standard_normal((nsets, nbins)))
    want = ora.chi2(vc, v_obs, sigma)
    ctx = q.Context(n=8, nboxes=1, L0=100.0)
    out = torch.full((nsets,), np.nan, dtype=torch.float64, device="cuda")
    ctx.qumond_chi2(to_dev(vc), to_dev(v_obs), to_dev(sigma), out)
    got = out.cpu().numpy()
    ctx.close()
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)


def test_chi2_invalid(q):
    ctx = q.Context(n=8, nboxes=1, L0=100.0)
    a = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QumondError):  # nbins = 0
        ctx.qumond_chi2(torch.empty(4, 0, dtype=torch.float64, device="cuda"), a[:0], a[:0], a)
    ctx.close()


def sweep_params(q, n, L0, prec, rel_tol):
    return q.default_params(n=n, nboxes=2, L0=L0, precision=prec, rel_tol=rel_tol, max_vcycles=40)


def oracle_curve(ora, gal, prm, n, L0, nbins, rmax, tol=1e-12):
    p = gal.particles(prm)
    boxes = ora.pipeline(p, n, L0, 2, tol=tol, max_vcycles=60)
    return ora.rotation_curve(n, L0, (0.0, 0.0, 0.0), [b.phi for b in boxes], nbins, rmax * prm[0])


def device_sets(gal, params):
    return [tuple(to_dev(a) for a in (p.x, p.y, p.z, p.m)) for p in (gal.particles(r) for r in params)]


@pytest.mark.parametrize("prec_name", ["MIXED_FIXED", "MIXED", "FP64"])
def test_sweep_small_matches_oracle(q, ora, prec_name):
    n, L0, nbins, rmax = 32, 80000.0, 24, 24000.0
    prec = getattr(q, "QUMOND_PREC_" + prec_name)
    gal = synth.SweepGalaxy(20000, seed=5)
    params = synth.fit_sweep_parameters(7, seed=6)
    rng = np.random.default_rng(7)
    v_obs = 80.0 + 40.0 * rng.random(nbins)
    sigma = 0.03 * v_obs
    sets = device_sets(gal, params)
    with q.FitSweep(sweep_params(q, n, L0, prec, 1e-10), nbins=nbins, rmax=rmax, workers=3) as sw:
        res = sw.run(sets, params[:, 0], to_dev(v_obs), to_dev(sigma), stats=True)
        torch.cuda.synchronize()
        vc = res.vc.cpu().numpy()
        chi2 = res.chi2.cpu().numpy()
        r = res.r.cpu().numpy()
    for s, prm in enumerate(params):
        assert all(ns.converged and ms.converged for ns, ms in res.stats[s])
        r_ref, v_ref = oracle_curve(ora, gal, prm, n, L0, nbins, rmax)
        np.testing.assert_allclose(r[s], r_ref, rtol=1e-15)
        assert np.max(np.abs(vc[s] - v_ref) / np.abs(v_ref)) <= VC_TOL, s
        want = ora.chi2(v_ref, v_obs, sigma)[0]
        assert abs(chi2[s] - want) <= chi2_bound(v_ref, v_obs, sigma), (s, chi2[s], want)


def test_sweep_independent_of_workers(q):
    n, L0, nbins, rmax = 32, 80000.0, 24, 24000.0
    gal = synth.SweepGalaxy(20000, seed=8)
    params = synth.fit_sweep_parameters(5, seed=9)
    v_obs = to_dev(np.linspace(60.0, 120.0, nbins))
    sigma = 0.03 * v_obs
    sets = device_sets(gal, params)
    out = []
    for workers in (1, 2, 5):
        with q.FitSweep(sweep_params(q, n, L0, q.QUMOND_PREC_MIXED_FIXED, 1e-8), nbins=nbins, rmax=rmax,
                        workers=workers) as sw:
            res = sw.run(sets, params[:, 0], v_obs, sigma)
            torch.cuda.synchronize()
            out.append((res.vc.cpu().numpy(), res.chi2.cpu().numpy()))
    for vc, chi2 in out[1:]:
        assert np.array_equal(vc, out[0][0])
        assert np.array_equal(chi2, out[0][1])


def test_sweep_empty(q):
    with q.FitSweep(sweep_params(q, 16, 80000.0, q.QUMOND_PREC_MIXED_FIXED, 1e-8), nbins=8, rmax=1e4,
                    workers=2) as sw:
        z = torch.zeros(8, dtype=torch.float64, device="cuda")
        res = sw.run([], [], z, z + 1.0)
        assert res.vc.shape == (0, 8) and res.chi2.shape == (0,)


def test_sweep_full_size(q, ora):
    """The fit-sweep workload as timed: 64 seeded parameter sets plus the
    target's own parameters, rel. residual 1e-8, fixed-point refinement."""
    doc = json.load(open(GOLDEN))
    s = doc["spec"]
    v_true, eps = np.array(doc["v_true"]), np.array(doc["eps"])
    v_obs, sigma = np.array(doc["v_obs"]), np.array(doc["sigma"])
    gal = synth.SweepGalaxy(s["particles"], s["galaxy_seed"])
    params = np.vstack([synth.fit_sweep_parameters(64, seed=2012), np.array(s["true_params"])[None, :]])
    sets = device_sets(gal, params)
    prm = sweep_params(q, s["n"], s["L0"], q.QUMOND_PREC_MIXED_FIXED, 1e-8)
    with q.FitSweep(prm, nbins=s["nbins"], rmax=s["rmax"], workers=16) as sw:
        res = sw.run(sets, params[:, 0], to_dev(v_obs), to_dev(sigma), stats=True)
        torch.cuda.synchronize()
        vc, chi2 = res.vc.cpu().numpy(), res.chi2.cpu().numpy()
    assert all(ns.converged and ms.converged for st in res.stats for ns, ms in st)
    assert np.all(np.isfinite(vc)) and np.all(chi2 > 0.0)
    # the target's own parameters reproduce the oracle's noiseless curve, so
    # their chi^2 is the mean square of the stored noise draws
    t = len(params) - 1
    assert np.max(np.abs(vc[t] - v_true) / v_true) <= VC_TOL
    want = float(np.mean(eps ** 2))
    assert abs(chi2[t] - want) <= chi2_bound(v_true, v_obs, sigma), (chi2[t], want)
    # the truth fits better than all but a few random sets (3% noise lets a neighbour win narrowly)
    assert chi2[t] < np.percentile(chi2[:t], 10)
    # one sampled random set, recomputed by the oracle
    k = 17
    _, v_ref = oracle_curve(ora, gal, params[k], s["n"], s["L0"], s["nbins"], s["rmax"])
    assert np.max(np.abs(vc[k] - v_ref) / np.abs(v_ref)) <= VC_TOL
