"""CPU checks of the fit-sweep inputs (Section 3.5): the parameter sets, the
galaxy realisation shared by all sets, and the oracle-made target curve."""
import json
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sweep_target_two_disk_129cube.json")


def test_parameter_ranges():
    p = synth.fit_sweep_parameters(4096, seed=1)
    lo = np.array([0.8, 0.3, 200.0, 50.0])
    hi = np.array([1.2, 1.2, 1000.0, 500.0])
    assert np.all(p >= lo) and np.all(p <= hi)
    assert np.all(np.abs(p.mean(axis=0) - 0.5 * (lo + hi)) < 0.03 * (hi - lo))


def test_sweep_galaxy_scaling():
    gal = synth.SweepGalaxy(20000, seed=3)
    a = gal.particles([1.0, 1.0, 400.0, 100.0])
    b = gal.particles([1.2, 0.5, 400.0, 300.0])
    ns = gal.ns
    # masses: stars M/L * 2 pi I0 (d Rd)^2, gas d^2 M_gas (Section 3.4: half the particles each)
    assert a.m[:ns].sum() == pytest.approx(2.0 * np.pi * 500.0 * 3000.0 ** 2, rel=1e-12)
    assert b.m[:ns].sum() == pytest.approx(0.5 * 2.0 * np.pi * 500.0 * 3600.0 ** 2, rel=1e-12)
    assert b.m[ns:].sum() == pytest.approx(1.44e9, rel=1e-12)
    # in-plane positions scale with the distance factor; the stellar heights are unchanged
    np.testing.assert_allclose(b.x, 1.2 * a.x, rtol=1e-13, atol=1e-9)
    np.testing.assert_allclose(b.y, 1.2 * a.y, rtol=1e-13, atol=1e-9)
    assert np.array_equal(b.z[:ns], a.z[:ns])
    assert np.all(np.abs(b.z[ns:]) >= np.abs(a.z[ns:]))  # thicker gas disk


def test_sweep_galaxy_profiles():
    gal = synth.SweepGalaxy(200000, seed=4)
    p = gal.particles([1.0, 1.0, 500.0, 100.0])
    ns = gal.ns
    R = np.hypot(p.x[:ns], p.y[:ns])
    # exponential disk truncated at 10 Rd: enclosed fraction 1 - (1+x) e^-x
    x = 2.0
    frac = (1.0 - (1.0 + x) * np.exp(-x)) / (1.0 - 11.0 * np.exp(-10.0))
    assert np.mean(R < x * 3000.0) == pytest.approx(frac, abs=4e-3)
    # sech^2(z/h): P(|z| < h) = tanh(1) / tanh(zmax/h)
    assert np.mean(np.abs(p.z[:ns]) < 500.0) == pytest.approx(np.tanh(1.0) / np.tanh(10.0), abs=4e-3)


def test_target_file_consistent(ora):
    doc = json.load(open(GOLDEN))
    s = doc["spec"]
    v_true, eps = np.array(doc["v_true"]), np.array(doc["eps"])
    v_obs, sigma = np.array(doc["v_obs"]), np.array(doc["sigma"])
    assert len(v_true) == s["nbins"]
    np.testing.assert_array_equal(eps, np.random.default_rng(s["noise_seed"]).standard_normal(s["nbins"]))
    np.testing.assert_allclose(v_obs, v_true * (1.0 + 0.03 * eps), rtol=1e-15)
    np.testing.assert_allclose(sigma, 0.03 * v_true, rtol=1e-15)
    assert ora.chi2(v_true, v_obs, sigma)[0] == pytest.approx(np.mean(eps ** 2), rel=1e-12)
    # a flat-ish MOND curve: rising inside 2 Rd, within 10% of its peak beyond it
    assert np.all(np.diff(v_true[:10]) > 0.0)
    assert np.min(v_true[10:]) > 0.9 * np.max(v_true)


def test_target_regenerates(ora):
    """The stored curve is what the oracle computes now."""
    doc = json.load(open(GOLDEN))
    s = doc["spec"]
    gal = synth.SweepGalaxy(s["particles"], s["galaxy_seed"])
    boxes = ora.pipeline(gal.particles(s["true_params"]), s["n"], s["L0"], s["nboxes"], G=s["G"], a0=s["a0"],
                         shift=s["shift"], ncycle=s["ncycle"], tol=s["tol"], max_vcycles=s["max_vcycles"],
                         ratio=s["ratio"])
    _, v = ora.rotation_curve(s["n"], s["L0"], (0.0, 0.0, 0.0), [b.phi for b in boxes], s["nbins"],
                              s["rmax"] * s["true_params"][0], s["nphi"], s["frac"], s["ratio"])
    np.testing.assert_allclose(v, doc["v_true"], rtol=1e-12)
