"""Writes sweep_target_two_disk_129cube.json: the synthetic "observed"
rotation curve of a fit sweep (Section 3.5), computed by the CPU oracle only.

The galaxy is the two-component disk at known parameters (distance scale 1,
stellar M/L 0.75, stellar scale height 450 pc, gas scale height 150 pc) from
the seeded draws of synth.SweepGalaxy; its QUMOND rotation curve on a 129^3
grid with two nested boxes (80 and 40 kpc) is the noiseless curve v_true.  The
observed curve is v_obs = v_true (1 + 0.03 eps) with eps standard normal
(seeded), and sigma_obs = 0.03 v_true.  Run from the repository root:

    python tests/golden/make_sweep_target.py
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

SPEC = dict(n=128, nboxes=2, L0=80000.0, ratio=2, particles=500_000, galaxy_seed=11, noise_seed=12,
            true_params=[1.0, 0.75, 450.0, 150.0], nbins=40, rmax=24000.0, nphi=64, frac=0.2, G=4.30e-3, a0=3.6,
            shift=24, ncycle=6, tol=1e-12, max_vcycles=60, sigma_frac=0.03)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sweep_target_two_disk_129cube.json")


def main():
    s = SPEC
    t0 = time.time()
    gal = synth.SweepGalaxy(s["particles"], s["galaxy_seed"])
    p = gal.particles(s["true_params"])
    boxes = oracle.pipeline(p, s["n"], s["L0"], s["nboxes"], G=s["G"], a0=s["a0"], shift=s["shift"],
                            ncycle=s["ncycle"], tol=s["tol"], max_vcycles=s["max_vcycles"], ratio=s["ratio"])
    r, v_true = oracle.rotation_curve(s["n"], s["L0"], (0.0, 0.0, 0.0), [b.phi for b in boxes], s["nbins"],
                                      s["rmax"] * s["true_params"][0], s["nphi"], s["frac"], s["ratio"])
    eps = np.random.default_rng(s["noise_seed"]).standard_normal(s["nbins"])
    v_obs = v_true * (1.0 + s["sigma_frac"] * eps)
    sigma = s["sigma_frac"] * v_true
    doc = dict(spec=s, r=r.tolist(), v_true=v_true.tolist(), eps=eps.tolist(), v_obs=v_obs.tolist(),
               sigma=sigma.tolist(), vcycles=[[b.newton_vcycles, b.mond_vcycles] for b in boxes],
               written_by="tests/golden/make_sweep_target.py (CPU oracle only)")
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print(f"wrote {OUT} in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
