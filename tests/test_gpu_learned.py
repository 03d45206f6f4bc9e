"""What the trained network (paper_1201_3185_gb300/weights, trained on the GPU
by `python -m paper_1201_3185_gb300.learned train`) gains over the method
without it, on galaxies it has not seen (129^3 x 2 boxes, two-disk galaxies,
QUMOND solves to rel. residual 1e-8 in the fixed-point mode).

Starting the QUMOND solve from Phi_N + network output instead of from Phi_N
alone must save V-cycles in every box, and the solve must end at the same
discrete solution as the FMG start.  FMG itself is the method's default
start; the comparison with it is printed (and recorded in the design notes),
not asserted."""
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_learned_start_saves_vcycles():
    import paper_1201_3185_gb300 as q
    from paper_1201_3185_gb300 import learned as L
    assert os.path.exists(L.WEIGHTS), "trained weights missing"
    dev = torch.device("cuda", 0)
    guess = q.Guess(128, L.PHI_SCALE)
    guess.qumond_guess_set_params(torch.from_numpy(L.load_weights()).to(dev))
    work = L.Workload(n=128, particles=200_000, seed=424242, device=dev)
    rows = L.evaluate(work, guess, 2)
    for r in rows:
        print("box %d h*=%.0f pc: " % (r["box"], r["h_star"]) +
              ", ".join("%s %d V-cycles (start residual %.2e, %.2f ms)" % (k, r[k]["vcycles"],
                                                                          r[k]["rel_residual_start"], r[k]["ms"])
                        for k in L.STARTS))
        assert r["learned"]["vcycles"] < r["phiN"]["vcycles"]
        assert r["learned"]["rel_residual"] <= 1e-8
        # the solve from the guess and the accurate (1e-10) solve agree to the path's potential bound
        assert r["learned"]["max_rel_diff_vs_accurate"] < 1e-6
    guess.close()
