"""Science extras on the GPU against the oracle: the algebraic MOND rotation
curve (Eq. 3, Section 3.3) and the vertical velocity dispersion of an
isothermal sech^2 layer (Section 5.6).

From identical potentials the two sides do the same FP64 operations up to
summation order: 1e-12.  End to end (each side's own potentials, 1e-10
residual) the curves inherit the v_c bound: 1e-5."""
import numpy as np
import pytest
import torch

import synth
from tests.analytic import node_coords
from tests.gpu_helpers import G, A0, gpu_pipeline, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import paper_1201_3185_gb300 as q
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return q


def smooth_potentials(n, L0, nb, seed):
    rng = np.random.default_rng(seed)
    out = []
    for b in range(nb):
        x, y, z = node_coords(n, L0 / 2 ** b, (0.0, 0.0, 0.0))
        r = np.sqrt(x * x + y * y + (3.0 * z) ** 2 + 1e6)
        out.append(-4e7 / r + 1e-3 * rng.standard_normal(x.shape) + 2e-4 * x)
    return out


@pytest.mark.parametrize("nb", [1, 3])
def test_profiles_match_oracle_on_identical_potentials(q, ora, nb):
    n, L0 = 32, 64000.0
    phis = smooth_potentials(n, L0, nb, nb)
    ctx = q.Context(n=n, nboxes=nb, L0=L0)
    dp = [to_dev(p) for p in phis]
    nbins, rmax = 37, 20000.0
    r, v = (torch.empty(nbins, dtype=torch.float64, device="cuda") for _ in range(2))
    ctx.qumond_rotation_curve_algebraic(dp, nbins, rmax, 48, r, v)
    r_o, v_o = ora.rotation_curve_algebraic(n, L0, (0.0, 0.0, 0.0), phis, nbins, rmax, 48, a0=A0)
    np.testing.assert_allclose(r.cpu().numpy(), r_o, rtol=1e-15)
    np.testing.assert_allclose(v.cpu().numpy(), v_o, rtol=1e-12)
    for z_eval, h in ((300.0, 400.0), (900.0, 300.0)):
        ctx.qumond_sigma_z(dp, nbins, rmax, 48, z_eval, h, r, v)
        _, s_o = ora.sigma_z(n, L0, (0.0, 0.0, 0.0), phis, nbins, rmax, z_eval, h, 48)
        np.testing.assert_allclose(v.cpu().numpy(), s_o, rtol=1e-12)
    with pytest.raises(q.QumondError):
        ctx.qumond_sigma_z(dp, nbins, rmax, 48, -1.0, h, r, v)
    ctx.close()


def test_profiles_end_to_end_two_disk(q, ora):
    n, L0, nb = 64, 60000.0, 2
    p = synth.two_component_disk(300_000, seed=3, rmax=25000.0, zmax=25000.0, h_star=500.0)
    out = gpu_pipeline(p, n, L0, nb, nbins=30, rmax=15000.0, rel_tol=1e-10, max_vcycles=40,
                       precision=q.QUMOND_PREC_MIXED_FIXED)
    boxes = ora.pipeline(p, n, L0, nb, tol=1e-12, max_vcycles=60)
    ctx = q.Context(n=n, nboxes=nb, L0=L0)
    r, v = (torch.empty(30, dtype=torch.float64, device="cuda") for _ in range(2))
    ctx.qumond_rotation_curve_algebraic([to_dev(a) for a in out["phiN"]], 30, 15000.0, 64, r, v)
    _, v_o = ora.rotation_curve_algebraic(n, L0, (0.0, 0.0, 0.0), [b.phiN for b in boxes], 30, 15000.0, 64, a0=A0)
    assert np.max(np.abs(v.cpu().numpy() / v_o - 1.0)) < 1e-5
    ctx.qumond_sigma_z([to_dev(a) for a in out["phi"]], 30, 15000.0, 64, 500.0, 500.0, r, v)
    _, s_o = ora.sigma_z(n, L0, (0.0, 0.0, 0.0), [b.phi for b in boxes], 30, 15000.0, 500.0, 500.0, 64)
    sel = np.abs(s_o) > 1.0
    assert np.max(np.abs(v.cpu().numpy()[sel] / s_o[sel] - 1.0)) < 1e-5
    # the stellar layer's dispersion falls with radius (Section 5.6's trend)
    assert s_o[2] > s_o[-1] > 0.0
    ctx.close()
