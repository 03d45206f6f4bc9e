"""The far-field boundary of box 0 (QUMOND_BC_MULTIPOLE) against the oracle.

* qumond_far_field on the GPU's own deposit (bit-exact with the oracle's)
  against ora_far_field: the QUMOND boundary values (FP64 on both sides, the
  sums in different orders) within 1e-12 of max|Phi|; the Newtonian ones
  within 1e-12 of max|Phi_N| plus 1e-5 of the largest contribution of the
  degrees 3..8 (the GPU evaluates those in FP32: a few roundings of 2^-24
  through the recurrence of depth 8, the sum over m and the FP32 moments,
  ~1e-6 of the terms, allowed ten times); interior untouched; every set of a
  context with several sets against its own oracle run.
* The whole path with the multipole boundary, two chains, graphs, fixed point,
  3 boxes: every potential within 1e-6 of max and the rotation curve within
  1e-5 of the oracle's pipeline with the same boundary.
"""
import numpy as np
import pytest
import torch

import synth
from tests import analytic as an
from tests.gpu_helpers import rel_max, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import paper_1201_3185_gb300 as q
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return q


@pytest.mark.parametrize("n,nsets", [(32, 1), (64, 1), (64, 3)])
def test_far_field_matches_oracle(q, ora, n, nsets):
    L0 = 120000.0
    gals = [synth.two_component_disk(40_000, seed=30 + s, rmax=0.45 * L0, zmax=0.45 * L0) for s in range(nsets)]
    # displace the sets so that their centres of mass differ
    gals = [synth.Particles(g.x + 3000.0 * s, g.y - 1500.0 * s, g.z, g.m * (1.0 + 0.5 * s)) for s, g in enumerate(gals)]
    ctx = q.Context(n=n, nboxes=1, L0=L0, bc_mode=q.QUMOND_BC_MULTIPOLE, nsets=nsets)
    N = (n + 1) ** 3
    x, y, z, m = (to_dev(np.concatenate([getattr(g, a) for g in gals])) for a in "xyzm")
    qf = torch.empty(nsets * N, dtype=torch.int64, device="cuda")
    rho = torch.empty(nsets * N, dtype=torch.float64, device="cuda")
    ctx.qumond_deposit(0, x, y, z, m, qf, rho)
    phiN = torch.full((nsets * N,), 7.0, dtype=torch.float64, device="cuda")
    phi = torch.full_like(phiN, 7.0)
    ctx.qumond_far_field(rho, phiN, phi)
    torch.cuda.synchronize()
    b = an.boundary_mask(n)
    for s, g in enumerate(gals):
        want_q, _ = ora.cic_deposit(n, L0, (0.0, 0.0, 0.0), 24, g.x, g.y, g.z, g.m)
        r_s = rho[s * N:(s + 1) * N].cpu().numpy()
        assert np.array_equal(qf[s * N:(s + 1) * N].cpu().numpy(), want_q)
        wN, wM, M = ora.far_field(n, L0, (0.0, 0.0, 0.0), r_s, lmax=8)
        w2, _, _ = ora.far_field(n, L0, (0.0, 0.0, 0.0), r_s, lmax=2)
        gN = phiN[s * N:(s + 1) * N].cpu().numpy()
        gM = phi[s * N:(s + 1) * N].cpu().numpy()
        assert M > 0.0
        high = np.max(np.abs(wN[b] - w2[b]))  # the degrees 3..8
        err = np.max(np.abs(gN[b] - wN[b]))
        print("set %d: Phi_N error %.2e of max, high degrees %.2e of max" % (s, err / np.max(np.abs(wN[b])),
                                                                           high / np.max(np.abs(wN[b]))))
        assert err < 1e-12 * np.max(np.abs(wN[b])) + 1e-5 * high, s
        assert np.max(np.abs(gM[b] - wM[b])) < 1e-12 * np.max(np.abs(wM[b])), s
        assert np.all(gN[~b] == 7.0) and np.all(gM[~b] == 7.0)
    ctx.close()


def test_far_field_needs_the_multipole_mode(q):
    ctx = q.Context(n=16, nboxes=1, L0=1000.0)
    a = torch.zeros(17 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QumondError):
        ctx.qumond_far_field(a, a.clone(), a.clone())
    ctx.close()


def test_far_field_zero_mass(q):
    ctx = q.Context(n=16, nboxes=1, L0=1000.0, bc_mode=q.QUMOND_BC_MULTIPOLE)
    rho = torch.zeros(17 ** 3, dtype=torch.float64, device="cuda")
    phiN = torch.full_like(rho, 3.0)
    phi = torch.full_like(rho, 3.0)
    ctx.qumond_far_field(rho, phiN, phi)
    torch.cuda.synchronize()
    b = torch.from_numpy(an.boundary_mask(16)).cuda()
    assert torch.all(phiN[b] == 0.0) and torch.all(phi[b] == 0.0) and torch.all(phiN[~b] == 3.0)
    ctx.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_multipole_pipeline_matches_oracle(q, ora, prec):
    n, L0, nb = 64, 120000.0, 3
    p = synth.two_component_disk(200_000, seed=33, rmax=0.45 * L0, zmax=0.45 * L0)
    kw = dict(n=n, nboxes=nb, L0=L0, rel_tol=1e-10, max_vcycles=40, ncycle=1, precision=prec,
              bc_mode=q.QUMOND_BC_MULTIPOLE)
    ca, cb = q.Context(**kw), q.Context(**kw)
    pipe = q.Pipeline(ca, ctx_mond=cb)
    x, y, z, m = (to_dev(a) for a in (p.x, p.y, p.z, p.m))
    for _ in range(2):
        res = pipe.run(x, y, z, m, nbins=40, rmax=25000.0, stats=True)
    torch.cuda.synchronize()
    boxes = ora.pipeline(p, n, L0, nb, ncycle=1, tol=1e-12, max_vcycles=40, far_field_lmax=8)
    for b, bx in enumerate(boxes):
        assert rel_max(pipe.phiN[b].cpu().numpy(), bx.phiN) < 1e-6, b
        assert rel_max(pipe.phi[b].cpu().numpy(), bx.phi) < 1e-6, b
    _, vc_w = ora.rotation_curve(n, L0, (0.0, 0.0, 0.0), [bx.phi for bx in boxes], 40, 25000.0)
    assert np.max(np.abs(res.vc.cpu().numpy() / vc_w - 1.0)) < 1e-5
    pipe.close()
    ca.close()
    cb.close()
