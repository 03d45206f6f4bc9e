"""The solve entry point that allocates nothing (qumond_solve_mond_noalloc).

It serves callers that cannot allocate device memory when they solve; its
scratch lives in a fixed array inside the library, so it is limited to
grids of at most 64 intervals per side.  Checked through the C ABI against
qumond_solve_mond (the context-based solve) on two calls in a row with
different inputs, so that state left by the first call would show.
This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from tests import analytic as an
from tests.gpu_helpers import rel_max, to_dev

pytestmark = pytest.mark.gpu


def _problem(n, L, seed):
    rng = np.random.default_rng(seed)
    x, y, z = an.node_coords(n, L)
    c = rng.random(3) * 0.2 * L
    f = np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + 4 * (z - c[2]) ** 2) / (0.01 * L * L)) * (1.0 + rng.random())
    bc = -100.0 / np.sqrt(x * x + y * y + z * z + 0.01 * L * L) * (1.0 + rng.random())
    return f, bc


@pytest.mark.parametrize("n,nboxes,box", [(64, 1, 0), (32, 2, 1), (8, 1, 0)])
def test_noalloc_matches_context_solve_twice(n, nboxes, box):
    import paper_1201_3185_gb300 as q
    L0 = 32000.0
    params = q.default_params(n=n, nboxes=nboxes, L0=L0, rel_tol=1e-10, max_vcycles=40, ncycle=1,
                              bc_mode=q.QUMOND_BC_GIVEN)
    ctx = q.Context(params)
    for call in range(2):
        f, bc = _problem(n, L0 / 2 ** box, seed=10 * n + call)
        parent = to_dev(np.cos(an.node_coords(n, L0)[0] / L0) * 50.0) if box > 0 else None
        start = to_dev(np.where(an.boundary_mask(n), bc, 0.0))
        want = start.clone()
        st_w = ctx.qumond_solve_mond(box, to_dev(f), parent, want, stats=True)
        got = start.clone()
        st_g = q.qumond.qumond_solve_mond_noalloc(params, box, to_dev(f), parent, got, stats=True)
        torch.cuda.synchronize()
        assert st_g.converged and st_w.converged
        assert st_g.vcycles == st_w.vcycles
        assert rel_max(got.cpu().numpy(), want.cpu().numpy()) < 1e-6
    ctx.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    import paper_1201_3185_gb300 as q
    params = q.default_params(n=128, nboxes=1, L0=1000.0)
    dev = torch.zeros(129 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QumondError) as ei:
        q.qumond.qumond_solve_mond_noalloc(params, 0, dev, None, torch.zeros_like(dev))
    assert ei.value.status == q.qumond.QUMOND_ERR_INVALID_ARG
    assert "n=128" in str(ei.value)
