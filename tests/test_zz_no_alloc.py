"""The solve entry point that allocates nothing (qumond_solve_mond_noalloc).

It serves callers that cannot allocate device memory when they solve; its
scratch lives in a fixed array inside the library, so it is limited to
grids of at most 64 intervals per side.  Checked through the C ABI against
qumond_solve_mond (the context-based solve) on two calls in a row with
different inputs, so that state left by the first call would show.
The entry point is meant for callers that never create a context, so one
case runs in a fresh process where the first call of the library is a
no-allocation solve (the one-time device set-up happens inside it).
This file is collected last on purpose.
"""
import os
import subprocess
import sys
import textwrap

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


_FRESH = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, sys.argv[1])
    from tests import analytic as an
    from tests.gpu_helpers import rel_max, to_dev
    import paper_1201_3185_gb300 as q

    L0 = 32000.0
    cases = [(64, 1, 0), (32, 2, 1)]
    got = []
    # no context exists in this process before these calls
    for n, nboxes, box in cases:
        params = q.default_params(n=n, nboxes=nboxes, L0=L0, rel_tol=1e-10, max_vcycles=40, ncycle=1,
                                  bc_mode=q.QUMOND_BC_GIVEN)
        x, y, z = an.node_coords(n, L0 / 2 ** box)
        f = np.exp(-(x * x + y * y + 4 * z * z) / (0.01 * (L0 / 2 ** box) ** 2))
        bc = -100.0 / np.sqrt(x * x + y * y + z * z + 1e6)
        parent = to_dev(np.cos(an.node_coords(n, L0)[0] / L0) * 50.0) if box > 0 else None
        start = to_dev(np.where(an.boundary_mask(n), bc, 0.0))
        u = start.clone()
        st = q.qumond.qumond_solve_mond_noalloc(params, box, to_dev(f), parent, u, stats=True)
        torch.cuda.synchronize()
        assert st.converged, (n, st.rel_residual)
        got.append((params, box, f, parent, start, u.cpu().numpy()))
    for params, box, f, parent, start, u in got:
        ctx = q.Context(params)
        want = start.clone()
        ctx.qumond_solve_mond(box, to_dev(f), parent, want, stats=True)
        torch.cuda.synchronize()
        err = rel_max(u, want.cpu().numpy())
        assert err < 1e-6, (params.n, err)
        ctx.close()
    print("fresh-process no-allocation solves ok")
""")


def test_noalloc_first_call_in_a_fresh_process():
    # n = 64 and n = 32 use the coarse-grid kernel's large shared-memory
    # configuration, which the first call must set up by itself
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no-allocation solves ok" in r.stdout
