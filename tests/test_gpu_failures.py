"""Failure paths of the solves, made on the host or through a wait limit
(no GPU fault is provoked).

* A grid barrier of the cooperative small-level V-cycle that runs out of
  polls: the kernel records the fault and returns, the solve reports
  QUMOND_ERR_TIMEOUT, and the context stays usable (the next solve is
  correct).  That wait has no asynchronous copies behind it.
* A NaN in the caller's density: the residual check sees a non-finite
  start, no V-cycle is trusted, and the solve reports
  QUMOND_ERR_NOT_CONVERGED in every precision; the next solve on the same
  context is correct.
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


def _rho(n, L, seed):
    p = synth.two_component_disk(50_000, seed=seed, rmax=0.45 * L, zmax=0.45 * L)
    import oracle
    qf, _ = oracle.cic_deposit(n, L, (0.0, 0.0, 0.0), 24, p.x, p.y, p.z, p.m)
    return oracle.rho_from_fixed(n, L, 24, qf)


@pytest.mark.parametrize("graphs", [1, 0])
def test_grid_barrier_timeout_is_reported_and_the_context_recovers(q, graphs):
    n, L = 128, 120000.0
    rho = to_dev(_rho(n, L, 21))
    kw = dict(n=n, nboxes=1, L0=L, rel_tol=1e-10, max_vcycles=40, precision=q.QUMOND_PREC_MIXED,
              persistent_vcycle=1, use_graphs=graphs)
    ctx = q.Context(**kw)
    if ctx_has_no_cooperative_kernel(q, ctx, rho):
        pytest.skip("device without cooperative launches: the small-level V-cycle is not one kernel")
    ctx.qumond_set_barrier_poll_limit(1)
    u = torch.zeros_like(rho)
    with pytest.raises(q.QumondError) as ei:
        ctx.qumond_solve_newton(0, rho, None, u, stats=True)
    assert ei.value.status == q.qumond.QUMOND_ERR_TIMEOUT
    # back to the default limit: the same context solves correctly
    ctx.qumond_set_barrier_poll_limit(1 << 26)
    u.zero_()
    st = ctx.qumond_solve_newton(0, rho, None, u, stats=True)
    assert st.converged and st.rel_residual <= 1e-10
    ref = q.Context(**dict(kw, persistent_vcycle=0))
    w = torch.zeros_like(rho)
    ref.qumond_solve_newton(0, rho, None, w, stats=True)
    torch.cuda.synchronize()
    assert torch.equal(u, w)  # the cooperative and per-step forms give the same bits
    ctx.close()
    ref.close()


def ctx_has_no_cooperative_kernel(q, ctx, rho):
    # a solve with tracing counts the kernel classes it launched
    u = torch.zeros_like(rho)
    ctx.qumond_trace_read(reset=True)
    ctx.qumond_solve_newton(0, rho, None, u, stats=True)
    stats, _, _ = ctx.qumond_trace_read(reset=True)
    return stats["vcycle_small_levels"].launches == 0


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_nan_density_gives_not_converged_then_recovers(q, prec):
    n, L = 64, 60000.0
    rho_np = _rho(n, L, 22)
    bad = rho_np.copy()
    i = (n // 2) + (n + 1) * ((n // 3) + (n + 1) * (n // 2))
    bad[i] = np.nan
    ctx = q.Context(n=n, nboxes=1, L0=L, rel_tol=1e-10, max_vcycles=20, precision=prec)
    u = torch.zeros((n + 1) ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(q.NotConverged) as ei:
        ctx.qumond_solve_newton(0, to_dev(bad), None, u, stats=True)
    assert ei.value.status == q.qumond.QUMOND_ERR_NOT_CONVERGED
    good = to_dev(rho_np)
    u.zero_()
    st = ctx.qumond_solve_newton(0, good, None, u, stats=True)
    assert st.converged and st.rel_residual <= 1e-10
    fresh = q.Context(n=n, nboxes=1, L0=L, rel_tol=1e-10, max_vcycles=20, precision=prec)
    w = torch.zeros_like(u)
    fresh.qumond_solve_newton(0, good, None, w, stats=True)
    torch.cuda.synchronize()
    assert torch.equal(u, w)  # nothing of the failed solve leaks into the next one
    ctx.close()
    fresh.close()
