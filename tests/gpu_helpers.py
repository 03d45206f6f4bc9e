"""Shared helpers of the GPU tests: run the CUDA path through the C ABI."""
import numpy as np
import torch

G, A0 = 4.30e-3, 3.6


def to_dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def gpu_pipeline(p, n, L0, nb, *, nbins=50, rmax=None, nphi=64, forces=False, bc_newton=None, bc_mond=None,
                 stats=True, **params):
    """Run the whole path on the GPU; returns a dict of numpy results."""
    import paper_1201_3185_gb300 as q
    from tests.analytic import boundary_mask, node_coords
    if bc_newton is not None:
        params["bc_mode"] = q.QUMOND_BC_GIVEN
    ctx = q.Context(n=n, nboxes=nb, L0=L0, **params)
    pipe = q.Pipeline(ctx)
    if bc_newton is not None:
        xs, ys, zs = node_coords(n, L0)
        bnd = boundary_mask(n)
        vn = np.zeros((n + 1) ** 3)
        vm = np.zeros((n + 1) ** 3)
        vn[bnd] = bc_newton(xs[bnd], ys[bnd], zs[bnd])
        vm[bnd] = bc_mond(xs[bnd], ys[bnd], zs[bnd])
        pipe.phiN[0].copy_(to_dev(vn))
        pipe.phi[0].copy_(to_dev(vm))
    x, y, z, m = (to_dev(a) for a in (p.x, p.y, p.z, p.m))
    out = {}
    gx = gy = gz = None
    if forces:
        gx, gy, gz = (torch.empty_like(x) for _ in range(3))
    ns, ms = [], []
    rho_fixed = []
    for b in range(nb):
        ctx.qumond_deposit(b, x, y, z, m, pipe.rho_fixed, pipe.rho)
        rho_fixed.append(pipe.rho_fixed.cpu().numpy().copy())
        ns.append(ctx.qumond_solve_newton(b, pipe.rho, pipe.phiN[b - 1] if b else None, pipe.phiN[b], stats=stats))
        ctx.qumond_source(b, pipe.phiN[b], pipe.src)
        out.setdefault("src", []).append(pipe.src.cpu().numpy().copy())
        ms.append(ctx.qumond_solve_mond(b, pipe.src, pipe.phi[b - 1] if b else None, pipe.phi[b], stats=stats))
    if forces:
        ctx.qumond_forces(pipe.phi, x, y, z, gx, gy, gz)
        out["g"] = (gx.cpu().numpy(), gy.cpu().numpy(), gz.cpu().numpy())
    if rmax is None:
        rmax = 0.4 * L0
    r = torch.empty(nbins, dtype=torch.float64, device="cuda")
    vc = torch.empty(nbins, dtype=torch.float64, device="cuda")
    ctx.qumond_rotation_curve(pipe.phi, nbins, rmax, nphi, r, vc)
    torch.cuda.synchronize()
    out.update(rho_fixed=rho_fixed, phiN=[t.cpu().numpy() for t in pipe.phiN], phi=[t.cpu().numpy() for t in pipe.phi],
               r=r.cpu().numpy(), vc=vc.cpu().numpy(), newton_stats=ns, mond_stats=ms)
    ctx.close()
    return out


def rel_max(a, b):
    """max|a - b| / max|b| (potential error measure)."""
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
