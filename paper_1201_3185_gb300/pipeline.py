"""One evaluation of the QUMOND path over all nested boxes (Section 2).

For b = 0 .. nboxes-1 (outermost first): deposit -> Newtonian solve ->
QUMOND source -> QUMOND solve, each box taking its boundary values from the
previous one; then the forces at the particles and the rotation curve.
Every step is a call into libqumond; this class only owns the device
buffers and orders the calls.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from .qumond import Context


@dataclass
class PipelineResult:
    r: torch.Tensor
    vc: torch.Tensor
    newton_stats: list = field(default_factory=list)
    mond_stats: list = field(default_factory=list)


class Pipeline:
    def __init__(self, ctx: Context, device=None):
        self.ctx = ctx
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nodes = ctx.nodes
        nb = ctx.params.nboxes
        self.device = dev
        self.rho_fixed = torch.empty(nodes, dtype=torch.int64, device=dev)
        self.rho = torch.empty(nodes, dtype=torch.float64, device=dev)
        self.src = torch.empty(nodes, dtype=torch.float64, device=dev)
        self.phiN = [torch.zeros(nodes, dtype=torch.float64, device=dev) for _ in range(nb)]
        self.phi = [torch.zeros(nodes, dtype=torch.float64, device=dev) for _ in range(nb)]

    def potentials(self, x, y, z, m, stats=False, stream=None):
        """Steps 1-4 for every box; fills self.phiN and self.phi."""
        c = self.ctx
        ns, ms = [], []
        for b in range(c.params.nboxes):
            c.qumond_deposit(b, x, y, z, m, self.rho_fixed, self.rho, stream=stream)
            par_n = self.phiN[b - 1] if b > 0 else None
            par_m = self.phi[b - 1] if b > 0 else None
            ns.append(c.qumond_solve_newton(b, self.rho, par_n, self.phiN[b], stats=stats, stream=stream))
            c.qumond_source(b, self.phiN[b], self.src, stream=stream)
            ms.append(c.qumond_solve_mond(b, self.src, par_m, self.phi[b], stats=stats, stream=stream))
        return ns, ms

    def run(self, x, y, z, m, *, nbins=50, rmax=30000.0, nphi=64, forces=None, stats=False, stream=None):
        """The whole path: potentials, then forces at (x, y, z) into `forces`
        (a tuple gx, gy, gz of tensors, or None to skip) and the rotation curve."""
        ns, ms = self.potentials(x, y, z, m, stats=stats, stream=stream)
        if forces is not None:
            self.ctx.qumond_forces(self.phi, x, y, z, *forces, stream=stream)
        r = torch.empty(nbins, dtype=torch.float64, device=self.device)
        vc = torch.empty(nbins, dtype=torch.float64, device=self.device)
        self.ctx.qumond_rotation_curve(self.phi, nbins, rmax, nphi, r, vc, stream=stream)
        return PipelineResult(r, vc, ns, ms)
