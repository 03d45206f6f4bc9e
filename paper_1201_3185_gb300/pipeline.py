"""One evaluation of the QUMOND path over all nested boxes (Section 2).

For b = 0 .. nboxes-1 (outermost first): deposit -> Newtonian solve ->
QUMOND source -> QUMOND solve, each box taking its boundary values from the
previous one; then the forces at the particles and the rotation curve.
Every step is a call into libqumond; this class only owns the device
buffers and orders the calls.

Concurrency: the QUMOND solve of box b needs box b's source and box b-1's
QUMOND potential, the Newtonian solve of box b+1 needs box b's Newtonian
potential -- so the two are independent.  With a second context
(`ctx_mond`), the Newtonian chain (deposits, Newtonian solves, sources) runs
on one stream from the calling thread and the QUMOND chain on another stream
from a worker thread, the source of each box handed over with a CUDA event.
Each solve spends a large part of its time on small multigrid levels that
leave most of the GPU idle, and the other chain fills it.  The kernels and
their order within each chain are unchanged, so the results are the same
bits as the sequential order.

Learned initial guess: with `guess` (a Guess for S = n) and `ctx_warm` (a
context with warm_start = 1), the QUMOND solve of each box starts from
Phi_N + the network's output instead of FMG (sequential order only).

Far-field boundary: with bc_mode QUMOND_BC_MULTIPOLE the boundary values of
box 0 (both potentials) come from qumond_far_field of box 0's density,
enqueued right after its deposit.

Sets: with a context of several sets (params.nsets > 1) every buffer holds
one grid per set and the particle arrays hold every set's particles, set
after set; each call then covers all sets.

Solve timing (measurement only): when `solve_events` is a list, the
sequential order appends one pair of CUDA timing events per solve, recorded
on the solve's stream right before and right after the call.
"""
from __future__ import annotations

import concurrent.futures as cf
import threading
from dataclasses import dataclass, field

import math

import torch

from .qumond import QUMOND_BC_MULTIPOLE, Context, Guess


@dataclass
class PipelineResult:
    r: torch.Tensor
    vc: torch.Tensor
    newton_stats: list = field(default_factory=list)
    mond_stats: list = field(default_factory=list)
    done: object = None  # run_many: CUDA event recorded once this evaluation's forces and curve are written


class Pipeline:
    def __init__(self, ctx: Context, device=None, ctx_mond: Context | None = None, guess: Guess | None = None,
                 ctx_warm: Context | None = None):
        self.ctx = ctx
        self.ctx_mond = ctx_mond
        if (guess is None) != (ctx_warm is None):
            raise ValueError("a learned guess needs both the network and a warm-start context")
        if guess is not None:
            if ctx_mond is not None:
                raise ValueError("the learned guess runs in the sequential order only")
            if guess.S != ctx.params.n or not ctx_warm.params.warm_start:
                raise ValueError("the network must match n and ctx_warm must have warm_start = 1")
        self.guess = guess
        self.ctx_warm = ctx_warm
        self.solve_events = None
        self.far_field = ctx.params.bc_mode == QUMOND_BC_MULTIPOLE
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nodes = ctx.nodes
        nb = ctx.params.nboxes
        self.device = dev
        self.rho_fixed = torch.empty(nodes, dtype=torch.int64, device=dev)
        self.rho = torch.empty(nodes, dtype=torch.float64, device=dev)
        nsrc = nb if ctx_mond is not None else 1  # concurrent chains: one source buffer per box
        self.srcs = [torch.empty(nodes, dtype=torch.float64, device=dev) for _ in range(nsrc)]
        self.src = self.srcs[0]
        self.phiN = [torch.zeros(nodes, dtype=torch.float64, device=dev) for _ in range(nb)]
        self.phi = [torch.zeros(nodes, dtype=torch.float64, device=dev) for _ in range(nb)]
        if ctx_mond is not None:
            if ctx_mond.nodes != nodes or ctx_mond.params.nboxes != nb:
                raise ValueError("the two contexts must describe the same boxes")
            self._streams = (torch.cuda.Stream(dev), torch.cuda.Stream(dev))
            self._pool = cf.ThreadPoolExecutor(max_workers=1, thread_name_prefix="qumond-mond")

    def close(self):
        if self.ctx_mond is not None:
            self._pool.shutdown(wait=True)

    def potentials(self, x, y, z, m, stats=False, stream=None):
        """Steps 1-4 for every box; fills self.phiN and self.phi."""
        if self.ctx_mond is not None:
            return self._potentials_concurrent(x, y, z, m, stats, stream)
        c = self.ctx
        ns, ms = [], []

        def timed(call):
            if self.solve_events is None:
                return call()
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record(stream)
            out = call()
            ev[1].record(stream)
            self.solve_events.append(ev)
            return out

        for b in range(c.params.nboxes):
            c.qumond_deposit(b, x, y, z, m, self.rho_fixed, self.rho, stream=stream)
            if b == 0 and self.far_field:
                c.qumond_far_field(self.rho, self.phiN[0], self.phi[0], stream=stream)
            par_n = self.phiN[b - 1] if b > 0 else None
            par_m = self.phi[b - 1] if b > 0 else None
            ns.append(timed(lambda: c.qumond_solve_newton(b, self.rho, par_n, self.phiN[b], stats=stats,
                                                          stream=stream)))
            c.qumond_source(b, self.phiN[b], self.src, stream=stream)
            if self.guess is not None:
                self.guess.qumond_guess_apply(self.rho_scale(b), float(b > 0), self.rho, self.phiN[b], self.phi[b],
                                              stream=stream)
                ms.append(timed(lambda: self.ctx_warm.qumond_solve_mond(b, self.src, par_m, self.phi[b], stats=stats,
                                                                        stream=stream)))
            else:
                ms.append(timed(lambda: c.qumond_solve_mond(b, self.src, par_m, self.phi[b], stats=stats,
                                                            stream=stream)))
        return ns, ms

    def rho_scale(self, b):
        """Density channel scale of the network for box b: 4 pi G h_b^2 / phi_scale."""
        p = self.ctx.params
        h = self.ctx.box_side(b) / p.n
        return 4.0 * math.pi * p.G * h * h / self.guess.phi_scale

    def _potentials_concurrent(self, x, y, z, m, stats, stream):
        caller = stream if stream is not None else torch.cuda.current_stream(self.device)
        sa, sb = self._streams
        nb = self.ctx.params.nboxes
        start = torch.cuda.Event()
        start.record(caller)
        sa.wait_event(start)
        sb.wait_event(start)
        ready = [threading.Event() for _ in range(nb)]
        src_done = [torch.cuda.Event() for _ in range(nb)]
        failed = []

        def mond_chain():
            out = []
            with torch.cuda.device(self.device):
                for b in range(nb):
                    ready[b].wait()
                    if failed:
                        return out
                    sb.wait_event(src_done[b])
                    par = self.phi[b - 1] if b > 0 else None
                    out.append(self.ctx_mond.qumond_solve_mond(b, self.srcs[b], par, self.phi[b], stats=stats,
                                                               stream=sb))
            return out

        fut = self._pool.submit(mond_chain)
        ns = []
        try:
            for b in range(nb):
                self.ctx.qumond_deposit(b, x, y, z, m, self.rho_fixed, self.rho, stream=sa)
                if b == 0 and self.far_field:  # before src_done[0], which the QUMOND chain waits for
                    self.ctx.qumond_far_field(self.rho, self.phiN[0], self.phi[0], stream=sa)
                par = self.phiN[b - 1] if b > 0 else None
                ns.append(self.ctx.qumond_solve_newton(b, self.rho, par, self.phiN[b], stats=stats, stream=sa))
                self.ctx.qumond_source(b, self.phiN[b], self.srcs[b], stream=sa)
                src_done[b].record(sa)
                ready[b].set()
        except Exception:
            failed.append(True)
            for e in ready:
                e.set()
            fut.result()
            raise
        ms = fut.result()
        end_a, end_b = torch.cuda.Event(), torch.cuda.Event()
        end_a.record(sa)
        end_b.record(sb)
        caller.wait_event(end_a)
        caller.wait_event(end_b)
        return ns, ms

    def run_many(self, inputs, *, nbins=50, rmax=30000.0, nphi=64, forces=None, stream=None, ready=None):
        """The whole path (as run()) for a sequence of evaluations, one (x, y,
        z, m) tuple of device tensors each, with the two chains pipelined
        across evaluations: the Newtonian chain of evaluation i+1 (deposits,
        far field, Newtonian solves, sources) runs while the QUMOND chain
        finishes evaluation i (its QUMOND solves, then the forces and the
        rotation curve, which this form runs on the QUMOND chain's context and
        stream).  Every evaluation runs the kernels of run() in the same order
        on the same data, so its results are the same bits.

        Ordering between the chains, with CUDA events: the source of box b of
        evaluation i+1 waits for the QUMOND solve of box b of evaluation i
        (they share the source buffer); with the far-field boundary, box 0's
        potential alternates between two buffers, and the far field of
        evaluation i+2 waits until evaluation i's forces and curve are done.
        forces: None, or one (gx, gy, gz) tuple per evaluation.  ready: None,
        or one CUDA event (or None) per evaluation that its first kernel waits
        for, e.g. the end of the copy of its particles on another stream, so
        that copies overlap the evaluations before it.  Needs two contexts
        (ctx_mond).  Returns one PipelineResult per evaluation (r, vc, and
        `done`, an event recorded once its forces and curve are written; no
        solve statistics)."""
        if self.ctx_mond is None:
            raise ValueError("run_many pipelines the two chains: it needs ctx_mond")
        if self.guess is not None:
            raise ValueError("the learned guess runs in the sequential order only")
        nev = len(inputs)
        if forces is not None and len(forces) != nev:
            raise ValueError("need one forces tuple per evaluation")
        if ready is not None and len(ready) != nev:
            raise ValueError("need one ready event (or None) per evaluation")
        nb = self.ctx.params.nboxes
        dev = self.device
        caller = stream if stream is not None else torch.cuda.current_stream(dev)
        sa, sb = self._streams
        if self.far_field and not hasattr(self, "_phi0_alt"):
            self._phi0_alt = torch.zeros_like(self.phi[0])
        phi0 = [self.phi[0], getattr(self, "_phi0_alt", self.phi[0])]
        results = [PipelineResult(torch.empty(nbins * self.ctx.nsets, dtype=torch.float64, device=dev),
                                  torch.empty(nbins * self.ctx.nsets, dtype=torch.float64, device=dev))
                   for _ in range(nev)]
        start = torch.cuda.Event()
        start.record(caller)
        sa.wait_event(start)
        sb.wait_event(start)
        src_done = [[torch.cuda.Event() for _ in range(nb)] for _ in range(nev)]
        mond_done = [[torch.cuda.Event() for _ in range(nb)] for _ in range(nev)]
        eval_done = [torch.cuda.Event() for _ in range(nev)]
        handoff = [[threading.Event() for _ in range(nb)] for _ in range(nev)]
        mond_rec = [[threading.Event() for _ in range(nb)] for _ in range(nev)]
        eval_rec = [threading.Event() for _ in range(nev)]
        failed = []

        def phis_of(i):
            return [phi0[i % 2] if self.far_field else self.phi[0]] + self.phi[1:]

        def mond_chain():
            with torch.cuda.device(dev):
                try:
                    for i in range(nev):
                        phis = phis_of(i)
                        for b in range(nb):
                            handoff[i][b].wait()
                            if failed:
                                return
                            sb.wait_event(src_done[i][b])
                            self.ctx_mond.qumond_solve_mond(b, self.srcs[b], phis[b - 1] if b > 0 else None, phis[b],
                                                            stream=sb)
                            mond_done[i][b].record(sb)
                            mond_rec[i][b].set()
                        x, y, z, _ = inputs[i]
                        if forces is not None:
                            self.ctx_mond.qumond_forces(phis, x, y, z, *forces[i], stream=sb)
                        self.ctx_mond.qumond_rotation_curve(phis, nbins, rmax, nphi, results[i].r, results[i].vc,
                                                            stream=sb)
                        eval_done[i].record(sb)
                        eval_rec[i].set()
                except Exception:
                    failed.append(True)
                    for ev in [e for row in mond_rec for e in row] + eval_rec:
                        ev.set()
                    raise

        fut = self._pool.submit(mond_chain)
        try:
            for i in range(nev):
                x, y, z, m = inputs[i]
                phis = phis_of(i)
                if ready is not None and ready[i] is not None:
                    sa.wait_event(ready[i])
                for b in range(nb):
                    self.ctx.qumond_deposit(b, x, y, z, m, self.rho_fixed, self.rho, stream=sa)
                    if b == 0 and self.far_field:
                        if i >= 2:  # box 0's potential buffer of evaluation i-2 is free once its forces and curve are
                            eval_rec[i - 2].wait()
                            if failed:
                                break
                            sa.wait_event(eval_done[i - 2])
                        self.ctx.qumond_far_field(self.rho, self.phiN[0], phis[0], stream=sa)
                    par = self.phiN[b - 1] if b > 0 else None
                    self.ctx.qumond_solve_newton(b, self.rho, par, self.phiN[b], stream=sa)
                    if i >= 1:  # the source buffer of box b is free once evaluation i-1's QUMOND solve has read it
                        mond_rec[i - 1][b].wait()
                        if failed:
                            break
                        sa.wait_event(mond_done[i - 1][b])
                    self.ctx.qumond_source(b, self.phiN[b], self.srcs[b], stream=sa)
                    src_done[i][b].record(sa)
                    handoff[i][b].set()
                if failed:
                    break
        except Exception:
            failed.append(True)
            for row in handoff:
                for e in row:
                    e.set()
            try:
                fut.result()
            except Exception:
                pass
            raise
        if failed:
            for row in handoff:
                for e in row:
                    e.set()
        fut.result()  # re-raises the QUMOND chain's error
        end_a, end_b = torch.cuda.Event(), torch.cuda.Event()
        end_a.record(sa)
        end_b.record(sb)
        caller.wait_event(end_a)
        caller.wait_event(end_b)
        if self.far_field and nev % 2 == 0:  # self.phi holds the last evaluation's potentials
            self.phi[0], self._phi0_alt = self._phi0_alt, self.phi[0]
        for res, ev in zip(results, eval_done):
            res.done = ev
        return results

    def run(self, x, y, z, m, *, nbins=50, rmax=30000.0, nphi=64, forces=None, stats=False, stream=None):
        """The whole path: potentials, then forces at (x, y, z) into `forces`
        (a tuple gx, gy, gz of tensors, or None to skip) and the rotation curve."""
        ns, ms = self.potentials(x, y, z, m, stats=stats, stream=stream)
        if forces is not None:
            self.ctx.qumond_forces(self.phi, x, y, z, *forces, stream=stream)
        r = torch.empty(nbins * self.ctx.nsets, dtype=torch.float64, device=self.device)
        vc = torch.empty(nbins * self.ctx.nsets, dtype=torch.float64, device=self.device)
        self.ctx.qumond_rotation_curve(self.phi, nbins, rmax, nphi, r, vc, stream=stream)
        return PipelineResult(r, vc, ns, ms)


def run_lanes(pipes, inputs, *, nbins=50, rmax=30000.0, nphi=64, forces=None, ready=None, stream=None):
    """Independent evaluations spread over several pipelines ("lanes", each
    with its own two contexts, buffers and streams) that run concurrently on
    the device: evaluation i goes to pipes[i % len(pipes)], and each lane
    pipelines its share as run_many does, from its own host thread (a solve
    call returns once its statistics are read, so every lane needs one).
    Each evaluation runs the kernels of run() on its own lane's buffers, so
    its results are the same bits.  forces / ready: as in run_many, one per
    evaluation (forces tuples of evaluations that run concurrently must be
    distinct).  Results in input order; every lane's work is ordered before
    later work on `stream` (the caller's current stream by default)."""
    nl = len(pipes)
    nev = len(inputs)
    caller = stream if stream is not None else torch.cuda.current_stream(pipes[0].device)
    results = [None] * nev
    errors = []
    # each lane starts after the caller's earlier work and ends on a stream of its own, which the caller waits
    # for once every lane is enqueued (a lane's end must not hold up another lane's start)
    start = torch.cuda.Event()
    start.record(caller)
    lane_streams = []
    for pp in pipes:
        if not hasattr(pp, "_lane_stream"):
            pp._lane_stream = torch.cuda.Stream(pp.device)
        pp._lane_stream.wait_event(start)
        lane_streams.append(pp._lane_stream)

    def lane(k):
        idx = list(range(k, nev, nl))
        if not idx:
            return
        try:
            with torch.cuda.device(pipes[k].device):
                rs = pipes[k].run_many([inputs[i] for i in idx], nbins=nbins, rmax=rmax, nphi=nphi,
                                       forces=None if forces is None else [forces[i] for i in idx],
                                       ready=None if ready is None else [ready[i] for i in idx],
                                       stream=lane_streams[k])
            for i, r in zip(idx, rs):
                results[i] = r
        except Exception as exc:  # re-raised in the calling thread
            errors.append(exc)

    threads = [threading.Thread(target=lane, args=(k,), name="qumond-lane-%d" % k) for k in range(1, nl)]
    for t in threads:
        t.start()
    lane(0)
    for t in threads:
        t.join()
    for ls in lane_streams:
        caller.wait_stream(ls)
    if errors:
        raise errors[0]
    return results
