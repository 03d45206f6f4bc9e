"""Rotation-curve fit sweep (Section 3.5): many parameter sets of one galaxy,
each run through the whole QUMOND path, scored by reduced chi^2 against an
observed curve.

The sets are independent, so they run side by side: `workers` contexts,
each with its own buffers and CUDA stream and driven by its own host thread,
take sets w, w + workers, w + 2 workers, ...  Every solve of a context is one
cached CUDA graph launch; one solve on 129^3 spends most of its time on
multigrid levels far too small to fill 152 SMs, and the other workers' solves
fill the rest.  Each set's kernels and their order are those of a single
pipeline on its own, so a set's rotation curve is the same bits whatever the
number of workers.  The rotation curve of set s is sampled at radii scaled by
that set's distance factor (the observed radii are fixed angles), written to
row s of one array, and one kernel computes every set's chi^2 at the end.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
from dataclasses import dataclass

import torch

from .pipeline import Pipeline
from .qumond import Context, qumond_params


@dataclass
class SweepResult:
    r: torch.Tensor      # nsets x nbins radii (pc)
    vc: torch.Tensor     # nsets x nbins circular speeds (km/s)
    chi2: torch.Tensor   # nsets reduced chi^2
    stats: list          # per set: [(newton SolveStats, mond SolveStats) per box], or None


class FitSweep:
    def __init__(self, params: qumond_params, *, nbins: int, rmax: float, nphi: int = 64, workers: int = 8,
                 device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.nbins, self.rmax, self.nphi = int(nbins), float(rmax), int(nphi)
        self.workers = int(workers)
        if self.workers < 1:
            raise ValueError("workers must be >= 1")
        with torch.cuda.device(self.device):
            self.ctxs = [Context(_copy(params)) for _ in range(self.workers)]
            self.pipes = [Pipeline(c, self.device) for c in self.ctxs]
            self.streams = [torch.cuda.Stream(self.device) for _ in range(self.workers)]
        self._pool = cf.ThreadPoolExecutor(max_workers=self.workers, thread_name_prefix="qumond-sweep")

    def close(self):
        self._pool.shutdown(wait=True)
        for c in self.ctxs:
            c.close()
        self.ctxs, self.pipes = [], []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, particles, distance, v_obs, sigma, *, stats=False, stream=None) -> SweepResult:
        """particles: one (x, y, z, m) tuple of device float64 tensors per set;
        distance: the sets' distance factors (the rotation curve of set s spans
        distance[s] * rmax); v_obs, sigma: the observed curve (device, nbins)."""
        nsets = len(particles)
        if len(distance) != nsets:
            raise ValueError("need one distance factor per set")
        dev = self.device
        caller = stream if stream is not None else torch.cuda.current_stream(dev)
        r = torch.empty(nsets, self.nbins, dtype=torch.float64, device=dev)
        vc = torch.empty(nsets, self.nbins, dtype=torch.float64, device=dev)
        chi2 = torch.empty(nsets, dtype=torch.float64, device=dev)
        start = torch.cuda.Event()
        start.record(caller)
        out_stats = [None] * nsets

        def work(w):
            with torch.cuda.device(dev):
                st = self.streams[w]
                st.wait_event(start)
                pipe, ctx = self.pipes[w], self.ctxs[w]
                for s in range(w, nsets, self.workers):
                    x, y, z, m = particles[s]
                    ns, ms = pipe.potentials(x, y, z, m, stats=stats, stream=st)
                    ctx.qumond_rotation_curve(pipe.phi, self.nbins, self.rmax * float(distance[s]), self.nphi,
                                              r[s], vc[s], stream=st)
                    if stats:
                        out_stats[s] = list(zip(ns, ms))
                done = torch.cuda.Event()
                done.record(st)
                return done

        futs = [self._pool.submit(work, w) for w in range(min(self.workers, nsets))]
        events = [f.result() for f in futs]  # re-raises a worker's error
        for e in events:
            caller.wait_event(e)
        if nsets:
            self.ctxs[0].qumond_chi2(vc, v_obs, sigma, chi2, stream=caller)
        return SweepResult(r, vc, chi2, out_stats if stats else None)


def _copy(p: qumond_params) -> qumond_params:
    q = qumond_params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(p))
    return q


def tune_workers(params: qumond_params, particles, distance, v_obs, sigma, *, nbins: int, rmax: float, nphi: int = 64,
                 candidates=(4, 8, 16, 24, 32), repeats: int = 2, device=None):
    """Picks the number of concurrent workers by timing: each candidate runs
    the given sweep once untimed (graph capture) and `repeats` times timed
    with CUDA events.  Results do not depend on the choice (each set's
    kernels are the same), only the time does.  Returns (best, {workers: ms})."""
    times = {}
    for k in candidates:
        if k > max(1, len(particles)):
            continue
        with FitSweep(params, nbins=nbins, rmax=rmax, nphi=nphi, workers=k, device=device) as sw:
            sw.run(particles, distance, v_obs, sigma)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record()
            for _ in range(repeats):
                sw.run(particles, distance, v_obs, sigma)
            t1.record()
            t1.synchronize()
            times[k] = t0.elapsed_time(t1) / repeats
        torch.cuda.empty_cache()
    best = min(times, key=times.get)
    return best, times
