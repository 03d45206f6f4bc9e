"""Rotation-curve fit sweep (Section 3.5): many parameter sets of one galaxy,
each run through the whole QUMOND path, scored by reduced chi^2 against an
observed curve.

The sets are independent problems of one shape (same grid and boxes,
different particles), so they are batched: a context with nsets = `batch`
holds a chunk of sets, and every kernel of the path is ONE launch for the
whole chunk (the set index is a grid dimension) -- the deposit, both solves
of every box (each a CUDA graph whose defect-correction loop runs until the
last set of the chunk has converged, converged sets being skipped), the
source and the rotation curve.  `lanes` such contexts run side by side, each
with its own stream and host thread, taking chunks lane, lane + lanes, ...;
the last chunk is padded with copies of its last set, whose results are
dropped.  Every set's kernels do that set's arithmetic in the same order as
a lone pipeline would, so a set's rotation curve is the same bits for any
batch size and number of lanes.  The rotation curve of set s is sampled at
radii scaled by that set's distance factor (the observed radii are fixed
angles) and one kernel computes every set's chi^2 at the end.

`autotune` picks the batch size, the number of lanes and the block shape of
the small-level kernels (params.tile_small), the form of the small-level
V-cycle (params.persistent_vcycle) and the V-cycles per defect-correction
step (params.dc_vcycles) by timing the sweep itself.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import itertools
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
    def __init__(self, params: qumond_params, *, nbins: int, rmax: float, nphi: int = 64, batch: int = 64,
                 lanes: int = 1, workers: int | None = None, device=None):
        """batch: sets per context (one launch per kernel covers them); lanes:
        contexts run side by side.  workers=K is the unbatched form: batch 1,
        K lanes."""
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.nbins, self.rmax, self.nphi = int(nbins), float(rmax), int(nphi)
        if workers is not None:
            batch, lanes = 1, int(workers)
        self.batch, self.lanes = int(batch), int(lanes)
        if self.batch < 1 or self.lanes < 1:
            raise ValueError("batch and lanes must be >= 1")
        with torch.cuda.device(self.device):
            p = _copy(params)
            p.nsets = self.batch
            self.ctxs = [Context(_copy(p)) for _ in range(self.lanes)]
            self.pipes = [Pipeline(c, self.device) for c in self.ctxs]
            self.streams = [torch.cuda.Stream(self.device) for _ in range(self.lanes)]
        self._pool = cf.ThreadPoolExecutor(max_workers=self.lanes, thread_name_prefix="qumond-sweep")

    @property
    def workers(self) -> int:
        return self.lanes

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
        """particles: one (x, y, z, m) tuple of device float64 tensors per set
        (the same count in every set), or one tuple of tensors holding every
        set's particles set after set; distance: the sets' distance factors
        (the rotation curve of set s spans distance[s] * rmax); v_obs, sigma:
        the observed curve (device, nbins)."""
        nsets = len(distance)
        stacked = isinstance(particles, tuple) and len(particles) == 4 and torch.is_tensor(particles[0])
        if not stacked and len(particles) != nsets:
            raise ValueError("need one distance factor per set")
        if stacked and particles[0].numel() % max(nsets, 1):
            raise ValueError("the stacked particle arrays must hold the same count for every set")
        np_set = (particles[0].numel() // max(nsets, 1)) if stacked else (particles[0][0].numel() if nsets else 0)
        if not stacked and any(p[0].numel() != np_set for p in particles):
            raise ValueError("every set must have the same number of particles (pad with particles outside the box)")
        dev = self.device
        B, K = self.batch, self.lanes
        caller = stream if stream is not None else torch.cuda.current_stream(dev)
        r = torch.empty(nsets, self.nbins, dtype=torch.float64, device=dev)
        vc = torch.empty(nsets, self.nbins, dtype=torch.float64, device=dev)
        chi2 = torch.empty(nsets, dtype=torch.float64, device=dev)
        nchunks = (nsets + B - 1) // B
        members = [[min(c * B + i, nsets - 1) for i in range(B)] for c in range(nchunks)]
        rmax_sets = torch.tensor([self.rmax * float(distance[s]) for mem in members for s in mem],
                                 dtype=torch.float64, device=dev)
        start = torch.cuda.Event()
        start.record(caller)
        out_stats = [None] * nsets

        def chunk_particles(c):
            mem = members[c]
            full = mem[-1] == c * B + B - 1
            if stacked and full:  # a contiguous run of sets: a view, no copy
                return tuple(a[c * B * np_set:(c + 1) * B * np_set] for a in particles)
            if stacked:
                return tuple(torch.cat([a[s * np_set:(s + 1) * np_set] for s in mem]) for a in particles)
            if B == 1:
                return particles[mem[0]]
            return tuple(torch.cat([particles[s][k] for s in mem]) for k in range(4))

        def work(lane):
            with torch.cuda.device(dev):
                st = self.streams[lane]
                st.wait_event(start)
                pipe, ctx = self.pipes[lane], self.ctxs[lane]
                with torch.cuda.stream(st):
                    for c in range(lane, nchunks, K):
                        x, y, z, m = chunk_particles(c)
                        ns, ms = pipe.potentials(x, y, z, m, stats=stats, stream=st)
                        n_real = min(B, nsets - c * B)
                        if n_real == B:
                            rr, vv = r[c * B:(c + 1) * B], vc[c * B:(c + 1) * B]
                        else:
                            rr = torch.empty(B, self.nbins, dtype=torch.float64, device=dev)
                            vv = torch.empty_like(rr)
                        ctx.qumond_rotation_curve_sets(pipe.phi, self.nbins, rmax_sets[c * B:(c + 1) * B], self.nphi,
                                                       rr, vv, stream=st)
                        if n_real < B:
                            r[c * B:].copy_(rr[:n_real])
                            vc[c * B:].copy_(vv[:n_real])
                        if stats:
                            for i in range(n_real):
                                pick = (lambda a: a) if B == 1 else (lambda a: a[i])
                                out_stats[c * B + i] = [(pick(a), pick(b)) for a, b in zip(ns, ms)]
                done = torch.cuda.Event()
                done.record(st)
                return done

        futs = [self._pool.submit(work, w) for w in range(min(K, nchunks))]
        events = [f.result() for f in futs]  # re-raises a lane's error
        for e in events:
            caller.wait_event(e)
        if nsets:
            self.ctxs[0].qumond_chi2(vc, v_obs, sigma, chi2, stream=caller)
        return SweepResult(r, vc, chi2, out_stats if stats else None)


def _copy(p: qumond_params) -> qumond_params:
    q = qumond_params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(p))
    return q


def autotune(params: qumond_params, particles, distance, v_obs, sigma, *, nbins: int, rmax: float, nphi: int = 64,
             batches=(8, 16, 32, 64), lanes=(1, 2, 4), tiles=(0, 1, 2), forms=(3, 0), dcs=(2, 3, 4), repeats: int = 2,
             device=None):
    """Picks the batch size, the number of lanes, the small-level block shape
    (params.tile_small), the form of the small-level V-cycle
    (params.persistent_vcycle: 3, one cluster per set holding the level n = 32
    in shared memory, or 0, one launch per step) and the V-cycles per
    defect-correction step (params.dc_vcycles) by timing: each candidate runs
    the given sweep once untimed (graph capture) and `repeats` times timed
    with CUDA events.  Batch and lanes are searched with params' own form and
    dc_vcycles and tile 0, the block shape at the best (batch, lanes), the
    form at the best of those, dc_vcycles last.  Batch, lanes, block shape and
    form do not change any set's results (each set's arithmetic is the same);
    dc_vcycles changes how many V-cycles a set makes before its residual meets
    the same tolerance.  Returns ({"batch", "lanes", "tile_small",
    "persistent_vcycle", "dc_vcycles"}, {(batch, lanes, tile, form, dc): ms})."""
    nsets = len(distance)
    times = {}
    form0 = params.persistent_vcycle
    dc0 = params.dc_vcycles

    def time_one(b, k, tile, form, dc):
        p = _copy(params)
        p.tile_small = tile
        p.persistent_vcycle = form
        p.dc_vcycles = dc
        with FitSweep(p, nbins=nbins, rmax=rmax, nphi=nphi, batch=b, lanes=k, device=device) as sw:
            sw.run(particles, distance, v_obs, sigma)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record()
            for _ in range(repeats):
                sw.run(particles, distance, v_obs, sigma)
            t1.record()
            t1.synchronize()
            ms = t0.elapsed_time(t1) / repeats
        torch.cuda.empty_cache()
        return ms

    for b, k in itertools.product(batches, lanes):
        if b > max(1, nsets) or (k > 1 and b * k > max(1, nsets) + b - 1):
            continue  # more lanes than chunks
        times[(b, k, 0, form0, dc0)] = time_one(b, k, 0, form0, dc0)
    b0, k0, _, _, _ = min(times, key=times.get)
    for tile in tiles:
        if (b0, k0, tile, form0, dc0) not in times:
            times[(b0, k0, tile, form0, dc0)] = time_one(b0, k0, tile, form0, dc0)
    _, _, t0, _, _ = min(times, key=times.get)
    for form in forms:
        if (b0, k0, t0, form, dc0) not in times:
            times[(b0, k0, t0, form, dc0)] = time_one(b0, k0, t0, form, dc0)
    _, _, _, f0, _ = min(times, key=times.get)
    for dc in dcs:
        if (b0, k0, t0, f0, dc) not in times:
            times[(b0, k0, t0, f0, dc)] = time_one(b0, k0, t0, f0, dc)
    best = min(times, key=times.get)
    return {"batch": best[0], "lanes": best[1], "tile_small": best[2], "persistent_vcycle": best[3],
            "dc_vcycles": best[4]}, times


def tune_workers(params: qumond_params, particles, distance, v_obs, sigma, *, nbins: int, rmax: float, nphi: int = 64,
                 candidates=(4, 8, 16, 24, 32), repeats: int = 2, device=None):
    """The unbatched form's choice: the number of one-set contexts run side by
    side.  Returns (best, {workers: ms})."""
    times = {}
    for k in candidates:
        if k > max(1, len(distance)):
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
