#!/usr/bin/env python
"""Throughput of the QUMOND particle-mesh path on GB300.

One step = one evaluation of the whole path for one galaxy: for each of the
3 nested boxes (120, 60, 30 kpc; 257^3 nodes each) the CIC deposit of 2e6
particles (box 0's outer boundary from the far field of its mass), the
Newtonian FMG solve, the QUMOND source and the QUMOND FMG solve (FP32
smoothing with defect correction to a relative residual of 1e-10, on a 64-bit
fixed-point iterate by default, in FP64 with --precision mixed), then the
forces at every particle and a 50-bin rotation curve.  The metric is QUMOND
solves per second (one solve = one such step); successive steps run with the
two solve chains pipelined across them (Pipeline.run_many), dealt to 1, 2 or
3 lanes of such pipelines (run_lanes), whichever a short timing picks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own replica of the workload (independent
galaxies; no data-path collective), the timed region is bracketed by a
barrier and a device synchronise, the maximum time over ranks is taken, and
rank 0 prints one JSON line.  --impl reference times the FP64 CPU oracle on
the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "QUMOND solves/sec and cell-updates/s at 256^3 (HBM % of peak) vs plain FMG"
PRECISION_NAMES = {
    "mixed": "FP32 smoothing + FP64 defect correction",
    "fixed": "FP32 smoothing + defect correction on a 64-bit fixed-point iterate (exact integer residual)",
    "fp64": "FP64 throughout",
}
UNIT = "solves/s"

WORKLOADS = {
    # the metric's configuration: 256^3 intervals, 3 nested boxes, two-disk galaxy
    # box 0's boundary: the far field of its own mass (multipole expansion to degree 8 for Phi_N, the point-mass
    # QUMOND potential of the total mass for Phi): the 120 kpc outer box is far smaller than the 2^10 x galaxy
    # box on which Section 2 sets Phi = 0
    "two-disk": dict(n=256, nboxes=3, L0=120000.0, particles=2_000_000, seed=1, rel_tol=1e-10, max_vcycles=40,
                     ncycle=1, npre=2, npost=2, nbins=50, rmax=30000.0, nphi=64, kind="two-disk", bc="multipole"),
    # the large grid: 512^3 intervals, 4 nested boxes (240/120/60/30 kpc), disks + Hernquist bulge
    "large": dict(n=512, nboxes=4, L0=240000.0, particles=20_000_000, seed=1, rel_tol=1e-10, max_vcycles=40,
                  ncycle=1, npre=2, npost=2, nbins=50, rmax=30000.0, nphi=64, kind="large", bc="multipole"),
}
# the fit sweep (Section 3.5): 64 parameter sets of the two-disk galaxy, 129^3 nodes x 2 boxes (80/40 kpc),
# 5e5 particles each, chi^2 against the oracle-made target curve; one step = the whole sweep
SWEEP = dict(n=128, nboxes=2, L0=80000.0, particles=500_000, galaxy_seed=11, sets=64, param_seed=2012,
             rel_tol=1e-8, max_vcycles=40, ncycle=1, npre=2, npost=2, nbins=40, rmax=24000.0, nphi=64, kind="sweep",
             target="tests/golden/sweep_target_two_disk_129cube.json")
WORKLOADS["sweep"] = SWEEP
# the learned initial guess: two-disk galaxies (stellar h in [0.3, 0.6] kpc) on 129^3 x 2 boxes (80/40 kpc),
# 2e5 particles; one step = the whole path of one galaxy with the QUMOND solves started from the network's
# guess, solves to rel. residual 1e-8
LEARNED = dict(n=128, nboxes=2, L0=80000.0, particles=200_000, galaxies=8, seed=7919, rel_tol=1e-8, max_vcycles=60,
               ncycle=1, npre=2, npost=2, nbins=40, rmax=24000.0, nphi=64, kind="learned")
WORKLOADS["learned"] = LEARNED
WORKLOAD = dict(WORKLOADS["two-disk"])


def workload_config(precision="FP32 smoothing + FP64 defect correction"):
    w = WORKLOAD
    sides = "/".join("%g" % (w["L0"] / 1000.0 / 2 ** b) for b in range(w["nboxes"]))
    galaxy = ("two-disk galaxy (stellar exponential disk Sigma0=500 Msun/pc^2, R_d=3 kpc, sech^2 h_* drawn in "
              "[0.3,0.6] kpc; gas disk 1e9 Msun, R_g=8 kpc, h_g=0.1 kpc)")
    if w["kind"] == "large":
        galaxy = ("stellar + gas exponential disks as the two-disk galaxy plus a Hernquist bulge (M_b=1e10 Msun, "
                  "a_b=0.5 kpc), a third of the particles each")
    return {
        "workload": "%s, %d particles, %d^3 nodes x %d nested boxes of %s kpc" % (galaxy, w["particles"], w["n"] + 1,
                                                                                   w["nboxes"], sides),
        "n_intervals": w["n"],
        "boxes_kpc": [w["L0"] / 1000.0 / 2 ** b for b in range(w["nboxes"])],
        "particles": w["particles"],
        "precision": precision,
        "rel_tol": w["rel_tol"],
        "fmg_vcycles_per_level": w["ncycle"],
        "npre_npost": [w["npre"], w["npost"]],
        "rotation_curve": "%d bins to %g kpc, %d azimuths" % (w["nbins"], w["rmax"] / 1000.0, w["nphi"]),
        "outer_boundary": ("far field of box 0's mass: multipole expansion to degree 8 (Phi_N), point-mass QUMOND "
                           "potential of the total mass (Phi)") if w.get("bc") == "multipole" else "Phi = 0",
        "seed": w["seed"],
        "l2": "inputs larger than L2: each 257^3 FP64 grid is 136 MB and one step streams tens of GB",
        "data": "synthetic (seeded generator)",
    }


def sweep_config(precision, choice):
    w = WORKLOAD
    return {
        "workload": "fit sweep: %d parameter sets (distance scale 0.8-1.2, stellar M/L 0.3-1.2, stellar h 0.2-1.0 kpc, "
                    "gas h 0.05-0.5 kpc; uniform, seed %d) of the two-disk galaxy (stellar disk I0=500 Lsun/pc^2, "
                    "R_d=3 kpc; gas 1e9 Msun, R_g=8 kpc), %d particles per set, %d^3 nodes x %d nested boxes of "
                    "%g/%g kpc, reduced chi^2 of each %d-bin rotation curve against a synthetic target with 3%% "
                    "Gaussian errors" % (w["sets"], w["param_seed"], w["particles"], w["n"] + 1, w["nboxes"],
                                         w["L0"] / 1000.0, w["L0"] / 2000.0, w["nbins"]),
        "sets_per_step": w["sets"],
        "n_intervals": w["n"],
        "particles_per_set": w["particles"],
        "precision": precision,
        "rel_tol": w["rel_tol"],
        "fmg_vcycles_per_level": w["ncycle"],
        "npre_npost": [w["npre"], w["npost"]],
        "batched_form": choice,
        "rotation_curve": "%d bins to %g kpc x distance factor, %d azimuths" % (w["nbins"], w["rmax"] / 1000.0,
                                                                                w["nphi"]),
        "l2": "inputs larger than L2: 64 sets x 5e5 particles x 32 B = 1 GB of particles, ~10 GB of grids per step",
        "data": "synthetic (seeded generator; target curve written by the oracle)",
    }


def make_particles():
    import synth
    w = WORKLOAD
    lim = 0.45 * w["L0"]
    if w["kind"] == "large":
        return synth.large_galaxy(w["particles"], seed=w["seed"], rmax=lim)
    return synth.two_component_disk(w["particles"], seed=w["seed"], rmax=lim, zmax=lim)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# --- clocks -------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "qumond_clocks_rank%d_%d.csv" % (index, os.getpid()))

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((int(f[0]), float(f[1]), float(f[2]), float(f[3]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        idx = self.index if any(r[0] == self.index for r in rows) else rows[0][0]
        rows = [r for r in rows if r[0] == idx]
        loaded = [r for r in rows if r[3] > 0.3 * max(x[3] for x in rows)] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in loaded for q, v in enumerate(r[4]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in loaded), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": reasons, "samples": len(loaded)}


# --- roofline helpers ------------------------------------------------------------
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def ncu_traffic(kernel: str, n: int, nsets: int = 1):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when there is none, it was taken on another grid size or number of
    sets (the write-back share depends on how much of a launch stays in L2),
    or the kernel's source file changed since."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    except (OSError, ValueError):
        return None
    k = t.get("kernels", {}).get(kernel)
    if not k or k.get("n") != n or k.get("nsets", 1) != nsets:
        return None
    src = os.path.join(ROOT, k["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != k.get("source_hash"):
        return None
    return k.get("dram_bytes_per_launch_full_size")


# kernel classes that belong to the solves (everything but the deposit, the source and the post-processing)
NOT_SOLVE = {"cic_deposit", "fixed_to_rho", "qumond_source", "forces", "rotation_curve", "chi2", "profile",
             "far_field"}


def solve_roofline(pipe1, ctx1, step, steps, peak, barrier, max_over_ranks):
    """Time every solve of `steps` whole steps run with one chain (the pipeline
    records a CUDA event pair around each solve call on its stream) and relate
    the solves' algorithmic bytes (the tracer's per-class counts of the solve
    kernels) to their summed event time."""
    import torch
    ctx1.qumond_trace_read(reset=True)
    pipe1.solve_events = []
    barrier()
    for _ in range(steps):
        step(pipe1)
    torch.cuda.synchronize()
    events, pipe1.solve_events = pipe1.solve_events, None
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in events))
    st, _, _ = ctx1.qumond_trace_read(reset=True)
    nbytes = sum(k.bytes for name, k in st.items() if name not in NOT_SOLVE)
    achieved = nbytes / ms / 1e6
    return {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "solves": len(events), "ms_per_solve": ms / len(events), "algorithmic_bytes_per_solve": nbytes / len(events),
            "timing": "CUDA events on the solve's stream around each qumond_solve_newton / qumond_solve_mond call "
                      "(boundary values, FMG, defect correction to the tolerance, output) over %d steps run with "
                      "one chain (no concurrent solve); bytes = the algorithmic bytes of the solve kernels" % steps}


class Contexts:
    """The contexts of a pipeline, read and driven as one (tracer counters merged)."""

    def __init__(self, ctxs):
        self.ctxs = ctxs

    def qumond_trace_timing(self, on, only=None):
        for c in self.ctxs:
            c.qumond_trace_timing(on, only=only)

    def qumond_trace_read(self, reset=False):
        merged, launches, cells = {}, 0, 0
        for c in self.ctxs:
            st, l, cu = c.qumond_trace_read(reset=reset)
            launches += l
            cells += cu
            for name, k in st.items():
                if name in merged:
                    a = merged[name]
                    a.launches += k.launches
                    a.bytes += k.bytes
                    a.ms += k.ms
                    a.timed += k.timed
                    a.timed_bytes += k.timed_bytes
                else:
                    merged[name] = k
        return merged, launches, cells

    def close(self):
        for c in self.ctxs:
            c.close()


# --- our arm -------------------------------------------------------------------------
def run_ours(args):
    import torch

    import paper_1201_3185_gb300 as q

    from paper_1201_3185_gb300.replicas import Replicas
    rep = Replicas.from_env()
    ws, rank, local = rep.world_size, rep.rank, rep.local_rank
    dev = rep.device
    barrier = rep.barrier
    max_over_ranks = rep.max

    w = WORKLOAD
    p = make_particles()
    prec = {"fp64": q.QUMOND_PREC_FP64, "mixed": q.QUMOND_PREC_MIXED, "fixed": q.QUMOND_PREC_MIXED_FIXED}[args.precision]

    def new_pipeline(precision):
        """A pipeline and its contexts: with two chains, the QUMOND solves run on their
        own context and stream, concurrently with the next box's Newtonian solve."""
        def make():
            return q.Context(n=w["n"], nboxes=w["nboxes"], L0=w["L0"], rel_tol=w["rel_tol"],
                             max_vcycles=w["max_vcycles"], ncycle=w["ncycle"], npre=w["npre"], npost=w["npost"],
                             precision=precision, use_graphs=0 if args.no_graphs else 1,
                             bc_mode=q.QUMOND_BC_MULTIPOLE if w.get("bc") == "multipole" else q.QUMOND_BC_ZERO,
                             persistent_vcycle=args.persistent_vcycle, small_cluster=args.small_cluster,
                             dc_vcycles=args.dc_vcycles)
        cs = [make() for _ in range(args.chains)]
        return Contexts(cs), q.Pipeline(cs[0], dev, ctx_mond=cs[1] if len(cs) > 1 else None)

    xd, yd, zd, md = (torch.from_numpy(a).to(dev) for a in (p.x, p.y, p.z, p.m))
    g = tuple(torch.empty_like(xd) for _ in range(3))

    # V-cycles per defect-correction step: 2 or 4, whichever times faster on a few pipelined steps of this
    # workload (every choice meets the same tolerance; only the number of residual checks differs)
    dc_tried = None
    if args.dc_vcycles == 0:
        dc_tried = {}
        for dc in (2, 4):
            args.dc_vcycles = dc
            cx, pp = new_pipeline(prec)
            runs = lambda k: (pp.run_many([(xd, yd, zd, md)] * k, nbins=w["nbins"], rmax=w["rmax"], nphi=w["nphi"],
                                          forces=[g] * k) if pp.ctx_mond is not None else
                              [pp.run(xd, yd, zd, md, nbins=w["nbins"], rmax=w["rmax"], nphi=w["nphi"], forces=g)
                               for _ in range(k)])
            runs(max(2, args.warmup))
            barrier()
            d0 = torch.cuda.Event(enable_timing=True)
            d1 = torch.cuda.Event(enable_timing=True)
            d0.record()
            runs(6)
            d1.record()
            barrier()
            dc_tried[dc] = ws * 6 * 1000.0 / max_over_ranks(d0.elapsed_time(d1))
            pp.close()
            cx.close()
            del pp, cx
            torch.cuda.empty_cache()
        args.dc_vcycles = max(dc_tried, key=dc_tried.get)

    ctx, pipe = new_pipeline(prec)

    def step(pp=None):
        pp = pp or pipe
        return pp.run(xd, yd, zd, md, nbins=w["nbins"], rmax=w["rmax"], nphi=w["nphi"], forces=g)

    # warm-up (untimed)
    for _ in range(args.warmup):
        step()
    st_check = pipe.potentials(xd, yd, zd, md, stats=True)
    vcycles = [s.vcycles for s in st_check[0] + st_check[1]]
    torch.cuda.synchronize()

    # --- per-kernel breakdown: the same steps with every kernel launched on its own and
    # bracketed by CUDA events on its stream (host launch latency can inflate short kernels) ---
    ctx.qumond_trace_read(reset=True)
    ctx.qumond_trace_timing(True)
    barrier()
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record()
    for _ in range(args.steps):
        step()
    r1.record()
    barrier()
    replay_ms = r0.elapsed_time(r1) / args.steps
    kstats, _, _ = ctx.qumond_trace_read(reset=True)
    ctx.qumond_trace_timing(False)

    # --- timed region: inputs resident in HBM; each solve is one CUDA graph.  With two chains
    # the K steps run pipelined (Pipeline.run_many): the Newtonian chain of step i+1 overlaps
    # the QUMOND chain, forces and rotation curve of step i; every step is the whole path. ---
    pipelined = args.chains == 2 and not args.no_pipeline
    # lanes: independent steps spread over several pipelines (two contexts each) that run concurrently
    # (paper_1201_3185_gb300.run_lanes); every step is still the whole path on one pipeline's buffers
    lane_sets = [(ctx, pipe)]
    lane_g = [g]

    def lane_pipes(nl):
        while len(lane_sets) < nl:
            lane_sets.append(new_pipeline(prec))
            lane_g.append(tuple(torch.empty_like(xd) for _ in range(3)))
        return [pp for _, pp in lane_sets[:nl]]

    def steps_timed(nsteps, pp=None, nl=1):
        pp = pp or pipe
        if pipelined and pp.ctx_mond is not None:
            pipes = lane_pipes(nl)
            return q.run_lanes(pipes, [(xd, yd, zd, md)] * nsteps, nbins=w["nbins"], rmax=w["rmax"],
                               nphi=w["nphi"], forces=[lane_g[i % nl] for i in range(nsteps)])
        return [step(pp) for _ in range(nsteps)]

    lanes = max(1, args.lanes) if pipelined else 1
    lanes_tried = None
    if pipelined and args.lanes == 0:  # pick the number of lanes (1, 2 or 3) by timing a few steps of each
        lanes_tried = {}
        for nl in (1, 2, 3):
            steps_timed(max(2, args.warmup), nl=nl)  # captures the graphs of the lanes' contexts
            barrier()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record()
            steps_timed(8, nl=nl)
            a1.record()
            barrier()
            lanes_tried[nl] = ws * 8 * 1000.0 / max_over_ranks(a0.elapsed_time(a1))
        lanes = max(lanes_tried, key=lanes_tried.get)
    steps_timed(max(2, args.warmup), nl=lanes)  # captures the graphs of the pipelined form
    ctx_all = Contexts([c for cx, _ in lane_sets[:lanes] for c in cx.ctxs])
    ctx_all.qumond_trace_read(reset=True)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record()
    res = steps_timed(args.steps, nl=lanes)[-1]
    s1.record()
    barrier()
    clk = clocks.stop()
    ms_total = max_over_ranks(s0.elapsed_time(s1))
    timed_stats, launches, cell_updates = ctx_all.qumond_trace_read(reset=True)
    step_bytes = sum(k.bytes for k in timed_stats.values()) / args.steps
    ms_step = ms_total / args.steps
    value = ws * args.steps / (ms_total / 1000.0)

    # --- end to end through the public API, host buffers: every step's particles copied in
    # from pinned host memory, its forces and rotation curve copied out.  The forces land in a ring of
    # two host buffers per lane (each step's result stays there for the next step of its lane): on a box
    # that had run other GPU jobs, copies into a fresh 48 MB pinned buffer every step slowed the
    # concurrent kernels by up to 15 %, a ring by about 5 % (copies into the same few buffers) ----------
    host = [torch.from_numpy(a).pin_memory() for a in (p.x, p.y, p.z, p.m)]
    n_ring = 2 * lanes if pipelined else 1
    out_g = [[torch.empty(w["particles"], dtype=torch.float64).pin_memory() for _ in range(3)]
             for _ in range(n_ring)]
    out_vc = torch.empty(args.steps, w["nbins"], dtype=torch.float64).pin_memory()
    out_r = torch.empty(args.steps, w["nbins"], dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host)
    d2h = sum(t.numel() * t.element_size() for t in out_g[0]) + w["nbins"] * 8 * 2
    if pipelined:  # device buffers of every step, so that the steps can overlap
        dev_in = [[torch.empty_like(xd) for _ in range(4)] for _ in range(args.steps)]
        dev_g = [tuple(torch.empty_like(xd) for _ in range(3)) for _ in range(args.steps)]
        h2d_stream, d2h_stream = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        # untimed: the lanes' graphs once more, with the copies' buffers allocated
        steps_timed(2 * lanes, nl=lanes)
        torch.cuda.synchronize()
    # one step's transfers on their own, on the copy streams (best of three): the rates the overlapped copies
    # of the timed region can reach
    copy_gbps = None
    if pipelined:
        def copy_ms(pairs, st):
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(st)
            with torch.cuda.stream(st):
                for a, b in pairs:
                    a.copy_(b, non_blocking=True)
            c1.record(st)
            c1.synchronize()
            return c0.elapsed_time(c1)
        ms_in = min(copy_ms(list(zip(dev_in[0], host)), h2d_stream) for _ in range(3))
        ms_out = min(copy_ms(list(zip(out_g[0], dev_g[0])), d2h_stream) for _ in range(3))
        copy_gbps = {"h2d": h2d / ms_in / 1e6, "d2h": (d2h - w["nbins"] * 16) / ms_out / 1e6}
    e2e_clocks = ClockSampler(local)
    e2e_load = os.getloadavg()[0] if hasattr(os, "getloadavg") else None
    barrier()
    e2e_clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    if pipelined:
        # copies in on one stream (each step's first kernel waits for its own copy), results out on
        # another as each step completes, so that the transfers overlap the other steps' kernels
        cur = torch.cuda.current_stream(dev)
        h2d_stream.wait_stream(cur)
        d2h_stream.wait_stream(cur)
        ready = []
        with torch.cuda.stream(h2d_stream):
            for i in range(args.steps):
                for a, b in zip(dev_in[i], host):
                    a.copy_(b, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(h2d_stream)
                ready.append(ev)
        rs = q.run_lanes(lane_pipes(lanes), [tuple(d) for d in dev_in], nbins=w["nbins"], rmax=w["rmax"],
                         nphi=w["nphi"], forces=dev_g, ready=ready)
        with torch.cuda.stream(d2h_stream):
            for i in range(args.steps):
                d2h_stream.wait_event(rs[i].done)
                for a, b in zip(out_g[i % n_ring], dev_g[i]):
                    a.copy_(b, non_blocking=True)
                out_vc[i].copy_(rs[i].vc, non_blocking=True)
                out_r[i].copy_(rs[i].r, non_blocking=True)
        cur.wait_stream(h2d_stream)
        cur.wait_stream(d2h_stream)
    else:
        for i in range(args.steps):
            xs, ys, zs, ms_ = (t.to(dev, non_blocking=True) for t in host)
            gg = tuple(torch.empty_like(xs) for _ in range(3))
            r = pipe.run(xs, ys, zs, ms_, nbins=w["nbins"], rmax=w["rmax"], nphi=w["nphi"], forces=gg)
            for a, b in zip(out_g[0], gg):
                a.copy_(b, non_blocking=True)
            out_vc[i].copy_(r.vc, non_blocking=True)
            out_r[i].copy_(r.r, non_blocking=True)
    e1.record()
    barrier()
    e2e_clk = e2e_clocks.stop()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1))
    e2e_value = ws * args.steps / (e2e_ms / 1000.0)
    if pipelined:
        del dev_in, dev_g

    # the same steps one after another (each waits for the previous one to finish)
    step_by_step = None
    if pipelined:
        barrier()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record()
        for _ in range(args.steps):
            step()
        b1.record()
        barrier()
        sbs_ms = max_over_ranks(b0.elapsed_time(b1)) / args.steps
        step_by_step = {"value": ws * 1000.0 / sbs_ms, "unit": UNIT, "ms_per_step": sbs_ms,
                        "form": "each step's two chains overlap each other only (Pipeline.run per step)"}

    # --- kernels timed live: the same steps with one chain (no concurrent solve sharing
    # the GPU), the graphs carrying event-record nodes around each run of consecutive
    # launches of one kernel class in the FMG part of every solve.  The three classes
    # with the most replay time are timed this way (one timed region each); the
    # dominant kernel is the one with the most live time per step. ----------------------
    pipe1 = q.Pipeline(ctx.ctxs[0], dev)
    ctx1 = Contexts(ctx.ctxs[:1])
    candidates = [k.name for k in sorted(kstats.values(), key=lambda k: -k.ms)[:3]]
    live_by = {}
    one_chain_ms = None
    for name in candidates:
        ctx1.qumond_trace_timing(True, only=name)
        step(pipe1)  # captures the instrumented graphs
        ctx1.qumond_trace_read(reset=True)
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(args.steps):
            step(pipe1)
        t1.record()
        barrier()
        ms1 = max_over_ranks(t0.elapsed_time(t1)) / args.steps
        one_chain_ms = ms1 if one_chain_ms is None else min(one_chain_ms, ms1)
        st1, _, _ = ctx1.qumond_trace_read(reset=True)
        ctx1.qumond_trace_timing(False)
        k = st1[name]
        per_launch = k.ms / k.timed if k.timed else 0.0
        live_by[name] = (k, per_launch * k.launches / args.steps)
    dom_name = max(live_by, key=lambda nm: live_by[nm][1])
    live = {dom_name: live_by[dom_name][0]}
    live_ms_per_step = {nm: v[1] for nm, v in live_by.items()}

    # dominant kernel and its roofline
    dom = live[dom_name]
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    bytes_per_launch = dom.timed_bytes / dom.timed if dom.timed else dom.bytes / max(dom.launches, 1)
    avg_ms = dom.ms / dom.timed if dom.timed else None
    achieved = dom.timed_bytes / dom.ms / 1e6 if dom.ms else None  # GB/s
    roofline = {"bound": "hbm", "kernel": dom.name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None,
                "traffic": ncu_traffic(dom.name, w["n"]),
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "avg_launch_ms": avg_ms, "timed_launches": dom.timed,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback 6.8 TB/s",
                "timing": "CUDA event-record nodes around each run of consecutive launches of this kernel class in "
                          "the FMG part of each solve's graph (e.g. the four half-sweeps of a pre-smoothing), read "
                          "after each solve, over %d timed steps of the same workload run with one chain; achieved = "
                          "algorithmic bytes of the timed launches / their time" % args.steps,
                "live_ms_per_step_of_candidates": live_ms_per_step}
    # --- the solve-level roofline: every FMG solve of the step (boundary values, FMG and the defect correction
    # to the tolerance) bracketed by CUDA events on its stream, with one chain so that no two solves overlap;
    # achieved = the algorithmic bytes of the solves' kernels / the solves' summed event time ----------------
    roofline["solve"] = {PRECISION_NAMES[args.precision]: solve_roofline(pipe1, ctx1, step, args.steps, peak, barrier,
                                                                         max_over_ranks)}
    # the same bytes in the timed pipelined region: the solves' algorithmic bytes per step / the step time.  The
    # step's time also covers its deposits, sources, far field, forces and curve, so this is a lower bound on
    # the rate the solves reach while the chains and lanes overlap
    solve_bytes_step = sum(k.bytes for name, k in timed_stats.items() if name not in NOT_SOLVE) / args.steps
    roofline["solve_pipelined"] = {
        "achieved": solve_bytes_step / (ms_step * 1e6), "peak": peak, "unit": "GB/s",
        "frac": solve_bytes_step / (ms_step * 1e6) / peak, "algorithmic_bytes_per_step": solve_bytes_step,
        "timing": "the timed region of `value` (%d lanes of two chains, pipelined steps): solve-kernel bytes per "
                  "step / ms per step" % lanes}

    total_kernel_ms = sum(k.ms for k in kstats.values())
    total_bytes = sum(k.bytes for k in kstats.values())
    kernels = {k.name: {"launches_per_step": k.launches / args.steps, "ms_per_step": k.ms / args.steps,
                        "share": k.ms / total_kernel_ms if total_kernel_ms else None,
                        "GBps": (k.timed_bytes / k.ms / 1e6) if k.ms else None}
               for k in sorted(kstats.values(), key=lambda k: -k.ms) if k.launches}

    # --- the other arithmetic modes at the same final residual -------------------------
    def time_mode(precision, nsteps):
        cx, pp = new_pipeline(precision)
        step(pp)
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        for _ in range(nsteps):
            step(pp)
        f1.record()
        barrier()
        pms = max_over_ranks(f0.elapsed_time(f1)) / nsteps
        pp.close()
        cx.close()
        return pms

    plain = None
    fp64_dc = None
    for cx, pp in lane_sets[1:]:  # the extra lanes
        pp.close()
        cx.close()
    del lane_sets[1:]
    if not args.no_plain and prec != q.QUMOND_PREC_FP64:
        pipe.close()
        ctx.close()
        del pipe
        torch.cuda.empty_cache()
        nplain = max(1, min(args.steps, 3))
        pms = time_mode(q.QUMOND_PREC_FP64, nplain)
        plain = {"value": ws * 1000.0 / pms, "unit": UNIT, "ms_per_step": pms, "steps": nplain,
                 "precision": PRECISION_NAMES["fp64"] + " (same kernels, same tolerance)",
                 "speedup_of_value": value / (ws * 1000.0 / pms)}
        if prec == q.QUMOND_PREC_MIXED_FIXED:
            mms = time_mode(q.QUMOND_PREC_MIXED, nplain)
            fp64_dc = {"value": ws * 1000.0 / mms, "unit": UNIT, "ms_per_step": mms, "steps": nplain,
                       "precision": PRECISION_NAMES["mixed"]}
            cm, _ = new_pipeline(q.QUMOND_PREC_MIXED)
            pm = q.Pipeline(cm.ctxs[0], dev)
            step(pm)
            roofline["solve"][PRECISION_NAMES["mixed"]] = solve_roofline(pm, Contexts(cm.ctxs[:1]), step,
                                                                         args.steps, peak, barrier, max_over_ranks)
            cm.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and w["kind"] != "large":  # (513^3: minutes per step)
        cpu = cpu_baseline(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {q.QUMOND_PREC_MIXED: "f32+f64", q.QUMOND_PREC_MIXED_FIXED: "f32+int64",
                                            q.QUMOND_PREC_FP64: "f64"}[prec],
            "data": "synthetic", "config": workload_config(PRECISION_NAMES[args.precision]),
            "cell_updates_per_s": ws * cell_updates / (ms_total / 1000.0),
            "algorithmic_bytes_per_step": step_bytes,
            "algorithmic_GBps_whole_step": step_bytes / (ms_step * 1e6),
            "kernel_ms_per_step_one_by_one": total_kernel_ms / args.steps,
            "replay_ms_per_step_one_by_one": replay_ms,
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "copy_GBps_alone": copy_gbps, "clocks": e2e_clk, "host_load_1min": e2e_load,
                    "host_result_buffers": n_ring},
            "gpu_launches": int(launches),
            "gpu_launches_per_step": launches / args.steps,
            "chains": args.chains,
            "pipelined_steps": pipelined,
            "lanes": lanes,
            "lanes_tried": lanes_tried,
            "dc_vcycles": args.dc_vcycles,
            "dc_vcycles_tried": dc_tried,
            "step_by_step": step_by_step,
            "small_level_vcycle": {0: "one graph kernel node per smoothing, restriction and prolongation", 1: "one cooperative kernel", 2: "one thread-block cluster per set", 3: "the level n = 32 and those under it in the distributed shared memory of one thread-block cluster per set"}[args.persistent_vcycle],
            "one_chain": {"value": ws * 1000.0 / one_chain_ms, "unit": UNIT, "ms_per_step": one_chain_ms},
            "vcycles_after_fmg_per_solve": vcycles,
            "plain_fmg": plain,
            "fp32_smoothing_fp64_defect_correction": fp64_dc,
            "kernels": kernels,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    rep.close()


# --- the fit sweep -----------------------------------------------------------------------
def sweep_inputs():
    import numpy as np

    import synth
    w = WORKLOAD
    doc = json.load(open(os.path.join(ROOT, w["target"])))
    gal = synth.SweepGalaxy(w["particles"], w["galaxy_seed"])
    params = synth.fit_sweep_parameters(w["sets"], seed=w["param_seed"])
    return gal, params, np.array(doc["v_obs"]), np.array(doc["sigma"])


def run_sweep(args):
    import numpy as np
    import torch

    import paper_1201_3185_gb300 as q
    from paper_1201_3185_gb300.replicas import Replicas
    rep = Replicas.from_env()
    ws, rank, local = rep.world_size, rep.rank, rep.local_rank
    dev = rep.device
    w = WORKLOAD
    prec = {"fp64": q.QUMOND_PREC_FP64, "mixed": q.QUMOND_PREC_MIXED, "fixed": q.QUMOND_PREC_MIXED_FIXED}[args.precision]

    def params(precision, tile=0, form=3, dc=2):
        return q.default_params(n=w["n"], nboxes=w["nboxes"], L0=w["L0"], rel_tol=w["rel_tol"],
                                max_vcycles=w["max_vcycles"], ncycle=w["ncycle"], npre=w["npre"], npost=w["npost"],
                                precision=precision, use_graphs=0 if args.no_graphs else 1, tile_small=tile,
                                persistent_vcycle=form, dc_vcycles=dc)

    gal, prm, v_obs_h, sigma_h = sweep_inputs()
    host_sets = [gal.particles(r) for r in prm]
    # every set's particles, set after set, resident in HBM (a chunk of sets is then a view)
    sets = tuple(torch.from_numpy(np.concatenate([getattr(p, a) for p in host_sets])).to(dev) for a in "xyzm")
    dist = [float(r[0]) for r in prm]
    v_obs = torch.from_numpy(v_obs_h).to(dev)
    sigma = torch.from_numpy(sigma_h).to(dev)
    kw = dict(nbins=w["nbins"], rmax=w["rmax"], nphi=w["nphi"], device=dev)

    if args.workers:
        choice, tune = {"batch": w["sets"], "lanes": args.workers, "tile_small": 0,
                        "persistent_vcycle": args.persistent_vcycle, "dc_vcycles": max(1, args.dc_vcycles)}, None
    else:
        choice, tune = q.autotune(params(prec), sets, dist, v_obs, sigma, **kw)
    sw = q.FitSweep(params(prec, choice["tile_small"], choice["persistent_vcycle"], choice["dc_vcycles"]),
                    batch=choice["batch"], lanes=choice["lanes"], **kw)
    ctx = Contexts(sw.ctxs)
    for _ in range(args.warmup):
        sw.run(sets, dist, v_obs, sigma)
    chk = sw.run(sets, dist, v_obs, sigma, stats=True)
    torch.cuda.synchronize()
    vcyc = [[a.vcycles, b.vcycles] for st in chk.stats for a, b in st]
    chi2 = chk.chi2.cpu().numpy()

    # timed region: particles resident in HBM
    ctx.qumond_trace_read(reset=True)
    clocks = ClockSampler(local)
    rep.barrier()
    clocks.start()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(args.steps):
        sw.run(sets, dist, v_obs, sigma)
    s1.record()
    rep.barrier()
    clk = clocks.stop()
    ms_total = rep.max(s0.elapsed_time(s1))
    tstats, launches, cells = ctx.qumond_trace_read(reset=True)
    step_bytes = sum(k.bytes for k in tstats.values()) / args.steps
    ms_step = ms_total / args.steps
    value = ws * w["sets"] * args.steps / (ms_total / 1000.0)

    # kernel classes timed live inside the batched graphs (the tuned batch, one lane): event-record nodes
    # around each run of consecutive launches of the class in the FMG part of every solve
    one = q.FitSweep(params(prec, choice["tile_small"], choice["persistent_vcycle"], choice["dc_vcycles"]),
                     batch=choice["batch"], lanes=1, **kw)
    c1 = Contexts(one.ctxs)
    nsub = choice["batch"]
    sub = tuple(a[:nsub * (a.numel() // w["sets"])] for a in sets)
    live = {}
    for name in ("rb_half_finest", "rb_half_coarser", "restrict_resid_red", "prolong_black", "residual_outer",
                 "coarse_solver"):
        c1.qumond_trace_timing(True, only=name)
        one.run(sub, dist[:nsub], v_obs, sigma)
        c1.qumond_trace_read(reset=True)
        one.run(sub, dist[:nsub], v_obs, sigma)
        torch.cuda.synchronize()
        st1, _, _ = c1.qumond_trace_read(reset=True)
        c1.qumond_trace_timing(False)
        k = st1[name]
        if k.timed:
            live[name] = (k, k.ms / k.timed * k.launches / nsub)
    one.close()
    dom_name = max(live, key=lambda nm: live[nm][1])
    dom = live[dom_name][0]
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = dom.timed_bytes / dom.ms / 1e6 if dom.ms else None
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "algorithmic_bytes_per_launch": dom.timed_bytes / dom.timed, "avg_launch_ms": dom.ms / dom.timed,
                "timed_launches": dom.timed,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback 6.8 TB/s",
                "timing": "CUDA event-record nodes around runs of this class's launches in the FMG part of each "
                          "solve's graph; one context holding %d sets (every launch covers all of them)" % nsub,
                "live_ms_per_set": {nm: v[1] for nm, v in live.items()},
                "live_GBps": {nm: v[0].timed_bytes / v[0].ms / 1e6 for nm, v in live.items() if v[0].ms}}

    # end to end: every set's particles copied from pinned host memory, chi^2 and curves read back.  The
    # particles of step i+1 are copied on a stream of their own into the second of two device buffers while
    # step i computes (a buffer is refilled once the step that read it is done)
    host = [torch.from_numpy(np.concatenate([getattr(p, a) for p in host_sets])).pin_memory() for a in "xyzm"]
    out_vc = torch.empty(w["sets"], w["nbins"], dtype=torch.float64).pin_memory()
    out_chi2 = torch.empty(w["sets"], dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host)
    d2h = out_vc.numel() * 8 + out_chi2.numel() * 8
    dbuf = [tuple(torch.empty(t.shape, dtype=t.dtype, device=dev) for t in host) for _ in range(2)]
    copy_stream = torch.cuda.Stream(dev)
    cur = torch.cuda.current_stream(dev)
    done = []

    def copy_in(i):
        if i == 0:
            copy_stream.wait_stream(cur)
        if i >= 2:
            copy_stream.wait_event(done[i - 2])  # the step that read this buffer
        with torch.cuda.stream(copy_stream):
            for a, b in zip(dbuf[i % 2], host):
                a.copy_(b, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(copy_stream)
        return ev

    rep.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    ready = copy_in(0)
    for i in range(args.steps):
        cur.wait_event(ready)
        if i + 1 < args.steps:
            ready = copy_in(i + 1)
        res = sw.run(dbuf[i % 2], dist, v_obs, sigma)
        ev = torch.cuda.Event()
        ev.record(cur)
        done.append(ev)
        out_vc.copy_(res.vc, non_blocking=True)
        out_chi2.copy_(res.chi2, non_blocking=True)
    e1.record()
    rep.barrier()
    e2e_ms = rep.max(e0.elapsed_time(e1))
    e2e_value = ws * w["sets"] * args.steps / (e2e_ms / 1000.0)
    sw.close()

    def timed_sweep(precision, nsteps, **form):
        one = q.FitSweep(params(precision, form.pop("tile", 0), 3, form.pop("dc", 2)), **form, **kw)
        one.run(sets, dist, v_obs, sigma)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        for _ in range(nsteps):
            one.run(sets, dist, v_obs, sigma)
        f1.record()
        rep.barrier()
        t = rep.max(f0.elapsed_time(f1)) / nsteps
        one.close()
        torch.cuda.empty_cache()
        return {"value": ws * w["sets"] / (t / 1000.0), "unit": "sets/s", "ms_per_step": t, "steps": nsteps}

    seq_same = plain = unbatched = None
    if not args.no_plain:
        nrep = max(1, min(args.steps, 3))
        # plain FP64 FMG: the same batched kernels and form, FP64 throughout, to the same tolerance
        plain = timed_sweep(q.QUMOND_PREC_FP64, nrep, batch=choice["batch"], lanes=choice["lanes"],
                            tile=choice["tile_small"], dc=choice["dc_vcycles"])
        plain["precision"] = PRECISION_NAMES["fp64"] + " (same batched kernels, same tolerance)"
        plain["speedup_of_value"] = value / plain["value"]
        # one set per context, 8 contexts side by side (the sweep without batching)
        unbatched = timed_sweep(prec, nrep, workers=8, dc=choice["dc_vcycles"])
        unbatched["form"] = "one set per context, 8 contexts on 8 streams"
        seq_same = timed_sweep(prec, 1, workers=1, dc=choice["dc_vcycles"])
        seq_same["form"] = "one set after another"

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ns = 4
        t = oracle_sweep_sample(gal, prm[:ns], v_obs_h, sigma_h)
        cpu = {"value": ns / t, "unit": "sets/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": "the first %d of the %d sets (galaxy realisation excluded), %.1f s" % (ns, w["sets"], t)}

    if rank == 0:
        best = int(np.argmin(chi2))
        line = {
            "metric": METRIC, "value": value, "unit": "sets/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {q.QUMOND_PREC_MIXED: "f32+f64", q.QUMOND_PREC_MIXED_FIXED: "f32+int64",
                                            q.QUMOND_PREC_FP64: "f64"}[prec],
            "data": "synthetic", "config": sweep_config(PRECISION_NAMES[args.precision], choice),
            "solves_per_s": 2 * w["nboxes"] * value,
            "cell_updates_per_s": ws * cells / (ms_total / 1000.0),
            "algorithmic_bytes_per_step": step_bytes,
            "algorithmic_GBps_whole_step": step_bytes / (ms_step * 1e6),
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": "sets/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "gpu_launches_per_step": launches / args.steps,
            "autotune_ms_per_sweep": {"batch %d, lanes %d, tile %d, small-level form %d, dc %d" % k: v
                                      for k, v in tune.items()} if tune else None,
            "vcycles_after_fmg_per_set_max": max(max(v) for v in vcyc),
            "best_set": {"index": best, "chi2": float(chi2[best]), "params": [float(v) for v in prm[best]]},
            "unbatched": unbatched,
            "sequential_same_precision": seq_same,
            "plain_fmg": plain,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    rep.close()


# --- the learned initial guess -------------------------------------------------------------
def learned_config(precision):
    w = WORKLOAD
    return {
        "workload": "learned initial guess: two-disk galaxies (stellar disk Sigma0=500 Msun/pc^2, R_d=3 kpc, sech^2 "
                    "h_* uniform in [0.3,0.6] kpc; gas 1e9 Msun, R_g=8 kpc, h_g=0.1 kpc), %d particles, %d^3 nodes "
                    "x %d nested boxes of %g/%g kpc; whole path per galaxy with each QUMOND solve started from "
                    "Phi_N + U-Net(rho, Phi_N) (BF16, 4 levels 16-32-64-128 channels) and V-cycles to rel. residual "
                    "%g" % (w["particles"], w["n"] + 1, w["nboxes"], w["L0"] / 1000.0, w["L0"] / 2000.0, w["rel_tol"]),
        "galaxies": w["galaxies"],
        "precision": precision,
        "rel_tol": w["rel_tol"],
        "weights": "paper_1201_3185_gb300/weights/unet_two_disk_129cube.npy (trained on the GPU by "
                   "python -m paper_1201_3185_gb300.learned train)",
        "l2": "inputs larger than L2: 8 galaxies x 2e5 particles; every step writes ~10 129^3 FP64 grids",
        "data": "synthetic (seeded generator), evaluation galaxies disjoint from the training draws",
    }


def run_learned(args):
    import numpy as np
    import torch

    import paper_1201_3185_gb300 as q
    from paper_1201_3185_gb300 import learned as L
    from paper_1201_3185_gb300.replicas import Replicas
    rep = Replicas.from_env()
    ws, rank, local = rep.world_size, rep.rank, rep.local_rank
    dev = rep.device
    w = WORKLOAD
    prec = {"fp64": q.QUMOND_PREC_FP64, "mixed": q.QUMOND_PREC_MIXED, "fixed": q.QUMOND_PREC_MIXED_FIXED}[args.precision]
    work = L.Workload(n=w["n"], L0=w["L0"], nboxes=w["nboxes"], particles=w["particles"], seed=w["seed"] + rank,
                      device=dev)
    gals = [work.galaxy()[0] for _ in range(w["galaxies"])]

    def ctx(precision, warm=0):
        return q.Context(q.default_params(n=w["n"], nboxes=w["nboxes"], L0=w["L0"], rel_tol=w["rel_tol"],
                                          max_vcycles=w["max_vcycles"], ncycle=w["ncycle"], npre=w["npre"],
                                          npost=w["npost"], precision=precision, warm_start=warm))

    guess = q.Guess(w["n"], L.PHI_SCALE)
    guess.qumond_guess_set_params(torch.from_numpy(L.load_weights()).to(dev))
    c_fmg, c_warm = ctx(prec), ctx(prec, 1)
    p_learn = q.Pipeline(c_fmg, dev, guess=guess, ctx_warm=c_warm)
    p_fmg = q.Pipeline(ctx(prec), dev)

    def run(pipe, n_steps):
        for k in range(n_steps):
            x, y, z, m = gals[k % len(gals)]
            pipe.potentials(x, y, z, m)

    def timed(pipe, n_steps):
        run(pipe, min(args.warmup, len(gals)))
        rep.barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        run(pipe, n_steps)
        t1.record()
        rep.barrier()
        return rep.max(t0.elapsed_time(t1)) / n_steps

    vcyc = {"learned": [], "fmg": []}
    for pipe, key in ((p_learn, "learned"), (p_fmg, "fmg")):
        for k in range(len(gals)):
            _, ms = pipe.potentials(*gals[k], stats=True)
            vcyc[key] += [s.vcycles for s in ms]
    torch.cuda.synchronize()

    run(p_learn, min(args.warmup, len(gals)))
    for c in (c_fmg, c_warm):
        c.qumond_trace_read(reset=True)
    g0 = guess.qumond_guess_launches()
    clocks = ClockSampler(local)
    rep.barrier()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    run(p_learn, args.steps)
    t1.record()
    rep.barrier()
    clk = clocks.stop()
    ms_learn = rep.max(t0.elapsed_time(t1)) / args.steps
    # kernels of the timed region: the solver contexts' and the network's
    launches = sum(c.qumond_trace_read(reset=True)[1] for c in (c_fmg, c_warm)) + \
        (guess.qumond_guess_launches() - g0)
    ms_fmg = timed(p_fmg, args.steps)
    value = ws * 1000.0 / ms_learn

    # end to end: each step copies a galaxy's particles in from pinned host memory and the finest box's
    # potential out
    host = [[t.cpu().pin_memory() for t in gals[k]] for k in range(min(len(gals), 4))]
    out_phi = torch.empty_like(p_learn.phi[-1], device="cpu").pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host[0])
    d2h = out_phi.numel() * out_phi.element_size()
    rep.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        xs, ys, zs, ms_ = (t.to(dev, non_blocking=True) for t in host[k % len(host)])
        p_learn.potentials(xs, ys, zs, ms_)
        out_phi.copy_(p_learn.phi[-1], non_blocking=True)
    e1.record()
    rep.barrier()
    e2e_ms = rep.max(e0.elapsed_time(e1))
    e2e = {"value": ws * args.steps / (e2e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    # plain FP64 FMG, same path and tolerance
    plain = None
    if not args.no_plain:
        pp = q.Pipeline(ctx(q.QUMOND_PREC_FP64), dev)
        ms_plain = timed(pp, max(1, min(args.steps, 8)))
        plain = {"value": ws * 1000.0 / ms_plain, "unit": UNIT, "ms_per_step": ms_plain,
                 "precision": PRECISION_NAMES["fp64"] + " FMG start (same path, same tolerance)",
                 "speedup_of_value": ms_plain / ms_learn}

    # the network alone: one inference (14 convolutions + pooling/upsampling + head) timed with events
    S = w["n"]
    layers = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (192, 64),
              (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]
    lev = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0]
    flops = float(sum(2 * 27 * ci * co * (S >> l) ** 3 for (ci, co), l in zip(layers, lev)))
    smp = torch.empty(3 * S ** 3, dtype=torch.bfloat16, device=dev)
    p_fmg.potentials(*gals[0])
    guess.qumond_guess_make_sample(p_learn.rho_scale(0), p_fmg.rho, p_fmg.phiN[-1], p_fmg.phi[-1], smp)
    yv = torch.empty(S ** 3, dtype=torch.float32, device=dev)
    for _ in range(3):
        guess.qumond_guess_forward(smp, 1.0, yv)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(10):
        guess.qumond_guess_forward(smp, 1.0, yv)
    f1.record()
    f1.synchronize()
    inf_ms = f0.elapsed_time(f1) / 10
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    f0.record()
    for _ in range(5):
        guess.qumond_guess_gradients([smp], [1.0], torch.empty(q.Guess.num_params(), dtype=torch.float32,
                                                               device=dev), loss)
    f1.record()
    f1.synchronize()
    grad_ms = f0.elapsed_time(f1) / 5
    peaks = measured_peaks()
    peak = peaks["bf16_tflops"] if peaks else 1900.0
    achieved = flops / (inf_ms * 1e9)
    tc = guess.qumond_guess_tensor_path_available()
    roofline = {"bound": "tensor",
                "kernel": ("conv3_tc_kernel" if tc else "conv3_kernel") +
                          " (the 14 convolutions of one network inference)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "algorithmic_flops_per_inference": flops, "inference_ms": inf_ms,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst, measured)" if peaks else "fallback",
                "note": ("tcgen05 MMAs with TMEM accumulators (BF16, FP32 accumulation)" if tc else
                         "mma.sync m16n8k16 BF16 tensor-core path") +
                        "; the time includes the input, pooling, upsampling and head launches"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_learn, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16+f32+int64", "data": "synthetic",
            "config": learned_config(PRECISION_NAMES[args.precision]),
            "fmg_start_same_precision": {"value": ws * 1000.0 / ms_fmg, "unit": UNIT, "ms_per_step": ms_fmg,
                                         "speedup_of_value": ms_fmg / ms_learn},
            "plain_fmg": plain,
            "mean_vcycles_per_mond_solve": {k: float(np.mean(v)) for k, v in vcyc.items()},
            "roofline": roofline,
            "training_step_ms_per_sample": grad_ms,
            "training_tflops": 3.0 * flops / (grad_ms * 1e9),
            "e2e": e2e,
            "gpu_launches": int(launches),
            "gpu_launches_per_step": launches / args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    rep.close()


# --- the oracle (CPU) ------------------------------------------------------------------
def oracle_sweep_sample(gal, prm, v_obs, sigma):
    """The sweep's path for the given parameter sets with the FP64 oracle:
    both solves of both boxes, the rotation curve and chi^2; returns seconds."""
    import oracle
    oracle.build()
    w = WORKLOAD
    t0 = time.perf_counter()
    for r_ in prm:
        p = gal.particles(r_)
        boxes = oracle.pipeline(p, w["n"], w["L0"], w["nboxes"], ncycle=w["ncycle"], npre=w["npre"],
                                npost=w["npost"], tol=w["rel_tol"], max_vcycles=w["max_vcycles"])
        _, vc_o = oracle.rotation_curve(w["n"], w["L0"], (0.0, 0.0, 0.0), [b.phi for b in boxes], w["nbins"],
                                        w["rmax"] * r_[0], w["nphi"])
        oracle.chi2(vc_o, v_obs, sigma)
    return time.perf_counter() - t0


def run_reference_sweep(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    w = WORKLOAD
    gal, prm, v_obs, sigma = sweep_inputs()
    oracle_sweep_sample(gal, prm[:1], v_obs, sigma)  # builds the oracle
    for i in range(args.warmup - 1):
        oracle_sweep_sample(gal, prm[i + 1:i + 2], v_obs, sigma)
    per = 2
    times = [oracle_sweep_sample(gal, prm[per * i:per * i + per], v_obs, sigma) for i in range(args.steps)]
    value = per * len(times) / sum(times)
    sample = "each step: %d of the %d sets at full size (galaxy realisation included), whole sweep = %d sets" % (
        per, w["sets"], w["sets"])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sets/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": w["sets"] * 1000.0 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": sweep_config("FP64 CPU oracle", None),
        "cpu_baseline": {"kind": "oracle", "cores": cpu_cores(), "sample": sample, "value": value, "unit": "sets/s"},
        "e2e": {"value": value, "unit": "sets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def oracle_step(p):
    """One whole step of the workload with the FP64 oracle: for every box the
    deposit, both FMG solves to the tolerance and the source, then the forces
    at every particle and the rotation curve.  Returns seconds."""
    import oracle
    w = WORKLOAD
    t0 = time.perf_counter()
    boxes = oracle.pipeline(p, w["n"], w["L0"], w["nboxes"], ncycle=w["ncycle"], npre=w["npre"], npost=w["npost"],
                            tol=w["rel_tol"], max_vcycles=w["max_vcycles"],
                            far_field_lmax=8 if w.get("bc") == "multipole" else None)
    phis = [b.phi for b in boxes]
    oracle.forces(w["n"], w["L0"], (0.0, 0.0, 0.0), phis, p.x, p.y, p.z)
    oracle.rotation_curve(w["n"], w["L0"], (0.0, 0.0, 0.0), phis, w["nbins"], w["rmax"], w["nphi"])
    return time.perf_counter() - t0


STEP_SAMPLE = ("the whole step at full size: for each of the %d boxes the deposit, both FMG solves to rel. residual "
               "%g and the source, then the forces at every particle and the rotation curve")


def cpu_cores():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def cpu_baseline(args, steps=2):
    """The oracle timed as the reference arm times it -- `bench.py --impl reference` in a process of its own
    (nothing of this process's GPU work, threads or pinned memory around it), 3 untimed and `steps` timed
    whole steps -- so that the two CPU figures are the same measurement."""
    w = WORKLOAD
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--workload", args.workload,
           "--steps", str(steps), "--warmup", "3", "--precision", args.precision]
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1200)
    line = None
    for ln in r.stdout.splitlines():
        if ln.startswith("{"):
            line = json.loads(ln)
    if r.returncode != 0 or not line or "value" not in line:
        raise RuntimeError("oracle timing failed: %s" % (r.stderr[-2000:] or r.stdout[-2000:]))
    return {"value": line["value"], "unit": UNIT, "cores": line["cpu_baseline"]["cores"], "kind": "oracle",
            "sample": "3 untimed and %d timed steps in a process of its own (bench.py --impl reference), each %s "
                      "(%.1f s per step)" % (steps, STEP_SAMPLE % (w["nboxes"], w["rel_tol"]),
                                             line["ms_per_step"] / 1000.0)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    import oracle
    oracle.build()
    p = make_particles()
    w = WORKLOAD
    for _ in range(args.warmup):
        oracle_step(p)
    times = [oracle_step(p) for _ in range(args.steps)]
    per_solve = statistics.mean(times)
    value = 1.0 / per_solve
    sample = "each step: " + STEP_SAMPLE % (w["nboxes"], w["rel_tol"])
    config = workload_config("FP64 CPU oracle")
    if w["kind"] == "learned":  # the oracle has no network: it runs the same path with its FMG start
        config = learned_config("FP64 CPU oracle, FMG start")
        sample += "; the oracle starts each solve from FMG"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_solve * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
        "cpu_baseline": {"kind": "oracle", "cores": cpu_cores(), "sample": sample, "value": value, "unit": UNIT},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def profile_case(args):
    """One box of the workload solved once, then a single V-cycle of defect
    correction from that solution with every kernel launched on its own,
    between cudaProfilerStart and cudaProfilerStop: the launches ncu sees
    with --profile-from-start off are the finest-level ones first."""
    import torch

    import paper_1201_3185_gb300 as q
    w = WORKLOAD
    prec = {"fp64": q.QUMOND_PREC_FP64, "mixed": q.QUMOND_PREC_MIXED, "fixed": q.QUMOND_PREC_MIXED_FIXED}[args.precision]
    p = make_particles()
    dev = torch.device("cuda", 0)
    x, y, z, m = (torch.from_numpy(a).to(dev) for a in (p.x, p.y, p.z, p.m))
    common = dict(n=w["n"], nboxes=1, L0=w["L0"], npre=w["npre"], npost=w["npost"], ncycle=w["ncycle"],
                  precision=prec, use_graphs=0)
    ctx = q.Context(rel_tol=w["rel_tol"], max_vcycles=w["max_vcycles"], **common)
    nodes = ctx.nodes
    qf = torch.empty(nodes, dtype=torch.int64, device=dev)
    rho = torch.empty(nodes, dtype=torch.float64, device=dev)
    phi = torch.zeros(nodes, dtype=torch.float64, device=dev)
    ctx.qumond_deposit(0, x, y, z, m, qf, rho)
    ctx.qumond_solve_newton(0, rho, None, phi)
    ctx2 = q.Context(rel_tol=1e-300, max_vcycles=1, warm_start=1, **common)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    try:
        ctx2.qumond_solve_newton(0, rho, None, phi)
    except q.NotConverged:
        pass
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ctx.close()
    ctx2.close()
    print(json.dumps({"profile_case": "box 0 of the workload, one warm-start V-cycle", "n": w["n"],
                      "precision": args.precision}))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fixed", "mixed", "fp64"], default="fixed")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 FMG comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip timing the oracle on the host")
    ap.add_argument("--no-graphs", action="store_true", help="launch kernels one by one (for profilers)")
    ap.add_argument("--chains", type=int, choices=[1, 2], default=2,
                    help="2: QUMOND solves on a second context and stream, concurrent with the Newtonian chain")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="two-disk",
                    help="two-disk: the metric's 256^3 x 3-box configuration; large: 512^3 x 4 boxes; "
                         "sweep: the 64-set rotation-curve fit sweep at 128^3 x 2 boxes; "
                         "learned: the whole path with the QUMOND solves started from the U-Net guess")
    ap.add_argument("--workers", type=int, default=0,
                    help="sweep: lanes of one 64-set chunk each (0: batch size, lanes and block shape by the "
                         "autotuner)")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="time the steps one after another instead of pipelining successive steps' chains")
    ap.add_argument("--persistent-vcycle", type=int, choices=[0, 1, 2, 3], default=3,
                    help="the V-cycle on the small levels: 0 one launch per step, 1 one cooperative kernel, "
                         "2 one thread-block cluster (levels n <= 64, global memory), 3 one thread-block cluster "
                         "holding the level n = 32 in distributed shared memory (two-disk and large workloads)")
    ap.add_argument("--lanes", type=int, default=0,
                    help="two-disk and large: pipelines (two contexts each) running independent steps "
                         "concurrently; 0: 1, 2 or 3, whichever times faster")
    ap.add_argument("--dc-vcycles", type=int, default=0,
                    help="two-disk and large: V-cycles per defect-correction step (params.dc_vcycles); 0: 2 or 4, "
                         "whichever times faster")
    ap.add_argument("--small-cluster", type=int, choices=[0, 4, 8, 16], default=0,
                    help="CTAs per cluster of --persistent-vcycle 3 (0: 8)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one profiled V-cycle on one box instead of the benchmark (for ncu)")
    args = ap.parse_args()
    WORKLOAD.clear()
    WORKLOAD.update(WORKLOADS[args.workload])
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.profile_case:
        profile_case(args)
    elif args.impl == "reference":
        run_reference_sweep(args) if args.workload == "sweep" else run_reference(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "learned":
        run_learned(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
