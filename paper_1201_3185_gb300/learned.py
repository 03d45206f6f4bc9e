"""Learned initial guess for the QUMOND solve (include/qumond_guess.h).

The network maps (rho, Phi_N) of a box to (Phi - Phi_N) / phi_scale; the
QUMOND solve of the box then starts from Phi_N + phi_scale * output and runs
V-cycles to the tolerance (warm start) instead of FMG.  This module builds the
training set with the method itself (every sample is one box of a galaxy run
through the whole path on the GPU), trains the network with the library's
own forward/backward kernels and Adam, and measures what the guess saves.

Input scaling: channel 0 = 4 pi G h_b^2 rho / phi_scale (the right-hand side
of the Newtonian equation in units of the potential per cell), channel 1 =
Phi_N / phi_scale; phi_scale = 1e5 (km/s)^2, the depth of the two-disk
galaxies' potentials.

    python -m paper_1201_3185_gb300.learned train --galaxies 4000 --epochs 3 --out weights.npy
    python -m paper_1201_3185_gb300.learned evaluate --eval-galaxies 8
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from .qumond import Context, Guess, default_params

PHI_SCALE = 1.0e5
G_NEWTON = 4.30e-3
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_two_disk_129cube.npy")


def rho_scale(L_box: float, n: int, phi_scale: float = PHI_SCALE, G: float = G_NEWTON) -> float:
    h = L_box / n
    return 4.0 * math.pi * G * h * h / phi_scale


def he_init(seed: int) -> np.ndarray:
    """He-normal convolution weights, zero biases, small head (FP32 parameter vector)."""
    from .qumond import _lib  # noqa: F401  (library must be loadable)
    rng = np.random.default_rng(seed)
    layers = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128),
              (192, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]
    p = []
    for ci, co in layers:
        p.append(rng.standard_normal(27 * ci * co) * math.sqrt(2.0 / (27 * ci)))
        p.append(np.zeros(co))
    p.append(rng.standard_normal(16) * math.sqrt(1.0 / 16))
    p.append(np.zeros(1))
    out = np.concatenate(p).astype(np.float32)
    assert out.size == Guess.num_params()
    return out


def load_weights(path: str = WEIGHTS) -> np.ndarray:
    return np.load(path).astype(np.float32)


class Workload:
    """Boxes and galaxies of the learned-guess workload: the two-disk galaxy
    (stellar h drawn in [300, 600] pc; gas h 100 pc), n^3 intervals x 2
    nested boxes of L0 and L0/2."""

    def __init__(self, n=128, L0=80000.0, nboxes=2, particles=200_000, draws=8, seed=0, rel_tol=1e-10,
                 precision=2, device=None):
        import synth
        self.n, self.L0, self.nboxes, self.particles = n, L0, nboxes, particles
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.gals = [synth.SweepGalaxy(particles, seed=1000 * seed + k) for k in range(draws)]
        self.rng = np.random.default_rng(seed)
        self.rel_tol = rel_tol
        self.precision = precision

    def context(self, **over):
        kw = dict(n=self.n, nboxes=self.nboxes, L0=self.L0, rel_tol=self.rel_tol, max_vcycles=60,
                  precision=self.precision, ncycle=1)
        kw.update(over)
        return Context(default_params(**kw))

    def galaxy(self):
        """A random two-disk galaxy: one of the seeded draws, its stellar scale
        height uniform in [300, 600] pc, rotated by a random angle."""
        g = self.gals[int(self.rng.integers(len(self.gals)))]
        h = 300.0 + 300.0 * float(self.rng.random())
        p = g.particles([1.0, 1.0, h, 100.0])
        a = 2.0 * math.pi * float(self.rng.random())
        c, s = math.cos(a), math.sin(a)
        x, y = c * p.x - s * p.y, s * p.x + c * p.y
        dev = self.device
        return tuple(torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (x, y, p.z, p.m)), h

    def rho_scales(self):
        return [rho_scale(self.L0 / 2 ** b, self.n) for b in range(self.nboxes)]


class Solver:
    """Whole-path buffers of one context, box by box, keeping every box's rho."""

    def __init__(self, ctx: Context, device):
        nodes = ctx.nodes
        nb = ctx.params.nboxes
        self.ctx = ctx
        self.rho_fixed = torch.empty(nodes, dtype=torch.int64, device=device)
        self.rho = [torch.empty(nodes, dtype=torch.float64, device=device) for _ in range(nb)]
        self.src = [torch.empty(nodes, dtype=torch.float64, device=device) for _ in range(nb)]
        self.phiN = [torch.zeros(nodes, dtype=torch.float64, device=device) for _ in range(nb)]
        self.phi = [torch.zeros(nodes, dtype=torch.float64, device=device) for _ in range(nb)]

    def newton_and_source(self, parts, b):
        c = self.ctx
        x, y, z, m = parts
        c.qumond_deposit(b, x, y, z, m, self.rho_fixed, self.rho[b])
        c.qumond_solve_newton(b, self.rho[b], self.phiN[b - 1] if b else None, self.phiN[b])
        c.qumond_source(b, self.phiN[b], self.src[b])

    def mond(self, b, ctx=None, stats=True):
        c = ctx or self.ctx
        return c.qumond_solve_mond(b, self.src[b], self.phi[b - 1] if b else None, self.phi[b], stats=stats)


def generate(work: Workload, guess: Guess, ngal: int, log_every=0):
    """Training samples from ngal galaxies, every box of each: list of
    (BF16 sample tensor, box flag)."""
    dev = work.device
    ctx = work.context()
    sol = Solver(ctx, dev)
    scales = work.rho_scales()
    out = []
    t0 = time.time()
    for i in range(ngal):
        parts, _ = work.galaxy()
        for b in range(work.nboxes):
            sol.newton_and_source(parts, b)
            sol.mond(b, stats=False)
            smp = torch.empty(3 * guess.voxels, dtype=torch.bfloat16, device=dev)
            guess.qumond_guess_make_sample(scales[b], sol.rho[b], sol.phiN[b], sol.phi[b], smp)
            out.append((smp, float(b > 0)))
        if log_every and (i + 1) % log_every == 0:
            print("generated %d galaxies in %.1f s" % (i + 1, time.time() - t0), flush=True)
    torch.cuda.synchronize()
    ctx.close()
    return out


def train(guess: Guess, samples, *, epochs=1, batch=4, lr=1e-3, lr_final=1e-4, seed=0, log_every=0):
    """Adam over shuffled mini-batches; the learning rate decays
    geometrically from lr to lr_final.  Returns the per-step losses."""
    dev = samples[0][0].device
    rng = np.random.default_rng(seed)
    nsteps = epochs * (len(samples) // batch)
    losses = torch.zeros(max(nsteps, 1), dtype=torch.float32, device=dev)
    step = 0
    t0 = time.time()
    for ep in range(epochs):
        order = rng.permutation(len(samples))
        for k in range(len(samples) // batch):
            idx = order[k * batch:(k + 1) * batch]
            rate = lr * (lr_final / lr) ** (step / max(nsteps - 1, 1))
            guess.qumond_guess_train_step([samples[i][0] for i in idx], [samples[i][1] for i in idx], rate,
                                          loss=losses[step:step + 1])
            step += 1
            if log_every and step % log_every == 0:
                torch.cuda.synchronize()
                print("step %d/%d loss %.4e (%.1f s)" % (step, nsteps, losses[step - 1].item(), time.time() - t0),
                      flush=True)
    torch.cuda.synchronize()
    return losses[:step].cpu().numpy()


STARTS = ("fmg", "learned", "phiN")


def evaluate(work: Workload, guess: Guess, ngal: int, rel_tol=1e-8):
    """For ngal fresh galaxies, every box: the QUMOND solve to rel_tol started
    from (a) FMG, (b) the network's guess, (c) Phi_N; V-cycles after the
    start, the start's relative residual, and CUDA-event times of the solve
    (with the guess's inference for (b)).  (A zero start is not offered: the
    fixed-point defect correction takes its scale from the starting iterate.)"""
    dev = work.device
    base = work.context(rel_tol=1e-10)
    fmg = work.context(rel_tol=rel_tol)
    warm = work.context(rel_tol=rel_tol, warm_start=1)
    sol = Solver(base, dev)
    scales = work.rho_scales()
    rows = []
    for _ in range(ngal):
        parts, h = work.galaxy()
        for b in range(work.nboxes):
            sol.newton_and_source(parts, b)
            sol.mond(b, stats=False)  # parent values for the next box come from an accurate solve
            keep = sol.phi[b].clone()
            row = {"box": b, "h_star": h}
            for name in STARTS:
                ctx = fmg if name == "fmg" else warm
                if name != "fmg":
                    sol.phi[b].copy_(sol.phiN[b])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                if name == "learned":
                    guess.qumond_guess_apply(scales[b], float(b > 0), sol.rho[b], sol.phiN[b], sol.phi[b])
                st = sol.mond(b, ctx=ctx)
                e1.record()
                e1.synchronize()
                row[name] = {"vcycles": st.vcycles, "rel_residual_start": st.rel_residual_fmg,
                             "rel_residual": st.rel_residual, "ms": e0.elapsed_time(e1),
                             "max_rel_diff_vs_accurate": float((sol.phi[b] - keep).abs().max() / keep.abs().max())}
            sol.phi[b].copy_(keep)
            rows.append(row)
    for c in (base, fmg, warm):
        c.close()
    return rows


def summarize(rows):
    out = {}
    for name in STARTS:
        out[name] = {"mean_vcycles": float(np.mean([r[name]["vcycles"] for r in rows])),
                     "mean_ms": float(np.mean([r[name]["ms"] for r in rows])),
                     "median_rel_residual_start": float(np.median([r[name]["rel_residual_start"] for r in rows]))}
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("cmd", choices=["train", "evaluate"])
    ap.add_argument("--galaxies", type=int, default=4000)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=5e-5)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--particles", type=int, default=200_000)
    ap.add_argument("--eval-galaxies", type=int, default=8)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="weights.npy")
    ap.add_argument("--report", default=None)
    ap.add_argument("--weights", default=WEIGHTS, help="evaluate: the parameter file")
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    guess = Guess(args.n, PHI_SCALE)
    if args.cmd == "evaluate":
        guess.qumond_guess_set_params(torch.from_numpy(load_weights(args.weights)).to(dev))
        ev = Workload(n=args.n, particles=args.particles, seed=args.seed + 7919, device=dev)
        rows = evaluate(ev, guess, args.eval_galaxies)
        rep = {"weights": args.weights, "eval": summarize(rows)}
        print(json.dumps(rep), flush=True)
        if args.report:
            with open(args.report, "w") as f:
                json.dump({"report": rep, "rows": rows}, f)
        return
    work = Workload(n=args.n, particles=args.particles, seed=args.seed, device=dev)
    p0 = torch.from_numpy(he_init(args.seed)).to(dev)
    guess.qumond_guess_set_params(p0)
    t0 = time.time()
    data = generate(work, guess, args.galaxies, log_every=500)
    t_gen = time.time() - t0
    t0 = time.time()
    losses = train(guess, data, epochs=args.epochs, batch=args.batch, lr=args.lr, lr_final=args.lr_final,
                   seed=args.seed, log_every=500)
    t_train = time.time() - t0
    p = torch.empty(Guess.num_params(), dtype=torch.float32, device=dev)
    guess.qumond_guess_get_params(p)
    torch.cuda.synchronize()
    np.save(args.out, p.cpu().numpy())
    ev = Workload(n=args.n, particles=args.particles, seed=args.seed + 7919, device=dev)
    rows = evaluate(ev, guess, args.eval_galaxies)
    rep = {"galaxies": args.galaxies, "samples": len(data), "epochs": args.epochs, "batch": args.batch,
           "generate_s": t_gen, "train_s": t_train, "steps": int(losses.size),
           "loss_first": float(losses[:50].mean()), "loss_last": float(losses[-50:].mean()),
           "eval": summarize(rows)}
    print(json.dumps(rep), flush=True)
    if args.report:
        with open(args.report, "w") as f:
            json.dump({"report": rep, "rows": rows, "losses": losses.tolist()}, f)


if __name__ == "__main__":
    main()
