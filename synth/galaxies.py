"""Static N-body realisations of the galaxies used by the QUMOND path.

* Kuzmin disk (Section 3.1): enclosed mass M(1 - a/sqrt(R^2+a^2)), so a mass
  fraction f sits inside R = a sqrt((1-f)^-2 - 1); azimuth uniform; z = 0.
* Exponential disk with sech^2 vertical profile (Sections 3.3-3.4): radius
  from the enclosed-mass fraction 1 - (1+x) e^-x, x = R/R_d (inverted on a
  fine table, which draws the distribution the paper's rejection sampler
  draws); z = h atanh(2u - 1) for rho ~ sech^2(z/h).
* Hernquist bulge: M(<r) = M r^2/(r+a)^2, so r = a sqrt(u)/(1 - sqrt(u)),
  isotropic direction.
* Two components (Section 3.4): stars and gas each get half of the particles,
  each particle weighted by its component's total mass.
* Fit sweeps (Section 3.5): every parameter set (distance, stellar M/L,
  stellar and gas scale heights) rescales one seeded set of draws (common
  random numbers), so the sets differ only through their parameters.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Particles:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    m: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def concat(self, other: "Particles") -> "Particles":
        return Particles(*(np.concatenate([a, b]) for a, b in
                           ((self.x, other.x), (self.y, other.y), (self.z, other.z), (self.m, other.m))))


def _rng(seed) -> np.random.Generator:
    return seed if isinstance(seed, np.random.Generator) else np.random.default_rng(seed)


def kuzmin_disk(n: int, M: float, a: float, seed=0, stratified: bool = False) -> Particles:
    """Razor-thin Kuzmin disk of total mass M and scale a, n particles of mass M/n.

    stratified=True places the mass fractions at (i+1/2)/n and the azimuths on
    a golden-angle sequence: a low-noise realisation for accuracy checks.
    The full (untruncated) disk is drawn; particles beyond a grid simply fall
    outside it."""
    rng = _rng(seed)
    if stratified:
        f = (np.arange(n, dtype=np.float64) + 0.5) / n
        phi = np.mod(np.arange(n, dtype=np.float64) * (np.pi * (3.0 - np.sqrt(5.0))), 2.0 * np.pi)
    else:
        f = rng.random(n)
        phi = 2.0 * np.pi * rng.random(n)
    R = a * np.sqrt((1.0 - f) ** -2 - 1.0)
    return Particles(R * np.cos(phi), R * np.sin(phi), np.zeros(n), np.full(n, M / n))


def _exp_radius(u: np.ndarray, Rd: float, rmax: float) -> np.ndarray:
    """Radius whose enclosed-mass fraction of an exponential disk truncated at
    rmax equals u: the fraction is inverted by bisection (60 halvings) on a
    table of 2^16+1 points and interpolated linearly in between."""
    xmax = rmax / Rd
    norm = 1.0 - (1.0 + xmax) * np.exp(-xmax)
    ut = np.linspace(0.0, 1.0, (1 << 16) + 1)
    target = ut * norm
    lo = np.zeros_like(ut)
    hi = np.full_like(ut, xmax)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        below = (1.0 - (1.0 + mid) * np.exp(-mid)) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    xt = 0.5 * (lo + hi)
    return np.interp(u, ut, xt) * Rd


def _sech2_height(u: np.ndarray, h: float, zmax: float) -> np.ndarray:
    """Height for rho ~ sech^2(z/h) truncated to |z| < zmax (inverse CDF)."""
    if h <= 0.0:
        return np.zeros_like(u)
    t = np.tanh(zmax / h)
    return h * np.arctanh((2.0 * u - 1.0) * t)


def exponential_disk(n: int, M: float, Rd: float, h: float, rmax: float, zmax: float, seed=0) -> Particles:
    """Exponential disk (scale length Rd) with a sech^2(z/h) vertical profile,
    truncated at R < rmax and |z| < zmax; n particles of mass M/n."""
    rng = _rng(seed)
    R = _exp_radius(rng.random(n), Rd, rmax)
    phi = 2.0 * np.pi * rng.random(n)
    z = _sech2_height(rng.random(n), h, zmax)
    return Particles(R * np.cos(phi), R * np.sin(phi), z, np.full(n, M / n))


def hernquist_bulge(n: int, M: float, a: float, rmax: float, seed=0) -> Particles:
    """Hernquist sphere of mass M and scale a truncated at r < rmax; n
    particles of mass M/n (the mass inside rmax is M)."""
    rng = _rng(seed)
    smax = rmax / (rmax + a)  # sqrt of the enclosed fraction at rmax
    s = np.sqrt(rng.random(n)) * smax
    r = a * s / (1.0 - s)
    cth = 2.0 * rng.random(n) - 1.0
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    phi = 2.0 * np.pi * rng.random(n)
    return Particles(r * sth * np.cos(phi), r * sth * np.sin(phi), r * cth, np.full(n, M / n))


def two_component_disk(n_total: int, seed=0, *, sigma0: float = 500.0, Rd: float = 3000.0,
                       h_star: float | None = None, M_gas: float = 1.0e9, Rg: float = 8000.0,
                       h_gas: float = 100.0, rmax: float = 54000.0, zmax: float = 54000.0,
                       mass_to_light: float = 1.0, distance_scale: float = 1.0) -> Particles:
    """Stellar + gas exponential disks, half of the particles each.

    Stellar mass 2 pi sigma0 Rd^2 (times mass_to_light); when h_star is None
    it is drawn uniformly from [300, 600] pc.  distance_scale multiplies every
    length (a fit's distance parameter rescales the galaxy)."""
    rng = _rng(seed)
    if h_star is None:
        h_star = 300.0 + 300.0 * float(rng.random())
    M_star = 2.0 * np.pi * sigma0 * Rd * Rd * mass_to_light
    ns = n_total // 2
    ng = n_total - ns
    d = distance_scale
    stars = exponential_disk(ns, M_star, Rd * d, h_star * d, rmax, zmax, rng)
    gas = exponential_disk(ng, M_gas, Rg * d, h_gas * d, rmax, zmax, rng)
    return stars.concat(gas)


def large_galaxy(n_total: int, seed=0, *, rmax: float = 108000.0) -> Particles:
    """Stellar disk + gas disk + Hernquist bulge (M_b = 1e10 Msun, a_b = 500 pc):
    a third of the particles in each component."""
    rng = _rng(seed)
    nb = n_total // 3
    disk = two_component_disk(n_total - nb, rng, rmax=rmax, zmax=rmax)
    bulge = hernquist_bulge(nb, 1.0e10, 500.0, rmax, rng)
    return disk.concat(bulge)


def fit_sweep_parameters(nsets: int, seed=0) -> np.ndarray:
    """Parameter sets of a rotation-curve fit sweep (Section 3.5): columns
    distance scale in [0.8, 1.2], stellar M/L in [0.3, 1.2], stellar scale
    height in [200, 1000] pc, gas scale height in [50, 500] pc; uniform."""
    rng = _rng(seed)
    u = rng.random((nsets, 4))
    lo = np.array([0.8, 0.3, 200.0, 50.0])
    hi = np.array([1.2, 1.2, 1000.0, 500.0])
    return lo + (hi - lo) * u


class SweepGalaxy:
    """Two-component disk of a rotation-curve fit (Section 3.5) for any
    parameter set (distance scale d, stellar M/L, stellar scale height h_star
    pc, gas scale height h_gas pc), from draws made once with `seed`.

    The fitted galaxy is the observed one seen at a distance d times the
    nominal one: every in-plane length scales by d (scale lengths, truncation
    radius), the stellar luminosity and the gas mass by d^2; the stellar mass
    is M/L times the luminosity 2 pi I0 (d Rd)^2.  Scale heights are free
    parameters in pc.  Half of the particles are stars, half gas."""

    def __init__(self, n_total: int, seed=0, *, I0: float = 500.0, Rd: float = 3000.0, M_gas: float = 1.0e9,
                 Rg: float = 8000.0, rmax: float = 30000.0, zmax: float = 5000.0):
        rng = _rng(seed)
        self.ns = n_total // 2
        self.ng = n_total - self.ns
        self.I0, self.Rd, self.M_gas, self.Rg, self.rmax, self.zmax = I0, Rd, M_gas, Rg, rmax, zmax
        # radii in units of the scale length at d = 1 (the truncation scales with d as well)
        self.Xs = _exp_radius(rng.random(self.ns), 1.0, rmax / Rd)
        ps = 2.0 * np.pi * rng.random(self.ns)
        self.us = rng.random(self.ns)
        self.Xg = _exp_radius(rng.random(self.ng), 1.0, rmax / Rg)
        pg = 2.0 * np.pi * rng.random(self.ng)
        self.ug = rng.random(self.ng)
        self.cs, self.ss = np.cos(ps), np.sin(ps)
        self.cg, self.sg = np.cos(pg), np.sin(pg)

    def particles(self, params) -> Particles:
        d, ml, h_star, h_gas = (float(v) for v in params)
        M_star = ml * 2.0 * np.pi * self.I0 * (d * self.Rd) ** 2
        Rs = self.Xs * (d * self.Rd)
        Rg = self.Xg * (d * self.Rg)
        x = np.concatenate([Rs * self.cs, Rg * self.cg])
        y = np.concatenate([Rs * self.ss, Rg * self.sg])
        z = np.concatenate([_sech2_height(self.us, h_star, self.zmax), _sech2_height(self.ug, h_gas, self.zmax)])
        m = np.concatenate([np.full(self.ns, M_star / self.ns), np.full(self.ng, d * d * self.M_gas / self.ng)])
        return Particles(x, y, z, m)
