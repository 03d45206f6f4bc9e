"""ctypes marshalling for the C oracle, plus the step order of Section 2."""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qumond_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_int64
_P = ctypes.c_void_p


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-std=c11"]
    tmp = _LIB + ".tmp.%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    sig = {
        "ora_cic_deposit": (_L, [_I, _D, _D, _D, _D, _I, _P, _P, _P, _P, _L, _P]),
        "ora_rho_from_fixed": (None, [_I, _D, _I, _P, _P]),
        "ora_relax_rbgs": (None, [_I, _D, _P, _P]),
        "ora_residual": (None, [_I, _D, _P, _P, _P]),
        "ora_interior_sumsq": (_D, [_I, _P]),
        "ora_restrict_fw": (None, [_I, _P, _P]),
        "ora_prolong": (None, [_I, _P, _P, _I]),
        "ora_coarsest": (None, [_D, _P, _P]),
        "ora_vcycle": (None, [_I, _D, _P, _P, _I, _I]),
        "ora_fmg": (None, [_I, _D, _P, _P, _I, _I, _I]),
        "ora_solve": (_I, [_I, _D, _P, _P, _I, _I, _I, _I, _D, _I, _P, _I]),
        "ora_source": (None, [_I, _D, _D, _P, _P]),
        "ora_boundary_fill": (None, [_I, _D, _D, _D, _D, _P, _D, _D, _D, _D, _P]),
        "ora_forces": (_L, [_I, _I, _D, _I, _D, _D, _D, _P, _P, _P, _P, _L, _P, _P, _P]),
        "ora_rotation_curve": (None, [_I, _I, _D, _I, _D, _D, _D, _P, _I, _D, _I, _D, _P, _P]),
        "ora_chi2": (None, [_P, _P, _P, _I, _I, _P]),
        "ora_rotation_curve_algebraic": (None, [_I, _I, _D, _I, _D, _D, _D, _P, _I, _D, _I, _D, _D, _P, _P]),
        "ora_sigma_z": (None, [_I, _I, _D, _I, _D, _D, _D, _P, _I, _D, _I, _D, _D, _D, _P, _P]),
        "ora_far_field": (_D, [_I, _D, _D, _D, _D, _P, _D, _D, _I, _P, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def grid_index(n: int, i, j, k):
    return i + (n + 1) * (j + (n + 1) * k)


def _check_grid(a: np.ndarray, n: int, dtype=np.float64):
    assert a.dtype == dtype and a.flags.c_contiguous and a.size == (n + 1) ** 3, (a.dtype, a.size, n)


# --- step 1 ----------------------------------------------------------------
def cic_deposit(n, L, center, shift, x, y, z, m, q=None):
    """Fixed-point CIC deposit (int64 grid, accumulated into q). Returns (q, kept)."""
    x, y, z, m = _f64(x), _f64(y), _f64(z), _f64(m)
    if q is None:
        q = np.zeros((n + 1) ** 3, dtype=np.int64)
    _check_grid(q, n, np.int64)
    kept = _load().ora_cic_deposit(n, L, center[0], center[1], center[2], shift,
                                   _ptr(x), _ptr(y), _ptr(z), _ptr(m), x.size, _ptr(q))
    return q, int(kept)


def rho_from_fixed(n, L, shift, q):
    rho = np.empty((n + 1) ** 3, dtype=np.float64)
    _load().ora_rho_from_fixed(n, L, shift, _ptr(q), _ptr(rho))
    return rho


# --- steps 2 and 4 -----------------------------------------------------------
def relax_rbgs(n, h, u, f):
    _check_grid(u, n); _check_grid(f, n)
    _load().ora_relax_rbgs(n, h, _ptr(u), _ptr(f))


def residual(n, h, u, f):
    r = np.empty_like(u)
    _load().ora_residual(n, h, _ptr(u), _ptr(f), _ptr(r))
    return r


def interior_sumsq(n, a):
    return float(_load().ora_interior_sumsq(n, _ptr(_f64(a))))


def restrict_fw(nf, fine):
    coarse = np.empty((nf // 2 + 1) ** 3, dtype=np.float64)
    _load().ora_restrict_fw(nf, _ptr(_f64(fine)), _ptr(coarse))
    return coarse


def prolong(nc, coarse, fine, add):
    _load().ora_prolong(nc, _ptr(_f64(coarse)), _ptr(fine), 1 if add else 0)


def coarsest(h, u, f):
    _load().ora_coarsest(h, _ptr(u), _ptr(f))


def vcycle(n, h, u, f, npre=2, npost=2):
    _check_grid(u, n); _check_grid(f, n)
    _load().ora_vcycle(n, h, _ptr(u), _ptr(f), npre, npost)


def fmg(n, h, u, f, ncycle=6, npre=2, npost=2):
    _check_grid(u, n); _check_grid(f, n)
    _load().ora_fmg(n, h, _ptr(u), _ptr(f), ncycle, npre, npost)


def solve(n, h, u, f, *, fmg=True, ncycle=6, npre=2, npost=2, tol=0.0, max_vcycles=0):
    """Solve in place. Returns (extra V-cycles made or -1, relative residual history)."""
    _check_grid(u, n); _check_grid(f, n)
    cap = max_vcycles + 1
    hist = np.zeros(cap, dtype=np.float64)
    made = _load().ora_solve(n, h, _ptr(u), _ptr(f), 1 if fmg else 0, ncycle, npre, npost,
                             tol, max_vcycles, _ptr(hist), cap)
    nh = (made if made >= 0 else max_vcycles) + 1
    return int(made), hist[:nh].copy()


# --- step 3 ----------------------------------------------------------------
def source(n, h, a0, phiN):
    phiN = _f64(phiN)
    _check_grid(phiN, n)
    src = np.empty_like(phiN)
    _load().ora_source(n, h, a0, _ptr(phiN), _ptr(src))
    return src


# --- nested boxes ------------------------------------------------------------
def boundary_fill(n, Lp, cp, up, L, c, u):
    _load().ora_boundary_fill(n, Lp, cp[0], cp[1], cp[2], _ptr(_f64(up)), L, c[0], c[1], c[2], _ptr(u))


def far_field(n, L, center, rho, G=4.30e-3, a0=3.6, lmax=8, phiN=None, phi=None):
    """Boundary values of the outermost box from the mass inside it: the
    multipole expansion (degree <= lmax) of the node masses for Phi_N and the
    point-mass QUMOND potential of the total mass for Phi.  Writes the
    boundary nodes of phiN and phi (new zero arrays when None).
    Returns (phiN, phi, total mass)."""
    rho = _f64(rho)
    _check_grid(rho, n)
    phiN = np.zeros((n + 1) ** 3) if phiN is None else phiN
    phi = np.zeros((n + 1) ** 3) if phi is None else phi
    _check_grid(phiN, n)
    _check_grid(phi, n)
    M = _load().ora_far_field(n, L, center[0], center[1], center[2], _ptr(rho), G, a0, lmax, _ptr(phiN), _ptr(phi))
    return phiN, phi, float(M)


# --- forces and rotation curve -------------------------------------------------
def _ptr_array(arrs):
    arr = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    return arr


def forces(n, L0, center, phis, qx, qy, qz, ratio=2):
    qx, qy, qz = _f64(qx), _f64(qy), _f64(qz)
    gx, gy, gz = np.empty_like(qx), np.empty_like(qx), np.empty_like(qx)
    pa = _ptr_array(phis)
    missed = _load().ora_forces(len(phis), n, L0, ratio, center[0], center[1], center[2], ctypes.cast(pa, _P),
                                _ptr(qx), _ptr(qy), _ptr(qz), qx.size, _ptr(gx), _ptr(gy), _ptr(gz))
    return gx, gy, gz, int(missed)


def rotation_curve(n, L0, center, phis, nbins, rmax, nphi=64, frac=0.2, ratio=2):
    r = np.empty(nbins, dtype=np.float64)
    vc = np.empty(nbins, dtype=np.float64)
    pa = _ptr_array(phis)
    _load().ora_rotation_curve(len(phis), n, L0, ratio, center[0], center[1], center[2], ctypes.cast(pa, _P),
                               nbins, rmax, nphi, frac, _ptr(r), _ptr(vc))
    return r, vc


def rotation_curve_algebraic(n, L0, center, phiNs, nbins, rmax, nphi=64, frac=0.2, ratio=2, a0=3.6):
    """Rotation curve of the algebraic MOND relation (Eq. 3) from the Newtonian potentials."""
    r = np.empty(nbins, dtype=np.float64)
    vc = np.empty(nbins, dtype=np.float64)
    pa = _ptr_array(phiNs)
    _load().ora_rotation_curve_algebraic(len(phiNs), n, L0, ratio, center[0], center[1], center[2],
                                         ctypes.cast(pa, _P), nbins, rmax, nphi, frac, a0, _ptr(r), _ptr(vc))
    return r, vc


def sigma_z(n, L0, center, phis, nbins, rmax, z_eval, h, nphi=64, frac=0.2, ratio=2):
    """Vertical velocity dispersion of an isothermal sech^2(z/h) layer (Section 5.6)."""
    r = np.empty(nbins, dtype=np.float64)
    sg = np.empty(nbins, dtype=np.float64)
    pa = _ptr_array(phis)
    _load().ora_sigma_z(len(phis), n, L0, ratio, center[0], center[1], center[2], ctypes.cast(pa, _P), nbins, rmax,
                        nphi, frac, z_eval, h, _ptr(r), _ptr(sg))
    return r, sg


def chi2(vc, v_obs, sigma):
    """Reduced chi^2 of each row of vc against (v_obs, sigma) (Section 3.5)."""
    vc = np.ascontiguousarray(np.atleast_2d(vc), dtype=np.float64)
    v_obs, sigma = _f64(v_obs), _f64(sigma)
    out = np.empty(vc.shape[0])
    _load().ora_chi2(_ptr(vc), _ptr(v_obs), _ptr(sigma), vc.shape[1], vc.shape[0], _ptr(out))
    return out


# --- the whole path, Section 2 ---------------------------------------------------
@dataclass
class Box:
    n: int
    L: float
    center: tuple
    rho_fixed: np.ndarray = None
    rho: np.ndarray = None
    phiN: np.ndarray = None
    src: np.ndarray = None
    phi: np.ndarray = None
    kept: int = 0
    newton_vcycles: int = 0
    mond_vcycles: int = 0
    newton_hist: np.ndarray = field(default=None)
    mond_hist: np.ndarray = field(default=None)

    @property
    def h(self):
        return self.L / self.n


def pipeline(particles, n, L0, nboxes, *, center=(0.0, 0.0, 0.0), G=4.30e-3, a0=3.6, shift=24,
             ncycle=6, npre=2, npost=2, tol=0.0, max_vcycles=0, bc_newton=None, bc_mond=None, ratio=2,
             far_field_lmax=None):
    """Steps 1-4 of Section 2 for every nested box, outermost first.

    Box b has side L0/ratio^b (ratio 2 in the paper).  Box 0 takes its boundary values from bc_newton /
    bc_mond (callables (x, y, z) -> value; None means zero, as in the paper's
    outermost box), or, with far_field_lmax set, from far_field() of its own
    density; box b >= 1 interpolates them from box b-1 (Section 2)."""
    boxes = []
    N = (n + 1) ** 3
    ii = np.arange(n + 1)
    kk, jj, i3 = np.meshgrid(ii, ii, ii, indexing="ij")
    on_bnd = ((i3 == 0) | (i3 == n) | (jj == 0) | (jj == n) | (kk == 0) | (kk == n)).ravel()
    for b in range(nboxes):
        L = L0 / ratio ** b
        bx = Box(n=n, L=L, center=tuple(center))
        bx.rho_fixed, bx.kept = cic_deposit(n, L, center, shift, particles.x, particles.y, particles.z, particles.m)
        bx.rho = rho_from_fixed(n, L, shift, bx.rho_fixed)
        f_newton = (4.0 * np.pi * G) * bx.rho
        if b == 0 and far_field_lmax is not None:
            ffN, ffM, _ = far_field(n, L, center, bx.rho, G=G, a0=a0, lmax=far_field_lmax)
        for kind in ("newton", "mond"):
            u = np.zeros(N)
            if b == 0 and far_field_lmax is not None:
                u[on_bnd] = (ffN if kind == "newton" else ffM)[on_bnd]
            elif b == 0:
                bc = bc_newton if kind == "newton" else bc_mond
                if bc is not None:
                    h = L / n
                    xs = center[0] - 0.5 * L + i3.ravel() * h
                    ys = center[1] - 0.5 * L + jj.ravel() * h
                    zs = center[2] - 0.5 * L + kk.ravel() * h
                    u[on_bnd] = bc(xs[on_bnd], ys[on_bnd], zs[on_bnd])
            else:
                parent = boxes[b - 1]
                up = parent.phiN if kind == "newton" else parent.phi
                boundary_fill(n, parent.L, center, up, L, center, u)
            if kind == "newton":
                made, hist = solve(n, L / n, u, f_newton, ncycle=ncycle, npre=npre, npost=npost,
                                   tol=tol, max_vcycles=max_vcycles)
                bx.phiN, bx.newton_vcycles, bx.newton_hist = u, made, hist
                bx.src = source(n, L / n, a0, bx.phiN)
            else:
                made, hist = solve(n, L / n, u, bx.src, ncycle=ncycle, npre=npre, npost=npost,
                                   tol=tol, max_vcycles=max_vcycles)
                bx.phi, bx.mond_vcycles, bx.mond_hist = u, made, hist
        boxes.append(bx)
    return boxes
