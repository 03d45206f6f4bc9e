"""Python binding of libqumond's C ABI (include/qumond.h).

Argument marshalling only: every function checks tensor placement, dtype,
shape and contiguity, then calls the C entry point of the same name with raw
device pointers and the current CUDA stream.  All arithmetic of the path runs
in the library's CUDA kernels; there is no fallback.  If the shared library
is missing or fails to load, importing this module raises.

Grids are 1-D tensors of (n+1)^3 elements (x fastest) or (n+1, n+1, n+1)
tensors indexed [k, j, i].
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

_LIB_PATH = _build.LIB

QUMOND_OK = 0
QUMOND_ERR_INVALID_ARG = 1
QUMOND_ERR_CUDA = 2
QUMOND_ERR_NOT_CONVERGED = 3
QUMOND_ERR_TIMEOUT = 4
QUMOND_ERR_OUT_OF_MEMORY = 5

QUMOND_PREC_FP64 = 0
QUMOND_PREC_MIXED = 1
QUMOND_PREC_MIXED_FIXED = 2
QUMOND_BC_ZERO = 0
QUMOND_BC_GIVEN = 1
QUMOND_BC_MULTIPOLE = 2

EXPORTED = (
    "qumond_default_params", "qumond_create", "qumond_destroy", "qumond_last_error", "qumond_deposit",
    "qumond_solve_newton", "qumond_source", "qumond_solve_mond", "qumond_forces", "qumond_rotation_curve",
    "qumond_chi2", "qumond_rotation_curve_algebraic", "qumond_sigma_z", "qumond_trace_classes", "qumond_trace_timing", "qumond_trace_read", "qumond_solve_mond_noalloc",
    "qumond_set_barrier_poll_limit", "qumond_rotation_curve_sets", "qumond_far_field",
    "qumond_guess_num_params", "qumond_guess_create", "qumond_guess_destroy", "qumond_guess_last_error",
    "qumond_guess_set_params", "qumond_guess_get_params", "qumond_guess_make_sample", "qumond_guess_forward",
    "qumond_guess_gradients", "qumond_guess_train_step", "qumond_guess_apply", "qumond_guess_tensor_path",
    "qumond_guess_tensor_path_available", "qumond_guess_status", "qumond_guess_launches", "qumond_guess_tc_selftest",
)
NOALLOC_MAX_N = 64


class qumond_params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("nboxes", ctypes.c_int),
        ("L0", ctypes.c_double),
        ("center", ctypes.c_double * 3),
        ("G", ctypes.c_double),
        ("a0", ctypes.c_double),
        ("npre", ctypes.c_int),
        ("npost", ctypes.c_int),
        ("ncycle", ctypes.c_int),
        ("rel_tol", ctypes.c_double),
        ("max_vcycles", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("bc_mode", ctypes.c_int),
        ("warm_start", ctypes.c_int),
        ("deposit_shift", ctypes.c_int),
        ("rc_box_frac", ctypes.c_double),
        ("box_ratio", ctypes.c_int),
        ("use_graphs", ctypes.c_int),
        ("persistent_vcycle", ctypes.c_int),
        ("nsets", ctypes.c_int),
        ("tile_small", ctypes.c_int),
        ("small_cluster", ctypes.c_int),
        ("dc_vcycles", ctypes.c_int),
    ]


class qumond_stats(ctypes.Structure):
    _fields_ = [
        ("vcycles", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("rel_residual_fmg", ctypes.c_double),
        ("rel_residual", ctypes.c_double),
    ]


class qumond_kernel_stat(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char_p),
        ("launches", ctypes.c_int64),
        ("bytes", ctypes.c_double),
        ("ms", ctypes.c_double),
        ("timed", ctypes.c_int64),
        ("timed_bytes", ctypes.c_double),
    ]


class qumond_counters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("cell_updates", ctypes.c_int64)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_int64
_D = ctypes.c_double


def load_library(path: str = _LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError("libqumond.so not built (%s): run paper_1201_3185_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    sigs = {
        "qumond_default_params": (None, [ctypes.POINTER(qumond_params)]),
        "qumond_create": (_I, [ctypes.POINTER(qumond_params), ctypes.POINTER(_P)]),
        "qumond_destroy": (None, [_P]),
        "qumond_last_error": (ctypes.c_char_p, [_P]),
        "qumond_deposit": (_I, [_P, _I, _P, _P, _P, _P, _L, _P, _P, _P]),
        "qumond_solve_newton": (_I, [_P, _I, _P, _P, _P, ctypes.POINTER(qumond_stats), _P]),
        "qumond_source": (_I, [_P, _I, _P, _P, _P]),
        "qumond_solve_mond": (_I, [_P, _I, _P, _P, _P, ctypes.POINTER(qumond_stats), _P]),
        "qumond_forces": (_I, [_P, _P, _P, _P, _P, _L, _P, _P, _P, _P]),
        "qumond_rotation_curve": (_I, [_P, _P, _I, _D, _I, _P, _P, _P]),
        "qumond_rotation_curve_sets": (_I, [_P, _P, _I, _P, _I, _P, _P, _P]),
        "qumond_far_field": (_I, [_P, _P, _P, _P, _P]),
        "qumond_chi2": (_I, [_P, _P, _P, _P, _I, _I, _P, _P]),
        "qumond_rotation_curve_algebraic": (_I, [_P, _P, _I, _D, _I, _P, _P, _P]),
        "qumond_sigma_z": (_I, [_P, _P, _I, _D, _I, _D, _D, _P, _P, _P]),
        "qumond_set_barrier_poll_limit": (_I, [_P, _L]),
        "qumond_trace_classes": (_I, []),
        "qumond_trace_timing": (_I, [_P, _I, _I]),
        "qumond_trace_read": (_I, [_P, ctypes.POINTER(qumond_kernel_stat), _I, ctypes.POINTER(qumond_counters), _I]),
        "qumond_solve_mond_noalloc": (_I, [ctypes.POINTER(qumond_params), _I, _P, _P, _P, ctypes.POINTER(qumond_stats),
                                           _P, ctypes.c_char_p, ctypes.c_size_t]),
        "qumond_guess_num_params": (ctypes.c_int64, []),
        "qumond_guess_create": (_I, [_I, _D, ctypes.POINTER(_P)]),
        "qumond_guess_destroy": (None, [_P]),
        "qumond_guess_last_error": (ctypes.c_char_p, [_P]),
        "qumond_guess_set_params": (_I, [_P, _P, _P]),
        "qumond_guess_get_params": (_I, [_P, _P, _P]),
        "qumond_guess_make_sample": (_I, [_P, _D, _P, _P, _P, _P, _P]),
        "qumond_guess_forward": (_I, [_P, _P, ctypes.c_float, _P, _P]),
        "qumond_guess_gradients": (_I, [_P, _P, _P, _I, _P, _P, _P]),
        "qumond_guess_train_step": (_I, [_P, _P, _P, _I, ctypes.c_float, _P, _P]),
        "qumond_guess_apply": (_I, [_P, _D, ctypes.c_float, _P, _P, _P, _P]),
        "qumond_guess_tensor_path": (_I, [_P, _I]),
        "qumond_guess_tensor_path_available": (_I, [_P]),
        "qumond_guess_tc_selftest": (_I, []),
        "qumond_guess_launches": (ctypes.c_int64, [_P]),
        "qumond_guess_status": (_I, [_P, _P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


class QumondError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("qumond status %d: %s" % (status, message))
        self.status = status


class NotConverged(QumondError):
    pass


def default_params(**overrides) -> qumond_params:
    p = qumond_params()
    _lib.qumond_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "center":
            p.center[0], p.center[1], p.center[2] = (float(c) for c in v)
        elif not hasattr(p, k):
            raise TypeError("unknown parameter %r" % k)
        else:
            setattr(p, k, v)
    return p


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, numel=None, name="tensor") -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if t.device.type != "cuda":
        raise ValueError("%s must live on a CUDA device" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (name, numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def qumond_solve_mond_noalloc(params: qumond_params, box, src, phi_parent, phi, stats=False, stream=None):
    """The solve of qumond_solve_mond for callers that cannot allocate device
    memory: no context, scratch in the library's fixed device array (n <= 64)."""
    nodes = (params.n + 1) ** 3
    a = _dev(src, torch.float64, nodes, "src")
    par = _dev(phi_parent, torch.float64, nodes, "phi_parent") if phi_parent is not None else None
    o = _dev(phi, torch.float64, nodes, "phi")
    st = qumond_stats()
    buf = ctypes.create_string_buffer(512)
    status = _lib.qumond_solve_mond_noalloc(ctypes.byref(params), box, a, par, o,
                                            ctypes.byref(st) if stats else None, _stream(stream), buf, 512)
    if status != QUMOND_OK:
        cls = NotConverged if status == QUMOND_ERR_NOT_CONVERGED else QumondError
        raise cls(status, buf.value.decode())
    if stats:
        return SolveStats(st.vcycles, bool(st.converged), st.rel_residual_fmg, st.rel_residual)
    return None


@dataclass
class KernelStat:
    name: str
    launches: int
    bytes: float
    ms: float
    timed: int
    timed_bytes: float


@dataclass
class SolveStats:
    vcycles: int
    converged: bool
    rel_residual_fmg: float
    rel_residual: float


class Context:
    """A qumond_ctx: parameters plus the multigrid scratch on the current device."""

    def __init__(self, params: qumond_params | None = None, **overrides):
        if params is None:
            params = default_params(**overrides)
        elif overrides:
            raise TypeError("give either params or keyword overrides")
        self.params = params
        self._ptr = ctypes.c_void_p()
        st = _lib.qumond_create(ctypes.byref(params), ctypes.byref(self._ptr))
        if st != QUMOND_OK:
            raise QumondError(st, "qumond_create failed (invalid parameters or out of memory)")

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if self._ptr:
            _lib.qumond_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n(self) -> int:
        return self.params.n

    @property
    def nsets(self) -> int:
        return max(1, self.params.nsets)

    @property
    def grid_nodes(self) -> int:
        """Nodes of one grid, (n+1)^3."""
        return (self.params.n + 1) ** 3

    @property
    def nodes(self) -> int:
        """Elements of a grid argument: one (n+1)^3 grid per set."""
        return self.nsets * (self.params.n + 1) ** 3

    def box_side(self, box: int) -> float:
        return self.params.L0 / self.params.box_ratio ** box

    def _check(self, st: int):
        if st == QUMOND_OK:
            return
        msg = _lib.qumond_last_error(self._ptr).decode()
        if st == QUMOND_ERR_NOT_CONVERGED:
            raise NotConverged(st, msg)
        raise QumondError(st, msg)

    # -- entry points -------------------------------------------------------------
    def qumond_deposit(self, box, x, y, z, mass, rho_fixed, rho=None, stream=None):
        """x, y, z, mass: the particles of every set, set s's np at s*np (np = numel / nsets)."""
        npart = x.numel()
        if npart % self.nsets:
            raise ValueError("the particle arrays must hold the same count for every set")
        args = [_dev(a, torch.float64, npart, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (mass, "mass"))]
        q = _dev(rho_fixed, torch.int64, self.nodes, "rho_fixed")
        r = _dev(rho, torch.float64, self.nodes, "rho") if rho is not None else None
        self._check(_lib.qumond_deposit(self._ptr, box, *args, npart // self.nsets, q, r, _stream(stream)))

    def _solve(self, fn, box, rhs, parent, out, want_stats, stream):
        a = _dev(rhs, torch.float64, self.nodes, "rhs")
        par = _dev(parent, torch.float64, self.nodes, "parent") if parent is not None else None
        o = _dev(out, torch.float64, self.nodes, "phi")
        st = (qumond_stats * self.nsets)()
        status = fn(self._ptr, box, a, par, o, ctypes.cast(st, ctypes.POINTER(qumond_stats)) if want_stats else None,
                    _stream(stream))
        self._check(status)
        if want_stats:
            out_st = [SolveStats(x.vcycles, bool(x.converged), x.rel_residual_fmg, x.rel_residual) for x in st]
            return out_st[0] if self.nsets == 1 else out_st
        return None

    def qumond_solve_newton(self, box, rho, phiN_parent, phiN, stats=False, stream=None):
        return self._solve(_lib.qumond_solve_newton, box, rho, phiN_parent, phiN, stats, stream)

    def qumond_source(self, box, phiN, src, stream=None):
        a = _dev(phiN, torch.float64, self.nodes, "phiN")
        b = _dev(src, torch.float64, self.nodes, "src")
        self._check(_lib.qumond_source(self._ptr, box, a, b, _stream(stream)))

    def qumond_solve_mond(self, box, src, phi_parent, phi, stats=False, stream=None):
        return self._solve(_lib.qumond_solve_mond, box, src, phi_parent, phi, stats, stream)

    def qumond_far_field(self, rho, phiN, phi, stream=None):
        """Boundary values of box 0 from its own mass (bc_mode QUMOND_BC_MULTIPOLE)."""
        self._check(_lib.qumond_far_field(self._ptr, _dev(rho, torch.float64, self.nodes, "rho"),
                                          _dev(phiN, torch.float64, self.nodes, "phiN"),
                                          _dev(phi, torch.float64, self.nodes, "phi"), _stream(stream)))

    def _phis(self, phis):
        if len(phis) != self.params.nboxes:
            raise ValueError("need one potential per box (%d)" % self.params.nboxes)
        ptrs = [_dev(p, torch.float64, self.nodes, "phi_boxes[%d]" % b).value for b, p in enumerate(phis)]
        return (ctypes.c_void_p * len(ptrs))(*ptrs)

    def qumond_forces(self, phis, qx, qy, qz, gx, gy, gz, stream=None):
        """Points and forces of every set, set s's nq at s*nq (nq = numel / nsets)."""
        nq = qx.numel()
        if nq % self.nsets:
            raise ValueError("the point arrays must hold the same count for every set")
        arr = self._phis(phis)
        pts = [_dev(a, torch.float64, nq, nm) for a, nm in ((qx, "qx"), (qy, "qy"), (qz, "qz"),
                                                             (gx, "gx"), (gy, "gy"), (gz, "gz"))]
        self._check(_lib.qumond_forces(self._ptr, ctypes.cast(arr, _P), *pts[:3], nq // self.nsets, *pts[3:],
                                       _stream(stream)))

    def qumond_rotation_curve(self, phis, nbins, rmax, nphi, r_out, vc_out, stream=None):
        arr = self._phis(phis)
        r = _dev(r_out, torch.float64, nbins * self.nsets, "r_out")
        v = _dev(vc_out, torch.float64, nbins * self.nsets, "vc_out")
        self._check(_lib.qumond_rotation_curve(self._ptr, ctypes.cast(arr, _P), nbins, float(rmax), nphi, r, v,
                                               _stream(stream)))

    def qumond_rotation_curve_sets(self, phis, nbins, rmax, nphi, r_out, vc_out, stream=None):
        """Every set's curve with its own outermost radius rmax[s] (device tensor of nsets)."""
        arr = self._phis(phis)
        rm = _dev(rmax, torch.float64, self.nsets, "rmax")
        r = _dev(r_out, torch.float64, nbins * self.nsets, "r_out")
        v = _dev(vc_out, torch.float64, nbins * self.nsets, "vc_out")
        self._check(_lib.qumond_rotation_curve_sets(self._ptr, ctypes.cast(arr, _P), nbins, rm, nphi, r, v,
                                                    _stream(stream)))

    def qumond_rotation_curve_algebraic(self, phiNs, nbins, rmax, nphi, r_out, vc_out, stream=None):
        arr = self._phis(phiNs)
        r = _dev(r_out, torch.float64, nbins * self.nsets, "r_out")
        v = _dev(vc_out, torch.float64, nbins * self.nsets, "vc_out")
        self._check(_lib.qumond_rotation_curve_algebraic(self._ptr, ctypes.cast(arr, _P), nbins, float(rmax), nphi, r,
                                                         v, _stream(stream)))

    def qumond_sigma_z(self, phis, nbins, rmax, nphi, z_eval, h, r_out, sigma_out, stream=None):
        arr = self._phis(phis)
        r = _dev(r_out, torch.float64, nbins * self.nsets, "r_out")
        v = _dev(sigma_out, torch.float64, nbins * self.nsets, "sigma_out")
        self._check(_lib.qumond_sigma_z(self._ptr, ctypes.cast(arr, _P), nbins, float(rmax), nphi, float(z_eval),
                                        float(h), r, v, _stream(stream)))

    def qumond_chi2(self, vc, v_obs, sigma, chi2_out, stream=None):
        """Reduced chi^2 of each row of vc (nsets x nbins) against v_obs, sigma."""
        nsets, nbins = (vc.shape[0], vc.shape[1]) if vc.dim() == 2 else (1, vc.numel())
        a = _dev(vc, torch.float64, nsets * nbins, "vc")
        b = _dev(v_obs, torch.float64, nbins, "v_obs")
        c = _dev(sigma, torch.float64, nbins, "sigma")
        d = _dev(chi2_out, torch.float64, nsets, "chi2")
        self._check(_lib.qumond_chi2(self._ptr, a, b, c, nbins, nsets, d, _stream(stream)))

    def qumond_set_barrier_poll_limit(self, polls: int):
        """Polls before a grid barrier of the cooperative small-level V-cycle
        gives up (the solve then fails with QUMOND_ERR_TIMEOUT)."""
        self._check(_lib.qumond_set_barrier_poll_limit(self._ptr, int(polls)))

    # -- tracing ------------------------------------------------------------------
    def qumond_trace_timing(self, on: bool, only: str | None = None):
        """Kernel timing with CUDA events; only=None times every launch (kernels
        launched one by one), only=<class name> times that class inside the graphs."""
        idx = -1
        if only is not None:
            names = self.trace_class_names()
            if only not in names:
                raise ValueError("unknown kernel class %r" % only)
            idx = names.index(only)
        self._check(_lib.qumond_trace_timing(self._ptr, 1 if on else 0, idx))

    def trace_class_names(self):
        k = _lib.qumond_trace_classes()
        arr = (qumond_kernel_stat * k)()
        self._check(_lib.qumond_trace_read(self._ptr, arr, k, None, 0))
        return [a.name.decode() for a in arr]

    def qumond_trace_read(self, reset: bool = False):
        """Returns ({class name: KernelStat}, total launches, cell updates)."""
        k = _lib.qumond_trace_classes()
        arr = (qumond_kernel_stat * k)()
        tot = qumond_counters()
        self._check(_lib.qumond_trace_read(self._ptr, arr, k, ctypes.byref(tot), 1 if reset else 0))
        stats = {a.name.decode(): KernelStat(a.name.decode(), a.launches, a.bytes, a.ms, a.timed, a.timed_bytes)
                 for a in arr}
        return stats, tot.launches, tot.cell_updates


# --- the learned initial guess (include/qumond_guess.h) ---------------------------------
class Guess:
    """A qumond_guess: the U-Net that maps (rho, Phi_N) of a box to Phi - Phi_N."""

    def __init__(self, S: int, phi_scale: float):
        self.S = int(S)
        self.phi_scale = float(phi_scale)
        self._ptr = ctypes.c_void_p()
        st = _lib.qumond_guess_create(self.S, self.phi_scale, ctypes.byref(self._ptr))
        if st != QUMOND_OK:
            raise QumondError(st, "qumond_guess_create failed (S must be a multiple of 16 in [16, 512]; "
                                  "or out of memory)")

    @staticmethod
    def num_params() -> int:
        return int(_lib.qumond_guess_num_params())

    @property
    def voxels(self) -> int:
        return self.S ** 3

    def close(self):
        if self._ptr:
            _lib.qumond_guess_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != QUMOND_OK:
            raise QumondError(st, _lib.qumond_guess_last_error(self._ptr).decode())

    def qumond_guess_tensor_path(self, mode: int):
        """1: tcgen05 convolutions where they apply (the default when available), 0: mma.sync everywhere."""
        self._check(_lib.qumond_guess_tensor_path(self._ptr, int(mode)))

    def qumond_guess_launches(self) -> int:
        """Kernels this network has enqueued since it was created."""
        return int(_lib.qumond_guess_launches(self._ptr))

    def qumond_guess_tensor_path_available(self) -> bool:
        return bool(_lib.qumond_guess_tensor_path_available(self._ptr))

    @staticmethod
    def qumond_guess_tc_selftest() -> int:
        """One tcgen05 MMA from the library's descriptors against a CPU product: 1 match, 0 mismatch, -1 error."""
        return int(_lib.qumond_guess_tc_selftest())

    def qumond_guess_status(self, stream=None):
        self._check(_lib.qumond_guess_status(self._ptr, _stream(stream)))

    def qumond_guess_set_params(self, params, stream=None):
        self._check(_lib.qumond_guess_set_params(self._ptr, _dev(params, torch.float32, self.num_params(), "params"),
                                                 _stream(stream)))

    def qumond_guess_get_params(self, params, stream=None):
        self._check(_lib.qumond_guess_get_params(self._ptr, _dev(params, torch.float32, self.num_params(), "params"),
                                                 _stream(stream)))

    def qumond_guess_make_sample(self, rho_scale, rho, phiN, phi, sample, stream=None):
        n = (self.S + 1) ** 3
        self._check(_lib.qumond_guess_make_sample(
            self._ptr, float(rho_scale), _dev(rho, torch.float64, n, "rho"), _dev(phiN, torch.float64, n, "phiN"),
            _dev(phi, torch.float64, n, "phi"), _dev(sample, torch.bfloat16, 3 * self.voxels, "sample"),
            _stream(stream)))

    def qumond_guess_forward(self, sample, box_flag, y, stream=None):
        self._check(_lib.qumond_guess_forward(self._ptr, _dev(sample, torch.bfloat16, 3 * self.voxels, "sample"),
                                              float(box_flag), _dev(y, torch.float32, self.voxels, "y"),
                                              _stream(stream)))

    def _batch(self, samples, flags):
        if len(samples) != len(flags) or not samples:
            raise ValueError("need one box flag per sample, at least one sample")
        ptrs = (ctypes.c_void_p * len(samples))(
            *[_dev(t, torch.bfloat16, 3 * self.voxels, "sample").value for t in samples])
        fl = (ctypes.c_float * len(flags))(*[float(f) for f in flags])
        return ptrs, fl

    def qumond_guess_gradients(self, samples, flags, grads, loss=None, stream=None):
        ptrs, fl = self._batch(samples, flags)
        lp = _dev(loss, torch.float32, 1, "loss") if loss is not None else None
        self._check(_lib.qumond_guess_gradients(self._ptr, ctypes.cast(ptrs, _P), ctypes.cast(fl, _P), len(samples),
                                                _dev(grads, torch.float32, self.num_params(), "grads"), lp,
                                                _stream(stream)))

    def qumond_guess_train_step(self, samples, flags, lr, loss=None, stream=None):
        ptrs, fl = self._batch(samples, flags)
        lp = _dev(loss, torch.float32, 1, "loss") if loss is not None else None
        self._check(_lib.qumond_guess_train_step(self._ptr, ctypes.cast(ptrs, _P), ctypes.cast(fl, _P), len(samples),
                                                 float(lr), lp, _stream(stream)))

    def qumond_guess_apply(self, rho_scale, box_flag, rho, phiN, phi, stream=None):
        n = (self.S + 1) ** 3
        self._check(_lib.qumond_guess_apply(self._ptr, float(rho_scale), float(box_flag),
                                            _dev(rho, torch.float64, n, "rho"), _dev(phiN, torch.float64, n, "phiN"),
                                            _dev(phi, torch.float64, n, "phi"), _stream(stream)))
