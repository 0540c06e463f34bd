"""Thin Python binding of the C ABI in ``include/lqcd.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: device buffers are torch tensors (used for memory and
streams only), scalars are passed through, and the status code is turned into
an exception.  The shared library must have been built (``build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

# --- enums (mirror lqcd.h) ---------------------------------------------------
LQCD_OK = 0
LQCD_ERR_INVALID = -1
LQCD_ERR_CUDA = -2
LQCD_ERR_NOCONV = -3
LQCD_ERR_NONFINITE = -4
LQCD_ERR_TIMEOUT = -5
LQCD_ERR_OOM = -6
LQCD_ERR_UNSUPPORTED = -7
LQCD_ERR_COMM = -8

LQCD_FULL, LQCD_EVEN, LQCD_ODD = 0, 1, 2
LQCD_F64, LQCD_DF64, LQCD_F32, LQCD_BF16S, LQCD_F16S = 0, 1, 2, 3, 4
LQCD_LAYOUT_LEXI, LQCD_LAYOUT_EO = 0, 1
LQCD_SOLVER_CG, LQCD_SOLVER_BICGSTAB = 0, 1

_STATUS_NAMES = {0: "LQCD_OK", -1: "LQCD_ERR_INVALID", -2: "LQCD_ERR_CUDA", -3: "LQCD_ERR_NOCONV",
                 -4: "LQCD_ERR_NONFINITE", -5: "LQCD_ERR_TIMEOUT", -6: "LQCD_ERR_OOM",
                 -7: "LQCD_ERR_UNSUPPORTED", -8: "LQCD_ERR_COMM"}


class LqcdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


# --- structs -------------------------------------------------------------------
class lqcd_geom(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32 * 4), ("antiperiodic_t", ctypes.c_int32)]


class lqcd_field(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("scale", ctypes.c_void_p), ("layout", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("nrhs", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class lqcd_cg_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("outer_prec", ctypes.c_int32), ("inner_prec", ctypes.c_int32),
                ("delta", ctypes.c_double), ("max_restarts", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("sloppy_recon", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("inner_tol", ctypes.c_double)]


class lqcd_cg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("reliable_updates", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("true_resid", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lqcd_counters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("hop_launches", ctypes.c_uint64),
                ("bytes", ctypes.c_double), ("hop_bytes", ctypes.c_double),
                ("hop_flops", ctypes.c_double), ("hop_sites", ctypes.c_double)]


class lqcd_hmc_params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("kappa", ctypes.c_double), ("mu", ctypes.c_double),
                ("tau", ctypes.c_double), ("nsteps", ctypes.c_int32), ("nf", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("traj", ctypes.c_uint32), ("integrator", ctypes.c_int32),
                ("c1", ctypes.c_double), ("nsteps_gauge", ctypes.c_int32), ("force_prec", ctypes.c_int32),
                ("lam", ctypes.c_double), ("mu2", ctypes.c_double), ("nsteps_mid", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("cg", lqcd_cg_params)]


class lqcd_hmc_stats(ctypes.Structure):
    _fields_ = [("dH", ctypes.c_double), ("H0", ctypes.c_double), ("H1", ctypes.c_double),
                ("plaquette", ctypes.c_double), ("accepted", ctypes.c_int32),
                ("cg_iters", ctypes.c_int32), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# caller allocator callbacks (lqcd_alloc_fn, lqcd_free_fn)
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

# communication hooks of the domain-decomposed solve (lqcd_dd_comm)
_EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t)
_ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int)


class lqcd_dd_comm(ctypes.Structure):
    _fields_ = [("user", ctypes.c_void_p), ("exchange", _EXCHANGE_FN), ("allreduce", _ALLREDUCE_FN)]


# --- library loading ------------------------------------------------------------
_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double

# (name, restype, argtypes) of every entry point declared in include/lqcd.h
SIGNATURES = [
    ("lqcd_abi_version", _i, []),
    ("lqcd_create", _i, [ctypes.POINTER(_vp), _i, _vp]),
    ("lqcd_destroy", _i, [_vp]),
    ("lqcd_set_stream", _i, [_vp, _vp]),
    ("lqcd_last_error", ctypes.c_char_p, [_vp]),
    ("lqcd_get_counters", _i, [_vp, _vp]),
    ("lqcd_set_autotune", _i, [_vp, _i, ctypes.c_char_p]),
    ("lqcd_set_launch_choice", _i, [_vp, _i]),
    ("lqcd_set_allocator", _i, [_vp, _ALLOC_FN, _FREE_FN, _vp]),
    ("lqcd_reset_counters", _i, [_vp]),
    ("lqcd_measure_peaks", _i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    ("lqcd_trim_memory", _i, [_vp]),
    ("lqcd_memory_stats", _i, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    ("lqcd_field_bytes", ctypes.c_size_t, [ctypes.POINTER(lqcd_geom), _i, _i, _i,
                                           ctypes.POINTER(ctypes.c_size_t)]),
    ("lqcd_gauge_import", _i, [_vp, _vp, ctypes.POINTER(lqcd_geom), _i, ctypes.POINTER(_vp)]),
    ("lqcd_gauge_export", _i, [_vp, _vp, _vp]),
    ("lqcd_gauge_free", _i, [_vp, _vp]),
    ("lqcd_spinor_pack", _i, [_vp, ctypes.POINTER(lqcd_geom), _vp, lqcd_field]),
    ("lqcd_spinor_unpack", _i, [_vp, ctypes.POINTER(lqcd_geom), lqcd_field, _vp]),
    ("lqcd_spinor_convert", _i, [_vp, ctypes.POINTER(lqcd_geom), _i, lqcd_field, lqcd_field]),
    ("lqcd_dslash", _i, [_vp, _vp, lqcd_field, lqcd_field, ctypes.POINTER(lqcd_geom), _i, _i]),
    ("lqcd_dd_face_bytes", ctypes.c_size_t, [ctypes.POINTER(lqcd_geom), _i]),
    ("lqcd_dd_pack", _i, [_vp, _vp, lqcd_field, _vp, _vp, ctypes.POINTER(lqcd_geom), _i, _i, _i, _i]),
    ("lqcd_dd_dslash", _i, [_vp, _vp, lqcd_field, lqcd_field, _vp, _vp, ctypes.POINTER(lqcd_geom), _i, _i]),
    ("lqcd_dd_face_bytes_dir", ctypes.c_size_t, [ctypes.POINTER(lqcd_geom), _i, _i]),
    ("lqcd_dd_pack_dir", _i, [_vp, _vp, lqcd_field, _i, _vp, _vp, ctypes.POINTER(lqcd_geom), _i, _i, _i, _i]),
    ("lqcd_dd_dslash_zt", _i, [_vp, _vp, lqcd_field, lqcd_field, _vp, _vp, _vp, _vp, ctypes.POINTER(lqcd_geom),
                               _i, _i]),
    ("lqcd_apply_M", _i, [_vp, _vp, lqcd_field, lqcd_field, ctypes.POINTER(lqcd_geom), _d, _d, _i]),
    ("lqcd_apply_Mdag", _i, [_vp, _vp, lqcd_field, lqcd_field, ctypes.POINTER(lqcd_geom), _d, _d,
                             _i]),
    ("lqcd_cg_solve", _i, [_vp, _vp, lqcd_field, lqcd_field, ctypes.POINTER(lqcd_geom), _d, _d,
                           ctypes.POINTER(lqcd_cg_params), ctypes.POINTER(lqcd_cg_stats)]),
    ("lqcd_dd_cg_solve", _i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(lqcd_field),
                              ctypes.POINTER(lqcd_field), ctypes.POINTER(_vp), ctypes.POINTER(lqcd_geom), _i, _i,
                              _i, _i, _d, _d, ctypes.POINTER(lqcd_cg_params), ctypes.POINTER(lqcd_dd_comm),
                              ctypes.POINTER(lqcd_cg_stats)]),
    ("lqcd_cg_solve_batch", _i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(lqcd_field),
                                 ctypes.POINTER(lqcd_field), ctypes.POINTER(_d), ctypes.POINTER(_d),
                                 ctypes.POINTER(lqcd_cg_params), ctypes.POINTER(lqcd_cg_stats)]),
    ("lqcd_fermion_force", _i, [_vp, _vp, lqcd_field, _vp, ctypes.POINTER(lqcd_field),
                                ctypes.POINTER(lqcd_geom), _d, _d, ctypes.POINTER(lqcd_cg_params),
                                ctypes.POINTER(lqcd_cg_stats), ctypes.POINTER(_d)]),
    ("lqcd_fermion_force_ratio", _i, [_vp, _vp, lqcd_field, _vp, ctypes.POINTER(lqcd_geom), _d, _d, _d,
                                      ctypes.POINTER(lqcd_cg_params), ctypes.POINTER(lqcd_cg_stats),
                                      ctypes.POINTER(_d)]),
    ("lqcd_gauge_force", _i, [_vp, _vp, _d, _d, _i, _vp, ctypes.POINTER(_d)]),
    ("lqcd_plaquette", _i, [_vp, _vp, ctypes.POINTER(_d)]),
    ("lqcd_heatbath_sweep", _i, [_vp, _vp, _d, ctypes.c_uint64, ctypes.c_uint64, _i, _i]),
    ("lqcd_overrelax_sweep", _i, [_vp, _vp, _i, _i]),
    ("lqcd_momenta_gaussian", _i, [_vp, ctypes.POINTER(lqcd_geom), _vp, ctypes.c_uint64,
                                   ctypes.c_uint32]),
    ("lqcd_spinor_gaussian", _i, [_vp, ctypes.POINTER(lqcd_geom), lqcd_field, _i, ctypes.c_uint64,
                                  ctypes.c_uint32]),
    ("lqcd_gauge_update", _i, [_vp, _vp, _vp, _d]),
    ("lqcd_gauge_update_prec", _i, [_vp, _vp, _vp, _d, _i]),
    ("lqcd_momenta_update", _i, [_vp, ctypes.POINTER(lqcd_geom), _vp, _vp, _d]),
    ("lqcd_momenta_kinetic", _i, [_vp, ctypes.POINTER(lqcd_geom), _vp, ctypes.POINTER(_d)]),
    ("lqcd_gauge_copy", _i, [_vp, _vp, _vp]),
    ("lqcd_hmc_trajectory", _i, [_vp, _vp, ctypes.POINTER(lqcd_hmc_params),
                                 ctypes.POINTER(lqcd_hmc_stats)]),
    ("lqcd_plaquette_noalloc", _i, [_vp, ctypes.POINTER(lqcd_geom), _vp, _vp]),
]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_1209_5942_gb300.build.build() first "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name, None)
        if f is None:
            continue  # optional entry points are checked by the export test
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def lib():
    return _load()


def declared_symbols() -> list[str]:
    """Names of every function declared in include/lqcd.h (parsed from the header)."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                       "lqcd.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(lqcd_[A-Za-z0-9_]+)\s*\(",
                                 txt, flags=re.M)))


# --- helpers ---------------------------------------------------------------------
def geom(L, antiperiodic_t=True) -> lqcd_geom:
    g = lqcd_geom()
    for k in range(4):
        g.L[k] = int(L[k])
    g.antiperiodic_t = 1 if antiperiodic_t else 0
    return g


def field(t: torch.Tensor, layout=LQCD_LAYOUT_EO, prec=LQCD_F64, nrhs=1,
          scale: torch.Tensor | None = None) -> lqcd_field:
    if not t.is_cuda:
        raise ValueError("fields must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("fields must be contiguous")
    f = lqcd_field()
    f.ptr = t.data_ptr()
    f.scale = scale.data_ptr() if scale is not None else None
    f.layout = layout
    f.prec = prec
    f.nrhs = nrhs
    f.reserved = 0
    f._keep = (t, scale)  # the descriptor keeps its buffers alive
    return f


def field_bytes(L, parity, prec, nrhs=1, antiperiodic_t=True):
    sb = ctypes.c_size_t(0)
    n = lib().lqcd_field_bytes(ctypes.byref(geom(L, antiperiodic_t)), parity, prec, nrhs,
                               ctypes.byref(sb))
    return int(n), int(sb.value)


def alloc_field(L, parity, prec, nrhs=1, device="cuda"):
    """Zeroed EO field buffers (data, scale or None) for the given shape."""
    n, sb = field_bytes(L, parity, prec, nrhs)
    data = torch.zeros(n // 8, dtype=torch.float64, device=device)
    scale = torch.zeros(max(sb // 4, 1), dtype=torch.float32, device=device) if sb else None
    return data, scale


class TorchAllocator:
    """The (alloc, free) pair of lqcd_set_allocator backed by PyTorch's caching
    allocator on one device and stream."""

    def __init__(self, device: int, stream: torch.cuda.Stream):
        self.device, self.stream = device, stream

        def _alloc(nbytes, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:  # out of memory: the library reports LQCD_ERR_OOM
                return None

        def _free(ptr, user):
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = _ALLOC_FN(_alloc)  # kept alive as long as this object
        self.free_fn = _FREE_FN(_free)


class Context:
    """An lqcd_ctx bound to a device and a stream (default: torch's current
    stream).  torch_allocator=True routes the library's device memory through
    PyTorch's caching allocator (lqcd_set_allocator)."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None, torch_allocator=False):
        self._h = _vp()
        self._allocator = None
        stream = stream or torch.cuda.current_stream(device)
        st = lib().lqcd_create(ctypes.byref(self._h), device, _vp(stream.cuda_stream))
        if st != LQCD_OK:
            raise LqcdError(st, "lqcd_create failed")
        self.device = device
        if torch_allocator:
            self._allocator = TorchAllocator(device, stream)
            lqcd_set_allocator(self, self._allocator.alloc_fn, self._allocator.free_fn)

    @property
    def handle(self):
        return self._h

    def check(self, status: int, allow=()):
        if status != LQCD_OK and status not in allow:
            raise LqcdError(status, lib().lqcd_last_error(self._h).decode())
        return status

    def set_stream(self, stream: torch.cuda.Stream):
        self.check(lib().lqcd_set_stream(self._h, _vp(stream.cuda_stream)))

    def close(self):
        if self._h:
            lib().lqcd_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Gauge:
    """Library-owned gauge field (lqcd_gauge*)."""

    def __init__(self, ctx: Context, handle, L, antiperiodic_t):
        self.ctx = ctx
        self._h = handle
        self.L = tuple(int(v) for v in L)
        self.antiperiodic_t = antiperiodic_t

    @property
    def handle(self):
        return self._h

    @property
    def geom(self):
        return geom(self.L, self.antiperiodic_t)

    def free(self):
        if self._h:
            lib().lqcd_gauge_free(self.ctx.handle, self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# --- entry points (same names as the C ABI) ----------------------------------------
def lqcd_abi_version() -> int:
    return lib().lqcd_abi_version()


def lqcd_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def lqcd_set_autotune(ctx: Context, enable=True, cache_path=None):
    ctx.check(lib().lqcd_set_autotune(ctx.handle, int(bool(enable)),
                                      cache_path.encode() if cache_path else None))


def lqcd_measure_peaks(ctx: Context) -> tuple[float, float]:
    """(FP64 FMA, FP32 FMA) peak of the context's GPU in TFLOP/s, measured."""
    a, b = _d(0.0), _d(0.0)
    ctx.check(lib().lqcd_measure_peaks(ctx.handle, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def lqcd_trim_memory(ctx: Context) -> None:
    """Returns the unused memory of the context's pool to the driver."""
    ctx.check(lib().lqcd_trim_memory(ctx.handle))


def lqcd_memory_stats(ctx: Context) -> tuple[int, int]:
    """(bytes the context's pool holds, bytes in live allocations)."""
    r, u = ctypes.c_uint64(0), ctypes.c_uint64(0)
    ctx.check(lib().lqcd_memory_stats(ctx.handle, ctypes.byref(r), ctypes.byref(u)))
    return r.value, u.value


def lqcd_set_allocator(ctx: Context, alloc_fn=None, free_fn=None):
    """Sets the caller's (alloc, free) pair (ctypes callbacks of the lqcd_alloc_fn /
    lqcd_free_fn types, e.g. a TorchAllocator's); None passes a NULL pointer."""
    a = alloc_fn if alloc_fn is not None else _ALLOC_FN()
    f = free_fn if free_fn is not None else _FREE_FN()
    ctx.check(lib().lqcd_set_allocator(ctx.handle, a, f, None))


def lqcd_set_launch_choice(ctx: Context, choice: int):
    ctx.check(lib().lqcd_set_launch_choice(ctx.handle, int(choice)))


def lqcd_gauge_import(ctx: Context, U_lexi: torch.Tensor, L, recon=18, antiperiodic_t=True) -> Gauge:
    if U_lexi.dtype != torch.complex128 or not U_lexi.is_cuda or not U_lexi.is_contiguous():
        raise ValueError("U must be a contiguous CUDA complex128 tensor [V,4,3,3]")
    h = _vp()
    g = geom(L, antiperiodic_t)
    ctx.check(lib().lqcd_gauge_import(ctx.handle, _vp(U_lexi.data_ptr()), ctypes.byref(g), recon,
                                      ctypes.byref(h)))
    return Gauge(ctx, h, L, antiperiodic_t)


def lqcd_gauge_export(ctx: Context, U: Gauge, out: torch.Tensor):
    ctx.check(lib().lqcd_gauge_export(ctx.handle, U.handle, _vp(out.data_ptr())))


def lqcd_spinor_pack(ctx: Context, L, lexi: torch.Tensor, eo: lqcd_field, antiperiodic_t=True):
    g = geom(L, antiperiodic_t)
    ctx.check(lib().lqcd_spinor_pack(ctx.handle, ctypes.byref(g), _vp(lexi.data_ptr()), eo))


def lqcd_spinor_unpack(ctx: Context, L, eo: lqcd_field, lexi: torch.Tensor, antiperiodic_t=True):
    g = geom(L, antiperiodic_t)
    ctx.check(lib().lqcd_spinor_unpack(ctx.handle, ctypes.byref(g), eo, _vp(lexi.data_ptr())))


def lqcd_spinor_convert(ctx: Context, L, parity, inp: lqcd_field, out: lqcd_field,
                        antiperiodic_t=True):
    g = geom(L, antiperiodic_t)
    ctx.check(lib().lqcd_spinor_convert(ctx.handle, ctypes.byref(g), parity, inp, out))


def lqcd_dslash(ctx: Context, U: Gauge, inp: lqcd_field, out: lqcd_field, out_parity, dagger=0):
    g = U.geom
    ctx.check(lib().lqcd_dslash(ctx.handle, U.handle, inp, out, ctypes.byref(g), out_parity,
                                int(dagger)))


def lqcd_dd_face_bytes(L_local, prec) -> int:
    return int(lib().lqcd_dd_face_bytes(ctypes.byref(geom(L_local, False)), prec))


def lqcd_dd_face_bytes_dir(L_local, mu, prec) -> int:
    return int(lib().lqcd_dd_face_bytes_dir(ctypes.byref(geom(L_local, False)), int(mu), prec))


def lqcd_dd_pack(ctx: Context, U: Gauge, inp: lqcd_field, face_to_prev: torch.Tensor, face_to_next: torch.Tensor,
                 out_parity, dagger=0, negate_to_prev=False, negate_to_next=False):
    g = U.geom
    ctx.check(lib().lqcd_dd_pack(ctx.handle, U.handle, inp, _vp(face_to_prev.data_ptr()),
                                 _vp(face_to_next.data_ptr()), ctypes.byref(g), out_parity, int(dagger),
                                 int(bool(negate_to_prev)), int(bool(negate_to_next))))


def lqcd_dd_pack_dir(ctx: Context, U: Gauge, inp: lqcd_field, mu, face_to_prev: torch.Tensor,
                     face_to_next: torch.Tensor, out_parity, dagger=0, negate_to_prev=False, negate_to_next=False):
    g = U.geom
    ctx.check(lib().lqcd_dd_pack_dir(ctx.handle, U.handle, inp, int(mu), _vp(face_to_prev.data_ptr()),
                                     _vp(face_to_next.data_ptr()), ctypes.byref(g), out_parity, int(dagger),
                                     int(bool(negate_to_prev)), int(bool(negate_to_next))))


def lqcd_dd_dslash(ctx: Context, U: Gauge, inp: lqcd_field, out: lqcd_field, face_from_next: torch.Tensor,
                   face_from_prev: torch.Tensor, out_parity, dagger=0):
    g = U.geom
    ctx.check(lib().lqcd_dd_dslash(ctx.handle, U.handle, inp, out, _vp(face_from_next.data_ptr()),
                                   _vp(face_from_prev.data_ptr()), ctypes.byref(g), out_parity, int(dagger)))


def lqcd_dd_dslash_zt(ctx: Context, U: Gauge, inp: lqcd_field, out: lqcd_field, t_from_next: torch.Tensor,
                      t_from_prev: torch.Tensor, z_from_next, z_from_prev, out_parity, dagger=0):
    """z_from_next / z_from_prev: tensors, or None for a lattice not split along z."""
    g = U.geom
    zn = None if z_from_next is None else _vp(z_from_next.data_ptr())
    zp = None if z_from_prev is None else _vp(z_from_prev.data_ptr())
    ctx.check(lib().lqcd_dd_dslash_zt(ctx.handle, U.handle, inp, out, _vp(t_from_next.data_ptr()),
                                      _vp(t_from_prev.data_ptr()), zn, zp, ctypes.byref(g), out_parity,
                                      int(dagger)))


def lqcd_apply_M(ctx: Context, U: Gauge, inp: lqcd_field, out: lqcd_field, kappa, mu,
                 parity=LQCD_FULL):
    g = U.geom
    ctx.check(lib().lqcd_apply_M(ctx.handle, U.handle, inp, out, ctypes.byref(g), kappa, mu,
                                 parity))


def lqcd_apply_Mdag(ctx: Context, U: Gauge, inp: lqcd_field, out: lqcd_field, kappa, mu,
                    parity=LQCD_FULL):
    g = U.geom
    ctx.check(lib().lqcd_apply_Mdag(ctx.handle, U.handle, inp, out, ctypes.byref(g), kappa, mu,
                                    parity))


def cg_params(tol=1e-10, max_iter=20000, outer_prec=LQCD_F64, inner_prec=None, delta=0.0,
              max_restarts=5, check_every=10, use_graph=1, sloppy_recon=0, solver=LQCD_SOLVER_CG,
              inner_tol=0.0) -> lqcd_cg_params:
    p = lqcd_cg_params()
    p.tol = tol
    p.max_iter = max_iter
    p.outer_prec = outer_prec
    p.inner_prec = outer_prec if inner_prec is None else inner_prec
    p.delta = delta
    p.max_restarts = max_restarts
    p.check_every = check_every
    p.use_graph = use_graph
    p.sloppy_recon = sloppy_recon
    p.solver = solver
    p.inner_tol = inner_tol
    return p


def lqcd_cg_solve(ctx: Context, U: Gauge, b: lqcd_field, x: lqcd_field, kappa, mu,
                  params: lqcd_cg_params, allow_noconv=False):
    nrhs = b.nrhs
    stats = (lqcd_cg_stats * nrhs)()
    g = U.geom
    ctx.check(lib().lqcd_cg_solve(ctx.handle, U.handle, b, x, ctypes.byref(g), kappa, mu,
                                  ctypes.byref(params), stats),
              allow=(LQCD_ERR_NOCONV,) if allow_noconv else ())
    return [s.as_dict() for s in stats]


def lqcd_dd_cg_solve(ctx: Context, Us, bs, xs, faces, first_domain, nt, kappa, mu,
                     params: lqcd_cg_params, antiperiodic_t=True, exchange=None, allreduce=None,
                     allow_noconv=False, nz=1):
    """Domain-decomposed CG (include/lqcd.h) on an nz x nt grid of domains:
    Us, bs, xs, faces for the held domains (faces: 4 device tensors per
    domain along t, then 4 along z when nz > 1); exchange(t_bytes, z_bytes)
    (move the leading bytes of each t and z face) / allreduce(list of floats)
    -> list: the communication hooks (None for all domains in this call).
    The hooks are called from inside the library call."""
    nd = len(Us)
    g = Us[0].geom
    U_arr = (_vp * nd)(*[u.handle for u in Us])
    b_arr = (lqcd_field * nd)(*bs)
    x_arr = (lqcd_field * nd)(*xs)
    ptrs = [t.data_ptr() for fs in faces for t in fs]
    if len(ptrs) != (8 if nz > 1 else 4) * nd:
        raise ValueError("faces: 4 tensors per domain (8 when nz > 1)")
    f_arr = (_vp * len(ptrs))(*ptrs)
    stats = lqcd_cg_stats()
    comm_p = None
    errors = []
    if exchange is not None:
        def _ex(_user, t_bytes, z_bytes):
            try:
                exchange(int(t_bytes), int(z_bytes))
                return 0
            except Exception as e:  # reported as LQCD_ERR_COMM; re-raised below
                errors.append(e)
                return 1

        def _ar(_user, vals, n):
            try:
                if allreduce is not None:
                    out = allreduce([vals[i] for i in range(n)])
                    for i in range(n):
                        vals[i] = float(out[i])
                return 0
            except Exception as e:
                errors.append(e)
                return 1
        ex_cb, ar_cb = _EXCHANGE_FN(_ex), _ALLREDUCE_FN(_ar)
        comm = lqcd_dd_comm(None, ex_cb, ar_cb)
        comm_p = ctypes.byref(comm)
    rc = lib().lqcd_dd_cg_solve(ctx.handle, nd, U_arr, b_arr, x_arr, f_arr, ctypes.byref(g), int(first_domain),
                                int(nz), int(nt), int(bool(antiperiodic_t)), kappa, mu, ctypes.byref(params),
                                comm_p, ctypes.byref(stats))
    if errors:
        raise errors[0]
    ctx.check(rc, allow=(LQCD_ERR_NOCONV,) if allow_noconv else ())
    return stats.as_dict()


def lqcd_cg_solve_batch(ctx: Context, Us, bs, xs, kappas, mus, params: lqcd_cg_params,
                        allow_noconv=False):
    n = len(Us)
    arrU = (_vp * n)(*[U.handle.value for U in Us])
    arrb = (lqcd_field * n)(*bs)
    arrx = (lqcd_field * n)(*xs)
    arrk = (_d * n)(*kappas)
    arrm = (_d * n)(*mus)
    stats = (lqcd_cg_stats * n)()
    ctx.check(lib().lqcd_cg_solve_batch(ctx.handle, n, arrU, arrb, arrx, arrk, arrm,
                                        ctypes.byref(params), stats),
              allow=(LQCD_ERR_NOCONV,) if allow_noconv else ())
    return [s.as_dict() for s in stats]


def lqcd_fermion_force(ctx: Context, U: Gauge, phi: lqcd_field, dSdw: torch.Tensor | None, kappa, mu,
                       params: lqcd_cg_params, X_cache: lqcd_field | None = None):
    """Returns (S, stats); dSdw (float64 [4, V, 8] CUDA) receives dS/domega
    (None: the action alone)."""
    st = lqcd_cg_stats()
    S = _d(0.0)
    g = U.geom
    ctx.check(lib().lqcd_fermion_force(ctx.handle, U.handle, phi,
                                       _vp(dSdw.data_ptr()) if dSdw is not None else None,
                                       ctypes.byref(X_cache) if X_cache is not None else None,
                                       ctypes.byref(g), kappa, mu, ctypes.byref(params),
                                       ctypes.byref(st), ctypes.byref(S)))
    return S.value, st.as_dict()


def lqcd_fermion_force_ratio(ctx: Context, U: Gauge, phi2: lqcd_field, dSdw: torch.Tensor, kappa, mu, mu2,
                             params: lqcd_cg_params):
    """Returns (S2, stats); dSdw receives dS2/domega of the mass-preconditioning ratio."""
    st = lqcd_cg_stats()
    S = _d(0.0)
    g = U.geom
    ctx.check(lib().lqcd_fermion_force_ratio(ctx.handle, U.handle, phi2, _vp(dSdw.data_ptr()), ctypes.byref(g),
                                             kappa, mu, mu2, ctypes.byref(params), ctypes.byref(st),
                                             ctypes.byref(S)))
    return S.value, st.as_dict()


def lqcd_gauge_force(ctx: Context, U: Gauge, beta, dSdw: torch.Tensor, want_action=True, c1=0.0,
                     prec=LQCD_F64):
    S = _d(0.0)
    ctx.check(lib().lqcd_gauge_force(ctx.handle, U.handle, beta, c1, prec, _vp(dSdw.data_ptr()),
                                     ctypes.byref(S) if want_action else None))
    return S.value if want_action else None


def lqcd_plaquette(ctx: Context, U: Gauge) -> float:
    p = _d(0.0)
    ctx.check(lib().lqcd_plaquette(ctx.handle, U.handle, ctypes.byref(p)))
    return p.value


def lqcd_heatbath_sweep(ctx: Context, U: Gauge, beta, seed, sweep_idx, n_or=0, prec=LQCD_F64):
    ctx.check(lib().lqcd_heatbath_sweep(ctx.handle, U.handle, beta, seed, sweep_idx, n_or, prec))


def lqcd_overrelax_sweep(ctx: Context, U: Gauge, n_or=1, prec=LQCD_F64):
    ctx.check(lib().lqcd_overrelax_sweep(ctx.handle, U.handle, n_or, prec))


def lqcd_momenta_gaussian(ctx: Context, L, P: torch.Tensor, seed, traj, antiperiodic_t=True):
    g = geom(L, antiperiodic_t)
    ctx.check(lib().lqcd_momenta_gaussian(ctx.handle, ctypes.byref(g), _vp(P.data_ptr()), seed,
                                          traj))


def lqcd_spinor_gaussian(ctx: Context, L, eta: lqcd_field, parity, seed, traj,
                         antiperiodic_t=True):
    g = geom(L, antiperiodic_t)
    ctx.check(lib().lqcd_spinor_gaussian(ctx.handle, ctypes.byref(g), eta, parity, seed, traj))


def lqcd_gauge_update(ctx: Context, U: Gauge, P: torch.Tensor, eps):
    ctx.check(lib().lqcd_gauge_update(ctx.handle, U.handle, _vp(P.data_ptr()), eps))


def lqcd_gauge_update_prec(ctx: Context, U: Gauge, P: torch.Tensor, eps, prec=LQCD_F64):
    ctx.check(lib().lqcd_gauge_update_prec(ctx.handle, U.handle, _vp(P.data_ptr()), eps, prec))


def lqcd_momenta_update(ctx: Context, L, P: torch.Tensor, dSdw: torch.Tensor, eps,
                        antiperiodic_t=True):
    g = geom(L, antiperiodic_t)
    ctx.check(lib().lqcd_momenta_update(ctx.handle, ctypes.byref(g), _vp(P.data_ptr()),
                                        _vp(dSdw.data_ptr()), eps))


def lqcd_momenta_kinetic(ctx: Context, L, P: torch.Tensor, antiperiodic_t=True) -> float:
    g = geom(L, antiperiodic_t)
    K = _d(0.0)
    ctx.check(lib().lqcd_momenta_kinetic(ctx.handle, ctypes.byref(g), _vp(P.data_ptr()),
                                         ctypes.byref(K)))
    return K.value


def lqcd_gauge_copy(ctx: Context, src: Gauge, dst: Gauge):
    ctx.check(lib().lqcd_gauge_copy(ctx.handle, src.handle, dst.handle))


LQCD_LEAPFROG, LQCD_2MN = 0, 1
TLSYM_C1 = -1.0 / 12.0


def hmc_params(beta, kappa, mu, tau=1.0, nsteps=20, nf=1, seed=1, traj=0, cg=None,
               integrator=LQCD_LEAPFROG, c1=0.0, nsteps_gauge=1, lam=0.0, force_prec=LQCD_F64, mu2=0.0,
               nsteps_mid=1):
    p = lqcd_hmc_params()
    p.beta, p.kappa, p.mu, p.tau = beta, kappa, mu, tau
    p.nsteps, p.nf, p.seed, p.traj = nsteps, nf, seed, traj
    p.integrator, p.c1, p.nsteps_gauge, p.lam = integrator, c1, nsteps_gauge, lam
    p.force_prec = force_prec
    p.mu2, p.nsteps_mid = mu2, nsteps_mid
    p.cg = cg if cg is not None else cg_params(tol=1e-10, outer_prec=LQCD_DF64,
                                               inner_prec=LQCD_F32)
    return p


def lqcd_hmc_trajectory(ctx: Context, U: Gauge, params: lqcd_hmc_params):
    st = lqcd_hmc_stats()
    ctx.check(lib().lqcd_hmc_trajectory(ctx.handle, U.handle, ctypes.byref(params),
                                        ctypes.byref(st)))
    return st.as_dict()
