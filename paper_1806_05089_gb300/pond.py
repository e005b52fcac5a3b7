"""Python binding of the PonD C ABI (include/pond.h), argument marshalling only.

Every entry point of libpond.so is exposed under its C name (``pond_create``,
``pond_set_state``, ``pond_step``, ``pond_moments``, ``pond_get_state``,
``pond_iterations``, ``pond_adjoint_step``, ``pond_destroy``, ...).  Arrays may
be NumPy arrays (host) or torch tensors (CUDA tensors are passed as device
pointers, CPU tensors as host pointers); every array is FP64 except the int32
iteration map.  All compute runs in the CUDA library: if it cannot be loaded
this module raises, there is no CPU fallback.

The library trusts the sizes behind its pointers, so the binding checks them:
``pond_create`` returns a ``PondCtx`` that records each grid's size, the
lattice's Q and the context's device, and every call that passes arrays
checks their dtype, element count, side (host or device) and device against
it before the C call (``TypeError`` / ``ValueError``; nothing reaches the
library when a check fails).

``Sim`` is a small convenience wrapper owning one context.
"""
from __future__ import annotations

import ctypes
import os
import sys
from dataclasses import dataclass

import numpy as np

from . import build as _build

POND_OK = 0
POND_ERR_ARG = 1
POND_ERR_OOM = 2
POND_ERR_CUDA = 3
POND_ERR_NONPHYSICAL = 4
POND_ERR_NOT_CONVERGED = 5
POND_ERR_TIMEOUT = 6
POND_ERR_STATE = 7
POND_FP64 = 0
POND_FP32_MIXED = 1
POND_D2Q16 = 0
POND_D2Q9 = 1
POND_KERNEL_DEFAULT = 0
POND_KERNEL_STAGED = 1
POND_KERNEL_DIRECT = 2
POND_PIPE_FP64 = 0
POND_PIPE_FP32 = 1
POND_PIPE_FP32X2 = 2
N_SPEEDS = {POND_D2Q16: 4, POND_D2Q9: 3}  # speeds per dimension; Q = n1^2

_STATUS = {0: "POND_OK", 1: "POND_ERR_ARG", 2: "POND_ERR_OOM", 3: "POND_ERR_CUDA",
           4: "POND_ERR_NONPHYSICAL", 5: "POND_ERR_NOT_CONVERGED", 6: "POND_ERR_TIMEOUT",
           7: "POND_ERR_STATE"}


class PondError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class pond_config(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("thermal", ctypes.c_int32),
        ("nu", ctypes.c_double),
        ("T_ref", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("eps_abs", ctypes.c_double),
        ("eps_rel", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("fixed_iter", ctypes.c_int32),
        ("ckpt_every", ctypes.c_int32),
        ("strict", ctypes.c_int32),
        ("seed_mode", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("tile_rows", ctypes.c_int32),
        ("lattice", ctypes.c_int32),
        ("nodes_per_warp", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
    ]


class pond_stats(ctypes.Structure):
    _fields_ = [
        ("node_updates", ctypes.c_int64),
        ("passes", ctypes.c_int64),
        ("max_passes", ctypes.c_int32),
        ("tile_rows", ctypes.c_int32),
        ("nonconverged", ctypes.c_int64),
        ("nonphysical", ctypes.c_int64),
        ("halo_fallback", ctypes.c_int64),
        ("index_faults", ctypes.c_int64),
        ("busy_ns", ctypes.c_int64),
        ("slot_ns", ctypes.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_LIB = None

# every symbol include/pond.h declares
EXPORTS = ["pond_config_default", "pond_create", "pond_set_stream", "pond_set_state",
           "pond_step", "pond_moments", "pond_get_state", "pond_iterations",
           "pond_adjoint_step", "pond_adjoint_step_given", "pond_adjoint_init",
           "pond_adjoint_nu_bar",
           "pond_step_fp64_noalloc", "pond_measure_peak", "pond_set_interior",
           "pond_pack_rect", "pond_unpack_rect", "pond_max_displacement", "pond_destroy",
           "pond_last_error", "pond_version"]

POND_NOALLOC_MAX_NODES = 262144


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True, path: str | None = None):
    """Load libpond.so (building it first if needed); ``path`` loads another
    build of the same library instead (tuning experiments)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if path is None:
        path = _build.LIB
        if not os.path.exists(path) or _build._stale():
            if not build_if_missing:
                raise RuntimeError("libpond.so is missing; build it with paper_1806_05089_gb300.build")
            _build.build()
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    i32 = ctypes.c_int32
    lib.pond_config_default.argtypes = [ctypes.POINTER(pond_config), i32]
    lib.pond_config_default.restype = None
    lib.pond_create.argtypes = [ctypes.POINTER(pond_config), i32, ctypes.POINTER(i32),
                                ctypes.POINTER(i32), vp, ctypes.POINTER(vp)]
    lib.pond_create.restype = i32
    lib.pond_set_stream.argtypes = [vp, vp]
    lib.pond_set_stream.restype = i32
    lib.pond_set_state.argtypes = [vp, i32, vp, vp, vp, vp, vp, i32]
    lib.pond_set_state.restype = i32
    lib.pond_step.argtypes = [vp, i32, ctypes.POINTER(pond_stats)]
    lib.pond_step.restype = i32
    lib.pond_moments.argtypes = [vp, i32, vp, vp, vp, vp, i32]
    lib.pond_moments.restype = i32
    lib.pond_get_state.argtypes = [vp, i32, vp, vp, vp, vp, i32]
    lib.pond_get_state.restype = i32
    lib.pond_iterations.argtypes = [vp, i32, vp, i32]
    lib.pond_iterations.restype = i32
    lib.pond_adjoint_step.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.pond_adjoint_step.restype = i32
    lib.pond_adjoint_step_given.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp,
                                            ctypes.POINTER(ctypes.c_double)]
    lib.pond_adjoint_step_given.restype = i32
    lib.pond_adjoint_init.argtypes = [vp, vp, vp]
    lib.pond_adjoint_init.restype = i32
    lib.pond_adjoint_nu_bar.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.pond_adjoint_nu_bar.restype = i32
    lib.pond_step_fp64_noalloc.argtypes = [ctypes.POINTER(pond_config), i32, i32,
                                           vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                           ctypes.POINTER(pond_stats), vp]
    lib.pond_step_fp64_noalloc.restype = i32
    lib.pond_measure_peak.argtypes = [i32, i32, vp, vp, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
    lib.pond_measure_peak.restype = i32
    lib.pond_set_interior.argtypes = [vp, i32, i32, i32, i32, i32]
    lib.pond_set_interior.restype = i32
    lib.pond_pack_rect.argtypes = [vp, i32, i32, i32, i32, i32, vp]
    lib.pond_pack_rect.restype = i32
    lib.pond_unpack_rect.argtypes = [vp, i32, i32, i32, i32, i32, vp]
    lib.pond_unpack_rect.restype = i32
    lib.pond_max_displacement.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double)]
    lib.pond_max_displacement.restype = i32
    lib.pond_destroy.argtypes = [vp]
    lib.pond_destroy.restype = None
    lib.pond_last_error.argtypes = [vp]
    lib.pond_last_error.restype = ctypes.c_char_p
    lib.pond_version.argtypes = []
    lib.pond_version.restype = ctypes.c_char_p
    _LIB = lib
    return lib


# ------------------------------------------------------------------ marshalling

class PondCtx(ctypes.c_void_p):
    """A pond_ctx handle: passed to the C calls as the pointer it holds, and
    carrying what the binding checks array arguments against: ``grids``, the
    (nx, ny) of each grid; ``q``, the populations per node; ``device``, the
    CUDA device index the context was created on (None when torch was not
    loaded then; the current device is assumed)."""


def _grid_nodes(ctx, grid):
    """Nodes of grid ``grid`` of a handle made by ``pond_create``; None for
    another handle or an index out of range (the library rejects that one
    itself with POND_ERR_ARG)."""
    grids = getattr(ctx, "grids", None)
    if grids is None or not 0 <= int(grid) < len(grids):
        return None
    nx, ny = grids[int(grid)]
    return nx * ny


def _counts(ctx, grid, *per_node):
    """Expected element counts for arrays of ``per_node`` values per node
    (1 for a field, 3 for a gauge triple, "q" for populations), or Nones
    when the handle does not know the grid."""
    n = _grid_nodes(ctx, grid)
    q = getattr(ctx, "q", None)
    if n is None or q is None:
        return [None] * len(per_node)
    return [n * (q if k == "q" else k) for k in per_node]


def _check_device(name, index, want):
    if index != want:
        raise ValueError("%s is on cuda:%s; the context's device is cuda:%s" % (name, index, want))


def _ptr(a, on_device: bool, count=None, kind: str = "f64", out: bool = False, device=None,
         name: str = "array"):
    """(pointer, keepalive) of one array argument, checked against what the
    header requires: ``kind`` "f64" (FP64) or "i32" (the iteration map);
    exactly ``count`` values when the grid is known; contiguous; on the side
    the call names; for CUDA tensors, on ``device`` (the current device when
    None).  Host inputs of another dtype are converted into a copy that the
    call reads; host outputs must already be writeable C-contiguous arrays of
    the right dtype, since the library would fill a converted copy that the
    caller never sees."""
    if a is None:
        return None, None
    torch = sys.modules.get("torch")
    if torch is not None and isinstance(a, torch.Tensor):
        want = torch.float64 if kind == "f64" else torch.int32
        if a.dtype != want:
            raise TypeError("%s must be %s, got %s" % (name, want, a.dtype))
        if not a.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if a.is_cuda != on_device:
            if on_device:
                raise ValueError("device call needs torch CUDA tensors (%s is on the host)" % name)
            raise ValueError("all arrays of one call must be on the same side (host or device)")
        if count is not None and a.numel() != count:
            raise ValueError("%s holds %d values; the grid needs %d" % (name, a.numel(), count))
        if a.is_cuda:
            _check_device(name, a.device.index,
                          device if device is not None else torch.cuda.current_device())
        return ctypes.c_void_p(a.data_ptr()), a
    if on_device:
        raise ValueError("device call needs torch CUDA tensors (%s is not one)" % name)
    want_np = np.dtype(np.float64 if kind == "f64" else np.int32)
    if out:
        if (not isinstance(a, np.ndarray) or a.dtype != want_np or not a.flags.c_contiguous
                or not a.flags.writeable):
            raise TypeError("%s is an output: it must be a writeable C-contiguous %s array"
                            % (name, want_np.name))
        arr = a
    else:
        arr = np.ascontiguousarray(a, dtype=want_np)
    if count is not None and arr.size != count:
        raise ValueError("%s holds %d values; the grid needs %d" % (name, arr.size, count))
    return ctypes.c_void_p(arr.ctypes.data), arr


def _is_device(*arrays) -> bool:
    for a in arrays:
        if a is None:
            continue
        try:
            import torch
            if isinstance(a, torch.Tensor):
                return a.is_cuda
        except ImportError:
            pass
        return False
    return False


def _check(ctx, status):
    if status != POND_OK:
        msg = load().pond_last_error(ctx).decode() if ctx else ""
        raise PondError(status, msg)


def pond_version() -> str:
    return load().pond_version().decode()


def pond_config_default(precision: int = POND_FP64) -> pond_config:
    cfg = pond_config()
    load().pond_config_default(ctypes.byref(cfg), precision)
    return cfg


def pond_create(cfg: pond_config, nx, ny, stream=None) -> PondCtx:
    nx = [int(v) for v in np.atleast_1d(nx)]
    ny = [int(v) for v in np.atleast_1d(ny)]
    n = len(nx)
    arr_x = (ctypes.c_int32 * n)(*nx)
    arr_y = (ctypes.c_int32 * n)(*ny)
    out = ctypes.c_void_p()
    st = load().pond_create(ctypes.byref(cfg), n, arr_x, arr_y,
                            ctypes.c_void_p(stream or 0), ctypes.byref(out))
    if st != POND_OK:
        raise PondError(st, "pond_create failed")
    ctx = PondCtx(out.value)
    ctx.grids = list(zip(nx, ny))
    n1 = N_SPEEDS.get(int(cfg.lattice))
    ctx.q = n1 * n1 if n1 is not None else None
    # the library binds the context to the device current at creation
    torch = sys.modules.get("torch")
    ctx.device = (torch.cuda.current_device()
                  if torch is not None and torch.cuda.is_available() else None)
    return ctx


def _marshal(ctx, grid, on_device, named, out=False):
    """Checked (pointer, keepalive) pairs of one call's arrays, ``named`` as
    (name, array, values per node, kind) with values per node 1, 3 or "q"."""
    device = getattr(ctx, "device", None)
    ps = []
    for name, a, per_node, kind in named:
        (count,) = _counts(ctx, grid, per_node)
        ps.append(_ptr(a, on_device, count, kind, out, device, name))
    return ps


def pond_set_stream(ctx, stream):
    _check(ctx, load().pond_set_stream(ctx, ctypes.c_void_p(stream or 0)))


def pond_set_state(ctx, grid, rho, ux, uy, T, f=None):
    dev = _is_device(ux, uy, T, rho, f)
    ps = _marshal(ctx, grid, dev, [("rho", rho, 1, "f64"), ("ux", ux, 1, "f64"),
                                   ("uy", uy, 1, "f64"), ("T", T, 1, "f64"),
                                   ("f", f, "q", "f64")])
    _check(ctx, load().pond_set_state(ctx, grid, *[p for p, _ in ps], int(dev)))


def pond_step(ctx, nsteps: int, want_stats: bool = True):
    stats = pond_stats()
    _check(ctx, load().pond_step(ctx, int(nsteps), ctypes.byref(stats) if want_stats else None))
    return stats.as_dict() if want_stats else None


def pond_moments(ctx, grid, rho=None, ux=None, uy=None, T=None):
    dev = _is_device(rho, ux, uy, T)
    ps = _marshal(ctx, grid, dev, [("rho", rho, 1, "f64"), ("ux", ux, 1, "f64"),
                                   ("uy", uy, 1, "f64"), ("T", T, 1, "f64")], out=True)
    _check(ctx, load().pond_moments(ctx, grid, *[p for p, _ in ps], int(dev)))


def pond_get_state(ctx, grid, f=None, ux=None, uy=None, T=None):
    dev = _is_device(f, ux, uy, T)
    ps = _marshal(ctx, grid, dev, [("f", f, "q", "f64"), ("ux", ux, 1, "f64"),
                                   ("uy", uy, 1, "f64"), ("T", T, 1, "f64")], out=True)
    _check(ctx, load().pond_get_state(ctx, grid, *[p for p, _ in ps], int(dev)))


def pond_iterations(ctx, grid, iters):
    dev = _is_device(iters)
    ((p, _k),) = _marshal(ctx, grid, dev, [("iters", iters, 1, "i32")], out=True)
    _check(ctx, load().pond_iterations(ctx, grid, p, int(dev)))


def _adjoint_arrays(ctx, f_bar_in, gauge_bar_in, f_bar_out, gauge_bar_out):
    return _marshal(ctx, 0, True, [("f_bar_in", f_bar_in, "q", "f64"),
                                   ("gauge_bar_in", gauge_bar_in, 3, "f64"),
                                   ("f_bar_out", f_bar_out, "q", "f64"),
                                   ("gauge_bar_out", gauge_bar_out, 3, "f64")])


def pond_adjoint_step(ctx, f_bar_in, gauge_bar_in, f_bar_out, gauge_bar_out,
                      nu_on_device: bool = False):
    """Device tensors only; returns d(loss)/d(nu) of this step, or, with
    nu_on_device, None: the contribution then accumulates on the device
    (read with pond_adjoint_nu_bar) and the call does not wait for the GPU."""
    nu_bar = ctypes.c_double(0.0)
    ps = _adjoint_arrays(ctx, f_bar_in, gauge_bar_in, f_bar_out, gauge_bar_out)
    acc = None if nu_on_device else ctypes.byref(nu_bar)
    _check(ctx, load().pond_adjoint_step(ctx, *[p for p, _ in ps], acc))
    return None if nu_on_device else nu_bar.value


def pond_adjoint_step_given(ctx, ux_out, uy_out, T_out, f_bar_in, gauge_bar_in, f_bar_out,
                            gauge_bar_out, nu_on_device: bool = False):
    """pond_adjoint_step with the step's output gauge (device tensors) given,
    so the forward step is not recomputed; returns d(loss)/d(nu) of this step
    (None with nu_on_device, as pond_adjoint_step)."""
    nu_bar = ctypes.c_double(0.0)
    ps = _marshal(ctx, 0, True, [("ux_out", ux_out, 1, "f64"), ("uy_out", uy_out, 1, "f64"),
                                 ("T_out", T_out, 1, "f64")])
    ps += _adjoint_arrays(ctx, f_bar_in, gauge_bar_in, f_bar_out, gauge_bar_out)
    acc = None if nu_on_device else ctypes.byref(nu_bar)
    _check(ctx, load().pond_adjoint_step_given(ctx, *[p for p, _ in ps], acc))
    return None if nu_on_device else nu_bar.value


def pond_adjoint_nu_bar(ctx) -> float:
    """The nu cotangent accumulated on the device since the last read (and
    clear it)."""
    v = ctypes.c_double(0.0)
    _check(ctx, load().pond_adjoint_nu_bar(ctx, ctypes.byref(v)))
    return v.value


def pond_adjoint_init(ctx, f_bar, rho_bar):
    """rho_bar = sum_q W_q f_bar_q (device tensors)."""
    ps = _marshal(ctx, 0, True, [("f_bar", f_bar, "q", "f64"), ("rho_bar", rho_bar, 1, "f64")])
    _check(ctx, load().pond_adjoint_init(ctx, *[p for p, _ in ps]))


def _check_noalloc_args(cfg, f_in, ux_in, uy_in, T_in, f_out, ux_out, uy_out, T_out, iters):
    """The C entry point trusts its pointers (it has no context that knows the
    grid), so the binding checks what the header requires before the call:
    float64 populations of shape (Q, ny, nx) with Q from cfg.lattice,
    float64 (ny, nx) gauges, an int32 (ny, nx) iteration map or None, all
    contiguous CUDA tensors on the current device.  Raises ValueError or
    TypeError; nothing reaches the GPU when a check fails."""
    import torch
    n1 = N_SPEEDS.get(int(cfg.lattice))
    if n1 is None:
        raise ValueError("unknown lattice %d" % int(cfg.lattice))
    named = [("f_in", f_in), ("ux_in", ux_in), ("uy_in", uy_in), ("T_in", T_in),
             ("f_out", f_out), ("ux_out", ux_out), ("uy_out", uy_out), ("T_out", T_out)]
    for name, a in named + [("iters", iters)]:
        if name == "iters" and a is None:
            continue
        if not isinstance(a, torch.Tensor):
            raise TypeError("%s must be a torch tensor" % name)
        if not a.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if ux_in.dim() != 2:
        raise ValueError("ux_in must be (ny, nx), got %s" % (tuple(ux_in.shape),))
    ny, nx = ux_in.shape
    for name, a in named:
        want = (n1 * n1, ny, nx) if name.startswith("f_") else (ny, nx)
        if tuple(a.shape) != want:
            raise ValueError("%s has shape %s; the lattice and grid need %s"
                             % (name, tuple(a.shape), want))
        if a.dtype != torch.float64:
            raise TypeError("%s must be float64, got %s" % (name, a.dtype))
    if iters is not None:
        if tuple(iters.shape) != (ny, nx):
            raise ValueError("iters has shape %s; the grid needs %s" % (tuple(iters.shape), (ny, nx)))
        if iters.dtype != torch.int32:
            raise TypeError("iters must be int32, got %s" % iters.dtype)
    arrays = [a for _, a in named] + ([iters] if iters is not None else [])
    if not all(a.is_cuda for a in arrays):
        raise ValueError("pond_step_fp64_noalloc takes CUDA tensors only")
    cur = torch.cuda.current_device()
    for name, a in named + [("iters", iters)]:
        if a is not None and a.device.index != cur:
            raise ValueError("%s is on cuda:%d but the current device is cuda:%d"
                             % (name, a.device.index, cur))


def pond_step_fp64_noalloc(cfg, f_in, ux_in, uy_in, T_in, f_out, ux_out, uy_out, T_out,
                           iters=None, want_stats=True, stream=None):
    """One FP64 step without a context or any allocation (CUDA float64
    tensors; see include/pond.h).  Returns the step counters."""
    _check_noalloc_args(cfg, f_in, ux_in, uy_in, T_in, f_out, ux_out, uy_out, T_out, iters)
    ny, nx = ux_in.shape
    ps = [_ptr(a, True) for a in (f_in, ux_in, uy_in, T_in, f_out, ux_out, uy_out, T_out)]
    ps.append(_ptr(iters, True, kind="i32", name="iters"))
    stats = pond_stats()
    st = load().pond_step_fp64_noalloc(ctypes.byref(cfg), nx, ny, *[p for p, _ in ps],
                                       ctypes.byref(stats) if want_stats else None,
                                       ctypes.c_void_p(stream or 0))
    if st != POND_OK:
        raise PondError(st, "pond_step_fp64_noalloc failed")
    return stats.as_dict() if want_stats else None


def pond_measure_peak(pipe: int, iters: int, sink, stream=None):
    """(TFLOP/s, seconds) of the FMA-chain probe of one arithmetic pipe
    (POND_PIPE_FP64, POND_PIPE_FP32, POND_PIPE_FP32X2) on the current device;
    ``sink`` is a CUDA tensor of at least 8 bytes."""
    tf = ctypes.c_double(0.0)
    secs = ctypes.c_double(0.0)
    st = load().pond_measure_peak(int(pipe), int(iters), ctypes.c_void_p(sink.data_ptr()),
                                  ctypes.c_void_p(stream or 0), ctypes.byref(tf),
                                  ctypes.byref(secs))
    if st != POND_OK:
        raise PondError(st, "pond_measure_peak failed")
    return tf.value, secs.value


def pond_set_interior(ctx, grid, x0, y0, w, h):
    _check(ctx, load().pond_set_interior(ctx, int(grid), int(x0), int(y0), int(w), int(h)))


def _rect_buffer(ctx, buf, q, w, h):
    """Pointer of a pack/unpack buffer: a contiguous CUDA float64 tensor on
    the context's device with at least (Q + 3) * w * h values, Q the
    context's populations per node (``q``, when given, must agree)."""
    import torch
    ctx_q = getattr(ctx, "q", None)
    if q is None:
        q = ctx_q if ctx_q is not None else 16
    elif ctx_q is not None and int(q) != ctx_q:
        raise ValueError("q = %d, but the context's lattice has Q = %d" % (int(q), ctx_q))
    if not isinstance(buf, torch.Tensor) or not buf.is_cuda or buf.dtype != torch.float64:
        raise TypeError("rectangle buffers are CUDA float64 tensors")
    if not buf.is_contiguous() or buf.numel() < (int(q) + 3) * int(w) * int(h):
        raise ValueError("rectangle buffer needs (Q + 3) * w * h contiguous values")
    device = getattr(ctx, "device", None)
    _check_device("buf", buf.device.index,
                  device if device is not None else torch.cuda.current_device())
    return ctypes.c_void_p(buf.data_ptr())


def pond_pack_rect(ctx, grid, x0, y0, w, h, buf, q=None):
    """Rectangle of the current state into a CUDA float64 buffer of
    (Q + 3) * w * h values (Q = populations of the context's lattice)."""
    _check(ctx, load().pond_pack_rect(ctx, int(grid), int(x0), int(y0), int(w), int(h),
                                      _rect_buffer(ctx, buf, q, w, h)))


def pond_unpack_rect(ctx, grid, x0, y0, w, h, buf, q=None):
    _check(ctx, load().pond_unpack_rect(ctx, int(grid), int(x0), int(y0), int(w), int(h),
                                        _rect_buffer(ctx, buf, q, w, h)))


def pond_max_displacement(ctx, grid=0) -> float:
    out = ctypes.c_double(0.0)
    _check(ctx, load().pond_max_displacement(ctx, int(grid), ctypes.byref(out)))
    return out.value


def pond_destroy(ctx):
    if ctx:
        load().pond_destroy(ctx)


# ------------------------------------------------------------------ convenience

@dataclass
class HostState:
    f: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    T: np.ndarray


class Sim:
    """One PonD context (one grid, or a batched ensemble of grids)."""

    def __init__(self, nx, ny, precision: int = POND_FP64, stream=None, **overrides):
        self.cfg = pond_config_default(precision)
        for k, v in overrides.items():
            if not hasattr(self.cfg, k):
                raise AttributeError("unknown config field %s" % k)
            setattr(self.cfg, k, v)
        self.nx = [int(v) for v in np.atleast_1d(nx)]
        self.ny = [int(v) for v in np.atleast_1d(ny)]
        self.Q = N_SPEEDS.get(int(self.cfg.lattice), 4) ** 2
        self.ctx = pond_create(self.cfg, self.nx, self.ny, stream)

    def close(self):
        if self.ctx:
            pond_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, rho, ux, uy, T, f=None, grid: int = 0):
        pond_set_state(self.ctx, grid, rho, ux, uy, T, f)

    def step(self, nsteps: int = 1, stats: bool = True):
        return pond_step(self.ctx, nsteps, stats)

    def moments(self, grid: int = 0):
        ny, nx = self.ny[grid], self.nx[grid]
        out = [np.zeros((ny, nx)) for _ in range(4)]
        pond_moments(self.ctx, grid, *out)
        return tuple(out)  # rho, ux, uy, T

    def state(self, grid: int = 0) -> HostState:
        ny, nx = self.ny[grid], self.nx[grid]
        f = np.zeros((self.Q, ny, nx))
        ux, uy, T = (np.zeros((ny, nx)) for _ in range(3))
        pond_get_state(self.ctx, grid, f, ux, uy, T)
        return HostState(f, ux, uy, T)

    def iterations(self, grid: int = 0) -> np.ndarray:
        it = np.zeros((self.ny[grid], self.nx[grid]), dtype=np.int32)
        pond_iterations(self.ctx, grid, it)
        return it
