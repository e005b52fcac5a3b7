"""FP64 CPU oracle of the Particles-on-Demand (PonD) time step (D2Q16 and D2Q9).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` import this package.  The
product library (``paper_1806_05089_gb300``) never imports it and shares no
code with it.

The arithmetic lives in ``pond_oracle.c`` (plain C, FP64, OpenMP over rows);
this module only marshals NumPy arrays through ctypes.  Each C function cites
the paper's equations it follows (Dorschner, Bosch, Karlin, arXiv 1806.05089).

State convention (shared with the CUDA library only through the plain array
shapes): ``f`` has shape (Q, ny, nx) with population index q = n1 k + l
(k: x-speed index, l: y-speed index, speeds ascending; n1 = 4, Q = 16 for
D2Q16, n1 = 3, Q = 9 for D2Q9); ``ux``, ``uy``, ``T`` have shape (ny, nx);
the grid is periodic.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_LIB = None

FLAG_NONCONVERGED = 1
FLAG_NONPHYSICAL = 2

D2Q16 = 0
D2Q9 = 1
_N1 = {D2Q16: 4, D2Q9: 3}


class _Params(ctypes.Structure):
    _fields_ = [
        ("nu", ctypes.c_double),
        ("T_ref", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("eps_abs", ctypes.c_double),
        ("eps_rel", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("fixed_iter", ctypes.c_int32),
        ("thermal", ctypes.c_int32),
        ("seed_mode", ctypes.c_int32),
        ("lattice", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


@dataclass
class Params:
    """Step parameters.  beta = 1 / (2 nu / (T_ref dt) + 1) (Eq. postcollision,
    nu = T (1/(2 beta) - 1/2) dt); tolerances of Eq. convergence (App. E);
    seed_mode 0: previous gauge (Eq. seed_gauge), 1: {0, T_L}, 2: {-u, T};
    lattice D2Q16 (default) or D2Q9 (App. A)."""
    nu: float = 0.01
    T_ref: float = 1.0
    dt: float = 1.0
    eps_abs: float = 1e-12
    eps_rel: float = 1e-10
    max_iter: int = 20
    fixed_iter: int = 0
    thermal: int = 1
    seed_mode: int = 0
    lattice: int = D2Q16

    def _c(self) -> _Params:
        return _Params(self.nu, self.T_ref, self.dt, self.eps_abs, self.eps_rel,
                       self.max_iter, self.fixed_iter, self.thermal, self.seed_mode,
                       self.lattice, 0)


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        ci = ctypes.c_int
        lib.oracle_lattice.argtypes = [ci, dp, dp, dp]
        lib.oracle_transfer.argtypes = [ci, dp, dp, dp, dp]
        lib.oracle_interp_weights.argtypes = [ctypes.c_double, dp]
        lib.oracle_init_equilibrium.argtypes = [ci, ctypes.c_int64, ctypes.c_int64, dp, dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_num_threads.restype = ctypes.c_int
        lib.oracle_step.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, dp, dp, dp,
                                    dp, dp, dp, dp, ip, ip,
                                    ctypes.POINTER(_Params), ctypes.c_int64,
                                    ctypes.c_int64]
        lib.oracle_step.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def num_threads() -> int:
    return int(_lib().oracle_num_threads())


def set_num_threads(n: int) -> int:
    """Threads (OpenMP) of later steps; returns the count in effect."""
    return int(_lib().oracle_set_num_threads(int(n)))


def lattice(kind: int = D2Q16):
    """(c[n1], w[n1], T_L) of the lattice as computed by the oracle."""
    c = np.zeros(4)
    w = np.zeros(4)
    tl = np.zeros(1)
    _lib().oracle_lattice(int(kind), _d(c), _d(w), _d(tl))
    n1 = _N1[kind]
    return c[:n1], w[:n1], float(tl[0])


def transfer(gauge_src, gauge_dst, f_src, lattice: int = D2Q16) -> np.ndarray:
    """f^{lambda'} = M_{lambda'}^{-1} M_lambda f^lambda (Eq. transform) for one
    node; gauges are (u_x, u_y, T)."""
    gs = np.ascontiguousarray(gauge_src, dtype=np.float64)
    gd = np.ascontiguousarray(gauge_dst, dtype=np.float64)
    Q = _N1[lattice] ** 2
    fs = np.zeros(16)
    fs[:Q] = np.asarray(f_src, dtype=np.float64)
    out = np.zeros(16)
    _lib().oracle_transfer(int(lattice), _d(gs), _d(gd), _d(fs), _d(out))
    return out[:Q]


def interp_weights(t: float) -> np.ndarray:
    """Cubic Lagrange weights l_0..l_3 at local coordinate t (App. C)."""
    out = np.zeros(4)
    _lib().oracle_interp_weights(float(t), _d(out))
    return out


@dataclass
class State:
    f: np.ndarray   # (Q, ny, nx)
    ux: np.ndarray  # (ny, nx)
    uy: np.ndarray
    T: np.ndarray

    @property
    def shape(self):
        return self.ux.shape

    def rho(self) -> np.ndarray:
        return self.f.sum(axis=0)

    def copy(self) -> "State":
        return State(self.f.copy(), self.ux.copy(), self.uy.copy(), self.T.copy())


def init_equilibrium(rho, ux, uy, T, lattice: int = D2Q16) -> State:
    """f = rho W in each node's own gauge (Eq. equilibrium)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    f = np.zeros((_N1[lattice] ** 2, ny, nx))
    _lib().oracle_init_equilibrium(int(lattice), nx, ny, _d(rho), _d(f))
    return State(f, np.ascontiguousarray(ux, dtype=np.float64).copy(),
                 np.ascontiguousarray(uy, dtype=np.float64).copy(),
                 np.ascontiguousarray(T, dtype=np.float64).copy())


def step(state: State, params: Params | None = None, rows=None):
    """One PonD time step.  Returns (new_state, iters, flags).  With ``rows``
    = (y0, y1) only those rows are computed (the rest of the returned state is
    left zero), which bounds the CPU cost of a sample."""
    params = params or Params()
    if state.f.shape[0] != _N1[params.lattice] ** 2:
        raise ValueError("f has %d populations; the lattice needs %d"
                         % (state.f.shape[0], _N1[params.lattice] ** 2))
    ny, nx = state.shape
    y0, y1 = (0, ny) if rows is None else rows
    fo = np.zeros_like(state.f)
    uxo = np.zeros_like(state.ux)
    uyo = np.zeros_like(state.uy)
    To = np.zeros_like(state.T)
    it = np.zeros((ny, nx), dtype=np.int32)
    fl = np.zeros((ny, nx), dtype=np.int32)
    cp = params._c()
    rc = _lib().oracle_step(nx, ny, _d(state.f), _d(state.ux), _d(state.uy),
                            _d(state.T), _d(fo), _d(uxo), _d(uyo), _d(To), _i(it),
                            _i(fl), ctypes.byref(cp), y0, y1)
    if rc != 0:
        raise RuntimeError("oracle_step failed: %d" % rc)
    return State(fo, uxo, uyo, To), it, fl


def run(state: State, nsteps: int, params: Params | None = None):
    """nsteps PonD steps; returns (state, total passes, max passes, flag-or)."""
    total = 0
    mx = 0
    flags = 0
    for _ in range(nsteps):
        state, it, fl = step(state, params)
        total += int(it.sum())
        mx = max(mx, int(it.max()))
        flags |= int(np.bitwise_or.reduce(fl, axis=None))
    return state, total, mx, flags
