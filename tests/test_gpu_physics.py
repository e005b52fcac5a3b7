"""Physics of the GPU step against the paper's claims (through the C ABI).

- Kinematic viscosity from a decaying pi/4-tilted shear wave is nu for
  advection Mach numbers up to 100 and temperatures T_L/2, T_L, 2 T_L
  (viscosity experiment, main text: Galilean invariance).
- The speed of sound is sqrt(2 T) for T from 1e-4 to 1e2, at rest and advected
  at Ma 10 (speed-of-sound experiment; gamma = 2 for the 2D ideal gas).
- The isothermal variant (main text after Eq. postcollision) matches the
  oracle's isothermal step.
- The Taylor-Green vortex converges with at least second order in the grid
  size at the paper's convergence-study parameters (App. D).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1806_05089_gb300 import pond

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("T", [0.5, 1.0, 2.0])
@pytest.mark.parametrize("mach", [0.0, 1.0, 10.0, 100.0])
def test_shear_wave_viscosity_is_galilean_invariant(T, mach):
    n, A, nu, steps, every = 200, 0.05, 0.02, 2000, 100
    X, Y = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float))
    k = 2 * np.pi / n * np.array([1.0, 1.0])         # wave vector along (1, 1)
    phase = k[0] * X + k[1] * Y
    u_long = mach * np.sqrt(T)                      # along k
    u_tr = A * np.sin(phase)                        # transverse, along (1, -1)
    ux = (u_long + u_tr) / np.sqrt(2.0)
    uy = (u_long - u_tr) / np.sqrt(2.0)
    k2 = float(k @ k)
    amps = []
    # nu = T (1/(2 beta) - 1/2) dt at the run's temperature: T_ref = T
    with pond.Sim(n, n, pond.POND_FP32_MIXED, thermal=0, nu=nu, T_ref=T, use_graph=1) as s:
        s.set_state(np.ones((n, n)), ux, uy, np.full((n, n), T))
        for t in range(0, steps, every):
            stats = s.step(every)
            assert stats["nonphysical"] == 0 and stats["nonconverged"] == 0
            _, vx, vy, _ = s.moments()
            tr = (vx - vy) / np.sqrt(2.0)
            amps.append(np.abs((tr * np.exp(-1j * phase)).sum()) * 2 / (n * n))
    t = np.arange(1, len(amps) + 1) * every
    rate = -np.polyfit(t, np.log(amps), 1)[0]
    assert abs(rate / (nu * k2) - 1) < 0.03, (rate, nu * k2)


@pytest.mark.parametrize("mach", [0.0, 10.0])
@pytest.mark.parametrize("T,nx", [(1e-4, 16), (1e-2, 64), (1.0, 256), (100.0, 2048)])
def test_speed_of_sound_over_six_decades(T, nx, mach):
    eps = 1e-3
    cs = np.sqrt(2.0 * T)
    k = 2 * np.pi / nx
    period = 2 * np.pi / (cs * k)
    steps = int(1.6 * period) + 2
    x = np.arange(nx, dtype=float)
    u = mach * np.sqrt(T)
    rho = (1.0 + eps * np.cos(k * x))[None, :]
    with pond.Sim(nx, 1, pond.POND_FP64, nu=0.01) as s:
        s.set_state(rho, np.full((1, nx), u), np.zeros((1, nx)), np.full((1, nx), T))
        a = []
        for t in range(1, steps + 1):
            s.step(1, stats=False)
            r, _, _, TT = s.moments()
            p = (r * TT)[0]
            # pressure mode in the frame moving with the flow
            a.append(((p - p.mean()) * np.exp(-1j * k * (x - u * t))).sum().real * 2 / nx)
    a = np.array(a)
    zc = [i + a[i] / (a[i] - a[i + 1]) for i in range(len(a) - 1) if a[i] * a[i + 1] < 0]
    assert len(zc) >= 2
    half = np.diff(zc).mean()
    cs_meas = np.pi / half / k
    assert abs(cs_meas / cs - 1) < 0.01, (cs_meas, cs)


@pytest.mark.parametrize("precision,tol", [(pond.POND_FP64, 1e-12), (pond.POND_FP32_MIXED, 1e-5)])
def test_isothermal_step_matches_oracle(precision, tol):
    n = 40
    X, Y = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float))
    ux = 0.8 + 0.05 * np.sin(2 * np.pi * Y / n)
    uy = -0.3 + 0.05 * np.cos(2 * np.pi * X / n)
    rho = 1.0 + 0.02 * np.cos(2 * np.pi * (X + Y) / n)
    T = np.full((n, n), 0.7)
    cfg = {"thermal": 0}
    if precision == pond.POND_FP64:
        cfg["fixed_iter"] = 5
    with pond.Sim(n, n, precision, **cfg) as s:
        s.set_state(rho, ux, uy, T)
        s.step(4)
        st = s.state()
    o = oracle.init_equilibrium(rho, ux, uy, T)
    p = oracle.Params(thermal=0, fixed_iter=5 if precision == pond.POND_FP64 else 0)
    for _ in range(4):
        o, _, fl = oracle.step(o, p)
        assert np.all(fl == 0)
    assert np.abs(st.T - T).max() <= 4e-16 * 0.7
    orho = o.f.sum(0)
    assert np.max(np.abs(st.f.sum(0) - orho) / orho) <= tol
    scale = max(np.abs(o.ux).max(), np.sqrt(0.7))
    assert np.abs(st.ux - o.ux).max() <= tol * scale
    assert np.abs(st.uy - o.uy).max() <= tol * scale


def _tg_error(L, lattice, T, ma, re):
    """Relative L2 error of u against the decaying Taylor-Green solution,
    averaged over five times in [0.9 t_h, 1.1 t_h] (App. D)."""
    u0 = ma * np.sqrt(T)
    nu = u0 * L / re
    k = 2 * np.pi / L
    X, Y = np.meshgrid(np.arange(L, dtype=float), np.arange(L, dtype=float))

    def exact(t):
        d = (u0 / np.sqrt(2)) * np.exp(-2 * nu * k * k * t)
        return -d * np.cos(k * X) * np.sin(k * Y), d * np.sin(k * X) * np.cos(k * Y)
    ux0, uy0 = exact(0.0)
    th = np.log(2.0) / (2 * nu * k * k)
    errs, done = [], 0
    with pond.Sim(L, L, pond.POND_FP64, lattice=lattice, T_ref=T, nu=nu, thermal=0) as s:
        s.set_state(np.ones((L, L)), ux0, uy0, np.full((L, L), T))
        for ts in np.linspace(0.9 * th, 1.1 * th, 5).round().astype(int):
            s.step(int(ts - done), stats=False)
            done = ts
            _, ux, uy, _ = s.moments()
            ex, ey = exact(ts)
            errs.append(np.sqrt(((ux - ex) ** 2 + (uy - ey) ** 2).sum() / (ex ** 2 + ey ** 2).sum()))
    return float(np.mean(errs))


@pytest.mark.parametrize("lattice,T_L", [(pond.POND_D2Q9, 1 / 3), (pond.POND_D2Q16, 1.0)])
def test_taylor_green_converges_at_second_order(lattice, T_L):
    """App. D: Taylor-Green at Re = u0 L / nu = 50 and Ma = u0 / sqrt(T) =
    0.001, isothermal at T = 1 (= 3 T_L on D2Q9), L = 35, 50, 70 (the low end
    of the paper's [35, 120], about 2e8 node-updates).  The fitted order is
    at least 2 (measured: 2.7 on D2Q9, 2.6 on D2Q16; the error is dominated
    by the cubic reconstruction's damping, (k dx)^4 per step over ~L steps)."""
    g = GOLD["tg_convergence"]["value"]
    Ls = [35, 50, 70]
    errs = [_tg_error(L, lattice, 1.0, g["Ma"], g["Re"]) for L in Ls]
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    order = -np.polyfit(np.log(Ls), np.log(errs), 1)[0]
    assert order >= g["order"] - 0.1, (order, errs)


@pytest.mark.parametrize("lattice,T_L", [(pond.POND_D2Q16, 1.0), (pond.POND_D2Q9, 1 / 3)])
def test_taylor_green_decay_rate_long_run(lattice, T_L):
    """App. D / configuration 1 run long: 64^2 Taylor-Green (u0 = 0.05 sqrt(T),
    nu = 0.01), 2000 steps.  The fitted decay rate of u lies within 3 % of
    2 nu k^2 (the oracle's 100-step pin allows 5 %).  Measured: D2Q16 2.3 %
    faster, D2Q9 under 2 %; the excess is the cubic reconstruction's
    numerical damping, the same effect the convergence test measures."""
    from paper_1806_05089_gb300 import workloads
    n, nu, steps, every = 64, 0.01, 2000, 100
    tg = workloads.taylor_green(n, n, 0.05)
    ux, uy = tg.ux * np.sqrt(T_L), tg.uy * np.sqrt(T_L)
    basis = ux / np.abs(ux).max()
    amps = []
    with pond.Sim(n, n, pond.POND_FP64, lattice=lattice, T_ref=T_L, nu=nu) as s:
        s.set_state(tg.rho, ux, uy, tg.T * T_L)
        for _ in range(steps // every):
            stats = s.step(every)
            assert stats["nonphysical"] == 0 and stats["nonconverged"] == 0
            amps.append((s.moments()[1] * basis).sum() / (basis * basis).sum())
    t = every * np.arange(1, len(amps) + 1)
    rate = -np.polyfit(t[1:], np.log(np.array(amps)[1:]), 1)[0]
    k = 2 * np.pi / n
    assert abs(rate / (2 * nu * k * k) - 1) < 0.03, rate / (2 * nu * k * k)
