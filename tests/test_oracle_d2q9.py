"""Pins of the oracle on the paper's own D2Q9 lattice (App. A, App. B), and
the thermal diffusivity of both lattices.

As for D2Q16, none of these compare the oracle with itself: the closed-form
transfer matrix of App. B (with the reading of its misprints stated below),
the Maxwell-Boltzmann moments of the equilibrium, brute force on tiny grids,
the uniform state, and the paper's D2Q9 thermal diffusivity.
"""
import json
import os

import numpy as np
import pytest

import oracle
from tests import bruteforce as bf

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
Q9 = oracle.D2Q9


def test_d2q9_lattice_constants():
    c, w, tl = oracle.lattice(Q9)
    assert np.array_equal(c, [-1.0, 0.0, 1.0])
    w0, w1 = GOLD["d2q9_weights"]["value"]
    assert np.allclose(w, [w1, w0, w1], rtol=0, atol=1e-16)
    assert abs(tl - GOLD["d2q9_T_L"]["value"]) < 1e-16
    assert abs((w * c * c).sum() - tl) < 1e-16  # T_L is the lattice's second moment


def test_d2q9_equilibrium_moments_are_maxwellian():
    """App. A: rho W_i W_j in gauge (u, T) carries the Maxwell-Boltzmann
    moments up to fourth order (m + n <= 4) for any u and T; the sixth
    order is not exact (so the check can fail)."""
    rho = 0.9
    x, wx = np.polynomial.hermite_e.hermegauss(20)
    wx = wx / wx.sum()
    for ux, uy, T in [(0.0, 0.0, 1 / 3), (1.5, -0.5, 0.3), (40.0, 7.0, 20.0), (0.2, 0.1, 1e-3)]:
        st = oracle.init_equilibrium(np.full((1, 1), rho), np.full((1, 1), ux),
                                     np.full((1, 1), uy), np.full((1, 1), T), lattice=Q9)
        f = st.f[:, 0, 0]
        vx, vy = bf.velocities(ux, uy, T, "d2q9")

        def mb(m, n):
            return rho * (wx * (np.sqrt(T) * x + ux) ** m).sum() * (wx * (np.sqrt(T) * x + uy) ** n).sum()
        for m in range(5):
            for n in range(5 - m):
                got = (f * vx ** m * vy ** n).sum()
                ref = mb(m, n)
                assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (m, n, ux, T)
        # sixth central moment: lattice 1/3 * ... vs Gaussian 15 theta^3 T_L^3
        c6 = (f * (vx - ux) ** 6).sum()
        assert abs(c6 - rho * 15 * T ** 3) > 0.1 * rho * 15 * T ** 3


def app_b_transfer(gs, gd, f):
    """App. B, Eq. transform2, as a closed-form dot product.  As printed the
    formula has misprints; the reading that makes it equal to the linear
    solve of Eq. invariance is: omega(0) = -1/T', omega(+-1) = +1/(2 T'),
    B(i, 0) = T' and B(i, j) = j sqrt(T') A(i) (T' the target temperature),
    with A(i) = (u' - u)/sqrt(3) - i sqrt(T) as printed."""
    us, vs, Ts = gs
    ut, vt, Tt = gd
    idx = (-1, 0, 1)

    def omega(j):
        return -1.0 / Tt if j == 0 else 0.5 / Tt

    def g(du, i, j):
        A = du / np.sqrt(3.0) - i * np.sqrt(Ts)
        B = Tt if j == 0 else j * np.sqrt(Tt) * A
        return A * A - B

    F = f.reshape(3, 3)
    out = np.zeros((3, 3))
    for a, k in enumerate(idx):
        for b, l in enumerate(idx):
            acc = 0.0
            for p, i in enumerate(idx):
                for q, j in enumerate(idx):
                    acc += g(ut - us, i, k) * g(vt - vs, j, l) * F[p, q]
            out[a, b] = omega(k) * omega(l) * acc
    return out.reshape(9)


GAUGES9 = [((0.0, 0.0, 1 / 3), (0.1, -0.05, 0.4)),
           ((0.3, -0.2, 0.5), (0.35, -0.1, 0.3)),
           ((-0.4, 0.2, 0.2), (0.0, 0.0, 1 / 3)),
           ((2.0, -1.0, 1.0), (2.2, -0.9, 1.3)),
           ((30.0, 5.0, 4.0), (30.4, 5.1, 4.4))]


@pytest.mark.parametrize("gs,gd", GAUGES9)
def test_d2q9_transfer_matches_app_b_closed_form(gs, gd):
    f = np.random.default_rng(11).random(9) + 0.1
    got = oracle.transfer(gs, gd, f, lattice=Q9)
    ref = app_b_transfer(gs, gd, f)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("gs,gd", GAUGES9[:4])
def test_d2q9_transfer_matches_raw_monomial_solve(gs, gd):
    """Eq. invariance with the 9 monomial moments of App. B, solved densely."""
    f = np.random.default_rng(12).random(9) + 0.1
    got = oracle.transfer(gs, gd, f, lattice=Q9)
    ref = bf.transfer(gs, gd, f, "d2q9")
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    # the nine moments M_mn, m, n <= 2, are the same in both gauges
    a = bf.moment_matrix(*gs, "d2q9") @ f
    b = bf.moment_matrix(*gd, "d2q9") @ got
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_d2q9_transfer_identity_and_round_trip():
    f = np.random.default_rng(13).random(9)
    for gs, gd in GAUGES9:
        assert np.abs(oracle.transfer(gs, gs, f, lattice=Q9) - f).max() < 1e-13 * (1 + abs(gs[0]) + abs(gs[1]))
        back = oracle.transfer(gd, gs, oracle.transfer(gs, gd, f, lattice=Q9), lattice=Q9)
        assert np.abs(back - f).max() < 1e-10


def test_d2q9_printed_app_b_is_not_the_transfer():
    """The formula exactly as printed (omega(0) = 1/T', omega(+-1) = -1/(2T'),
    T in B) does not match the moments: the reading above is needed."""
    gs, gd = GAUGES9[1]
    f = np.random.default_rng(14).random(9) + 0.1
    us, vs, Ts = gs
    ut, vt, Tt = gd

    def g(du, i, j):
        A = du / np.sqrt(3.0) - i * np.sqrt(Ts)
        return A * A - (Ts if j == 0 else j * np.sqrt(Ts) * A)
    om = {0: 1.0 / Tt, -1: -0.5 / Tt, 1: -0.5 / Tt}
    idx = (-1, 0, 1)
    F = f.reshape(3, 3)
    printed = np.array([[om[k] * om[l] * sum(g(ut - us, i, k) * g(vt - vs, j, l) * F[p, q]
                                             for p, i in enumerate(idx) for q, j in enumerate(idx))
                         for l in idx] for k in idx]).reshape(9)
    assert np.abs(printed - oracle.transfer(gs, gd, f, lattice=Q9)).max() > 1e-3


def _tiny_state9(nx, ny, seed, mach=0.2):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.05 * rng.standard_normal((ny, nx))
    ux = mach + 0.05 * rng.standard_normal((ny, nx))
    uy = -0.5 * mach + 0.05 * rng.standard_normal((ny, nx))
    T = 1 / 3 + 0.03 * rng.random((ny, nx))
    st = oracle.init_equilibrium(rho, ux, uy, T, lattice=Q9)
    st.f = st.f * (1.0 + 0.05 * rng.standard_normal(st.f.shape))
    return st


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 1), (3, 2), (4, 4)])
@pytest.mark.parametrize("thermal", [1, 0])
def test_d2q9_step_matches_bruteforce_tiny(nx, ny, thermal):
    st = _tiny_state9(nx, ny, seed=nx * 10 + ny)
    p = oracle.Params(fixed_iter=3, lattice=Q9, thermal=thermal, T_ref=1 / 3)
    got, it, _ = oracle.step(st, p)
    fo, uxo, uyo, To = bf.step(st.f, st.ux, st.uy, st.T, passes=3, thermal=bool(thermal),
                               T_ref=1 / 3, lattice="d2q9")
    assert np.all(it == 3)
    assert np.abs(got.f - fo).max() <= 1e-11 * np.abs(fo).max()
    assert np.abs(got.ux - uxo).max() <= 1e-11
    assert np.abs(got.uy - uyo).max() <= 1e-11
    assert np.abs(got.T - To).max() <= 1e-11


@pytest.mark.parametrize("mach,T", [(0.0, 1 / 3), (10.0, 0.01), (100.0, 1.0), (3.0, 100.0)])
def test_d2q9_uniform_state_is_a_fixed_point(mach, T):
    n = 5
    ux = np.full((n, n), mach * np.sqrt(T) * np.cos(0.7))
    uy = np.full((n, n), mach * np.sqrt(T) * np.sin(0.7))
    st = oracle.init_equilibrium(np.full((n, n), 0.8), ux, uy, np.full((n, n), T), lattice=Q9)
    f0 = st.f.copy()
    p = oracle.Params(lattice=Q9, T_ref=T)
    for _ in range(10):
        st, it, fl = oracle.step(st, p)
        assert np.all(it == 1) and np.all(fl == 0)
    rel = max(1e-13, 10 * 9 * 1.11e-16 * (1.0 + 3 * mach * mach))
    speed = np.hypot(ux, uy).max() + np.sqrt(T)
    assert np.abs(st.f - f0).max() <= rel * np.abs(f0).max()
    assert np.abs(st.ux - ux).max() <= rel * speed
    assert np.abs(st.T - T).max() <= rel * T


def test_d2q9_stored_gauge_is_comoving_frame():
    rng = np.random.default_rng(15)
    n = 10
    X = np.arange(n)[None, :] + 0 * np.arange(n)[:, None]
    st = oracle.init_equilibrium(1 + 0.05 * np.sin(2 * np.pi * X / n), np.full((n, n), 1.2),
                                 0.1 * rng.standard_normal((n, n)), 0.3 + 0.02 * rng.random((n, n)),
                                 lattice=Q9)
    for _ in range(2):
        st, _, fl = oracle.step(st, oracle.Params(lattice=Q9, T_ref=1 / 3))
        assert np.all(fl == 0)
    for Y in range(n):
        for Xn in range(n):
            g = (st.ux[Y, Xn], st.uy[Y, Xn], st.T[Y, Xn])
            vx, vy = bf.velocities(*g, "d2q9")
            fq = st.f[:, Y, Xn]
            rho = fq.sum()
            assert abs((vx * fq).sum() / rho - g[0]) < 1e-12
            assert abs((vy * fq).sum() / rho - g[1]) < 1e-12
            e = ((vx ** 2 + vy ** 2) * fq).sum() / rho - g[0] ** 2 - g[1] ** 2
            assert abs(e / 2 - g[2]) < 1e-12


def _entropy_mode_decay(lattice, L, nu, T0, U, steps):
    """Decay rate of a density wave at constant pressure rho T = T0 (thermal
    diffusivity experiment: amplitude 1e-3)."""
    A = 1e-3
    X = np.arange(L, dtype=float)[None, :]
    rho = 1 + A * np.sin(2 * np.pi * X / L)
    st = oracle.init_equilibrium(rho, np.full((1, L), U), np.zeros((1, L)), T0 / rho,
                                 lattice=lattice)
    p = oracle.Params(nu=nu, T_ref=T0, lattice=lattice)
    k = 2 * np.pi / L
    amps = []
    for _ in range(steps):
        st, _, fl = oracle.step(st, p)
        assert np.all(fl == 0)
        r = st.f.sum(axis=0)[0]
        amps.append(abs((r * np.exp(-1j * k * X[0])).sum()) * 2 / L)
    t = np.arange(1, steps + 1)
    sel = t > steps // 5
    return -np.polyfit(t[sel], np.log(np.array(amps)[sel]), 1)[0] / (k * k)


@pytest.mark.parametrize("U", [0.0, 2.0])
def test_d2q9_thermal_diffusivity(U):
    """Thermal diffusivity experiment: for D2Q9 alpha = (T/4)(1/(2 beta) -
    1/2) dt, independent of the advection speed."""
    T0, nu = 1 / 3, 0.1
    alpha = _entropy_mode_decay(Q9, 64, nu, T0, U, 1500)
    beta = 1.0 / (2.0 * nu / T0 + 1.0)
    theory = (T0 / 4) * (1 / (2 * beta) - 0.5)
    assert abs(alpha / theory - 1) < 0.01, (alpha, theory)


def test_d2q16_thermal_diffusivity_is_bgk_prandtl_one():
    """On D2Q16 the equilibrium carries the fourth-order moments the heat flux
    needs, so the BGK collision gives the kinetic-theory Prandtl number 1:
    alpha = nu (unlike D2Q9, whose alpha is a quarter of that)."""
    nu = 0.1
    alpha = _entropy_mode_decay(oracle.D2Q16, 64, nu, 1.0, 0.0, 700)
    assert abs(alpha / nu - 1) < 0.01, alpha


@pytest.mark.parametrize("mach", [0.0, 1.5, 10.0])
def test_d2q9_shear_wave_galilean_invariance(mach):
    """Viscosity experiment on D2Q9: an isothermal shear wave u_y = A sin(2 pi
    x/L) at T = T_L, advected along x at Mach Ma_a, decays at nu k^2 (within
    3 %, independent of Ma_a) and moves with the flow."""
    T = GOLD["d2q9_T_L"]["value"]
    L, A, nu, steps = 64, 0.05 * np.sqrt(T), 0.05, 60
    X = np.arange(L, dtype=float)[None, :]
    U = mach * np.sqrt(T)
    st = oracle.init_equilibrium(np.ones((1, L)), np.full((1, L), U),
                                 A * np.sin(2 * np.pi * X / L), np.full((1, L), T), lattice=Q9)
    p = oracle.Params(nu=nu, thermal=0, lattice=Q9, T_ref=T)
    k = 2 * np.pi / L
    amps = []
    for _ in range(steps):
        st, _, fl = oracle.step(st, p)
        assert np.all(fl == 0)
        amps.append((st.uy[0] * np.exp(-1j * k * X[0])).sum() * 2 / L)
    amps = np.array(amps)
    t = np.arange(1, steps + 1)
    rate = -np.polyfit(t[10:], np.log(np.abs(amps[10:])), 1)[0]
    assert abs(rate / (nu * k * k) - 1) < 0.03, rate
    phase = np.unwrap(np.angle(amps))
    speed = -np.polyfit(t[10:], phase[10:], 1)[0] / k
    assert abs(speed - U) < 1e-3 * max(1.0, U), speed


@pytest.mark.parametrize("T_over_TL", [0.5, 2.0])
def test_d2q9_speed_of_sound(T_over_TL):
    """Speed-of-sound experiment on D2Q9: a standing acoustic wave oscillates
    at c_s = sqrt(gamma T), gamma = 2, within 1 %; the lattice's T_L = 1/3
    does not enter (T at half and twice T_L)."""
    T = T_over_TL * GOLD["d2q9_T_L"]["value"]
    L, eps, steps = 64, 1e-3, 200
    X = np.arange(L, dtype=float)[None, :]
    st = oracle.init_equilibrium(1 + eps * np.cos(2 * np.pi * X / L), np.zeros((1, L)),
                                 np.zeros((1, L)), np.full((1, L), T), lattice=Q9)
    k = 2 * np.pi / L
    basis = np.cos(k * X[0])
    a = []
    for _ in range(steps):
        st, _, fl = oracle.step(st, oracle.Params(nu=0.01, lattice=Q9, T_ref=T))
        assert np.all(fl == 0)
        p = st.f.sum(axis=0)[0] * st.T[0]  # pressure p = rho T
        a.append(((p - p.mean()) * basis).sum() * 2 / L)
    a = np.array(a)
    zc = [i + a[i] / (a[i] - a[i + 1]) for i in range(len(a) - 1) if a[i] * a[i + 1] < 0]
    assert len(zc) >= 3
    cs = np.pi / np.diff(zc).mean() / k
    assert abs(cs / np.sqrt(GOLD["gamma_2d"]["value"] * T) - 1) < 0.01, cs


def test_d2q9_taylor_green_decay_rate():
    """App. D on the paper's own lattice: the 64^2 Taylor-Green vortex at the
    same Mach number as the D2Q16 pin (u0 = 0.05 sqrt(T_L), T = T_L,
    nu = 0.01) decays at 2 nu k^2 within 5 %."""
    from paper_1806_05089_gb300 import workloads
    T_L = GOLD["d2q9_T_L"]["value"]
    n, nu, steps = 64, 0.01, 100
    tg = workloads.tg64(n)
    st = oracle.init_equilibrium(tg.rho, tg.ux * np.sqrt(T_L), tg.uy * np.sqrt(T_L),
                                 tg.T * T_L, lattice=Q9)
    basis = tg.ux / np.abs(tg.ux).max()
    amps = []
    for _ in range(steps):
        st, _, fl = oracle.step(st, oracle.Params(nu=nu, lattice=Q9, T_ref=T_L))
        assert np.all(fl == 0)
        amps.append((st.ux * basis).sum() / (basis * basis).sum())
    t = np.arange(1, steps + 1)
    sel = t >= 10
    rate = -np.polyfit(t[sel], np.log(amps)[sel], 1)[0]
    k = 2 * np.pi / n
    theory = GOLD["tg_decay_factor"]["value"] * nu * k * k
    assert abs(rate / theory - 1) < 0.05, (rate, theory)
