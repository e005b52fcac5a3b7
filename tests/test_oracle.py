"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

None of these compare the oracle with itself: each checks a closed form, an
invariant, a special case or an independent brute force (tests/bruteforce.py).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1806_05089_gb300 import workloads
from tests import bruteforce as bf

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def raw_moments(f, g):
    """Raw moments sum_q f_q v_x^m v_y^n, m,n = 0..3 (Eq. moments)."""
    return bf.moment_matrix(*g) @ f


# ---------------------------------------------------------------- lattice

def test_lattice_is_hermite_quadrature():
    c, w, tl = oracle.lattice()
    # speeds are the roots of He4(x) = x^4 - 6x^2 + 3
    assert np.allclose(c ** 4 - 6 * c ** 2 + 3, 0, atol=1e-13)
    assert np.all(np.diff(c) > 0)
    # Gauss-Hermite: sum_i w_i c_i^m = standard-normal moments up to m = 7
    gauss = [1, 0, 1, 0, 3, 0, 15, 0]
    for m, g in enumerate(gauss):
        assert abs((w * c ** m).sum() - g) < 1e-12, m
    # order 8 is no longer exact (105 for a Gaussian)
    assert abs((w * c ** 8).sum() - 105) > 1
    assert tl == 1.0  # T_L = sum w c^2


def test_equilibrium_moments_are_maxwellian():
    """rho W in gauge (u, T) carries the Maxwell-Boltzmann moments (App. A):
    1D factor exact to order 7, so all m, n <= 3 moments are exact."""
    c, w, _ = oracle.lattice()
    rho = 1.3
    for ux, uy, T in [(0.0, 0.0, 1.0), (1.5, -0.5, 0.3), (40.0, 7.0, 20.0)]:
        st = oracle.init_equilibrium(np.full((1, 1), rho), np.full((1, 1), ux),
                                     np.full((1, 1), uy), np.full((1, 1), T))
        f = st.f[:, 0, 0]
        vx, vy = bf.velocities(ux, uy, T)
        for m in range(4):
            for n in range(4):
                # exact Gaussian moment by a fine Gauss-Hermite rule (numpy)
                x, wx = np.polynomial.hermite_e.hermegauss(20)
                wx = wx / wx.sum()
                ex = (wx * (np.sqrt(T) * x + ux) ** m).sum()
                ey = (wx * (np.sqrt(T) * x + uy) ** n).sum()
                got = (f * vx ** m * vy ** n).sum()
                ref = rho * ex * ey
                assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (m, n)


# ---------------------------------------------------------------- transform

GAUGES = [((0.0, 0.0, 1.0), (0.1, -0.05, 1.2)),
          ((0.3, -0.2, 1.1), (0.35, -0.1, 0.9)),
          ((-0.4, 0.2, 0.7), (0.0, 0.0, 1.0)),
          ((0.2, 0.1, 0.5), (0.25, 0.05, 2.0))]


@pytest.mark.parametrize("gs,gd", GAUGES)
def test_transfer_matches_raw_monomial_solve(gs, gd):
    """Eq. transform with the paper's literal monomial moments, solved densely."""
    f = np.random.default_rng(1).random(16) + 0.1
    got = oracle.transfer(gs, gd, f)
    ref = bf.transfer(gs, gd, f)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("gs,gd", GAUGES + [((10.0, -3.0, 4.0), (10.2, -3.1, 4.3)),
                                            ((100.0, 0.0, 1.0), (100.01, 0.0, 1.001))])
def test_transfer_matches_lagrange_closed_form(gs, gd):
    """On a tensor lattice M_{l'}^{-1} M_l factorises into 1D Lagrange maps
    G[k][a] = L_k(xi_a) with xi = (sqrt(theta_s) c_a + u_s - u')/sqrt(theta')."""
    c = bf.C
    f = np.random.default_rng(2).random(16) + 0.1

    def G1(us, ut, sts, stt):
        xi = (sts * c + us - ut) / stt
        G = np.ones((4, 4))
        for k in range(4):
            for j in range(4):
                if j != k:
                    G[k, :] *= (xi - c[j]) / (c[k] - c[j])
        return G
    sts, stt = np.sqrt(gs[2]), np.sqrt(gd[2])
    Gx = G1(gs[0], gd[0], sts, stt)
    Gy = G1(gs[1], gd[1], sts, stt)
    ref = (Gx @ f.reshape(4, 4) @ Gy.T).reshape(16)
    got = oracle.transfer(gs, gd, f)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(f).max() * max(1, np.abs(Gx).max() ** 2)


@pytest.mark.parametrize("gs,gd", GAUGES)
def test_transfer_matches_moments(gs, gd):
    """Eq. match: the Q moments are the same in both gauges."""
    f = np.random.default_rng(3).random(16)
    f2 = oracle.transfer(gs, gd, f)
    a = raw_moments(f, gs)
    b = raw_moments(f2, gd)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_transfer_identity_and_round_trip():
    f = np.random.default_rng(4).random(16)
    for gs, gd in GAUGES + [((50.0, -20.0, 9.0), (50.5, -19.0, 10.0))]:
        assert np.abs(oracle.transfer(gs, gs, f) - f).max() < 1e-13 * (1 + abs(gs[0]) + abs(gs[1]))
        back = oracle.transfer(gd, gs, oracle.transfer(gs, gd, f))
        assert np.abs(back - f).max() < 1e-11
        assert abs(oracle.transfer(gs, gd, f).sum() - f.sum()) < 1e-13


# ---------------------------------------------------------------- interpolation

def test_interp_weights_exact_for_cubics():
    rng = np.random.default_rng(5)
    for t in [1.0, 1.25, 1.5, 1.999, 1.0 + 1e-9] + list(rng.uniform(1, 2, 8)):
        a = oracle.interp_weights(t)
        assert np.allclose(a, bf.interp_weights(t), atol=1e-14)
        for p in range(4):
            assert abs(sum(a[j] * j ** p for j in range(4)) - t ** p) < 1e-13
    assert np.allclose(oracle.interp_weights(1.0), [0, 1, 0, 0], atol=1e-15)


# ---------------------------------------------------------------- whole step

def _tiny_state(nx, ny, seed, mach=0.2):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.05 * rng.standard_normal((ny, nx))
    ux = mach + 0.05 * rng.standard_normal((ny, nx))
    uy = -0.5 * mach + 0.05 * rng.standard_normal((ny, nx))
    T = 1.0 + 0.1 * rng.random((ny, nx))
    st = oracle.init_equilibrium(rho, ux, uy, T)
    # add a non-equilibrium part so the step is not trivial
    st.f = st.f * (1.0 + 0.05 * rng.standard_normal(st.f.shape))
    return st


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 1), (3, 2), (4, 4)])
def test_step_matches_bruteforce_tiny(nx, ny):
    st = _tiny_state(nx, ny, seed=nx * 10 + ny)
    p = oracle.Params(fixed_iter=3)
    got, it, _ = oracle.step(st, p)
    fo, uxo, uyo, To = bf.step(st.f, st.ux, st.uy, st.T, passes=3)
    assert np.all(it == 3)
    assert np.abs(got.f - fo).max() <= 1e-11 * np.abs(fo).max()
    assert np.abs(got.ux - uxo).max() <= 1e-11
    assert np.abs(got.uy - uyo).max() <= 1e-11
    assert np.abs(got.T - To).max() <= 1e-11


def test_single_node_limit_is_own_moments():
    """On a 1x1 periodic grid the reconstruction reduces to the node itself,
    the transform preserves moments, so the limit gauge is the node's own
    moments after the second pass."""
    st = _tiny_state(1, 1, seed=9)
    f = st.f[:, 0, 0]
    g = (st.ux[0, 0], st.uy[0, 0], st.T[0, 0])
    vx, vy = bf.velocities(*g)
    rho = f.sum()
    ux = (vx * f).sum() / rho
    uy = (vy * f).sum() / rho
    T = (((vx ** 2 + vy ** 2) * f).sum() / rho - ux ** 2 - uy ** 2) / 2
    out, it, _ = oracle.step(st, oracle.Params())
    assert it[0, 0] == 2
    assert abs(out.ux[0, 0] - ux) < 1e-13 and abs(out.uy[0, 0] - uy) < 1e-13
    assert abs(out.T[0, 0] - T) < 1e-13


@pytest.mark.parametrize("mach,T", [(0.0, 1.0), (1.58, 1.0), (10.0, 0.01), (100.0, 1.0),
                                    (3.0, 100.0), (100.0, 100.0)])
def test_uniform_state_is_a_fixed_point(mach, T):
    """A uniform state stays uniform at any Mach number and temperature, in one
    predictor-corrector pass (G = I, interpolation weights sum to 1, f = rho W)."""
    n = 6
    ux = np.full((n, n), mach * np.sqrt(T) * np.cos(0.3))
    uy = np.full((n, n), mach * np.sqrt(T) * np.sin(0.3))
    st = oracle.init_equilibrium(np.full((n, n), 1.2), ux, uy, np.full((n, n), T))
    f0 = st.f.copy()
    for _ in range(20):
        st, it, fl = oracle.step(st, oracle.Params())
        assert np.all(it == 1) and np.all(fl == 0)
    # rounding bound: the energy moment of Eq. conservation_T is formed from
    # |v|^2 ~ |u|^2 + 2T, so each step may move T by ~16 eps (|u|^2 + 2T);
    # 20 steps of that, relative to T (and likewise for f and u)
    rel = max(1e-13, 20 * 16 * 1.11e-16 * (1.0 + mach * mach))
    speed = np.hypot(ux, uy).max() + np.sqrt(T)
    assert np.abs(st.f - f0).max() <= rel * np.abs(f0).max()
    assert np.abs(st.ux - ux).max() <= rel * speed
    assert np.abs(st.uy - uy).max() <= rel * speed
    assert np.abs(st.T - T).max() <= rel * T


def test_seed_independence():
    """The converged limit does not depend on the seed gauge (main text after
    the vortex benchmark): previous gauge, {0, T_L} and {-u, T}."""
    f = workloads.supersonic(nx=24, ny=20)
    st = oracle.init_equilibrium(f.rho, 0.3 * f.ux, 0.3 * f.uy, f.T)
    st, _, _ = oracle.step(st)  # develop a non-equilibrium part
    outs = []
    for seed in (0, 1, 2):
        p = oracle.Params(seed_mode=seed, max_iter=60)
        o, it, fl = oracle.step(st, p)
        assert np.all(fl == 0), seed
        outs.append(o)
    for o in outs[1:]:
        for a, b in [(o.ux, outs[0].ux), (o.uy, outs[0].uy), (o.T, outs[0].T)]:
            assert np.abs(a - b).max() <= 1e-9


@pytest.mark.parametrize("passes", [1, 2, 40])
def test_stored_gauge_is_comoving_frame(passes):
    """The stored gauge is the co-moving frame of the stored populations
    (remark after Eq. precollision), after any number of passes: the BGK step
    then keeps rho, rho u and energy exactly."""
    f = workloads.supersonic(nx=16, ny=12)
    st = oracle.init_equilibrium(f.rho, f.ux, f.uy, f.T)
    for _ in range(2):
        st, _, _ = oracle.step(st, oracle.Params(fixed_iter=passes))
    for Y in range(st.shape[0]):
        for X in range(st.shape[1]):
            g = (st.ux[Y, X], st.uy[Y, X], st.T[Y, X])
            vx, vy = bf.velocities(*g)
            fq = st.f[:, Y, X]
            rho = fq.sum()
            assert abs((vx * fq).sum() / rho - g[0]) < 1e-12
            assert abs((vy * fq).sum() / rho - g[1]) < 1e-12
            e = ((vx ** 2 + vy ** 2) * fq).sum() / rho - g[0] ** 2 - g[1] ** 2
            assert abs(e / 2 - g[2]) < 1e-11


def test_iteration_counts_match_paper_range():
    """Two to three passes past the predictor on a smooth low-Mach flow, at
    most five in all (App. E); a supersonic advected field needs more passes
    because the seed (the previous step's gauge at the node) is further from
    the limit, but still converges well inside max_iter."""
    tg = workloads.tg64(32)
    st = oracle.init_equilibrium(tg.rho, tg.ux, tg.uy, tg.T)
    for _ in range(4):
        st, it, fl = oracle.step(st)
    assert np.all(fl == 0)
    assert 2.0 <= it.mean() <= 4.0
    assert it.max() <= GOLD["max_iterations_observed"]["value"]
    f = workloads.supersonic(nx=64, ny=64)
    st = oracle.init_equilibrium(f.rho, f.ux, f.uy, f.T)
    for _ in range(2):
        st, it, fl = oracle.step(st)
    assert np.all(fl == 0) and it.max() < 12


def test_nonphysical_input_is_flagged():
    st = _tiny_state(4, 4, seed=3)
    st.T[1, 2] = -1.0
    _, _, fl = oracle.step(st)
    assert fl.max() & oracle.FLAG_NONPHYSICAL


# ---------------------------------------------------------------- physics pins

def _amplitude(field, basis):
    return (field * basis).sum() / (basis * basis).sum()


def test_taylor_green_decay_rate():
    """App. D: u decays as exp(-2 nu k^2 t); the fitted rate over 100 steps on
    64^2 (u0 = 0.05, nu = 0.01) lies within 5 % of 2 nu k^2."""
    n = 64
    tg = workloads.tg64(n)
    st = oracle.init_equilibrium(tg.rho, tg.ux, tg.uy, tg.T)
    basis = tg.ux / np.abs(tg.ux).max()
    nu = 0.01
    amps = []
    steps = 100
    for t in range(steps):
        st, _, fl = oracle.step(st, oracle.Params(nu=nu))
        assert np.all(fl == 0)
        amps.append(_amplitude(st.ux, basis))
    t = np.arange(1, steps + 1)
    sel = t >= 10
    rate = -np.polyfit(t[sel], np.log(amps)[sel], 1)[0]
    k = 2 * np.pi / n
    theory = GOLD["tg_decay_factor"]["value"] * nu * k * k
    assert abs(rate / theory - 1) < 0.05, (rate, theory)


@pytest.mark.parametrize("mach", [0.0, 1.5, 10.0])
def test_shear_wave_galilean_invariance(mach):
    """Isothermal shear wave u_y = A sin(2 pi x/L) advected along x at Mach
    Ma_a (main text, viscosity experiment): decay rate nu k^2 independent of
    Ma_a, and the wave moves with the flow."""
    L, A, nu, T, steps = 64, 0.05, 0.05, 1.0, 60
    X = np.arange(L, dtype=float)[None, :]
    U = mach * np.sqrt(T)
    st = oracle.init_equilibrium(np.ones((1, L)), np.full((1, L), U),
                                 A * np.sin(2 * np.pi * X / L), np.full((1, L), T))
    p = oracle.Params(nu=nu, thermal=0)
    k = 2 * np.pi / L
    amps = []
    for t in range(steps):
        st, _, fl = oracle.step(st, p)
        assert np.all(fl == 0)
        z = (st.uy[0] * np.exp(-1j * k * X[0])).sum() * 2 / L  # = A e^{-i phase}/i
        amps.append(z)
    amps = np.array(amps)
    t = np.arange(1, steps + 1)
    rate = -np.polyfit(t[10:], np.log(np.abs(amps[10:])), 1)[0]
    assert abs(rate / (nu * k * k) - 1) < 0.03, rate
    phase = np.unwrap(np.angle(amps))
    speed = -np.polyfit(t[10:], phase[10:], 1)[0] / k
    assert abs(speed - U) < 1e-3 * max(1.0, U), speed


@pytest.mark.parametrize("T", [0.5, 2.0])
def test_speed_of_sound(T):
    """Thermal mode: a standing acoustic wave oscillates with c_s = sqrt(gamma T),
    gamma = 2 (speed-of-sound experiment)."""
    L, eps, steps = 64, 1e-3, 120
    X = np.arange(L, dtype=float)[None, :]
    st = oracle.init_equilibrium(1 + eps * np.cos(2 * np.pi * X / L), np.zeros((1, L)),
                                 np.zeros((1, L)), np.full((1, L), T))
    k = 2 * np.pi / L
    basis = np.cos(k * X[0])
    a = []
    for _ in range(steps):
        st, _, fl = oracle.step(st, oracle.Params(nu=0.01))
        assert np.all(fl == 0)
        p = st.f.sum(axis=0)[0] * st.T[0]  # pressure p = rho T; the entropy mode has none
        a.append(((p - p.mean()) * basis).sum() * 2 / L)
    a = np.array(a)
    # zero crossings of the pressure mode -> half periods
    zc = [i + a[i] / (a[i] - a[i + 1]) for i in range(len(a) - 1) if a[i] * a[i + 1] < 0]
    half = np.diff(zc).mean()
    omega = np.pi / half
    cs = omega / k
    assert abs(cs / np.sqrt(GOLD["gamma_2d"]["value"] * T) - 1) < 0.01, cs


@pytest.mark.parametrize("lattice,T_L", [(oracle.D2Q16, 1.0), (oracle.D2Q9, 1.0 / 3.0)])
def test_one_pass_from_a_uniform_gauge_conserves_globally(lattice, T_L):
    """From a uniform gauge, a step of one pass conserves total mass, momentum
    and energy to rounding: every node then shares the departure offsets, so
    the interpolation (App. C) is a periodic convolution with weights summing
    to one and keeps each population's total; the re-gauge (Eq. transform)
    keeps each node's moments and BGK (Eq. postcollision) conserves them.
    The stored gauge moves by a few percent, so neither part is trivial.  A
    second pass, in node-dependent gauges, is not conservative (the paper
    claims no global conservation), which the last check confirms."""
    rng = np.random.default_rng(4)
    ny, nx = 20, 24
    rho = 1 + 0.2 * rng.random((ny, nx))
    shape = (ny, nx)
    ux, uy = np.full(shape, 1.3 * np.sqrt(T_L)), np.full(shape, -0.4 * np.sqrt(T_L))
    T = np.full(shape, 0.8 * T_L)
    st = oracle.init_equilibrium(rho, ux, uy, T, lattice=lattice)

    def totals(s):
        r = s.f.sum(axis=0)
        return np.array([r.sum(), (r * s.ux).sum(), (r * s.uy).sum(),
                         (r * (s.ux ** 2 + s.uy ** 2 + 2 * s.T)).sum()])

    before = totals(st)
    one, _, fl = oracle.step(st, oracle.Params(nu=0.01, fixed_iter=1, lattice=lattice, T_ref=T_L))
    assert np.all(fl == 0)
    assert np.abs(one.ux - ux).max() > 1e-2 * np.sqrt(T_L)
    assert np.all(np.abs(totals(one) - before) <= 1e-13 * np.abs(before))
    two, _, _ = oracle.step(st, oracle.Params(nu=0.01, fixed_iter=2, lattice=lattice, T_ref=T_L))
    assert np.abs(totals(two) - before).max() > 1e-6 * np.abs(before).max()
