"""More pins of the FP64 CPU oracle: the stop test of the predictor-corrector,
the whole step at high Mach number and T != 1, and the composition of the
gauge transform that the staged kernel's reformulation rests on.

The stop test (App. E, Eq. convergence) is pinned through whole oracle steps
on a 1 x 1 grid whose stored populations are built so that the first pass
moves the gauge by a chosen amount (tests/convergence_cases.py): the pass
count then shows which test the oracle applied.  The high-Mach step is
checked against the brute force of tests/bruteforce.py in 40-digit mpmath
arithmetic, which solves the paper's raw monomial Eq. transform literally
where the FP64 solve is too ill-conditioned to use.
"""
import numpy as np
import pytest

import oracle
from tests import bruteforce as bf
from tests import convergence_cases as cc

LAT = {"d2q16": oracle.D2Q16, "d2q9": oracle.D2Q9}


@pytest.mark.parametrize("case", cc.cases(), ids=lambda c: c.name)
def test_stop_test_decision(case):
    f = cc.populations(case)
    # the construction gives the intended moments (checked independently)
    got = cc.moments(case, f)
    for a, b in zip(got, case.gauge1):
        assert abs(a - b) <= 1e-13 * max(1.0, abs(b))
    Q = f.size
    st = oracle.State(f.reshape(Q, 1, 1).copy(), np.full((1, 1), case.gauge0[0]),
                      np.full((1, 1), case.gauge0[1]), np.full((1, 1), case.gauge0[2]))
    p = oracle.Params(eps_abs=case.eps_abs, eps_rel=case.eps_rel, lattice=LAT[case.lattice],
                      T_ref=bf.LATTICES[case.lattice][2])
    out, it, fl = oracle.step(st, p)
    assert fl[0, 0] == 0
    assert it[0, 0] == case.passes
    # after the stop, the stored gauge is the populations' own moments
    assert abs(out.ux[0, 0] - case.gauge1[0]) <= 1e-12 * max(1.0, abs(case.gauge1[0]))
    assert abs(out.T[0, 0] - case.gauge1[2]) <= 1e-12 * case.gauge1[2]


def _fast_state(nx, ny, seed, mach, T0, lattice="d2q16"):
    """Tiny state moving at `mach` times the adiabatic sound speed sqrt(2 T0)
    (gamma = 2 in 2D), with 5 % noise on every field and a non-equilibrium
    part, in a direction that is not a lattice axis."""
    rng = np.random.default_rng(seed)
    U = mach * np.sqrt(2.0 * T0)
    rho = 1.0 + 0.05 * rng.standard_normal((ny, nx))
    ux = U * np.cos(0.4) * (1.0 + 0.05 * rng.standard_normal((ny, nx)))
    uy = U * np.sin(0.4) * (1.0 + 0.05 * rng.standard_normal((ny, nx)))
    T = T0 * (1.0 + 0.05 * rng.random((ny, nx)))
    st = oracle.init_equilibrium(rho, ux, uy, T, lattice=LAT[lattice])
    st.f = st.f * (1.0 + 0.05 * rng.standard_normal(st.f.shape))
    return st


@pytest.mark.parametrize("nx,ny,mach,T0,lattice", [
    (2, 1, 3.0, 4.0, "d2q16"),
    (2, 2, 3.0, 0.25, "d2q16"),
    (3, 2, 5.0, 2.5, "d2q16"),
    (2, 2, 4.0, 0.2, "d2q9"),
])
def test_step_matches_high_precision_bruteforce_at_high_mach(nx, ny, mach, T0, lattice):
    st = _fast_state(nx, ny, 100 * nx + ny, mach, T0, lattice)
    tl = bf.LATTICES[lattice][2]
    p = oracle.Params(fixed_iter=3, lattice=LAT[lattice], T_ref=tl)
    got, it, fl = oracle.step(st, p)
    assert np.all(it == 3) and np.all(fl == 0)
    fo, uxo, uyo, To = bf.step_mp(st.f, st.ux, st.uy, st.T, passes=3, T_ref=tl, lattice=lattice)
    speed = np.hypot(uxo, uyo).max()
    assert np.abs(got.f - fo).max() <= 1e-11 * np.abs(fo).max()
    assert np.abs(got.ux - uxo).max() <= 1e-12 * speed
    assert np.abs(got.uy - uyo).max() <= 1e-12 * speed
    assert np.max(np.abs(got.T - To) / To) <= 1e-11


def test_high_precision_bruteforce_agrees_with_fp64_bruteforce_at_low_mach():
    """The mpmath brute force is the FP64 brute force in more digits: where
    the FP64 solve is well conditioned (low Mach) the two agree."""
    st = _fast_state(2, 2, 5, 0.1, 1.0)
    a = bf.step(st.f, st.ux, st.uy, st.T, passes=2)
    b = bf.step_mp(st.f, st.ux, st.uy, st.T, passes=2)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() <= 1e-11 * np.abs(y).max()


def _gauge_near(rng, base, spread, T_L):
    """A gauge within `spread` thermal speeds and a factor 1.5 in T of base."""
    ux, uy, T = base
    c = np.sqrt(T / T_L)
    return (ux + spread * c * rng.uniform(-1, 1), uy + spread * c * rng.uniform(-1, 1),
            T * np.exp(rng.uniform(np.log(1 / 1.5), np.log(1.5))))


@pytest.mark.parametrize("lattice", ["d2q16", "d2q9"])
def test_transfer_composes_through_a_reference_gauge(lattice):
    """Eq. transform composes: the Q matched moments fix the Q populations,
    so moving f from gauge s to gauge t equals moving it to any third gauge r
    and then on to t.  With the linearity of Eq. interpolation this makes
    f_q = sum_s a_s [G(s -> t) f_s]_q = [G(r -> t) sum_s a_s G(s -> r) f_s]_q
    for each population q with its own weights a_s, the exact reformulation
    the staged kernel computes (sources moved once into a tile's reference
    gauge r).  Checked on the oracle's transfer for gauges spread as in a
    staged window (a few thermal speeds, T within a factor 1.5)."""
    lat = LAT[lattice]
    T_L = bf.LATTICES[lattice][2]
    n1 = 4 if lattice == "d2q16" else 3
    Q = n1 * n1
    rng = np.random.default_rng(11)
    for trial in range(20):
        t = (rng.uniform(-3, 3) * np.sqrt(T_L), rng.uniform(-3, 3) * np.sqrt(T_L),
             T_L * rng.uniform(0.5, 2.0))
        r = _gauge_near(rng, t, 2.0, T_L)
        s = _gauge_near(rng, t, 3.0, T_L)
        f = rng.uniform(0.1, 1.0, Q)
        direct = oracle.transfer(s, t, f, lat)
        via = oracle.transfer(r, t, oracle.transfer(s, r, f, lat), lat)
        assert np.abs(direct - via).max() <= 1e-11 * np.abs(direct).max(), trial

        # one target's reconstruction from a 4 x 4 stencil of sources
        src = [_gauge_near(rng, t, 1.0, T_L) for _ in range(16)]
        fs = [rng.uniform(0.1, 1.0, Q) for _ in range(16)]
        to_t = [oracle.transfer(g, t, fj, lat) for g, fj in zip(src, fs)]
        to_r = [oracle.transfer(g, r, fj, lat) for g, fj in zip(src, fs)]
        for q in range(Q):
            a = np.outer(oracle.interp_weights(rng.uniform(1, 2)),
                         oracle.interp_weights(rng.uniform(1, 2))).ravel()  # a_s of population q
            lhs = sum(a[j] * to_t[j][q] for j in range(16))
            rhs = oracle.transfer(r, t, sum(a[j] * to_r[j] for j in range(16)), lat)[q]
            scale = max(abs(lhs), np.abs(np.array(to_t)).max())
            assert abs(lhs - rhs) <= 1e-11 * scale, (trial, q)
