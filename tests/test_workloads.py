"""The seeded synthetic inputs match their stated recipe.

Every GPU parity case, physics test and bench line runs on these fields, so
their shapes, ranges and spectra are pinned here: the mode content of the
sinusoid sums, the supersonic base flow and its 0.1 perturbation, the
ratio-4 isobaric temperature of the precision workload, the Taylor-Green
field of App. D, the adjoint pulse and target, the isentropic vortex and the
256-grid ensemble.  All are deterministic.
"""
import numpy as np
import pytest

from paper_1806_05089_gb300 import workloads as wl


def test_sinusoid_sum_holds_only_the_stated_modes():
    n, kmax = 32, 3
    s = wl.sinusoids(n, n, wl.rng(99), modes=8, kmax=kmax)
    F = np.fft.fft2(s) / (n * n)
    ky, kx = np.nonzero(np.abs(F) > 1e-9)
    kx = np.where(kx > n // 2, kx - n, kx)
    ky = np.where(ky > n // 2, ky - n, ky)
    assert np.all(np.abs(kx) <= kmax) and np.all(np.abs(ky) <= kmax)
    assert np.all(np.maximum(np.abs(kx), np.abs(ky)) >= 1)   # no mean shift
    assert len(kx) <= 2 * 8                                    # each mode at +-k
    assert abs(s.mean()) < 1e-12
    assert np.abs(s).max() <= 8.0


def test_supersonic_field():
    f = wl.supersonic(nx=64, ny=48)
    assert f.shape == (48, 64)
    assert np.all(f.ux == 1.5) and np.all(f.uy == 0.5)       # (1.5, 0.5) sqrt(T) at T = 1
    for a in (f.rho, f.T):
        assert np.abs(a - 1.0).max() <= 0.1 + 1e-12          # total amplitude 0.1 over 8 modes
        assert abs(a.mean() - 1.0) < 1e-12
    g = wl.supersonic(nx=64, ny=48)
    assert np.array_equal(f.rho, g.rho) and np.array_equal(f.T, g.T)


def test_precision_field_is_isobaric_with_temperature_ratio_four():
    f = wl.precision(128)
    lt = np.log2(f.T)
    assert np.abs(lt).max() == pytest.approx(1.0, abs=1e-15)  # T = 2^s, max|s| = 1
    assert f.T.min() >= 0.5 - 1e-15 and f.T.max() <= 2.0 + 1e-15
    assert f.T.max() / f.T.min() >= 2.0                         # a ratio up to 4 across the field
    p = f.rho * f.T
    assert np.abs(p - 1.0).max() <= 0.1 + 1e-12                 # pressure carries the 0.1 modes


def test_taylor_green_field_is_app_d():
    n, u0 = 64, 0.05
    f = wl.taylor_green(n, n, u0)
    k = 2 * np.pi / n
    y, x = 5, 11
    assert f.ux[y, x] == pytest.approx(-(u0 / np.sqrt(2)) * np.cos(k * x) * np.sin(k * y), abs=1e-17)
    assert f.uy[y, x] == pytest.approx((u0 / np.sqrt(2)) * np.sin(k * x) * np.cos(k * y), abs=1e-17)
    assert np.mean(f.ux ** 2 + f.uy ** 2) == pytest.approx(u0 * u0 / 4, rel=1e-12)
    # divergence-free: spectral derivative of the periodic field
    kk = 2 * np.pi * np.fft.fftfreq(n)
    div = np.fft.ifft2(1j * kk[None, :] * np.fft.fft2(f.ux) + 1j * kk[:, None] * np.fft.fft2(f.uy))
    assert np.abs(div).max() < 1e-15
    assert np.all(f.rho == 1.0) and np.all(f.T == 1.0)


def test_adjoint_pulse_and_target():
    f, target = wl.adjoint(64)
    assert (f.rho - 1.0).max() == pytest.approx(0.2, abs=1e-15)   # Gaussian pulse peak at the centre
    assert f.rho[32, 32] == pytest.approx(1.2, abs=1e-15)
    assert f.rho[32, 32 + 16] - 1.0 == pytest.approx(0.2 * np.exp(-0.5), abs=1e-15)  # width 16
    assert np.abs(f.ux).max() == pytest.approx(0.3 / np.sqrt(2), rel=1e-2)           # TG u0 = 0.3
    assert np.abs(target - 1.0).max() <= 0.08


def test_isentropic_vortex():
    n, R, mv, ma = 96, 12.0, 0.8, 2.0
    f = wl.vortex(n, R, mv, ma)
    ratio = f.rho / f.T
    assert np.abs(ratio - ratio[0, 0]).max() < 1e-15                 # rho ~ T (gamma = 2)
    c = np.sqrt(2.0)
    assert f.T[n // 2, n // 2] == pytest.approx(1.0 - 0.5 * mv * mv * np.e, rel=1e-12)
    # swirl speed Ma_v c r e^{(1 - r^2)/2}: at r = 1 it is Ma_v c, on top of U = Ma_a c
    x = n // 2 + int(R)
    assert f.uy[n // 2, x] == pytest.approx(mv * c, rel=1e-12)
    assert f.ux[n // 2, x] == pytest.approx(ma * c, rel=1e-12)


def test_ensemble_recipe():
    nxs, nys = wl.ensemble_sizes(256)
    assert len(nxs) == len(nys) == 256
    assert min(nxs + nys) >= 32 and max(nxs + nys) <= 512
    assert (nxs, nys) == wl.ensemble_sizes(256)
    for i in (0, 17, 255):
        m = wl.ensemble_member(i, 40, 36)
        speed = np.hypot(m.ux, m.uy)
        assert np.ptp(speed) == 0.0 and speed.max() <= 3.0           # uniform Mach up to 3 at T = 1
        assert m.T.min() > 0 and m.T.max() / m.T.min() <= 4.0 + 1e-12
        assert min(abs(m.T.min() - 1.0), abs(m.T.max() - 1.0)) < 1e-12  # T spans [1, r] or [r, 1]
        assert np.abs(m.rho - 1.0).max() <= 0.1 + 1e-12
