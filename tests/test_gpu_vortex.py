"""Isentropic vortex on the GPU (main text, vortex benchmark; App. E).

- A standing vortex (Ma_v = 0.8) needs only a few predictor-corrector passes,
  with the most where the flow changes fastest (App. E, the iteration-map
  figure; App. E reports three on average and five at most for D2Q9).
- Advected through the periodic box at Ma_a up to about 10, the vortex keeps
  its shape: after whole box traversals its pressure field matches the vortex
  at rest after the same number of steps (no deformation with the flow speed,
  the method's Galilean invariance at high Mach).
"""
import numpy as np
import pytest

from paper_1806_05089_gb300 import pond, workloads

pytestmark = pytest.mark.gpu


def test_standing_vortex_iteration_map():
    n, R = 128, 16.0
    f = workloads.vortex(n, R, 0.8, 0.0)
    with pond.Sim(n, n, pond.POND_FP64, nu=0.01) as s:
        s.set_state(f.rho, f.ux, f.uy, f.T)
        s.step(10)
        stats = s.step(10)
        it = s.iterations()
    # every node converges well inside max_iter; the D2Q16 step needs about
    # one pass more than the paper's D2Q9 figure (4 on average, up to ~12 in
    # the core while the start-up transient lasts)
    assert stats["nonconverged"] == 0 and stats["nonphysical"] == 0
    assert it.max() <= 12
    assert it.mean() <= 5.0
    X, Y = np.meshgrid(np.arange(n), np.arange(n))
    r = np.hypot(X - n / 2, Y - n / 2) / R
    assert it[r < 1.5].mean() >= it[r > 3.0].mean()


@pytest.mark.parametrize("traversals,steps", [(1, 113), (5, 57)])
def test_advected_vortex_keeps_its_shape(traversals, steps):
    n, R, mach_v = 160, 16.0, 0.5
    U = traversals * n / steps                       # whole box traversals in `steps`
    mach_a = U / np.sqrt(2.0)
    rest = workloads.vortex(n, R, mach_v, 0.0)
    moving = workloads.vortex(n, R, mach_v, mach_a)
    out = []
    for f in (rest, moving):
        with pond.Sim(n, n, pond.POND_FP64, nu=0.01) as s:
            s.set_state(f.rho, f.ux, f.uy, f.T)
            stats = s.step(steps)
            assert stats["nonconverged"] == 0 and stats["nonphysical"] == 0
            rho, ux, uy, T = s.moments()
            out.append((rho * T, ux, uy))
    p_rest, p_mov = out[0][0], out[1][0]
    depth = 1.0 - (rest.rho * rest.T).min()
    assert np.abs(p_mov - p_rest).max() <= 0.02 * depth, (mach_a, np.abs(p_mov - p_rest).max() / depth)
    # the swirl is unchanged too (velocity relative to the flow)
    du = np.hypot(out[1][1] - U - out[0][1], out[1][2] - out[0][2]).max()
    assert du <= 0.02 * mach_v * np.sqrt(2.0)


def _vortex64(mach_a=1.0, mach_v=0.5):
    # diagonal advection, so both departure directions carry the flow
    return workloads.vortex(64, 8.0, mach_v, mach_a, angle=0.6)


@pytest.mark.parametrize("kernel", [pond.POND_KERNEL_STAGED, pond.POND_KERNEL_DIRECT])
def test_vortex_fp64_matches_oracle(kernel):
    """64^2 advected vortex (Ma_a 1, Ma_v 0.5), 3 steps with 4 passes each:
    the GPU FP64 step against the FP64 CPU oracle at 1e-12."""
    import oracle
    f = _vortex64()
    cfg = {"kernel": kernel}
    if kernel == pond.POND_KERNEL_DIRECT:
        cfg["nodes_per_warp"] = 32
    with pond.Sim(64, 64, pond.POND_FP64, fixed_iter=4, **cfg) as s:
        s.set_state(f.rho, f.ux, f.uy, f.T)
        s.step(3)
        g = s.state()
        rho = g.f.sum(axis=0)
    st = oracle.init_equilibrium(f.rho, f.ux, f.uy, f.T)
    for _ in range(3):
        st, it, fl = oracle.step(st, oracle.Params(fixed_iter=4))
        assert not fl.any()
    orho = st.f.sum(axis=0)
    umax = np.hypot(st.ux, st.uy).max()
    assert np.max(np.abs(rho - orho) / orho) <= 1e-12
    assert np.max(np.abs(g.T - st.T) / st.T) <= 1e-12
    assert max(np.abs(g.ux - st.ux).max(), np.abs(g.uy - st.uy).max()) <= 1e-12 * umax
    assert np.abs(g.f - st.f).max() <= 1e-12 * np.abs(st.f).max()


@pytest.mark.parametrize("kernel", [pond.POND_KERNEL_STAGED, pond.POND_KERNEL_DIRECT])
def test_vortex_mixed_matches_oracle(kernel):
    """The same vortex in the mixed form with adaptive passes, 6 steps,
    against the oracle at the mixed form's 1e-5."""
    import oracle
    f = _vortex64()
    with pond.Sim(64, 64, pond.POND_FP32_MIXED, kernel=kernel) as s:
        s.set_state(f.rho, f.ux, f.uy, f.T)
        stats = s.step(6)
        rho, ux, uy, T = s.moments()
    assert stats["nonconverged"] == 0
    st = oracle.init_equilibrium(f.rho, f.ux, f.uy, f.T)
    for _ in range(6):
        st, it, fl = oracle.step(st)
    orho = st.f.sum(axis=0)
    speed = max(np.hypot(st.ux, st.uy).max(), np.sqrt(st.T.mean()))
    assert np.max(np.abs(rho - orho) / orho) <= 1e-5
    assert np.max(np.abs(T - st.T) / st.T) <= 1e-5
    assert max(np.abs(ux - st.ux).max(), np.abs(uy - st.uy).max()) <= 1e-5 * speed


@pytest.mark.parametrize("kernel", [pond.POND_KERNEL_STAGED, pond.POND_KERNEL_DIRECT])
def test_vortex_mixed_halo_fallback_run_matches_fp64(kernel):
    """An advected vortex (Ma_a 1.2, |u| about 1.7) seeded with {-u, T}: every
    tile plans its staged window around departures 2|u| dt on the wrong
    side, so stencils leave the window and take the global-memory path
    (halo_fallback > 0).  The mixed run still matches the FP64 run of the
    same steps to the mixed form's 1e-5.  (At Ma_a 3 that seed is so far
    from the fixed point that the first pass's moments are non-physical, in
    FP64 as well: the seed-independence the paper reports holds near the
    limit, not from any seed.)"""
    f = _vortex64(mach_a=1.2)
    out = {}
    for prec in (pond.POND_FP64, pond.POND_FP32_MIXED):
        with pond.Sim(64, 64, prec, seed_mode=2, max_iter=60, kernel=kernel) as s:
            s.set_state(f.rho, f.ux, f.uy, f.T)
            stats = s.step(2)
            out[prec] = (s.moments(), stats)
    (r64, x64, y64, t64), s64 = out[pond.POND_FP64]
    (r32, x32, y32, t32), s32 = out[pond.POND_FP32_MIXED]
    assert s32["halo_fallback"] > 0
    assert s32["nonconverged"] == 0 and s64["nonconverged"] == 0
    speed = max(np.hypot(x64, y64).max(), np.sqrt(t64.mean()))
    assert np.max(np.abs(r32 - r64) / r64) <= 1e-5
    assert np.max(np.abs(t32 - t64) / t64) <= 1e-5
    assert max(np.abs(x32 - x64).max(), np.abs(y32 - y64).max()) <= 1e-5 * speed
