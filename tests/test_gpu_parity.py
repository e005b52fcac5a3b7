"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances:
  FP64 step, fixed pass count: 1e-12 relative (rho, T per node; u relative to
    max|u|; f relative to max f).  With adaptive passes a node whose update
    lands within rounding of the App. E threshold may stop one pass earlier on
    one side; the two results then differ by about the threshold itself, so
    adaptive runs compare pass maps (equal at >= 99.9 % of nodes) and values
    at 1e-9.
  Mixed FP32/FP64 step: 1e-5 relative (FP32 populations; the convergence
    tolerance of that form is 1e-6); velocity errors against the larger of
    the flow speed and the thermal speed sqrt(T).
"""
import numpy as np
import pytest

import oracle
from paper_1806_05089_gb300 import pond, workloads

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def gpu_run(fields, steps, precision=pond.POND_FP64, f=None, **cfg):
    ny, nx = fields.shape
    with pond.Sim(nx, ny, precision, **cfg) as s:
        s.set_state(fields.rho, fields.ux, fields.uy, fields.T, f)
        stats = s.step(steps) if steps else None
        st = s.state()
        rho, ux, uy, T = s.moments()
        it = s.iterations()
    return st, rho, it, stats


def oracle_run(fields, steps, f=None, **params):
    st = oracle.init_equilibrium(fields.rho, fields.ux, fields.uy, fields.T)
    if f is not None:
        st.f = f.copy()
    p = oracle.Params(**params)
    it = None
    for _ in range(steps):
        st, it, fl = oracle.step(st, p)
        assert np.all(fl == 0)
    return st, it


def rel_errors(g, grho, o, speed_scale=False):
    """Relative errors of (rho, u, T, f).  rho and T per node; f against max f;
    u against max|u| -- or, with speed_scale, against the larger of max|u|
    and the thermal speed sqrt(T): FP32 rounding of the populations moves u by
    an amount set by the particle speeds, not by the flow speed alone."""
    orho = o.f.sum(axis=0)
    e_rho = np.max(np.abs(grho - orho) / np.abs(orho))
    umax = max(np.abs(o.ux).max(), np.abs(o.uy).max(), 1e-300)
    if speed_scale:
        umax = max(umax, float(np.sqrt(o.T.mean())))
    e_u = max(np.abs(g.ux - o.ux).max(), np.abs(g.uy - o.uy).max()) / umax
    e_T = np.max(np.abs(g.T - o.T) / np.abs(o.T))
    e_f = np.abs(g.f - o.f).max() / np.abs(o.f).max()
    return e_rho, e_u, e_T, e_f


def small_fields(name, nx, ny):
    if name == "tg":
        return workloads.taylor_green(nx, ny, 0.05)
    if name == "supersonic":
        return workloads.supersonic(nx=nx, ny=ny)
    if name == "hot":
        f = workloads.supersonic(nx=nx, ny=ny)
        f.T = 1.0 + 0.5 * (f.T - 1.0) / np.abs(f.T - 1.0).max()
        f.ux = -0.7 * f.ux
        return f
    raise KeyError(name)


# ------------------------------------------------------------------ FP64

# FP64 kernels: the direct per-pair kernel in its three mappings (one and two
# nodes per warp, one node per thread) and the reference-gauge staged tile
# kernel (the default) with both tile shapes
FP64_KERNELS = {
    "direct_npw1": {"kernel": pond.POND_KERNEL_DIRECT, "nodes_per_warp": 1},
    "direct_npw2": {"kernel": pond.POND_KERNEL_DIRECT, "nodes_per_warp": 2},
    "direct_node": {"kernel": pond.POND_KERNEL_DIRECT, "nodes_per_warp": 32},
    "staged_32x4": {"kernel": pond.POND_KERNEL_STAGED, "tile_rows": 4},
    "staged_32x8": {"kernel": pond.POND_KERNEL_STAGED, "tile_rows": 8},
}


@pytest.mark.parametrize("kern", list(FP64_KERNELS))
@pytest.mark.parametrize("name,nx,ny,steps", [("tg", 64, 64, 12), ("supersonic", 37, 29, 6),
                                              ("hot", 48, 40, 5), ("supersonic", 1, 1, 3),
                                              ("tg", 3, 5, 4), ("supersonic", 2, 7, 3)])
def test_fp64_fixed_passes_matches_oracle(name, nx, ny, steps, kern):
    fields = small_fields(name, nx, ny)
    g, grho, git, _ = gpu_run(fields, steps, fixed_iter=4, **FP64_KERNELS[kern])
    o, oit = oracle_run(fields, steps, fixed_iter=4)
    assert np.all(git == 4) and np.all(oit == 4)
    e = rel_errors(g, grho, o)
    assert max(e) <= TOL64, e


@pytest.mark.parametrize("kern", list(FP64_KERNELS))
def test_fp64_taylor_green_full_config_adaptive(kern):
    """64^2 Taylor-Green, u0 = 0.05, nu = 0.01, 100 steps, adaptive passes,
    every FP64 kernel."""
    fields = workloads.tg64()
    g, grho, git, stats = gpu_run(fields, 100, **FP64_KERNELS[kern])
    o, oit = oracle_run(fields, 100)
    assert stats["nonconverged"] == 0 and stats["nonphysical"] == 0
    assert np.mean(git == oit) >= 0.999
    e = rel_errors(g, grho, o)
    assert max(e) <= 1e-9, e


@pytest.mark.parametrize("kern", list(FP64_KERNELS))
def test_fp64_supersonic_adaptive_pass_map(kern):
    # 63 x 47: an odd node count leaves the last warp of the two-node mapping
    # with one node, the last block of the node-per-thread mapping part
    # filled, and the last tiles of the staged kernel ragged in x and y
    fields = small_fields("supersonic", 63, 47)
    g, grho, git, stats = gpu_run(fields, 4, **FP64_KERNELS[kern])
    o, oit = oracle_run(fields, 4)
    assert np.mean(git == oit) >= 0.999
    assert max(rel_errors(g, grho, o)) <= 1e-9


@pytest.mark.parametrize("seed_mode", [1, 2])
def test_fp64_seed_modes_match_oracle(seed_mode):
    fields = small_fields("supersonic", 24, 20)
    fields.ux = 0.3 * fields.ux
    fields.uy = 0.3 * fields.uy
    g, grho, git, _ = gpu_run(fields, 2, seed_mode=seed_mode, fixed_iter=30)
    o, _ = oracle_run(fields, 2, seed_mode=seed_mode, fixed_iter=30)
    assert max(rel_errors(g, grho, o)) <= 1e-11


@pytest.mark.parametrize("mach,T", [(100.0, 1.0), (3.0, 100.0), (10.0, 0.01)])
def test_fp64_uniform_state_fixed_point(mach, T):
    n = 16
    f = workloads.Fields(np.full((n, n), 1.1), np.full((n, n), mach * np.sqrt(T) * 0.8),
                         np.full((n, n), mach * np.sqrt(T) * 0.6), np.full((n, n), T))
    g, grho, git, stats = gpu_run(f, 20)
    assert np.all(git == 1) and stats["max_passes"] == 1
    speed = mach * np.sqrt(T) + np.sqrt(T)
    assert np.abs(grho - 1.1).max() <= 1e-13
    assert np.abs(g.ux - f.ux).max() <= 1e-13 * speed
    assert np.abs(g.uy - f.uy).max() <= 1e-13 * speed
    assert np.abs(g.T - T).max() <= 1e-13 * T


@pytest.mark.parametrize("fixed", [4, 0])
def test_fp64_full_size_sampled_rows(fixed):
    """2048^2 supersonic field (the at-scale FP64 workload), one step in the
    benchmark's launch configuration; oracle recomputes sampled rows."""
    fields = workloads.supersonic(2048)
    g, grho, git, stats = gpu_run(fields, 1, fixed_iter=fixed)
    st0 = oracle.init_equilibrium(fields.rho, fields.ux, fields.uy, fields.T)
    for r0 in (0, 777, 2047):
        o, oit, fl = oracle.step(st0, oracle.Params(fixed_iter=fixed), rows=(r0, r0 + 1))
        sl = slice(r0, r0 + 1)
        orho = o.f[:, sl].sum(axis=0)
        tol = TOL64 if fixed else 1e-9
        assert np.max(np.abs(grho[sl] - orho) / orho) <= tol
        assert np.max(np.abs(g.T[sl] - o.T[sl]) / o.T[sl]) <= tol
        assert np.abs(g.ux[sl] - o.ux[sl]).max() <= tol * 1.6
        assert np.abs(g.f[:, sl] - o.f[:, sl]).max() <= tol * np.abs(o.f[:, sl]).max()
        if not fixed:
            assert np.mean(git[sl] == oit[sl]) >= 0.99


def test_state_round_trip_is_bit_exact():
    fields = small_fields("supersonic", 19, 11)
    rng = np.random.default_rng(0)
    f = rng.random((16, 11, 19)) + 0.01
    with pond.Sim(19, 11) as s:
        s.set_state(None, fields.ux, fields.uy, fields.T, f)
        st = s.state()
    assert np.array_equal(st.f, f)
    assert np.array_equal(st.ux, fields.ux) and np.array_equal(st.uy, fields.uy)
    assert np.abs(st.T - fields.T).max() <= 4e-16 * fields.T.max()


def test_device_pointers_through_torch():
    torch = pytest.importorskip("torch")
    fields = small_fields("tg", 32, 32)
    dev = [torch.tensor(a, device="cuda") for a in (fields.rho, fields.ux, fields.uy, fields.T)]
    with pond.Sim(32, 32, stream=torch.cuda.current_stream().cuda_stream) as s:
        s.set_state(*dev)
        s.step(3)
        out = [torch.empty((32, 32), dtype=torch.float64, device="cuda") for _ in range(4)]
        pond.pond_moments(s.ctx, 0, *out)
        torch.cuda.synchronize()
        host = s.moments()
    for a, b in zip(out, host):
        assert np.array_equal(a.cpu().numpy(), b)


def test_errors_are_reported_not_trapped():
    fields = small_fields("tg", 8, 8)
    with pond.Sim(8, 8) as s:
        with pytest.raises(pond.PondError) as e:
            s.step(1)
        assert e.value.status == pond.POND_ERR_STATE
        bad = fields.T.copy()
        bad[2, 3] = -1.0
        with pytest.raises(pond.PondError) as e:
            s.set_state(fields.rho, fields.ux, fields.uy, bad)
        assert e.value.status == pond.POND_ERR_NONPHYSICAL
        # negative populations: the moments give rho < 0 -> counted, reported
        f = -np.ones((16, 8, 8))
        s.set_state(None, fields.ux, fields.uy, fields.T, f)
        with pytest.raises(pond.PondError) as e:
            s.step(1)
        assert e.value.status == pond.POND_ERR_NONPHYSICAL
        # the context stays usable
        s.set_state(fields.rho, fields.ux, fields.uy, fields.T)
        assert s.step(1)["nonphysical"] == 0


@pytest.mark.parametrize("on_device", [False, True])
def test_set_state_refuses_bad_gauges(on_device):
    """T <= 0 or a non-finite gauge at any node is refused (checked on the
    device in the set_state bounds pass, for host and device input); the
    refused grid takes no step until a valid set_state."""
    import torch
    fields = small_fields("tg", 24, 16)
    dev = torch.device("cuda")

    def side(a):
        return torch.tensor(a, device=dev) if on_device else a

    cases = [("T", 0.0), ("T", -2.0), ("T", np.nan), ("ux", np.inf), ("uy", np.nan)]
    with pond.Sim(24, 16) as s:
        for name, v in cases:
            s.set_state(side(fields.rho), side(fields.ux), side(fields.uy), side(fields.T))
            s.step(1)
            arrs = {"ux": fields.ux.copy(), "uy": fields.uy.copy(), "T": fields.T.copy()}
            arrs[name][7, 13] = v
            with pytest.raises(pond.PondError) as e:
                s.set_state(side(fields.rho), side(arrs["ux"]), side(arrs["uy"]), side(arrs["T"]))
            assert e.value.status == pond.POND_ERR_NONPHYSICAL, (name, v)
            with pytest.raises(pond.PondError) as e:
                s.step(1)
            assert e.value.status == pond.POND_ERR_STATE, (name, v)
        s.set_state(side(fields.rho), side(fields.ux), side(fields.uy), side(fields.T))
        assert s.step(1)["nonphysical"] == 0


def test_strict_mode_reports_nonconvergence():
    fields = small_fields("supersonic", 16, 16)
    with pond.Sim(16, 16, max_iter=1, strict=1) as s:
        s.set_state(fields.rho, fields.ux, fields.uy, fields.T)
        with pytest.raises(pond.PondError) as e:
            s.step(1)
        assert e.value.status == pond.POND_ERR_NOT_CONVERGED


# ------------------------------------------------------------------ mixed

MIXED_KERNELS = [(pond.POND_KERNEL_STAGED, 4), (pond.POND_KERNEL_STAGED, 8),
                 (pond.POND_KERNEL_STAGED, 16), (pond.POND_KERNEL_DIRECT, 4),
                 (pond.POND_KERNEL_DIRECT, 8), (pond.POND_KERNEL_DIRECT, 16),
                 (pond.POND_KERNEL_DIRECT, -16)]


@pytest.mark.parametrize("kernel,tile_rows", MIXED_KERNELS)
@pytest.mark.parametrize("name,nx,ny,steps", [("tg", 64, 64, 20), ("supersonic", 70, 45, 8),
                                              ("hot", 40, 33, 6), ("supersonic", 5, 3, 3),
                                              ("tg", 1, 1, 2)])
def test_mixed_matches_oracle(name, nx, ny, steps, kernel, tile_rows):
    fields = small_fields(name, nx, ny)
    g, grho, git, stats = gpu_run(fields, steps, pond.POND_FP32_MIXED, tile_rows=tile_rows,
                                  kernel=kernel)
    assert stats["tile_rows"] == tile_rows
    o, _ = oracle_run(fields, steps)
    assert stats["nonconverged"] == 0
    e = rel_errors(g, grho, o, speed_scale=True)
    assert max(e[:3]) <= TOL32, e


def test_mixed_halo_fallback_path():
    """Seed {-u, T}: the staged window is planned around the wrong
    departures, so stencils fall back to global reads; results still match."""
    fields = small_fields("supersonic", 64, 24)
    g, grho, git, stats = gpu_run(fields, 2, pond.POND_FP32_MIXED, seed_mode=2, max_iter=40)
    assert stats["halo_fallback"] > 0
    o, _ = oracle_run(fields, 2, seed_mode=2, max_iter=40)
    assert max(rel_errors(g, grho, o, speed_scale=True)[:3]) <= TOL32


@pytest.mark.parametrize("kernel,tile_rows", [(pond.POND_KERNEL_STAGED, 8),
                                              (pond.POND_KERNEL_STAGED, 16),
                                              (pond.POND_KERNEL_DIRECT, 8),
                                              (pond.POND_KERNEL_DIRECT, -16)])
def test_batched_matches_single_grid_runs(kernel, tile_rows):
    sizes = [(37, 23), (64, 40), (33, 70), (32, 32), (50, 45), (96, 17), (1, 1), (5, 9)]
    members = [workloads.ensemble_member(i, nx, ny) for i, (nx, ny) in enumerate(sizes)]
    nxs = [s[0] for s in sizes]
    nys = [s[1] for s in sizes]
    with pond.Sim(nxs, nys, pond.POND_FP32_MIXED, tile_rows=tile_rows, kernel=kernel) as b:
        for i, m in enumerate(members):
            b.set_state(m.rho, m.ux, m.uy, m.T, grid=i)
        b.step(3)
        batched = [b.state(i) for i in range(len(sizes))]
    for i, m in enumerate(members):
        with pond.Sim(nxs[i], nys[i], pond.POND_FP32_MIXED, tile_rows=tile_rows,
                      kernel=kernel) as s:
            s.set_state(m.rho, m.ux, m.uy, m.T)
            s.step(3)
            single = s.state()
        assert np.array_equal(batched[i].f, single.f), i
        assert np.array_equal(batched[i].ux, single.ux), i
        if min(nxs[i], nys[i]) < 16:
            continue  # wavenumber-2 modes are not resolved on so few cells
        o, _ = oracle_run(m, 3, max_iter=60)
        assert np.max(np.abs(batched[i].T - o.T) / o.T) <= TOL32
        assert np.max(np.abs(batched[i].f.sum(0) - o.f.sum(0)) / o.f.sum(0)) <= TOL32


@pytest.mark.parametrize("tile_rows", [4, 8])
def test_fp64_batched_matches_single_grid_runs(tile_rows):
    """FP64 ensembles on the staged kernel's persistent work list: every
    grid bit-identical to its own single-grid run (which the FP64 parity
    tests pin to the oracle)."""
    sizes = [(37, 23), (64, 40), (33, 70), (1, 1), (50, 45), (5, 9)]
    members = [workloads.ensemble_member(i, nx, ny) for i, (nx, ny) in enumerate(sizes)]
    nxs = [s[0] for s in sizes]
    nys = [s[1] for s in sizes]
    with pond.Sim(nxs, nys, pond.POND_FP64, tile_rows=tile_rows) as b:
        for i, m in enumerate(members):
            b.set_state(m.rho, m.ux, m.uy, m.T, grid=i)
        st = b.step(2)
        batched = [b.state(i) for i in range(len(sizes))]
    assert st["nonphysical"] == 0
    for i, m in enumerate(members):
        with pond.Sim(nxs[i], nys[i], pond.POND_FP64, tile_rows=tile_rows) as s:
            s.set_state(m.rho, m.ux, m.uy, m.T)
            s.step(2)
            single = s.state()
        assert np.array_equal(batched[i].f, single.f), i
        assert np.array_equal(batched[i].ux, single.ux), i
        assert np.array_equal(batched[i].T, single.T), i


def test_graph_replay_matches_plain_launches():
    fields = small_fields("supersonic", 80, 40)
    out = []
    for use_graph in (0, 1):
        with pond.Sim(80, 40, pond.POND_FP32_MIXED, use_graph=use_graph) as s:
            s.set_state(fields.rho, fields.ux, fields.uy, fields.T)
            s.step(5)
            out.append(s.state())
    assert np.array_equal(out[0].f, out[1].f)
    assert np.array_equal(out[0].T, out[1].T)


def test_stream_switch_keeps_results():
    """pond_set_stream between graph-replayed steps: the steps queued on the
    first stream finish first and the graphs are captured again, so the run
    equals one that stays on a single stream."""
    import torch
    fields = small_fields("supersonic", 80, 40)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    out = []
    for switch in (False, True):
        with pond.Sim(80, 40, pond.POND_FP32_MIXED, stream=s1.cuda_stream, use_graph=1) as s:
            s.set_state(fields.rho, fields.ux, fields.uy, fields.T)
            pond.pond_step(s.ctx, 4, want_stats=False)
            if switch:
                pond.pond_set_stream(s.ctx, s2.cuda_stream)
            pond.pond_step(s.ctx, 4, want_stats=False)
            out.append(s.state())
    assert np.array_equal(out[0].f, out[1].f)
    assert np.array_equal(out[0].ux, out[1].ux)


def test_autotune_picks_a_tile_shape_and_matches_oracle(tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("POND_AUTOTUNE_CACHE", str(cache))
    sizes = [(70, 45), (33, 90), (128, 40)]
    members = [workloads.ensemble_member(10 + i, nx, ny) for i, (nx, ny) in enumerate(sizes)]
    nxs = [s[0] for s in sizes]
    nys = [s[1] for s in sizes]
    with pond.Sim(nxs, nys, pond.POND_FP32_MIXED, autotune=1) as b:
        for i, m in enumerate(members):
            b.set_state(m.rho, m.ux, m.uy, m.T, grid=i)
        stats = b.step(3)
        out = [b.state(i) for i in range(len(sizes))]
    assert stats["tile_rows"] in (4, 8, 16, -16)
    for i, m in enumerate(members):
        o, _ = oracle_run(m, 3, max_iter=60)
        assert np.max(np.abs(out[i].T - o.T) / o.T) <= TOL32
        assert np.max(np.abs(out[i].f.sum(0) - o.f.sum(0)) / o.f.sum(0)) <= TOL32
    import json
    saved = json.load(open(cache))
    assert stats["tile_rows"] in saved.values()
