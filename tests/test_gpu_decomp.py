"""GPU tests of the spatial domain decomposition, on one GPU: the blocks are
separate library contexts on the same device and the halo messages are
handed over in-process (LocalTransport), so every kernel, the interior
launch and the strip packing run as they would with one block per GPU;
only the transport differs (its NCCL/gloo form is tested on the CPU).

A split whose block origins fall on the staged kernel's tile grid runs the
same arithmetic on every node as the single-grid step and must match it bit
for bit; an unaligned split moves the tiles' reference gauges and matches to
rounding.
"""
import numpy as np
import pytest
import torch

from paper_1806_05089_gb300 import decomp, pond, workloads

pytestmark = pytest.mark.gpu


def single_grid(fields, steps, precision, tile_rows):
    ny, nx = fields.shape
    with pond.Sim(nx, ny, precision, kernel=pond.POND_KERNEL_STAGED, tile_rows=tile_rows) as s:
        s.set_state(fields.rho, fields.ux, fields.uy, fields.T)
        s.step(steps)
        st = s.state()
    return st.f, [st.ux, st.uy, st.T]


def split_run(fields, steps, precision, px, py, tile_rows, halo=None):
    ny, nx = fields.shape
    if halo is None:
        with pond.Sim(nx, ny, precision) as probe:
            probe.set_state(fields.rho, fields.ux, fields.uy, fields.T)
            halo = decomp.halo_width(pond.pond_max_displacement(probe.ctx) * 1.2)
    with decomp.DecomposedSim(nx, ny, px, py, halo, precision=precision,
                              tile_rows=tile_rows) as d:
        d.set_state(fields.rho, fields.ux, fields.uy, fields.T)
        stats = d.step(steps)
        f, g = d.gather_state()
    return f, g, stats


@pytest.mark.parametrize("precision", [pond.POND_FP64, pond.POND_FP32_MIXED])
@pytest.mark.parametrize("px,py", [(2, 1), (1, 2), (2, 2)])
def test_aligned_split_is_bit_identical_to_single_grid(precision, px, py):
    fields = workloads.supersonic(nx=128, ny=64)
    f1, g1 = single_grid(fields, 4, precision, 8)
    f2, g2, stats = split_run(fields, 4, precision, px, py, 8)
    assert np.array_equal(f1, f2)
    for a, b in zip(g1, g2):
        assert np.array_equal(a, b)
    # every block updated exactly its interior
    for per_step in stats:
        assert sum(s["node_updates"] for s in per_step.values()) == 128 * 64
        assert all(s["halo_fallback"] == 0 for s in per_step.values())


def test_unaligned_split_matches_to_rounding():
    fields = workloads.supersonic(nx=100, ny=70)
    f1, g1 = single_grid(fields, 3, pond.POND_FP64, 4)
    f2, g2, _ = split_run(fields, 3, pond.POND_FP64, 3, 2, 4)
    assert np.abs(f2 - f1).max() <= 1e-12 * np.abs(f1).max()
    for a, b in zip(g2, g1):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_rectangle_pack_unpack_round_trip_is_exact():
    fields = workloads.supersonic(nx=48, ny=40)
    for precision in (pond.POND_FP64, pond.POND_FP32_MIXED):
        with pond.Sim(48, 40, precision) as a, pond.Sim(48, 40, precision) as b:
            a.set_state(fields.rho, fields.ux, fields.uy, fields.T)
            a.step(2)
            b.set_state(fields.rho, 0.5 * fields.ux, fields.uy, fields.T)
            buf = torch.empty((a.Q + 3) * 48 * 40, dtype=torch.float64, device="cuda")
            pond.pond_pack_rect(a.ctx, 0, 0, 0, 48, 40, buf, q=a.Q)
            pond.pond_unpack_rect(b.ctx, 0, 0, 0, 48, 40, buf, q=a.Q)
            torch.cuda.synchronize()
            sa, sb = a.state(), b.state()
            assert np.array_equal(sa.f, sb.f)
            assert np.array_equal(sa.ux, sb.ux) and np.array_equal(sa.T, sb.T)


def test_halo_narrower_than_the_displacement_is_refused():
    fields = workloads.supersonic(nx=128, ny=64)
    with pytest.raises(RuntimeError, match="halo"):
        split_run(fields, 1, pond.POND_FP64, 2, 1, 8, halo=4)


def test_interior_needs_the_staged_kernel_and_a_rectangle_inside_the_grid():
    with pond.Sim(32, 16, pond.POND_FP64, kernel=pond.POND_KERNEL_DIRECT) as s:
        with pytest.raises(pond.PondError):
            pond.pond_set_interior(s.ctx, 0, 4, 4, 8, 8)
    with pond.Sim(32, 16, pond.POND_FP64) as s:
        with pytest.raises(pond.PondError):
            pond.pond_set_interior(s.ctx, 0, 30, 4, 8, 8)
