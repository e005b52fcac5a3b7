"""The context-free FP64 step that allocates nothing (pond_step_fp64_noalloc).

Some callers cannot allocate device memory where they run the step: a host
callback, a custom allocator or memory pool, a framework that has already
reserved the device's memory, a real-time loop that must not enter the
allocator.  For them the library offers one FP64 step that works only on the
caller's own input and output arrays plus a fixed scratch array compiled into
the library.  This test drives it through the C ABI with device arrays owned
by the test, for two calls in a row (the second fed with the first call's
output, while the shared scratch still holds the first call's contents), and
checks each result against what the context-based entry points
(pond_create / pond_set_state / pond_step / pond_get_state) give for the same
steps, within the FP64 parity tolerance of the other GPU tests (1e-12).
"""
import numpy as np
import pytest
import torch

from paper_1806_05089_gb300 import pond, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-12


def test_noalloc_step_matches_context_step_on_two_calls():
    ny, nx = 40, 48
    fields = workloads.supersonic(nx=nx, ny=ny)
    with pond.Sim(nx, ny, pond.POND_FP64) as s:
        s.set_state(fields.rho, fields.ux, fields.uy, fields.T)
        start = s.state()
        refs = []
        for _ in range(2):
            stats = s.step(1)
            refs.append((s.state(), s.iterations(), stats))

    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    cfg = pond.pond_config_default(pond.POND_FP64)
    cur = [torch.tensor(a, device=dev) for a in (start.f, start.ux, start.uy, start.T)]
    for ref, ref_iters, ref_stats in refs:
        out = [torch.empty_like(a) for a in cur]
        iters = torch.zeros((ny, nx), dtype=torch.int32, device=dev)
        stats = pond.pond_step_fp64_noalloc(cfg, *cur, *out, iters=iters, stream=stream)
        torch.cuda.synchronize()
        f, ux, uy, T = (a.cpu().numpy() for a in out)
        assert np.abs(f - ref.f).max() <= TOL * np.abs(ref.f).max()
        umax = max(np.abs(ref.ux).max(), np.abs(ref.uy).max())
        assert np.abs(ux - ref.ux).max() <= TOL * umax
        assert np.abs(uy - ref.uy).max() <= TOL * umax
        assert np.max(np.abs(T - ref.T) / ref.T) <= TOL
        assert np.mean(iters.cpu().numpy() == ref_iters) >= 0.999
        assert stats["node_updates"] == nx * ny
        assert abs(stats["passes"] - ref_stats["passes"]) <= 0.001 * ref_stats["passes"]
        assert stats["nonphysical"] == 0
        cur = out


def test_noalloc_step_rejects_grids_above_its_scratch():
    dev = torch.device("cuda")
    ny, nx = 8, pond.POND_NOALLOC_MAX_NODES // 8 + 1
    cfg = pond.pond_config_default(pond.POND_FP64)
    f = torch.zeros((16, ny, nx), dtype=torch.float64, device=dev)
    g = [torch.ones((ny, nx), dtype=torch.float64, device=dev) for _ in range(3)]
    with pytest.raises(pond.PondError) as e:
        pond.pond_step_fp64_noalloc(cfg, f, *g, f.clone(), *[a.clone() for a in g])
    assert e.value.status == pond.POND_ERR_ARG
