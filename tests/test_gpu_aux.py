"""GPU tests of the failure paths that need no GPU fault: a device
allocation larger than the GPU's memory is refused with POND_ERR_OOM by
pond_create (the CUDA allocator's own refusal, provoked on the host side by
the size asked for), partial allocations are released, and the process
stays usable for the next context."""
import numpy as np
import pytest
import torch

from paper_1806_05089_gb300 import pond, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [pond.POND_FP64, pond.POND_FP32_MIXED])
def test_create_larger_than_device_memory_reports_oom(precision):
    free, total = torch.cuda.mem_get_info()
    # populations alone: 2 buffers x 16 x nodes x (8 or 4) bytes > 4 x total
    side = int(np.sqrt(4 * total / (2 * 16 * 4))) + 1
    with pytest.raises(pond.PondError) as e:
        pond.Sim(side, side, precision)
    assert e.value.status == pond.POND_ERR_OOM
    # nothing leaked: the free memory is back where it was (within the
    # allocator's granularity), and a normal context still works
    free2, _ = torch.cuda.mem_get_info()
    assert free2 >= free - (64 << 20)
    f = workloads.supersonic(nx=32, ny=24)
    with pond.Sim(32, 24, precision) as s:
        s.set_state(f.rho, f.ux, f.uy, f.T)
        st = s.step(2)
    assert st["nonphysical"] == 0 and st["node_updates"] == 2 * 32 * 24


@pytest.mark.parametrize("precision", [pond.POND_FP64, pond.POND_FP32_MIXED])
def test_persistent_launch_idle_accounting(precision):
    """The batched (persistent) staged launches report their CTA busy time
    and CTA-slot time; busy never exceeds the slots, both grow with the
    number of steps, and single-grid contexts report neither."""
    nxs, nys = workloads.ensemble_sizes(12, 32, 96)
    mem = workloads.ensemble(12, 32, 96)
    with pond.Sim(nxs, nys, precision) as s:
        for i, m in enumerate(mem):
            s.set_state(m.rho, m.ux, m.uy, m.T, grid=i)
        st1 = s.step(1)
        st3 = s.step(3)
    for st in (st1, st3):
        assert 0 < st["busy_ns"] <= st["slot_ns"]
    assert st3["busy_ns"] > st1["busy_ns"] and st3["slot_ns"] > st1["slot_ns"]
    f = workloads.supersonic(nx=64, ny=40)
    with pond.Sim(64, 40, precision) as s:
        s.set_state(f.rho, f.ux, f.uy, f.T)
        st = s.step(2)
    assert st["busy_ns"] == 0 and st["slot_ns"] == 0
