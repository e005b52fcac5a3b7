"""The binding's array checks with real CUDA tensors on a live context: the
handle from pond_create records the grid, Q and device, arrays of the wrong
size, dtype or lattice are refused before the library is called, and the
context stays usable.  (The same paths run on the CPU in
test_binding_args.py.)  The file sorts after the parity and physics files."""
import numpy as np
import pytest

from paper_1806_05089_gb300 import pond, workloads

pytestmark = pytest.mark.gpu


def test_context_calls_check_arrays_before_the_library():
    """The handle records the grid, Q and device; CUDA tensors of the wrong
    size, dtype or lattice are refused in the binding, and the context stays
    usable."""
    import torch
    fields = workloads.taylor_green(24, 16, 0.05)
    dev = torch.device("cuda")
    with pond.Sim(24, 16) as s:
        assert s.ctx.grids == [(24, 16)] and s.ctx.q == 16
        assert s.ctx.device == torch.cuda.current_device()
        s.set_state(fields.rho, fields.ux, fields.uy, fields.T)
        s.step(1)
        with pytest.raises(ValueError, match="the grid needs 384"):
            s.set_state(fields.rho[:8], fields.ux, fields.uy, fields.T)
        with pytest.raises(ValueError, match="f holds"):
            pond.pond_get_state(s.ctx, 0, torch.empty((9, 16, 24), dtype=torch.float64,
                                                      device=dev))
        with pytest.raises(TypeError, match="iters must be torch.int32"):
            pond.pond_iterations(s.ctx, 0, torch.empty((16, 24), dtype=torch.float64,
                                                       device=dev))
        fbar = torch.zeros((16, 16, 24), dtype=torch.float64, device=dev)
        with pytest.raises(ValueError, match="gauge_bar_in holds"):
            pond.pond_adjoint_step(s.ctx, fbar, torch.zeros((2, 16, 24), dtype=torch.float64,
                                                            device=dev),
                                   torch.empty_like(fbar),
                                   torch.empty((3, 16, 24), dtype=torch.float64, device=dev))
        f = torch.empty((16, 16, 24), dtype=torch.float64, device=dev)
        it = torch.empty((16, 24), dtype=torch.int32, device=dev)
        pond.pond_get_state(s.ctx, 0, f)
        pond.pond_iterations(s.ctx, 0, it)
        torch.cuda.synchronize()
        assert np.array_equal(f.cpu().numpy(), s.state().f)
        assert np.array_equal(it.cpu().numpy(), s.iterations())
        assert s.step(1)["nonphysical"] == 0
