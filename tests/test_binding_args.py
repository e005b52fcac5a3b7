"""Array checks of the binding's context calls, on the CPU.

The library takes raw pointers and trusts the sizes behind them, so the
binding checks every array against the handle ``pond_create`` returns (each
grid's size, the lattice's Q, the context's device) before the C call.  These
tests drive the checks with a handle whose pointer is NULL: an array the
binding rejects raises TypeError / ValueError, and arrays it accepts reach the
library, which answers POND_ERR_ARG for the NULL context without touching
them.  The device-side checks and the marshalling itself (which pointer
lands in which slot) are driven with tensors that report a CUDA device,
against a stand-in library that only records its calls.  So no test here
needs a GPU, and none can write through a pointer."""
import numpy as np
import pytest
import torch

from paper_1806_05089_gb300 import pond

NX, NY = 8, 6


def _handle(q=16, grids=((NX, NY),)):
    ctx = pond.PondCtx(None)
    ctx.grids = list(grids)
    ctx.q = q
    ctx.device = None
    return ctx


def _fields(ny=NY, nx=NX):
    return [np.ones((ny, nx)) for _ in range(4)]  # rho, ux, uy, T


def _reaches_library(call):
    """The binding accepted the arrays: the library refused the NULL context."""
    with pytest.raises(pond.PondError) as e:
        call()
    assert e.value.status == pond.POND_ERR_ARG


def test_valid_host_arrays_reach_the_library():
    ctx = _handle()
    rho, ux, uy, T = _fields()
    _reaches_library(lambda: pond.pond_set_state(ctx, 0, rho, ux, uy, T))
    f = np.ones((16, NY, NX))
    _reaches_library(lambda: pond.pond_set_state(ctx, 0, None, ux, uy, T, f))
    _reaches_library(lambda: pond.pond_moments(ctx, 0, np.zeros((NY, NX))))
    # flat arrays of the right length are accepted as well as (ny, nx) ones
    _reaches_library(lambda: pond.pond_get_state(ctx, 0, np.zeros(16 * NY * NX)))
    _reaches_library(lambda: pond.pond_iterations(ctx, 0, np.zeros((NY, NX), np.int32)))


def test_field_of_the_wrong_size_is_rejected():
    ctx = _handle()
    rho, ux, uy, T = _fields()
    with pytest.raises(ValueError, match="ux holds 42 values; the grid needs 48"):
        pond.pond_set_state(ctx, 0, rho, np.ones((6, 7)), uy, T)
    with pytest.raises(ValueError, match="T holds"):
        pond.pond_moments(ctx, 0, None, None, None, np.zeros((NY + 1, NX)))


def test_populations_of_another_lattice_are_rejected():
    rho, ux, uy, T = _fields()
    with pytest.raises(ValueError, match="f holds 432 values; the grid needs 768"):
        pond.pond_set_state(_handle(q=16), 0, None, ux, uy, T, np.ones((9, NY, NX)))
    with pytest.raises(ValueError, match="f holds 768 values; the grid needs 432"):
        pond.pond_get_state(_handle(q=9), 0, np.zeros((16, NY, NX)))


def test_each_grid_of_an_ensemble_has_its_own_size():
    ctx = _handle(grids=((NX, NY), (5, 3)))
    _reaches_library(lambda: pond.pond_moments(ctx, 1, np.zeros((3, 5))))
    with pytest.raises(ValueError, match="the grid needs 15"):
        pond.pond_moments(ctx, 1, np.zeros((NY, NX)))


def test_grid_index_out_of_range_is_left_to_the_library():
    ctx = _handle()
    _reaches_library(lambda: pond.pond_moments(ctx, 3, np.zeros((2, 2))))


def test_host_inputs_of_another_dtype_are_converted():
    """An int32 field is read as FP64 only after conversion (passing it as is
    would make the library read 4-byte integers as 8-byte doubles)."""
    ctx = _handle()
    rho, ux, uy, T = _fields()
    ptr, keep = pond._ptr(np.ones((NY, NX), np.int32), False, NX * NY, name="rho")
    assert keep.dtype == np.float64 and keep.size == NX * NY
    _reaches_library(lambda: pond.pond_set_state(ctx, 0, rho.astype(np.int32), ux, uy, T))


def test_host_outputs_must_be_filled_in_place():
    """A converted or contiguous copy of an output would be filled instead of
    the caller's array, so outputs of the wrong dtype or layout are refused."""
    ctx = _handle()
    with pytest.raises(TypeError, match="rho is an output"):
        pond.pond_moments(ctx, 0, np.zeros((NY, NX), np.float32))
    with pytest.raises(TypeError, match="ux is an output"):
        pond.pond_moments(ctx, 0, None, np.zeros((NX, NY)).T)
    ro = np.zeros((NY, NX))
    ro.flags.writeable = False
    with pytest.raises(TypeError, match="T is an output"):
        pond.pond_get_state(ctx, 0, None, None, None, ro)
    with pytest.raises(TypeError, match="iters is an output: it must be a writeable "
                                        "C-contiguous int32 array"):
        pond.pond_iterations(ctx, 0, np.zeros((NY, NX)))
    with pytest.raises(TypeError, match="rho is an output"):
        pond.pond_moments(ctx, 0, [[0.0] * NX] * NY)


def test_torch_tensors_keep_their_dtype_rule():
    ctx = _handle()
    rho, ux, uy, T = (torch.from_numpy(a) for a in _fields())
    with pytest.raises(TypeError, match="ux must be torch.float64"):
        pond.pond_set_state(ctx, 0, rho, ux.to(torch.int32), uy, T)
    with pytest.raises(TypeError, match="iters must be torch.int32"):
        pond.pond_iterations(ctx, 0, torch.zeros((NY, NX), dtype=torch.float64))
    with pytest.raises(ValueError, match="rho holds"):
        pond.pond_moments(ctx, 0, torch.zeros((NY, NX + 1), dtype=torch.float64))
    _reaches_library(lambda: pond.pond_set_state(ctx, 0, rho, ux, uy, T))


def test_adjoint_calls_take_device_tensors_only():
    ctx = _handle()
    f = torch.zeros((16, NY, NX), dtype=torch.float64)
    g = torch.zeros((3, NY, NX), dtype=torch.float64)
    with pytest.raises(ValueError, match="device call needs torch CUDA tensors"):
        pond.pond_adjoint_step(ctx, f, g, f.clone(), g.clone())
    with pytest.raises(ValueError, match="device call needs torch CUDA tensors"):
        pond.pond_adjoint_init(ctx, f, g[0])


def test_adjoint_array_counts():
    """Populations take Q values per node, gauge cotangents three, fields one."""
    assert pond._counts(_handle(q=9), 0, "q", 3, 1) == [9 * NX * NY, 3 * NX * NY, NX * NY]
    assert pond._counts(pond.PondCtx(None), 0, "q", 1) == [None, None]


def test_rectangle_buffer_follows_the_context_lattice():
    ctx = _handle(q=16)
    with pytest.raises(ValueError, match="q = 9, but the context's lattice has Q = 16"):
        pond._rect_buffer(ctx, None, 9, 4, 4)
    with pytest.raises(TypeError, match="CUDA float64"):
        pond._rect_buffer(ctx, torch.zeros(19 * 16, dtype=torch.float64), None, 4, 4)


def test_device_of_a_tensor_must_be_the_context_device():
    pond._check_device("f", 0, 0)
    with pytest.raises(ValueError, match="f is on cuda:1; the context's device is cuda:0"):
        pond._check_device("f", 1, 0)


class _ReportsCuda(torch.Tensor):
    """A CPU tensor that reports itself as a CUDA tensor on device 0, so the
    binding's device-side checks and marshalling run without a GPU."""

    @property
    def is_cuda(self):
        return True

    @property
    def device(self):
        return torch.device("cuda", 0)


def _cuda(shape, dtype=torch.float64):
    return torch.Tensor._make_subclass(_ReportsCuda, torch.zeros(shape, dtype=dtype))


def test_device_tensors_are_checked_and_marshalled(monkeypatch):
    """Context calls with (reported) CUDA tensors against a library that only
    records its calls: the handle from pond_create carries the grid, Q and
    device; the call patterns of the autograd rollout, the adjoint and the
    decomposition reach the library with each tensor's own data pointer and
    on_device = 1; wrong sizes, dtypes and lattices are refused first."""
    real = pond.load()
    calls = []

    class Recording:
        def __getattr__(self, name):
            if name in ("pond_config_default", "pond_version"):
                return getattr(real, name)

            def call(*args):
                calls.append((name, args))
                if name == "pond_create":
                    args[-1]._obj.value = 4096          # a handle nothing dereferences
                return b"" if name == "pond_last_error" else 0
            return call

    monkeypatch.setattr(pond, "_LIB", Recording())
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)

    def last(name):
        return [a for n, a in calls if n == name][-1]

    ny, nx = 16, 24
    with pond.Sim(nx, ny) as s, pond.Sim(8, 6, lattice=pond.POND_D2Q9) as s9:
        assert (s.ctx.grids, s.ctx.q, s.ctx.device) == ([(nx, ny)], 16, 0)
        assert (s9.ctx.grids, s9.ctx.q) == ([(8, 6)], 9)
        f = _cuda((16, ny, nx))
        ux, uy, T = (_cuda((ny, nx)) for _ in range(3))
        pond.pond_get_state(s.ctx, 0, f, ux, uy, T)
        args = last("pond_get_state")
        assert [a.value for a in args[2:6]] == [t.data_ptr() for t in (f, ux, uy, T)]
        assert args[6] == 1
        pond.pond_set_state(s.ctx, 0, None, ux, uy, T, f)          # the rollout's restore
        args = last("pond_set_state")
        assert args[2] is None and args[6].value == f.data_ptr() and args[7] == 1
        gbar = _cuda((3, ny, nx))
        pond.pond_adjoint_step_given(s.ctx, ux, uy, T, f, gbar, _cuda((16, ny, nx)),
                                     _cuda((3, ny, nx)), nu_on_device=True)
        assert last("pond_adjoint_step_given")[-1] is None        # the device accumulator
        pond.pond_adjoint_init(s.ctx, f, _cuda((ny, nx)))
        it = _cuda((ny, nx), torch.int32)
        pond.pond_iterations(s.ctx, 0, it)
        assert last("pond_iterations")[2].value == it.data_ptr()
        buf = _cuda(((16 + 3) * nx * ny,))
        pond.pond_pack_rect(s.ctx, 0, 0, 0, nx, ny, buf)
        pond.pond_set_state(s9.ctx, 0, None, *(_cuda((6, 8)) for _ in range(3)), _cuda((9, 6, 8)))

        n = len(calls)
        with pytest.raises(ValueError, match="gauge_bar_in holds 768 values; the grid needs 1152"):
            pond.pond_adjoint_step(s.ctx, f, _cuda((2, ny, nx)), _cuda((16, ny, nx)), gbar)
        with pytest.raises(ValueError, match="f holds 3456 values; the grid needs 6144"):
            pond.pond_get_state(s.ctx, 0, _cuda((9, ny, nx)))
        with pytest.raises(ValueError, match="f holds 768 values; the grid needs 432"):
            pond.pond_set_state(s9.ctx, 0, None, *(_cuda((6, 8)) for _ in range(3)),
                                _cuda((16, 6, 8)))
        with pytest.raises(TypeError, match="iters must be torch.int32"):
            pond.pond_iterations(s.ctx, 0, _cuda((ny, nx)))
        with pytest.raises(ValueError, match="q = 9, but the context's lattice has Q = 16"):
            pond.pond_unpack_rect(s.ctx, 0, 0, 0, nx, ny, buf, q=9)
        with pytest.raises(ValueError, match=r"device call needs torch CUDA tensors \(ux is not one\)"):
            pond.pond_moments(s.ctx, 0, _cuda((ny, nx)), np.zeros((ny, nx)))
        assert len(calls) == n                  # nothing refused reached the library
