"""Argument checks of the binding of pond_step_fp64_noalloc, on the CPU.

The C entry point has no context that knows the grid, so it trusts the
caller's pointers; the Python binding checks shapes, dtypes and the device
before calling it.  Every rejection here happens before any GPU work, so the
checks run without a GPU (CPU tensors of the right shape fail last, on the
device check)."""
import pytest
import torch

from paper_1806_05089_gb300 import pond


def _args(Q=16, ny=6, nx=8, dtype=torch.float64, idtype=torch.int32):
    f = torch.zeros((Q, ny, nx), dtype=dtype)
    g = [torch.ones((ny, nx), dtype=dtype) for _ in range(3)]
    return [f, *g, f.clone(), *[a.clone() for a in g]], torch.zeros((ny, nx), dtype=idtype)


def _call(cfg, arrays, iters):
    pond.pond_step_fp64_noalloc(cfg, *arrays, iters=iters)


def test_d2q9_populations_with_a_d2q16_config_are_rejected():
    cfg = pond.pond_config_default(pond.POND_FP64)
    arrays, iters = _args(Q=9)
    with pytest.raises(ValueError, match="shape"):
        _call(cfg, arrays, iters)
    cfg.lattice = pond.POND_D2Q9
    arrays, iters = _args(Q=16)
    with pytest.raises(ValueError, match="shape"):
        _call(cfg, arrays, iters)


def test_wrong_dtypes_are_rejected():
    cfg = pond.pond_config_default(pond.POND_FP64)
    arrays, iters = _args()
    arrays[0] = arrays[0].to(torch.int32)
    with pytest.raises(TypeError, match="f_in"):
        _call(cfg, arrays, iters)
    arrays, iters = _args(dtype=torch.float32)
    with pytest.raises(TypeError):
        _call(cfg, arrays, iters)
    arrays, iters = _args(idtype=torch.int64)
    with pytest.raises(TypeError, match="iters"):
        _call(cfg, arrays, iters)


def test_mismatched_gauge_and_output_shapes_are_rejected():
    cfg = pond.pond_config_default(pond.POND_FP64)
    for i in (2, 3, 4, 5, 6, 7):
        arrays, iters = _args()
        arrays[i] = arrays[i][..., :-1].contiguous()
        with pytest.raises(ValueError, match="shape"):
            _call(cfg, arrays, iters)
    arrays, iters = _args()
    with pytest.raises(ValueError, match="iters"):
        _call(cfg, arrays, iters[:, :-1].contiguous())


def test_non_contiguous_and_host_tensors_are_rejected():
    cfg = pond.pond_config_default(pond.POND_FP64)
    arrays, iters = _args()
    arrays[1] = torch.ones((8, 6), dtype=torch.float64).t()
    with pytest.raises(ValueError, match="contiguous"):
        _call(cfg, arrays, iters)
    arrays, iters = _args()
    with pytest.raises(ValueError, match="CUDA"):
        _call(cfg, arrays, iters)
    with pytest.raises(ValueError, match="CUDA"):
        _call(cfg, arrays, None)
