"""Adjoint of the PonD step.

CPU: the plain-PyTorch reference step (oracle/torch_ref.py) matches the C
oracle, and its autograd gradient matches central finite differences of the
C oracle -- this pins the reference gradient.
GPU: the CUDA adjoint (pond_adjoint_step through PondRollout) matches the
reference gradient, and central finite differences of the GPU forward, up to
the 512^2 / 200-step / checkpoint-20 workload; on D2Q16 and on D2Q9.

Loss throughout: L = 1/2 sum (rho_T - rho*)^2 with a seeded target rho*.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import torch_ref as tr
from paper_1806_05089_gb300 import workloads


def small_case(nx, ny, seed=0, T_L=1.0):
    """Taylor-Green (u0 = 0.3) with seeded density and temperature; on D2Q9
    (T_L = 1/3) T and u are rescaled to the same Mach numbers."""
    tg = workloads.taylor_green(nx, ny, 0.3)
    rng = np.random.default_rng(seed)
    rho0 = 1.0 + 0.05 * rng.standard_normal((ny, nx))
    target = 1.0 + 0.01 * rng.standard_normal((ny, nx))
    T0 = (1.0 + 0.1 * rng.random((ny, nx))) * T_L
    return rho0, tg.ux * np.sqrt(T_L), tg.uy * np.sqrt(T_L), T0, target


def fast_case(nx, ny, seed=0, T_L=1.0):
    """The supersonic field (u = (1.5, 0.5), Mach 1.6) with a Taylor-Green
    swirl (u0 = 0.3) on top, so the particle velocities span a wide, varying
    range: the adjoint gathers' candidate windows are wide."""
    f = workloads.supersonic(nx=nx, ny=ny)
    tg = workloads.taylor_green(nx, ny, 0.3)
    rng = np.random.default_rng(seed)
    rho0 = f.rho * (1.0 + 0.02 * rng.standard_normal((ny, nx)))
    target = 1.0 + 0.01 * rng.standard_normal((ny, nx))
    return (rho0, (f.ux + tg.ux) * np.sqrt(T_L), (f.uy + tg.uy) * np.sqrt(T_L), f.T * T_L,
            target)


CASES = {"tg": small_case, "fast": fast_case}


def oracle_loss(rho0, ux, uy, T, target, nu, steps, passes, lattice=0, T_ref=1.0):
    st = oracle.init_equilibrium(rho0, ux, uy, T, lattice=lattice)
    p = oracle.Params(nu=nu, fixed_iter=passes, lattice=lattice, T_ref=T_ref)
    for _ in range(steps):
        st, _, _ = oracle.step(st, p)
    return 0.5 * ((st.f.sum(0) - target) ** 2).sum()


def reference_grad(rho0, ux, uy, T, target, nu, steps, passes, lattice=0, T_ref=1.0):
    r = torch.tensor(rho0, requires_grad=True)
    n = torch.tensor(nu, dtype=torch.float64, requires_grad=True)
    rho = tr.rollout(r, torch.tensor(ux), torch.tensor(uy), torch.tensor(T), n, steps, passes,
                     T_ref=T_ref, lattice_kind=lattice)
    loss = 0.5 * ((rho - torch.tensor(target)) ** 2).sum()
    loss.backward()
    return float(loss.detach()), r.grad.numpy(), float(n.grad)


LATTICES = [(0, 1.0), (1, 1.0 / 3.0)]  # (lattice, T_L): D2Q16, D2Q9


@pytest.mark.parametrize("lattice,T_L", LATTICES)
def test_reference_step_matches_oracle(lattice, T_L):
    rho0, ux, uy, T, _ = small_case(7, 5, T_L=T_L)
    st = oracle.init_equilibrium(rho0, ux, uy, T, lattice=lattice)
    f = torch.tensor(st.f)
    g = [torch.tensor(a) for a in (st.ux, st.uy, st.T)]
    o = st
    for _ in range(2):
        o, _, _ = oracle.step(o, oracle.Params(nu=0.02, fixed_iter=5, lattice=lattice, T_ref=T_L))
        f, *g = tr.step(f, *g, 0.02, 5, T_ref=T_L, lattice_kind=lattice)
    assert np.abs(f.numpy() - o.f).max() <= 1e-13
    assert np.abs(g[0].numpy() - o.ux).max() <= 1e-13
    assert np.abs(g[2].numpy() - o.T).max() <= 1e-13


@pytest.mark.parametrize("lattice,T_L", LATTICES)
def test_reference_gradient_matches_oracle_fd(lattice, T_L):
    rho0, ux, uy, T, target = small_case(6, 5, seed=1, T_L=T_L)
    nu, steps, passes = 0.02, 2, 20
    kw = dict(lattice=lattice, T_ref=T_L)
    L, grho, gnu = reference_grad(rho0, ux, uy, T, target, nu, steps, passes, **kw)
    assert abs(L - oracle_loss(rho0, ux, uy, T, target, nu, steps, passes, **kw)) <= 1e-12 * L
    rng = np.random.default_rng(7)
    for _ in range(2):
        d = rng.standard_normal(rho0.shape)
        h = 1e-5
        fd = (oracle_loss(rho0 + h * d, ux, uy, T, target, nu, steps, passes, **kw)
              - oracle_loss(rho0 - h * d, ux, uy, T, target, nu, steps, passes, **kw)) / (2 * h)
        assert abs(fd - (grho * d).sum()) <= 1e-6 * abs(fd)
    h = 1e-6
    fd = (oracle_loss(rho0, ux, uy, T, target, nu + h, steps, passes, **kw)
          - oracle_loss(rho0, ux, uy, T, target, nu - h, steps, passes, **kw)) / (2 * h)
    assert abs(fd - gnu) <= 1e-6 * abs(fd)


# ------------------------------------------------------------------ GPU


def gpu_grad(rho0, ux, uy, T, target, nu, steps, ckpt, **cfg):
    from paper_1806_05089_gb300.autograd import pond_rollout
    dev = torch.device("cuda")
    r = torch.tensor(rho0, device=dev, requires_grad=True)
    n = torch.tensor(nu, dtype=torch.float64, device=dev, requires_grad=True)
    rho = pond_rollout(r, n, *(torch.tensor(a, device=dev) for a in (ux, uy, T)), steps, ckpt,
                       **cfg)
    loss = 0.5 * ((rho - torch.tensor(target, device=dev)) ** 2).sum()
    loss.backward()
    return float(loss.detach()), r.grad.cpu().numpy(), float(n.grad)


def gpu_loss(rho0, ux, uy, T, target, nu, steps, **cfg):
    from paper_1806_05089_gb300 import pond
    ny, nx = rho0.shape
    with pond.Sim(nx, ny, pond.POND_FP64, nu=nu, **cfg) as s:
        s.set_state(rho0, ux, uy, T)
        s.step(steps, stats=False)
        rho = s.moments()[0]
    return 0.5 * ((rho - target) ** 2).sum()


@pytest.mark.gpu
@pytest.mark.parametrize("lattice,T_L", LATTICES)
def test_adjoint_matches_reference_gradient(lattice, T_L):
    rho0, ux, uy, T, target = small_case(10, 8, seed=2, T_L=T_L)
    nu, steps, passes = 0.02, 3, 24
    L, grho, gnu = reference_grad(rho0, ux, uy, T, target, nu, steps, passes, lattice=lattice,
                                  T_ref=T_L)
    Lg, grho_g, gnu_g = gpu_grad(rho0, ux, uy, T, target, nu, steps, 2, fixed_iter=passes,
                                 lattice=lattice, T_ref=T_L)
    assert abs(Lg - L) <= 1e-12 * L
    assert np.abs(grho_g - grho).max() <= 1e-9 * np.abs(grho).max()
    assert abs(gnu_g - gnu) <= 1e-9 * abs(gnu)


@pytest.mark.gpu
@pytest.mark.parametrize("lattice,T_L", LATTICES)
@pytest.mark.parametrize("fixed", [30, 0])
def test_adjoint_matches_gpu_finite_differences(fixed, lattice, T_L):
    rho0, ux, uy, T, target = small_case(32, 24, seed=3, T_L=T_L)
    if lattice == 1:
        # D2Q9 has a zero speed: its populations depart from x - u dt, which
        # lies exactly on a node where the Taylor-Green u vanishes (whole
        # rows), the kink of the piecewise-cubic reconstruction.  A central
        # difference straddling the kink differs from the one-sided
        # derivative by ~1e-4 at h = 1e-5 (the C oracle's differences do too,
        # against the reference gradient); a mean flow moves those departures
        # off the nodes.
        ux = ux + 0.37 * np.sqrt(T_L)
        uy = uy - 0.185 * np.sqrt(T_L)
    nu, steps, ckpt = 0.01, 6, 4
    cfg = {"fixed_iter": fixed} if fixed else {}
    cfg.update(lattice=lattice, T_ref=T_L)
    L, grho, gnu = gpu_grad(rho0, ux, uy, T, target, nu, steps, ckpt, **cfg)
    rng = np.random.default_rng(11)
    for _ in range(4):
        d = rng.standard_normal(rho0.shape)
        h = 1e-5
        fd = (gpu_loss(rho0 + h * d, ux, uy, T, target, nu, steps, **cfg)
              - gpu_loss(rho0 - h * d, ux, uy, T, target, nu, steps, **cfg)) / (2 * h)
        assert abs(fd - (grho * d).sum()) <= 1e-6 * abs(fd), (fd, (grho * d).sum())
    h = 1e-6
    fd = (gpu_loss(rho0, ux, uy, T, target, nu + h, steps, **cfg)
          - gpu_loss(rho0, ux, uy, T, target, nu - h, steps, **cfg)) / (2 * h)
    assert abs(fd - gnu) <= 1e-6 * abs(fd), (fd, gnu)


@pytest.mark.gpu
def test_adjoint_full_workload_512():
    """512^2 Taylor-Green (u0 = 0.3) plus a Gaussian pulse, 200 steps,
    checkpoints every 20; gradient w.r.t. rho0 (8 seeded directions) and nu
    against central finite differences of the GPU forward."""
    f, target = workloads.adjoint(512)
    nu, steps, ckpt = 0.01, 200, 20
    L, grho, gnu = gpu_grad(f.rho, f.ux, f.uy, f.T, target, nu, steps, ckpt)
    rng = np.random.default_rng(1806050894)
    for _ in range(8):
        d = rng.standard_normal(f.rho.shape)
        h = 1e-6
        fd = (gpu_loss(f.rho + h * d, f.ux, f.uy, f.T, target, nu, steps)
              - gpu_loss(f.rho - h * d, f.ux, f.uy, f.T, target, nu, steps)) / (2 * h)
        assert abs(fd - (grho * d).sum()) <= 1e-6 * abs(fd), (fd, (grho * d).sum())
    h = 1e-7
    fd = (gpu_loss(f.rho, f.ux, f.uy, f.T, target, nu + h, steps)
          - gpu_loss(f.rho, f.ux, f.uy, f.T, target, nu - h, steps)) / (2 * h)
    assert abs(fd - gnu) <= 1e-6 * abs(fd), (fd, gnu)


@pytest.mark.gpu
@pytest.mark.parametrize("lattice,T_L", LATTICES)
@pytest.mark.parametrize("nx,ny", [(48, 40), (37, 29)])
def test_mixed_adjoint_matches_fp64_adjoint(nx, ny, lattice, T_L):
    """The FP32 adjoint (mixed context) against the FP64 adjoint on the same
    rollout: the gradients agree to the accuracy of the FP32 forward.  37 x 29
    leaves a partly filled last block of the one-thread-per-node kernels."""
    from paper_1806_05089_gb300 import pond
    rho0, ux, uy, T, target = small_case(nx, ny, seed=5, T_L=T_L)
    nu, steps, ckpt = 0.01, 8, 4
    kw = dict(lattice=lattice, T_ref=T_L)
    L64, g64, n64 = gpu_grad(rho0, ux, uy, T, target, nu, steps, ckpt, **kw)
    L32, g32, n32 = gpu_grad(rho0, ux, uy, T, target, nu, steps, ckpt,
                             precision=pond.POND_FP32_MIXED, **kw)
    assert abs(L32 - L64) <= 1e-4 * L64
    assert np.abs(g32 - g64).max() <= 1e-4 * np.abs(g64).max()
    assert abs(n32 - n64) <= 1e-4 * abs(n64)


@pytest.mark.gpu
@pytest.mark.parametrize("lattice,T_L", LATTICES)
@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_given_output_gauge_matches_recomputed(precision, lattice, T_L):
    """pond_adjoint_step_given (the step's output gauge handed in) gives the
    same VJP as pond_adjoint_step (forward step recomputed inside), FP64 and
    mixed, both lattices; a NULL output gauge is refused."""
    from paper_1806_05089_gb300 import pond
    rho0, ux, uy, T, _ = small_case(40, 36, seed=7, T_L=T_L)
    dev = torch.device("cuda")
    rng = np.random.default_rng(8)
    Q = 16 if lattice == 0 else 9
    fbar = torch.tensor(rng.standard_normal((Q, 36, 40)), device=dev)
    gbar = torch.tensor(rng.standard_normal((3, 36, 40)), device=dev)
    with pond.Sim(40, 36, precision, nu=0.01, lattice=lattice, T_ref=T_L) as s:
        s.set_state(rho0, ux, uy, T)
        s.step(2)                         # a state with a non-equilibrium part
        st0 = s.state()
        s.step(1)
        st1 = s.state()                   # the step's output
        s.set_state(None, st0.ux, st0.uy, st0.T, st0.f)
        outs = []
        for given in (False, True):
            fo = torch.empty_like(fbar)
            go = torch.empty_like(gbar)
            if given:
                g1 = [torch.tensor(a, device=dev) for a in (st1.ux, st1.uy, st1.T)]
                nb = pond.pond_adjoint_step_given(s.ctx, *g1, fbar, gbar, fo, go)
            else:
                nb = pond.pond_adjoint_step(s.ctx, fbar, gbar, fo, go)
            outs.append((fo.cpu().numpy(), go.cpu().numpy(), nb))
        with pytest.raises(pond.PondError) as e:
            pond.pond_adjoint_step_given(s.ctx, None, g1[1], g1[2], fbar, gbar, fo, go)
        assert e.value.status == pond.POND_ERR_ARG
    (f_a, g_a, n_a), (f_b, g_b, n_b) = outs
    assert np.abs(f_a - f_b).max() <= 1e-14 * np.abs(f_a).max()
    assert np.abs(g_a - g_b).max() <= 1e-14 * np.abs(g_a).max()
    # nu_bar is a sum of per-node double atomics whose order varies from run
    # to run: equal to rounding of that sum
    assert abs(n_a - n_b) <= 1e-12 * abs(n_a)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_nu_cotangent_on_device_matches_host(precision):
    """With nu_bar_accum NULL the nu cotangent accumulates on the device and
    pond_adjoint_nu_bar returns (and clears) the sum: the same value as the
    host accumulator, over several calls, and the same f / gauge cotangents."""
    from paper_1806_05089_gb300 import pond
    rho0, ux, uy, T, _ = small_case(40, 36, seed=3)
    dev = torch.device("cuda")
    rng = np.random.default_rng(4)
    fbar = torch.tensor(rng.standard_normal((16, 36, 40)), device=dev)
    gbar = torch.tensor(rng.standard_normal((3, 36, 40)), device=dev)
    with pond.Sim(40, 36, precision, nu=0.01) as s:
        s.set_state(rho0, ux, uy, T)
        s.step(2)
        assert pond.pond_adjoint_nu_bar(s.ctx) == 0.0  # before any adjoint call
        outs = []
        for on_device in (False, True):
            tot = 0.0
            for _ in range(3):
                fo = torch.empty_like(fbar)
                go = torch.empty_like(gbar)
                nb = pond.pond_adjoint_step(s.ctx, fbar, gbar, fo, go, nu_on_device=on_device)
                if on_device:
                    assert nb is None
                else:
                    tot += nb
            if on_device:
                tot = pond.pond_adjoint_nu_bar(s.ctx)
                assert pond.pond_adjoint_nu_bar(s.ctx) == 0.0  # cleared by the read
            outs.append((fo.cpu().numpy(), go.cpu().numpy(), tot))
    (f_a, g_a, n_a), (f_b, g_b, n_b) = outs
    assert np.abs(f_a - f_b).max() <= 1e-14 * np.abs(f_a).max()
    assert np.abs(g_a - g_b).max() <= 1e-14 * np.abs(g_a).max()
    assert n_a != 0.0 and abs(n_a - n_b) <= 1e-12 * abs(n_a)


@pytest.mark.gpu
def test_mixed_adjoint_rollout_length_bound():
    """The stated accuracy of the FP32 adjoint over a long rollout: on the
    512^2 adjoint workload, 200 steps with checkpoints every 20, its gradient
    w.r.t. rho0 stays within 3e-5 (max-norm relative) of the FP64 adjoint's
    and its nu gradient within 1e-2.  nu_bar sums 200 steps of per-node beta
    cotangents that largely cancel, so it is the sensitive one (measured
    7.4e-6 and 1.7e-3)."""
    from paper_1806_05089_gb300 import pond
    f, target = workloads.adjoint(512)
    nu, steps, ckpt = 0.01, 200, 20
    L64, g64, n64 = gpu_grad(f.rho, f.ux, f.uy, f.T, target, nu, steps, ckpt)
    L32, g32, n32 = gpu_grad(f.rho, f.ux, f.uy, f.T, target, nu, steps, ckpt,
                             precision=pond.POND_FP32_MIXED)
    assert np.abs(g32 - g64).max() <= 3e-5 * np.abs(g64).max()
    assert abs(n32 - n64) <= 1e-2 * abs(n64)
    assert abs(L32 - L64) <= 1e-4 * L64


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["tg", "fast"])
@pytest.mark.parametrize("lattice,T_L", LATTICES)
@pytest.mark.parametrize("nx,ny", [(40, 36), (37, 29), (3, 5)])
def test_staged_adjoint_matches_direct_adjoint(nx, ny, lattice, T_L, case):
    """The FP64 adjoint step of a staged-kernel context (phase A through the
    tile's reference gauge, the target-centric gather) and of a direct-kernel
    context give the same VJP to rounding, on a full, a ragged and a tiny
    grid, at low and at supersonic speed."""
    from paper_1806_05089_gb300 import pond
    rho0, ux, uy, T, _ = CASES[case](nx, ny, seed=11, T_L=T_L)
    dev = torch.device("cuda")
    rng = np.random.default_rng(12)
    Q = 16 if lattice == 0 else 9
    fbar = torch.tensor(rng.standard_normal((Q, ny, nx)), device=dev)
    gbar = torch.tensor(rng.standard_normal((3, ny, nx)), device=dev)
    outs = []
    for kernel in (pond.POND_KERNEL_STAGED, pond.POND_KERNEL_DIRECT):
        with pond.Sim(nx, ny, pond.POND_FP64, nu=0.01, lattice=lattice, T_ref=T_L,
                      kernel=kernel) as s:
            s.set_state(rho0, ux, uy, T)
            s.step(2)
            fo = torch.empty_like(fbar)
            go = torch.empty_like(gbar)
            nb = pond.pond_adjoint_step(s.ctx, fbar, gbar, fo, go)
            outs.append((fo.cpu().numpy(), go.cpu().numpy(), nb))
    (f_a, g_a, n_a), (f_b, g_b, n_b) = outs
    assert np.abs(f_a - f_b).max() <= 1e-11 * np.abs(f_b).max()
    assert np.abs(g_a - g_b).max() <= 1e-11 * np.abs(g_b).max()
    assert abs(n_a - n_b) <= 1e-11 * abs(n_b)


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["tg", "fast"])
@pytest.mark.parametrize("lattice,T_L", LATTICES)
@pytest.mark.parametrize("nx,ny", [(40, 36), (37, 29), (3, 5)])
def test_staged_mixed_adjoint_matches_direct_mixed_adjoint(nx, ny, lattice, T_L, case):
    """The FP32 adjoint step with the staged phase A (sources staged in the
    tile's reference gauge, epilogue fused) and with the per-pair phase A,
    both handed the same input state and output gauge, agree to FP32
    rounding, and both with the FP64 adjoint step, on a full, a ragged and a
    tiny grid."""
    from paper_1806_05089_gb300 import pond
    rho0, ux, uy, T, _ = CASES[case](nx, ny, seed=13, T_L=T_L)
    dev = torch.device("cuda")
    rng = np.random.default_rng(14)
    Q = 16 if lattice == 0 else 9
    fbar = torch.tensor(rng.standard_normal((Q, ny, nx)), device=dev)
    gbar = torch.tensor(rng.standard_normal((3, ny, nx)), device=dev)
    with pond.Sim(nx, ny, pond.POND_FP64, nu=0.01, lattice=lattice, T_ref=T_L) as s:
        s.set_state(rho0, ux, uy, T)
        s.step(2)
        st0 = s.state()
        s.step(1)
        st1 = s.state()
    g1 = [torch.tensor(a, device=dev) for a in (st1.ux, st1.uy, st1.T)]
    outs = {}
    for name, prec, kernel in (("staged", pond.POND_FP32_MIXED, pond.POND_KERNEL_STAGED),
                               ("direct", pond.POND_FP32_MIXED, pond.POND_KERNEL_DIRECT),
                               ("fp64", pond.POND_FP64, pond.POND_KERNEL_STAGED)):
        with pond.Sim(nx, ny, prec, nu=0.01, lattice=lattice, T_ref=T_L, kernel=kernel) as s:
            s.set_state(None, st0.ux, st0.uy, st0.T, st0.f)
            fo = torch.empty_like(fbar)
            go = torch.empty_like(gbar)
            nb = pond.pond_adjoint_step_given(s.ctx, *g1, fbar, gbar, fo, go)
            outs[name] = (fo.cpu().numpy(), go.cpu().numpy(), nb)
    for a, b in (("staged", "direct"), ("staged", "fp64"), ("direct", "fp64")):
        (f_a, g_a, n_a), (f_b, g_b, n_b) = outs[a], outs[b]
        assert np.abs(f_a - f_b).max() <= 1e-4 * np.abs(f_b).max(), (a, b)
        assert np.abs(g_a - g_b).max() <= 1e-4 * np.abs(g_b).max(), (a, b)
        assert abs(n_a - n_b) <= 1e-4 * abs(n_b), (a, b)
