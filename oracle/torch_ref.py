"""Plain PyTorch FP64 (CPU) restatement of the PonD step, for autograd.

TEST INFRASTRUCTURE ONLY: it gives the reference gradient that the CUDA
adjoint is checked against.  It follows the same reading of the paper as
pond_oracle.c, written independently with tensor operations: a fixed number
of predictor-corrector passes (each one: departures of Eqs. advection and vi,
the reconstruction of Eq. interpolation with the cubic weights of App. C, the
gauge transform of Eq. transform solved in the target-centred moment basis,
the raw moments of Eqs. conservation_rho/rhou/T), then the last pass's
populations re-expressed in the gauge their moments define, and the BGK
relaxation of Eq. postcollision.  Unrolling enough passes reaches the fixed
point to round-off, so autograd through the unrolled passes gives the
derivative of the converged step.  The floor() of the departure point is
piecewise constant and carries no gradient.  Lattices: D2Q16 (lattice=0, the
four roots of He4, T_L = 1) and D2Q9 (lattice=1, App. A: c = -1, 0, 1,
W = 1/6, 2/3, 1/6, T_L = 1/3); populations q = n1 k + l.
"""
from __future__ import annotations

import math

import torch

DT = torch.float64


def lattice(kind: int = 0):
    """(c, w, T_L): 1D speeds (ascending), weights and lattice temperature."""
    if kind == 1:
        return (torch.tensor([-1.0, 0.0, 1.0], dtype=DT),
                torch.tensor([1 / 6, 2 / 3, 1 / 6], dtype=DT), 1.0 / 3.0)
    s6 = math.sqrt(6.0)
    c = torch.tensor([-math.sqrt(3 + s6), -math.sqrt(3 - s6), math.sqrt(3 - s6),
                      math.sqrt(3 + s6)], dtype=DT)
    w = torch.tensor([(3 - s6) / 12, (3 + s6) / 12, (3 + s6) / 12, (3 - s6) / 12], dtype=DT)
    return c, w, 1.0


def moment_inverse(c):
    """Inverse of M[(m,n),(k,l)] = c_k^m c_l^n, m, n < n1 (target-centred
    moment basis)."""
    n1 = len(c)
    rows = []
    for m in range(n1):
        for n in range(n1):
            rows.append(torch.stack([c[k] ** m * c[l] ** n for k in range(n1) for l in range(n1)]))
    return torch.linalg.inv(torch.stack(rows))


def transfer(f, gs, gd, c, minv, T_L: float = 1.0):
    """Eq. transform: f (..., Q) from gauge gs = (ux, uy, T) to gauge gd."""
    n1 = len(c)
    sts = torch.sqrt(gs[2] / T_L)
    stt = torch.sqrt(gd[2] / T_L)
    xi_x = ((sts[..., None] * c + gs[0][..., None]) - gd[0][..., None]) / stt[..., None]
    xi_y = ((sts[..., None] * c + gs[1][..., None]) - gd[1][..., None]) / stt[..., None]
    p = torch.arange(n1, dtype=DT)
    px = xi_x[..., None, :] ** p[:, None]   # (..., m, a)
    py = xi_y[..., None, :] ** p[:, None]   # (..., n, b)
    mom = torch.einsum("...ma,...nb,...ab->...mn", px, py, f.reshape(*f.shape[:-1], n1, n1))
    return torch.einsum("qr,...r->...q", minv, mom.reshape(*mom.shape[:-2], n1 * n1))


def interp_weights(t):
    """Cubic Lagrange weights on nodes 0..3 at t (..., 4) (App. C)."""
    out = []
    for j in range(4):
        r = torch.ones_like(t)
        for k in range(4):
            if k != j:
                r = r * (t - k) / (j - k)
        out.append(r)
    return torch.stack(out, dim=-1)


def step(f, ux, uy, T, nu, passes: int, dt: float = 1.0, T_ref: float = 1.0, lattice_kind: int = 0):
    """One step with a fixed number of passes.  f: (Q, ny, nx); gauge (ny, nx)."""
    ny, nx = ux.shape
    c, w, T_L = lattice(lattice_kind)
    n1 = len(c)
    Q = n1 * n1
    minv = moment_inverse(c)
    beta = 1.0 / (2.0 * nu / (T_ref * dt) + 1.0)
    kq = torch.arange(Q) // n1
    lq = torch.arange(Q) % n1
    Y, X = torch.meshgrid(torch.arange(ny, dtype=DT), torch.arange(nx, dtype=DT), indexing="ij")
    fsrc = f.permute(1, 2, 0)  # (ny, nx, Q)
    g = (ux, uy, T)
    A = None
    for p in range(passes):
        st = torch.sqrt(g[2] / T_L)
        vx = st[None] * c[kq][:, None, None] + g[0][None]   # (Q, ny, nx)
        vy = st[None] * c[lq][:, None, None] + g[1][None]
        dx = X[None] - vx * dt
        dy = Y[None] - vy * dt
        fx = torch.floor(dx).detach()
        fy = torch.floor(dy).detach()
        ax = interp_weights(dx - fx + 1.0)  # (Q, ny, nx, 4)
        ay = interp_weights(dy - fy + 1.0)
        off = torch.arange(4)
        ix = torch.remainder(fx.long()[..., None] - 1 + off, nx)  # (Q, ny, nx, 4)
        iy = torch.remainder(fy.long()[..., None] - 1 + off, ny)
        SY = iy[..., :, None].expand(Q, ny, nx, 4, 4)
        SX = ix[..., None, :].expand(Q, ny, nx, 4, 4)
        fs = fsrc[SY, SX]                                   # (Q, ny, nx, 4, 4, Q)
        gsrc = (ux[SY, SX], uy[SY, SX], T[SY, SX])
        gdst = tuple(v[None, :, :, None, None].expand(Q, ny, nx, 4, 4) for v in g)
        ft = transfer(fs, gsrc, gdst, c, minv, T_L)       # (Q, ny, nx, 4, 4, Q)
        idx = torch.arange(Q).view(Q, 1, 1, 1, 1, 1).expand(Q, ny, nx, 4, 4, 1)
        fq = torch.gather(ft, -1, idx)[..., 0]              # (Q, ny, nx, 4, 4)
        A = (ay[..., :, None] * ax[..., None, :] * fq).sum(dim=(-1, -2))  # (Q, ny, nx)
        rho = A.sum(0)
        ux1 = (vx * A).sum(0) / rho
        uy1 = (vy * A).sum(0) / rho
        T1 = (((vx * vx + vy * vy) * A).sum(0) / rho - ux1 * ux1 - uy1 * uy1) / 2.0
        g_next = (ux1, uy1, T1)
        if p == passes - 1:
            A = transfer(A.permute(1, 2, 0), g, g_next, c, minv, T_L).permute(2, 0, 1)
        g = g_next
    rho = A.sum(0)
    W = (w[kq] * w[lq])[:, None, None]
    return A + 2.0 * beta * (rho[None] * W - A), g[0], g[1], g[2]


def rollout(rho0, ux0, uy0, T0, nu, steps: int, passes: int, T_ref: float = 1.0,
            lattice_kind: int = 0):
    """Final density after ``steps`` steps from f = rho0 W (Eq. equilibrium)."""
    c, w, _ = lattice(lattice_kind)
    n1 = len(c)
    kq = torch.arange(n1 * n1) // n1
    lq = torch.arange(n1 * n1) % n1
    f = rho0[None] * (w[kq] * w[lq])[:, None, None]
    ux, uy, T = ux0, uy0, T0
    for _ in range(steps):
        f, ux, uy, T = step(f, ux, uy, T, nu, passes, T_ref=T_ref, lattice_kind=lattice_kind)
    return f.sum(0)
