"""Brute-force NumPy restatement of the PonD step for tiny grids.

Independent of the C oracle: the gauge transform is the paper's literal
Eq. transform with the raw monomial moment matrices M_lambda (Eq. moments),
solved densely with numpy.linalg.solve; interpolation weights come from
solving the 4x4 Vandermonde system that makes the reconstruction exact for
cubics (App. C), not from the product formula.  Only usable at low Mach
number (the raw monomial basis is ill-conditioned at large |u|) and on a
handful of nodes.
"""
import numpy as np

S6 = np.sqrt(6.0)
C = np.array([-np.sqrt(3 + S6), -np.sqrt(3 - S6), np.sqrt(3 - S6), np.sqrt(3 + S6)])
W1 = np.array([(3 - S6) / 12, (3 + S6) / 12, (3 + S6) / 12, (3 - S6) / 12])
T_L = 1.0


def velocities(ux, uy, T):
    st = np.sqrt(T / T_L)
    vx = np.repeat(st * C + ux, 4)          # q = 4k + l -> k
    vy = np.tile(st * C + uy, 4)            # -> l
    return vx, vy


def moment_matrix(ux, uy, T):
    """M_lambda[(m,n), q] = v_x(q)^m v_y(q)^n, m, n = 0..3 (Eq. moments)."""
    vx, vy = velocities(ux, uy, T)
    return np.array([vx ** m * vy ** n for m in range(4) for n in range(4)])


def transfer(gs, gd, f):
    return np.linalg.solve(moment_matrix(*gd), moment_matrix(*gs) @ f)


def interp_weights(t):
    """Weights a_j with sum_j a_j p(j) = p(t) for every cubic p."""
    V = np.array([[float(j) ** p for j in range(4)] for p in range(4)])
    return np.linalg.solve(V, np.array([t ** p for p in range(4)]))


def step(f, ux, uy, T, nu=0.01, passes=3, thermal=True, dt=1.0, T_ref=1.0):
    """One step with a fixed number of predictor-corrector passes."""
    _, ny, nx = f.shape
    beta = 1.0 / (2.0 * nu / (T_ref * dt) + 1.0)
    fo = np.zeros_like(f)
    uxo = np.zeros_like(ux)
    uyo = np.zeros_like(uy)
    To = np.zeros_like(T)
    for Y in range(ny):
        for X in range(nx):
            g = (ux[Y, X], uy[Y, X], T[Y, X])
            for _ in range(passes):
                vx, vy = velocities(*g)
                fq = np.zeros(16)
                for q in range(16):
                    dx = X - vx[q] * dt
                    dy = Y - vy[q] * dt
                    x0 = np.floor(dx) - 1
                    y0 = np.floor(dy) - 1
                    ax = interp_weights(dx - x0)
                    ay = interp_weights(dy - y0)
                    for m in range(4):
                        for n in range(4):
                            sx = int(x0 + n) % nx
                            sy = int(y0 + m) % ny
                            gs = (ux[sy, sx], uy[sy, sx], T[sy, sx])
                            fq[q] += ax[n] * ay[m] * transfer(gs, g, f[:, sy, sx])[q]
                rho = fq.sum()
                u1x = (vx * fq).sum() / rho
                u1y = (vy * fq).sum() / rho
                T1 = g[2]
                if thermal:
                    T1 = (((vx ** 2 + vy ** 2) * fq).sum() / rho - u1x ** 2 - u1y ** 2) / 2.0
                last = (fq, g)
                g = (u1x, u1y, T1)
            fq, g_last = last
            fq = transfer(g_last, g, fq)  # into the gauge its moments define
            rho = fq.sum()
            W = np.outer(W1, W1).reshape(16)
            fo[:, Y, X] = fq + 2 * beta * (rho * W - fq)
            uxo[Y, X], uyo[Y, X], To[Y, X] = g
    return fo, uxo, uyo, To
