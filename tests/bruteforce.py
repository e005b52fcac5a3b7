"""Brute-force NumPy restatement of the PonD step for tiny grids.

Independent of the C oracle: the gauge transform is the paper's literal
Eq. transform with the raw monomial moment matrices M_lambda (Eq. moments),
solved densely with numpy.linalg.solve; interpolation weights come from
solving the 4x4 Vandermonde system that makes the reconstruction exact for
cubics (App. C), not from the product formula.  Only usable at low Mach
number (the raw monomial basis is ill-conditioned at large |u|) and on a
handful of nodes.

Two lattices: ``"d2q16"`` (the four roots of He4, T_L = 1) and ``"d2q9"``
(App. A: c = -1, 0, 1, W = 1/6, 2/3, 1/6, T_L = 1/3).
"""
import numpy as np

S6 = np.sqrt(6.0)
C = np.array([-np.sqrt(3 + S6), -np.sqrt(3 - S6), np.sqrt(3 - S6), np.sqrt(3 + S6)])
W1 = np.array([(3 - S6) / 12, (3 + S6) / 12, (3 + S6) / 12, (3 - S6) / 12])
T_L = 1.0

LATTICES = {
    "d2q16": (C, W1, T_L),
    "d2q9": (np.array([-1.0, 0.0, 1.0]), np.array([1 / 6, 2 / 3, 1 / 6]), 1.0 / 3.0),
}


def velocities(ux, uy, T, lattice="d2q16"):
    c, _, tl = LATTICES[lattice]
    n1 = len(c)
    st = np.sqrt(T / tl)
    vx = np.repeat(st * c + ux, n1)         # q = n1 k + l -> k
    vy = np.tile(st * c + uy, n1)           # -> l
    return vx, vy


def moment_matrix(ux, uy, T, lattice="d2q16"):
    """M_lambda[(m,n), q] = v_x(q)^m v_y(q)^n, m, n < n1 (Eq. moments)."""
    vx, vy = velocities(ux, uy, T, lattice)
    n1 = len(LATTICES[lattice][0])
    return np.array([vx ** m * vy ** n for m in range(n1) for n in range(n1)])


def transfer(gs, gd, f, lattice="d2q16"):
    return np.linalg.solve(moment_matrix(*gd, lattice), moment_matrix(*gs, lattice) @ f)


def interp_weights(t):
    """Weights a_j with sum_j a_j p(j) = p(t) for every cubic p."""
    V = np.array([[float(j) ** p for j in range(4)] for p in range(4)])
    return np.linalg.solve(V, np.array([t ** p for p in range(4)]))


def step(f, ux, uy, T, nu=0.01, passes=3, thermal=True, dt=1.0, T_ref=1.0,
         lattice="d2q16"):
    """One step with a fixed number of predictor-corrector passes."""
    Q, ny, nx = f.shape
    W1_ = LATTICES[lattice][1]
    beta = 1.0 / (2.0 * nu / (T_ref * dt) + 1.0)
    fo = np.zeros_like(f)
    uxo = np.zeros_like(ux)
    uyo = np.zeros_like(uy)
    To = np.zeros_like(T)
    for Y in range(ny):
        for X in range(nx):
            g = (ux[Y, X], uy[Y, X], T[Y, X])
            for _ in range(passes):
                vx, vy = velocities(*g, lattice)
                fq = np.zeros(Q)
                for q in range(Q):
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
                            fq[q] += ax[n] * ay[m] * transfer(gs, g, f[:, sy, sx], lattice)[q]
                rho = fq.sum()
                u1x = (vx * fq).sum() / rho
                u1y = (vy * fq).sum() / rho
                T1 = g[2]
                if thermal:
                    T1 = (((vx ** 2 + vy ** 2) * fq).sum() / rho - u1x ** 2 - u1y ** 2) / 2.0
                last = (fq, g)
                g = (u1x, u1y, T1)
            fq, g_last = last
            fq = transfer(g_last, g, fq, lattice)  # into the gauge its moments define
            rho = fq.sum()
            W = np.outer(W1_, W1_).reshape(Q)
            fo[:, Y, X] = fq + 2 * beta * (rho * W - fq)
            uxo[Y, X], uyo[Y, X], To[Y, X] = g
    return fo, uxo, uyo, To


# ---------------------------------------------------------------- high precision

def step_mp(f, ux, uy, T, nu=0.01, passes=3, thermal=True, dt=1.0, T_ref=1.0,
            lattice="d2q16", dps=40):
    """``step`` in mpmath arithmetic at ``dps`` decimal digits, for any Mach
    number: the raw monomial matrices of Eq. moments grow like |v|^(2 n1 - 2)
    and make the FP64 solve of ``transfer`` useless beyond Ma ~ 1, but at
    40 digits Eq. transform solved literally stays exact to far below FP64
    rounding.  Same algorithm and pairing as ``step`` (fixed pass count, the
    last pass's populations re-expressed in the gauge their moments define,
    BGK); returns FP64 arrays.  The lattice speeds are recomputed in mpmath
    from their definitions (roots of He4, or App. A's D2Q9)."""
    import mpmath as mp

    mp.mp.dps = dps
    if lattice == "d2q16":
        s6 = mp.sqrt(6)
        c = [-mp.sqrt(3 + s6), -mp.sqrt(3 - s6), mp.sqrt(3 - s6), mp.sqrt(3 + s6)]
        w = [(3 - s6) / 12, (3 + s6) / 12, (3 + s6) / 12, (3 - s6) / 12]
        tl = mp.mpf(1)
    else:
        c = [mp.mpf(-1), mp.mpf(0), mp.mpf(1)]
        w = [mp.mpf(1) / 6, mp.mpf(2) / 3, mp.mpf(1) / 6]
        tl = mp.mpf(1) / 3
    n1 = len(c)
    Q, ny, nx = f.shape
    beta = 1 / (2 * mp.mpf(nu) / (mp.mpf(T_ref) * mp.mpf(dt)) + 1)

    def vel(g):
        st = mp.sqrt(g[2] / tl)
        return ([st * c[k] + g[0] for k in range(n1) for _ in range(n1)],
                [st * c[l] + g[1] for _ in range(n1) for l in range(n1)])

    def mmat(g):
        vx, vy = vel(g)
        return mp.matrix([[vx[q] ** m * vy[q] ** n for q in range(Q)]
                          for m in range(n1) for n in range(n1)])

    def weights(t):
        V = mp.matrix([[mp.mpf(j) ** p for j in range(4)] for p in range(4)])
        return mp.lu_solve(V, mp.matrix([t ** p for p in range(4)]))

    fm = [[[mp.mpf(float(f[q, y, x])) for x in range(nx)] for y in range(ny)] for q in range(Q)]
    gm = [[(mp.mpf(float(ux[y, x])), mp.mpf(float(uy[y, x])), mp.mpf(float(T[y, x])))
           for x in range(nx)] for y in range(ny)]
    src_mom = {}
    for y in range(ny):
        for x in range(nx):
            src_mom[(y, x)] = mmat(gm[y][x]) * mp.matrix([fm[q][y][x] for q in range(Q)])
    fo = np.zeros_like(f)
    uxo = np.zeros_like(ux)
    uyo = np.zeros_like(uy)
    To = np.zeros_like(T)
    Wq = [w[q // n1] * w[q % n1] for q in range(Q)]
    for Y in range(ny):
        for X in range(nx):
            g = gm[Y][X]
            for _ in range(passes):
                vx, vy = vel(g)
                Mt = mmat(g)
                cache = {}
                fq = [mp.mpf(0)] * Q
                for q in range(Q):
                    dx = X - vx[q] * dt
                    dy = Y - vy[q] * dt
                    x0 = mp.floor(dx) - 1
                    y0 = mp.floor(dy) - 1
                    ax = weights(dx - x0)
                    ay = weights(dy - y0)
                    for m in range(4):
                        for n in range(4):
                            sx = int(x0 + n) % nx
                            sy = int(y0 + m) % ny
                            if (sy, sx) not in cache:
                                cache[(sy, sx)] = mp.lu_solve(Mt, src_mom[(sy, sx)])
                            fq[q] += ax[n] * ay[m] * cache[(sy, sx)][q]
                rho = sum(fq)
                u1x = sum(vx[q] * fq[q] for q in range(Q)) / rho
                u1y = sum(vy[q] * fq[q] for q in range(Q)) / rho
                T1 = g[2]
                if thermal:
                    T1 = (sum((vx[q] ** 2 + vy[q] ** 2) * fq[q] for q in range(Q)) / rho
                          - u1x ** 2 - u1y ** 2) / 2
                last = (fq, g)
                g = (u1x, u1y, T1)
            fq, g_last = last
            fq = mp.lu_solve(mmat(g), mmat(g_last) * mp.matrix(fq))
            rho = sum(fq[q] for q in range(Q))
            for q in range(Q):
                fo[q, Y, X] = float(fq[q] + 2 * beta * (rho * Wq[q] - fq[q]))
            uxo[Y, X], uyo[Y, X], To[Y, X] = (float(v) for v in g)
    return fo, uxo, uyo, To
