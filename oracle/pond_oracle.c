/*
 * pond_oracle.c -- plain FP64 CPU oracle of one Particles-on-Demand (PonD)
 * time step on the D2Q16 lattice (Dorschner, Bosch, Karlin, "Particles-on-
 * Demand for Kinetic Theory", arXiv 1806.05089).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library: every constant below is derived here from its
 * definition.
 *
 * The step follows the paper's order:
 *   seed gauge                       (Eqs. seed_gauge, vi)
 *   semi-Lagrangian propagation      (Eq. advection)
 *     reconstruction                 (Eq. interpolation; App. C)
 *     gauge transform by moment matching (Eqs. moments, match, transform)
 *   moments of the propagated populations (Eqs. conservation_rho/rhou/T)
 *   predictor-corrector until the convergence test holds (Eqs. density..
 *     precollision; App. E, Eq. convergence)
 *   BGK relaxation to the co-moving equilibrium (Eqs. equilibrium,
 *     postcollision)
 *
 * Readings taken where the paper is silent or specific to D2Q9:
 *  - lattice: D2Q16 by default, the tensor product of the four roots of the
 *    Hermite polynomial He4 (c^2 = 3 -+ sqrt 6), weights (3 -+ sqrt 6)/12,
 *    T_L = 1 (the paper's general theory, Eq. peculiar and App. A, is
 *    lattice-agnostic); or the paper's own D2Q9 (App. A: c in {0, +-1},
 *    W = 2/3, 1/6, T_L = 1/3), matching its 9 moments m, n <= 2 (App. B).
 *  - moments for the transform are taken in the monomial basis centred and
 *    scaled on the TARGET gauge, ((v_x-u'_x)/sqrt(theta'))^m ((v_y-u'_y)/
 *    sqrt(theta'))^n, m,n = 0..3.  These 16 polynomials are an invertible
 *    triangular recombination of the paper's v_x^m v_y^n (Eq. moments), so
 *    matching them (Eq. match) gives the same f^{lambda'}; the target-side
 *    matrix becomes the constant c_k^m c_l^n and stays well conditioned at
 *    any Mach number.
 *  - after the last predictor-corrector pass n, whose populations
 *    f^{lambda_n} have the moments lambda_{n+1}, the populations are
 *    re-expressed in lambda_{n+1} (Eq. transform at the node itself) and
 *    stored with that gauge: the stored gauge is then exactly the co-moving
 *    frame of the stored populations (remark after Eq. precollision), and
 *    both tend to the limits of Eqs. density..precollision.
 *  - convergence: |phi_{n+1}-phi_n| < eps_abs + eps_rel |phi_{n+1}| for
 *    phi in {u_x, u_y, sqrt(theta)}; at most max_iter passes; fixed_iter > 0
 *    runs exactly that many passes.
 *  - beta from nu = T_ref (1/(2 beta) - 1/2) dt with a global T_ref.
 *  - periodic wrap in both directions.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see build.py).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_Q 16

typedef struct {
    double nu, T_ref, dt, eps_abs, eps_rel;
    int32_t max_iter, fixed_iter, thermal, seed_mode;
    int32_t lattice; /* 0: D2Q16 (default), 1: D2Q9 (the paper's App. A lattice) */
    int32_t pad;
} oracle_params;

/* per-node flags written by oracle_step */
#define ORACLE_FLAG_NONCONVERGED 1
#define ORACLE_FLAG_NONPHYSICAL 2

typedef struct {
    int n1;             /* speeds per dimension (4: D2Q16, 3: D2Q9) */
    int q;              /* populations, n1 * n1 */
    double c[4];        /* 1D peculiar speeds, ascending */
    double w[4];        /* 1D weights */
    double T_L;         /* lattice temperature */
    double minv[16][16];/* inverse of the target-side moment matrix */
} lattice_t;

/* One-dimensional speeds and weights.  D2Q16: the four roots of He4 with
 * their Gauss-Hermite weights, T_L = 1 (App. A generalised to a fourth-order
 * set).  D2Q9: c in {-1, 0, 1}, W = {1/6, 2/3, 1/6}, T_L = 1/3 (App. A). */
static void lattice_1d(int lattice, lattice_t *L) {
    if (lattice == 1) {
        L->n1 = 3;
        L->c[0] = -1.0;
        L->c[1] = 0.0;
        L->c[2] = 1.0;
        L->w[0] = 1.0 / 6.0;
        L->w[1] = 2.0 / 3.0;
        L->w[2] = 1.0 / 6.0;
        L->c[3] = 0.0;
        L->w[3] = 0.0;
        L->T_L = 1.0 / 3.0;
    } else {
        const double s6 = sqrt(6.0);
        L->n1 = 4;
        L->c[0] = -sqrt(3.0 + s6);
        L->c[1] = -sqrt(3.0 - s6);
        L->c[2] = sqrt(3.0 - s6);
        L->c[3] = sqrt(3.0 + s6);
        L->w[0] = (3.0 - s6) / 12.0;
        L->w[1] = (3.0 + s6) / 12.0;
        L->w[2] = (3.0 + s6) / 12.0;
        L->w[3] = (3.0 - s6) / 12.0;
        L->T_L = 1.0;
    }
    L->q = L->n1 * L->n1;
}

/* Gauss-Jordan inversion with partial pivoting of an n x n matrix. */
static int invert(int n, double *a, double *inv) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r * n + col]) > fabs(a[piv * n + col])) piv = r;
        if (a[piv * n + col] == 0.0) return -1;
        if (piv != col) {
            for (int j = 0; j < n; ++j) {
                double t = a[col * n + j];
                a[col * n + j] = a[piv * n + j];
                a[piv * n + j] = t;
                t = inv[col * n + j];
                inv[col * n + j] = inv[piv * n + j];
                inv[piv * n + j] = t;
            }
        }
        double d = a[col * n + col];
        for (int j = 0; j < n; ++j) {
            a[col * n + j] /= d;
            inv[col * n + j] /= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double m = a[r * n + col];
            if (m == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                a[r * n + j] -= m * a[col * n + j];
                inv[r * n + j] -= m * inv[col * n + j];
            }
        }
    }
    return 0;
}

static double ipow(double x, int p) {
    double r = 1.0;
    for (int i = 0; i < p; ++i) r *= x;
    return r;
}

static void lattice_init(lattice_t *L, int lattice) {
    lattice_1d(lattice, L);
    const int n1 = L->n1, Q = L->q;
    /* Target-side moment matrix: row (m,n) = n1 m + n, column (k,l) =
     * n1 k + l, entry c_k^m c_l^n (Eq. moments in the target-centred basis,
     * m, n < n1: the Q moments of App. B for D2Q9). */
    double m[16 * 16], inv[16 * 16];
    for (int mm = 0; mm < n1; ++mm)
        for (int nn = 0; nn < n1; ++nn)
            for (int k = 0; k < n1; ++k)
                for (int l = 0; l < n1; ++l) {
                    m[(n1 * mm + nn) * Q + (n1 * k + l)] =
                        ipow(L->c[k], mm) * ipow(L->c[l], nn);
                }
    invert(Q, m, inv);
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) L->minv[i][j] = inv[i * Q + j];
}

/* Gauge transform f^{lambda'} = M_{lambda'}^{-1} M_{lambda} f^{lambda}
 * (Eq. transform) of one node's 16 populations from the source gauge
 * (usx, usy, Ts) to the target gauge (utx, uty, Tt). */
static void transfer(const lattice_t *L, double usx, double usy, double Ts,
                     double utx, double uty, double Tt, const double *fs,
                     double *ft) {
    const double sts = sqrt(Ts / L->T_L), stt = sqrt(Tt / L->T_L);
    const int n1 = L->n1, Q = L->q;
    double xi_x[4], xi_y[4];
    for (int a = 0; a < n1; ++a) {
        /* source particle velocity (Eq. peculiar) seen from the target frame */
        xi_x[a] = ((sts * L->c[a] + usx) - utx) / stt;
        xi_y[a] = ((sts * L->c[a] + usy) - uty) / stt;
    }
    double mom[16];
    for (int mm = 0; mm < n1; ++mm)
        for (int nn = 0; nn < n1; ++nn) {
            double acc = 0.0;
            for (int a = 0; a < n1; ++a)
                for (int b = 0; b < n1; ++b) {
                    acc += fs[n1 * a + b] * ipow(xi_x[a], mm) * ipow(xi_y[b], nn);
                }
            mom[n1 * mm + nn] = acc;
        }
    for (int q = 0; q < Q; ++q) {
        double acc = 0.0;
        for (int r = 0; r < Q; ++r) acc += L->minv[q][r] * mom[r];
        ft[q] = acc;
    }
}

/* Cubic Lagrange basis on the nodes 0,1,2,3 (App. C). */
static double lagrange_weight(int j, double t) {
    double r = 1.0;
    for (int k = 0; k < 4; ++k)
        if (k != j) r *= (t - (double)k) / (double)(j - k);
    return r;
}

static int64_t wrap(int64_t i, int64_t n) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

/* ------------------------------------------------------------------ */
/* exported helpers (for pinning the oracle's parts in tests)          */

void oracle_lattice(int lattice, double *c, double *w, double *T_L) {
    lattice_t L;
    lattice_init(&L, lattice);
    memcpy(c, L.c, sizeof L.c);
    memcpy(w, L.w, sizeof L.w);
    *T_L = L.T_L;
}

void oracle_transfer(int lattice, const double *gauge_src, const double *gauge_dst,
                     const double *f_src, double *f_dst) {
    lattice_t L;
    lattice_init(&L, lattice);
    transfer(&L, gauge_src[0], gauge_src[1], gauge_src[2], gauge_dst[0],
             gauge_dst[1], gauge_dst[2], f_src, f_dst);
}

void oracle_interp_weights(double t, double *w4) {
    for (int j = 0; j < 4; ++j) w4[j] = lagrange_weight(j, t);
}

/* f_q = rho W_q in each node's own gauge (Eq. equilibrium); the gauge
 * arrays need no change. */
void oracle_init_equilibrium(int lattice, int64_t nx, int64_t ny, const double *rho,
                             double *f) {
    lattice_t L;
    lattice_init(&L, lattice);
    const int64_t N = nx * ny;
    const int n1 = L.n1;
    for (int k = 0; k < n1; ++k)
        for (int l = 0; l < n1; ++l)
            for (int64_t i = 0; i < N; ++i)
                f[(n1 * k + l) * N + i] = rho[i] * L.w[k] * L.w[l];
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following oracle_step calls (n >= 1); returns the count in
 * effect afterwards. */
int oracle_set_num_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* One PonD time step for rows [y_begin, y_end) of a periodic nx x ny grid.
 * State arrays: f[Q][ny][nx] (q = n1 k + l; k: x speed index, l: y speed
 * index), ux, uy, T [ny][nx].  Outputs are written for the given rows only.
 * iters[i] = predictor-corrector passes taken at node i; flags[i] holds
 * ORACLE_FLAG_* bits.  Returns 0. */
int oracle_step(int64_t nx, int64_t ny, const double *f_in, const double *ux_in,
                const double *uy_in, const double *T_in, double *f_out,
                double *ux_out, double *uy_out, double *T_out, int32_t *iters,
                int32_t *flags, const oracle_params *p, int64_t y_begin,
                int64_t y_end) {
    lattice_t L;
    lattice_init(&L, p->lattice);
    const int n1 = L.n1, Q = L.q;
    const int64_t N = nx * ny;
    const double beta = 1.0 / (2.0 * p->nu / (p->T_ref * p->dt) + 1.0);
    const double D = 2.0;

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t node = y_begin * nx; node < y_end * nx; ++node) {
        {
            const int64_t X = node % nx, Y = node / nx;
            /* seed gauge (Eqs. seed_gauge, seed_gauge_T) */
            double ux = ux_in[node], uy = uy_in[node], T = T_in[node];
            if (p->seed_mode == 1) {
                ux = 0.0;
                uy = 0.0;
                T = L.T_L;
            } else if (p->seed_mode == 2) {
                ux = -ux;
                uy = -uy;
            }
            double fq[16];
            double ux1 = ux, uy1 = uy, T1 = T; /* gauge defined by the last pass */
            int flag = 0, pass = 0;
            for (;;) {
                const double st = sqrt(T / L.T_L);
                double vx[16], vy[16];
                /* propagation in gauge (ux, uy, T): Eq. advection */
                for (int k = 0; k < n1; ++k)
                    for (int l = 0; l < n1; ++l) {
                        const int q = n1 * k + l;
                        vx[q] = st * L.c[k] + ux; /* Eq. vi */
                        vy[q] = st * L.c[l] + uy;
                        const double dep_x = (double)X - vx[q] * p->dt;
                        const double dep_y = (double)Y - vy[q] * p->dt;
                        const double x0 = floor(dep_x) - 1.0;
                        const double y0 = floor(dep_y) - 1.0;
                        const double tx = dep_x - x0, ty = dep_y - y0;
                        double acc = 0.0;
                        for (int m = 0; m < 4; ++m)     /* y offset */
                            for (int n = 0; n < 4; ++n) { /* x offset */
                                const int64_t sx = wrap((int64_t)x0 + n, nx);
                                const int64_t sy = wrap((int64_t)y0 + m, ny);
                                const int64_t s = sy * nx + sx;
                                double fs[16], ft[16];
                                for (int r = 0; r < Q; ++r) fs[r] = f_in[r * N + s];
                                transfer(&L, ux_in[s], uy_in[s], T_in[s], ux, uy, T,
                                         fs, ft);
                                acc += lagrange_weight(n, tx) *
                                       lagrange_weight(m, ty) * ft[q];
                            }
                        fq[q] = acc;
                    }
                ++pass;
                /* moments with the pass's discrete velocities:
                 * Eqs. conservation_rho, conservation_rhou, conservation_T */
                double rho = 0.0, jx = 0.0, jy = 0.0, e = 0.0;
                for (int q = 0; q < Q; ++q) {
                    rho += fq[q];
                    jx += vx[q] * fq[q];
                    jy += vy[q] * fq[q];
                    e += (vx[q] * vx[q] + vy[q] * vy[q]) * fq[q];
                }
                ux1 = jx / rho;
                uy1 = jy / rho;
                T1 = T;
                if (p->thermal) T1 = (e / rho - (ux1 * ux1 + uy1 * uy1)) / D;
                if (!(rho > 0.0) || !(T1 > 0.0) || !isfinite(ux1) ||
                    !isfinite(uy1)) {
                    flag |= ORACLE_FLAG_NONPHYSICAL;
                    break;
                }
                const double st1 = sqrt(T1 / L.T_L);
                /* Eq. convergence for phi in {u_x, u_y, sqrt(theta)} */
                const int conv =
                    fabs(ux1 - ux) < p->eps_abs + p->eps_rel * fabs(ux1) &&
                    fabs(uy1 - uy) < p->eps_abs + p->eps_rel * fabs(uy1) &&
                    fabs(st1 - st) < p->eps_abs + p->eps_rel * fabs(st1);
                int stop;
                if (p->fixed_iter > 0) {
                    stop = pass >= p->fixed_iter;
                } else {
                    stop = conv || pass >= p->max_iter;
                    if (!conv && pass >= p->max_iter) flag |= ORACLE_FLAG_NONCONVERGED;
                }
                if (stop) break;
                ux = ux1;
                uy = uy1;
                T = T1;
            }
            /* The pass's populations f^{lambda_n} have the moments lambda_{n+1};
             * re-expressed in that gauge (Eq. transform at the node itself)
             * the gauge is exactly their co-moving frame, as the limit of
             * Eqs. density..precollision is.  Skipped if the moments were
             * non-physical. */
            if (!(flag & ORACLE_FLAG_NONPHYSICAL)) {
                double fr[16];
                transfer(&L, ux, uy, T, ux1, uy1, T1, fq, fr);
                for (int q = 0; q < Q; ++q) fq[q] = fr[q];
                ux = ux1;
                uy = uy1;
                T = T1;
            }
            /* BGK relaxation toward rho W in the co-moving gauge
             * (Eqs. equilibrium, postcollision) */
            double rho = 0.0;
            for (int q = 0; q < Q; ++q) rho += fq[q];
            for (int k = 0; k < n1; ++k)
                for (int l = 0; l < n1; ++l) {
                    const int q = n1 * k + l;
                    const double feq = rho * L.w[k] * L.w[l];
                    f_out[q * N + node] = fq[q] + 2.0 * beta * (feq - fq[q]);
                }
            ux_out[node] = ux;
            uy_out[node] = uy;
            T_out[node] = T;
            if (iters) iters[node] = pass;
            if (flags) flags[node] = flag;
        }
    }
    return 0;
}
