// pond_adjoint.cu -- vector-Jacobian product of one PonD step (FP64).
//
// The step maps the input state S = {f_s, lambda_s} to, at every node x,
//   lambda*(x) = the fixed point of Phi(lambda) = M(A(lambda), lambda)
//                (Eqs. conservation_*, density..T),
//   A*(x)      = A(lambda*), A_q(lambda) = sum_j a_j(lambda) (G_{lambda_j}^{lambda} f_j)_q
//                (Eqs. advection, interpolation, transform),
//   f_out      = A* + 2 beta (rho W - A*)   (Eq. postcollision),  gauge_out = lambda*.
// The fixed point is differentiated implicitly.  In the parametrisation
// lambda = (u_x, u_y, s = sqrt(theta)) the moment map M has, at the fixed point,
// dM/dlambda = I (its explicit gauge dependence cancels there), so
// I - dPhi/dlambda = -M_A A_lambda, a 3 x 3 matrix per node, with
//   M_A[u_x][q] = s c_k / rho,  M_A[u_y][q] = s c_l / rho,
//   M_A[s][q]   = s (|c_q|^2 - 2 T_L) / (4 rho T_L).
// Given cotangents (fbar, lambdabar) of the output:
//   Abar   = (1 - 2 beta) fbar + 2 beta (W . fbar) 1,   betabar = sum 2 (rho W - A) fbar
//   g      = A_lambda^T Abar + lambdabar
//   mu     = (I - dPhi/dlambda)^{-T} g = -(M_A A_lambda)^{-T} g
//   w      = Abar + M_A^T mu
//   Sbar   = A_S^T w   (transpose of the reconstruction: onto the source
//                       populations f_j and source gauges lambda_j)
// The seed gauge gets no gradient: the limit does not depend on it.
//
// Phase A forms A*, the JVP A_lambda in three directions, the 3 x 3 solve
// and w.  Contexts on the staged forward kernel run it staged
// (k_adjoint_jvp_staged: one thread per target node, the sources staged per
// tile in a reference gauge, then k_adjoint_epilogue); contexts on the
// direct kernels run k_adjoint_targets (one warp per target node, lane =
// population).  Phase B (one warp per source node) gathers the transpose
// over the targets whose departure stencils can contain the source (a
// window bounded by the particle-velocity range), so the result is
// deterministic and needs no atomics: per population in the direct
// contexts (k_adjoint_sources), per target with the target's hit set
// K x L in the staged ones (k_adjoint_sources_t).
#include <cmath>

#include "pond_device.cuh"
#include "pond_staged.cuh"

namespace pond {

// Lattice constants of the adjoint kernels, slot lattice_slot(n1).
__constant__ Lattice c_La[2];

cudaError_t upload_lattice_adjoint() {
    const Lattice L[2] = {make_lattice(POND_D2Q16), make_lattice(POND_D2Q9)};
    return cudaMemcpyToSymbol(c_La, L, sizeof(L));
}

struct AdjointScratch {
    int64_t N = 0;
    StateBuf<double> fwd{};   // forward step output: gauge = lambda*
    double* w = nullptr;      // [Q][N] (allocated for 16)
    int32_t* iters = nullptr;
    DevStats* stats = nullptr;
    double* beta_bar = nullptr;  // device accumulator
    double* minmax = nullptr;    // 6 doubles: min/max of ux*, uy*, s*
    int2* org = nullptr;         // [16][N] stencil origin of (q, t), relative to t
    double* lw = nullptr;        // [16][N][8] cubic weights of (q, t): x 0..3, y 0..3
    double* inv_st = nullptr;    // [N] 1 / s* at every target
    double* jvp = nullptr;       // [4][16][N] A*, dA/du_x, dA/du_y, dA/ds (staged phase A)
    double* nu_dev = nullptr;    // nu cotangent of calls with nu_bar_accum == NULL
    double host_minmax[6];
};

// Cubic Lagrange weights on 0..3 and their derivatives at t (App. C).
__device__ __forceinline__ void lagrange4_d(double t, double l[4], double dl[4]) {
    const double a = t, b = t - 1.0, c = t - 2.0, d = t - 3.0;
    l[0] = -(b * c * d) / 6.0;
    l[1] = (a * c * d) / 2.0;
    l[2] = -(a * b * d) / 2.0;
    l[3] = (a * b * c) / 6.0;
    dl[0] = -(c * d + b * d + b * c) / 6.0;
    dl[1] = (c * d + a * d + a * c) / 2.0;
    dl[2] = -(b * d + a * d + a * b) / 2.0;
    dl[3] = (b * c + a * c + a * b) / 6.0;
}

// L_k(c_a + de) and its derivative in xi, from the Taylor coefficients.
__device__ __forceinline__ void lag_taylor(const Lattice& L, int k, int a, double de, double& g,
                                          double& gd) {
    const double d1 = L.d1[k][a], d2 = L.d2[k][a], d3 = L.d3[k];
    g = fma(fma(fma(d3, de, d2), de, d1), de, (k == a) ? 1.0 : 0.0);
    gd = fma(fma(3.0 * d3, de, 2.0 * d2), de, d1);
}

struct AdjArgs {
    StateBuf<double> in;     // input state S
    const double* ux_s;      // lambda* (forward output gauge)
    const double* uy_s;
    const double* st_s;
    const double* fbar;      // [Q][N]
    const double* gbar;      // [3][N]  (u_x, u_y, T)
    double* w;               // [Q][N]
    double* fbar_in;         // [Q][N]
    double* gbar_in;         // [3][N]
    double* beta_bar;
    // per (population, target), written by the target kernel for the gather:
    // stencil origin relative to the target, cubic weights, and 1 / s*
    int2* org;
    double* lw;
    double* inv_st;
    int nx, ny;
    long long N;
    double beta, dt, T_L;
    double vlo_x[4], vhi_x[4], vlo_y[4], vhi_y[4];  // particle-velocity bounds per speed
};

constexpr int ADJ_WARPS = 4;

template <int N1>
__global__ void __launch_bounds__(ADJ_WARPS * 32, 2) k_adjoint_targets(AdjArgs A) {
    constexpr int Q = N1 * N1;
    const Lattice& L = c_La[lattice_slot(N1)];
    const int lane = threadIdx.x & 31;
    const long long node = (long long)blockIdx.x * ADJ_WARPS + (threadIdx.x >> 5);
    if (node >= A.N) return;  // warp-uniform
    const int X = (int)(node % A.nx), Y = (int)(node / A.nx);
    // lane = (population q, half); on D2Q9 lanes with q >= 9 hold no
    // population: they contribute zeros to the 16-lane sums and read nothing
    const int q = lane & 15, half = lane >> 4;
    const bool act = q < Q;
    const int qa = act ? q : 0, k = qa / N1, l = qa % N1;
    const double ck = act ? L.c[k] : 0.0, cl = act ? L.c[l] : 0.0;
    const double ux = A.ux_s[node], uy = A.uy_s[node], st = A.st_s[node];
    const double inv = 1.0 / st;

    // departure of population q at lambda*
    const double vx = fma(st, ck, ux), vy = fma(st, cl, uy);
    const double depx = (double)X - vx * A.dt, depy = (double)Y - vy * A.dt;
    const double flx = floor(depx), fly = floor(depy);
    double lx[4], dlx[4], ly[4], dly[4];
    lagrange4_d(depx - flx + 1.0, lx, dlx);
    lagrange4_d(depy - fly + 1.0, ly, dly);
    const int x0 = wrap_idx((long long)flx - 1, A.nx);
    const int y0 = wrap_idx((long long)fly - 1, A.ny);
    // what the gather needs of (q, target): the stencil origin relative to
    // the target and the cubic weights; and 1 / s* of the target
    if (act) {
        const long long o = (long long)q * A.N + node;
        double2* pw = reinterpret_cast<double2*>(A.lw + 8 * o + 4 * half);
        if (half == 0) {
            A.org[o] = make_int2((int)((long long)flx - 1 - X), (int)((long long)fly - 1 - Y));
            pw[0] = make_double2(lx[0], lx[1]);
            pw[1] = make_double2(lx[2], lx[3]);
        } else {
            pw[0] = make_double2(ly[0], ly[1]);
            pw[1] = make_double2(ly[2], ly[3]);
        }
    }
    if (lane == 0) A.inv_st[node] = inv;

    double Aq = 0.0, dAux = 0.0, dAuy = 0.0, dAst = 0.0;
    if (act) {
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
        const int jy = 2 * half + jj;
        const double wy = half ? ly[2 + jj] : ly[jj];
        const double dwy = half ? dly[2 + jj] : dly[jj];
        const int sy = wrap_inc(y0, jy, A.ny);
#pragma unroll
        for (int jx = 0; jx < 4; ++jx) {
            const int sx = wrap_inc(x0, jx, A.nx);
            const long long s = (long long)sy * A.nx + sx;
            const double r = fma(A.in.st[s], inv, -1.0);
            const double dx = (A.in.ux[s] - ux) * inv;
            const double dy = (A.in.uy[s] - uy) * inv;
            double gx[N1], gdx[N1], gy[N1], gdy[N1], xix[N1], xiy[N1];
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                const double ex = fma(L.c[a], r, dx), ey = fma(L.c[a], r, dy);
                xix[a] = L.c[a] + ex;
                xiy[a] = L.c[a] + ey;
                lag_taylor(L, k, a, ex, gx[a], gdx[a]);
                lag_taylor(L, l, a, ey, gy[a], gdy[a]);
            }
            double g = 0.0, gux = 0.0, guy = 0.0, gst = 0.0;
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                double h = 0.0, hp = 0.0, hq = 0.0;
#pragma unroll
                for (int b = 0; b < N1; ++b) {
                    const double fv = A.in.f[(long long)(N1 * a + b) * A.N + s];
                    h = fma(gy[b], fv, h);
                    hp = fma(gdy[b], fv, hp);
                    hq = fma(gdy[b] * xiy[b], fv, hq);
                }
                g = fma(gx[a], h, g);
                gux = fma(gdx[a], h, gux);
                guy = fma(gx[a], hp, guy);
                gst = fma(gdx[a] * xix[a], h, fma(gx[a], hq, gst));
            }
            // d xi / d(target u) = -1/s ; d xi / d(target s) = -xi / s
            gux *= -inv;
            guy *= -inv;
            gst *= -inv;
            const double wx = lx[jx], dwx = dlx[jx];
            const double a_w = wx * wy;
            // d t / d u = -dt ; d t / d s = -c dt
            const double da_ux = -A.dt * dwx * wy;
            const double da_uy = -A.dt * wx * dwy;
            const double da_st = -A.dt * (ck * dwx * wy + cl * wx * dwy);
            Aq = fma(a_w, g, Aq);
            dAux = fma(a_w, gux, fma(da_ux, g, dAux));
            dAuy = fma(a_w, guy, fma(da_uy, g, dAuy));
            dAst = fma(a_w, gst, fma(da_st, g, dAst));
        }
    }
    }
    Aq += __shfl_xor_sync(0xffffffffu, Aq, 16);
    dAux += __shfl_xor_sync(0xffffffffu, dAux, 16);
    dAuy += __shfl_xor_sync(0xffffffffu, dAuy, 16);
    dAst += __shfl_xor_sync(0xffffffffu, dAst, 16);

    auto sum16 = [](double v) {
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    const double Wq = act ? L.w[k] * L.w[l] : 0.0;
    const double fb = act ? A.fbar[(long long)q * A.N + node] : 0.0;
    const double rho = sum16(Aq);
    const double wf = sum16(Wq * fb);
    const double Abar = (1.0 - 2.0 * A.beta) * fb + 2.0 * A.beta * wf;
    const double bb = sum16(2.0 * (rho * Wq - Aq) * fb);

    // moment-map rows at the fixed point
    const double c2 = ck * ck + cl * cl;
    const double mux = st * ck / rho, muy = st * cl / rho;
    const double mst = st * (c2 - 2.0 * A.T_L) / (4.0 * rho * A.T_L);
    double J[3][3];
    J[0][0] = sum16(mux * dAux);
    J[0][1] = sum16(mux * dAuy);
    J[0][2] = sum16(mux * dAst);
    J[1][0] = sum16(muy * dAux);
    J[1][1] = sum16(muy * dAuy);
    J[1][2] = sum16(muy * dAst);
    J[2][0] = sum16(mst * dAux);
    J[2][1] = sum16(mst * dAuy);
    J[2][2] = sum16(mst * dAst);
    // output-gauge cotangent, T -> s: dL/ds = dL/dT * 2 s T_L
    double g0 = sum16(Abar * dAux) + A.gbar[node];
    double g1 = sum16(Abar * dAuy) + A.gbar[A.N + node];
    double g2 = sum16(Abar * dAst) + A.gbar[2 * A.N + node] * 2.0 * st * A.T_L;
    // solve J^T mu = -g (Cramer's rule on the transpose)
    const double a00 = J[0][0], a01 = J[1][0], a02 = J[2][0];
    const double a10 = J[0][1], a11 = J[1][1], a12 = J[2][1];
    const double a20 = J[0][2], a21 = J[1][2], a22 = J[2][2];
    const double det = a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) +
                       a02 * (a10 * a21 - a11 * a20);
    const double idet = 1.0 / det;
    const double r0 = -g0, r1 = -g1, r2 = -g2;
    const double mu0 = (r0 * (a11 * a22 - a12 * a21) - a01 * (r1 * a22 - a12 * r2) +
                        a02 * (r1 * a21 - a11 * r2)) * idet;
    const double mu1 = (a00 * (r1 * a22 - a12 * r2) - r0 * (a10 * a22 - a12 * a20) +
                        a02 * (a10 * r2 - r1 * a20)) * idet;
    const double mu2 = (a00 * (a11 * r2 - r1 * a21) - a01 * (a10 * r2 - r1 * a20) +
                        r0 * (a10 * a21 - a11 * a20)) * idet;
    const double wq = Abar + mux * mu0 + muy * mu1 + mst * mu2;
    if (half == 0 && act) A.w[(long long)q * A.N + node] = wq;
    if (lane == 0) atomicAdd(A.beta_bar, bb);
}

// Warp reduce-scatter of 16 per-lane partial sums by recursive halving: at
// distance 2h each lane keeps the h slots its lane bit selects and adds its
// partner's copy of them.  Returns, in lanes 2p and 2p + 1, the warp total of
// slot p (16 additions per lane, against 16 x 5 for a full all-reduce).
__device__ __forceinline__ double warp_reduce_scatter16(double (&v)[16], int lane) {
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const bool up = (lane & (2 * h)) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double keep = up ? v[i + h] : v[i];
            const double send = up ? v[i] : v[i + h];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * h);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Transpose of the reconstruction, gathered at each source node.
template <int N1>
__global__ void __launch_bounds__(ADJ_WARPS * 32, 2) k_adjoint_sources(AdjArgs A) {
    constexpr int Q = N1 * N1;
    const Lattice& L = c_La[lattice_slot(N1)];
    const int lane = threadIdx.x & 31;
    const long long src = (long long)blockIdx.x * ADJ_WARPS + (threadIdx.x >> 5);
    if (src >= A.N) return;  // warp-uniform
    const int JX = (int)(src % A.nx), JY = (int)(src / A.nx);
    // lane = (population q, half); on D2Q9 lanes with q >= 9 hold no
    // population: they contribute zeros to the 16-lane sums and read nothing
    const int q = lane & 15, half = lane >> 4;
    const bool act = q < Q;
    const int qa = act ? q : 0, k = qa / N1, l = qa % N1;
    double fj[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fj[i] = A.in.f[(long long)i * A.N + src];
    const double uxj = A.in.ux[src], uyj = A.in.uy[src], stj = A.in.st[src];

    double fb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fb[i] = 0.0;
    double bux = 0.0, buy = 0.0, bst = 0.0;

    // candidate targets: J is in the stencil of the target at x when
    // floor(x - v dt) is in [J - 2, J + 1], i.e. x in [J - 2 + v dt, J + 2 + v dt);
    // over v in [vlo, vhi] the integers x from ceil(J - 2 + vlo dt) to
    // ceil(J + 2 + vhi dt) - 1, widened by a rounding margin (the exact test
    // below decides).  ceil(J + a) = J + ceil(a) for integer J, so the bounds
    // are formed relative to J.
    const double ex = 1e-9 * (1.0 + fabs(A.vlo_x[k]) + fabs(A.vhi_x[k])) * A.dt;
    const double ey = 1e-9 * (1.0 + fabs(A.vlo_y[l]) + fabs(A.vhi_y[l])) * A.dt;
    const int xlo = JX + (int)ceil(-2.0 + A.vlo_x[k] * A.dt - ex);
    const int xhi = JX + (int)ceil(2.0 + A.vhi_x[k] * A.dt + ex) - 1;
    const int ylo = JY + (int)ceil(-2.0 + A.vlo_y[l] * A.dt - ey);
    const int yhi = JY + (int)ceil(2.0 + A.vhi_y[l] * A.dt + ey) - 1;
    for (int yy = ylo + half; act && yy <= yhi; yy += 2) {
        const int ty = wrap_idx(yy, A.ny);
        for (int xx = xlo; xx <= xhi; ++xx) {
            const int tx = wrap_idx(xx, A.nx);
            const long long t = (long long)ty * A.nx + tx;
            // the target's stencil origin for population q, as the target
            // kernel found it (at the target's own, wrapped position)
            const long long o = (long long)q * A.N + t;
            const int2 og = A.org[o];
            const int jx = JX - (xx + og.x), jy = JY - (yy + og.y);
            if (jx < 0 || jx > 3 || jy < 0 || jy > 3) continue;
            const double wgt = A.lw[8 * o + jx] * A.lw[8 * o + 4 + jy];
            const double coef = A.w[o] * wgt;
            const double ux = A.ux_s[t], uy = A.uy_s[t];
            const double inv = A.inv_st[t];
            const double r = fma(stj, inv, -1.0);
            const double dx = (uxj - ux) * inv, dy = (uyj - uy) * inv;
            double gx[N1], gdx[N1], gy[N1], gdy[N1];
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                lag_taylor(L, k, a, fma(L.c[a], r, dx), gx[a], gdx[a]);
                lag_taylor(L, l, a, fma(L.c[a], r, dy), gy[a], gdy[a]);
            }
            double sux = 0.0, suy = 0.0, sst = 0.0;
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                const double cgx = coef * gx[a];
                double h = 0.0, hp = 0.0, hq = 0.0;
#pragma unroll
                for (int b = 0; b < N1; ++b) {
                    fb[N1 * a + b] = fma(cgx, gy[b], fb[N1 * a + b]);
                    const double fv = fj[N1 * a + b];
                    h = fma(gy[b], fv, h);
                    hp = fma(gdy[b], fv, hp);
                    hq = fma(gdy[b] * L.c[b], fv, hq);
                }
                sux = fma(gdx[a], h, sux);
                suy = fma(gx[a], hp, suy);
                sst = fma(gdx[a] * L.c[a], h, fma(gx[a], hq, sst));
            }
            // d xi / d(source u) = 1/s ; d xi / d(source s) = c / s
            const double ci = coef * inv;
            bux = fma(ci, sux, bux);
            buy = fma(ci, suy, buy);
            bst = fma(ci, sst, bst);
        }
    }
    // reduce over the warp (all populations and both halves): lanes 2p and
    // 2p + 1 get population p's total, every lane the gauge cotangents
    double v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = i < Q ? fb[i] : 0.0;
    const double tot = warp_reduce_scatter16(v, lane);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        bux += __shfl_xor_sync(0xffffffffu, bux, o);
        buy += __shfl_xor_sync(0xffffffffu, buy, o);
        bst += __shfl_xor_sync(0xffffffffu, bst, o);
    }
    const int p = lane >> 1;
    if ((lane & 1) == 0 && p < Q) A.fbar_in[(long long)p * A.N + src] = tot;
    if (lane == 1) {
        A.gbar_in[src] = bux;
        A.gbar_in[A.N + src] = buy;
        // s = sqrt(T / T_L): dL/dT = dL/ds / (2 s T_L)
        A.gbar_in[2 * A.N + src] = bst / (2.0 * stj * A.T_L);
    }
}

// The gather of the staged contexts takes the source-gauge derivatives out
// of the hit loop.  G(j -> t) = G(r -> t) G(j -> r) for any fixed r (the matched
// moments determine the populations), so with r held at the source's own
// gauge lambda_j,
//   d/dlambda_j [G(j -> t) f_j]_q = [G(r -> t) dG(j -> r)/dlambda_j f_j]_q,
// and summed over the hits (target t, population q) with their weights,
//   lambda_j_bar = sum_{a,b} h[a][b] (dG(j -> r)/dlambda_j f_j)[a][b],
//   h = sum_hits coef G(j -> t)[q, :]  (= the populations' cotangent f_j_bar).
// At r = lambda_j the map G(j -> r) is the identity and its derivatives are
// the constants L_k'(c_a) = d1[k][a] over s_j (x: d xi/d u = 1/s_j; s:
// d xi/d s = c_a/s_j).  A hit then needs only the two rows of G(j -> t) and a
// rank-one update, about a third of the direct gather's FP64 work.
//
// It is organised by target.  For a source j and a candidate
// target t, population (k, l) hits when j lies in both its x-stencil and its
// y-stencil; the x-stencil's origin depends on k alone and the y-stencil's
// on l alone, so the hits of (j, t) are a product set K x L.  The rows
// G(j -> t)_x[k][.] (k in K) and G_y[l][.] (l in L) are then evaluated once
// per target, not once per hit, and a hit costs its weight and a rank-one
// update.  Each round, every lane of the source's warp takes one candidate
// target and writes its gauge offsets and stencil positions to a
// shared-memory slot, its rows to a job queue and its hits to a hit queue
// (offsets by a warp prefix sum); the warp then evaluates the rows and does
// the hits 32 at a time.  Work per lane thus does not depend on how many
// rows and hits its own target has: the FP64 pipe serves full warps.
constexpr int ADJ_GATHER_WARPS = 2;

struct GatherSlot {
    double gx[4][4];   // G_x(j -> t)[k][a]
    double gy[4][4];   // G_y(j -> t)[l][b]
    double lx[4];      // x-weight of j in the stencil of x-speed k
    double ly[4];      // y-weight of j in the stencil of y-speed l
    double r, dx, dy;  // gauge offsets of j from t (r: s_j / s_t - 1)
    long long t;
    signed char jx[4], jy[4];  // j's position in the x- and y-stencils
};

template <int N1>
__global__ void __launch_bounds__(ADJ_GATHER_WARPS * 32) k_adjoint_sources_t(AdjArgs A) {
    constexpr int Q = N1 * N1;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ GatherSlot s_slot[ADJ_GATHER_WARPS][32];
    __shared__ unsigned short s_hit[ADJ_GATHER_WARPS][32 * Q];
    __shared__ unsigned short s_job[ADJ_GATHER_WARPS][32 * 2 * N1];
    const Lattice& L = c_La[lattice_slot(N1)];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long src = (long long)blockIdx.x * ADJ_GATHER_WARPS + wid;
    if (src >= A.N) return;  // warp-uniform
    const int JX = (int)(src % A.nx), JY = (int)(src / A.nx);
    const double uxj = A.in.ux[src], uyj = A.in.uy[src], stj = A.in.st[src];
    GatherSlot& my = s_slot[wid][lane];
    unsigned short* hitq = s_hit[wid];
    unsigned short* jobq = s_job[wid];

    // candidate targets: the union over the speeds of the windows of
    // k_adjoint_sources (J in the stencil of the target at x when
    // floor(x - v dt) is in [J - 2, J + 1], v within the speed's bounds)
    int xlo = 0x7fffffff, xhi = -0x7fffffff, ylo = 0x7fffffff, yhi = -0x7fffffff;
#pragma unroll
    for (int i = 0; i < N1; ++i) {
        const double ex = 1e-9 * (1.0 + fabs(A.vlo_x[i]) + fabs(A.vhi_x[i])) * A.dt;
        const double ey = 1e-9 * (1.0 + fabs(A.vlo_y[i]) + fabs(A.vhi_y[i])) * A.dt;
        xlo = min(xlo, (int)ceil(-2.0 + A.vlo_x[i] * A.dt - ex));
        xhi = max(xhi, (int)ceil(2.0 + A.vhi_x[i] * A.dt + ex) - 1);
        ylo = min(ylo, (int)ceil(-2.0 + A.vlo_y[i] * A.dt - ey));
        yhi = max(yhi, (int)ceil(2.0 + A.vhi_y[i] * A.dt + ey) - 1);
    }
    const int wx = xhi - xlo + 1;
    const int nc = wx * (yhi - ylo + 1);

    double fb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fb[i] = 0.0;
    for (int c0 = 0; c0 < nc; c0 += 32) {
        // 1. this lane's candidate: its hit set K x L and gauge offsets
        const int c = c0 + lane;
        unsigned kmask = 0u, lmask = 0u;
        if (c < nc) {
            const int xx = JX + xlo + c % wx, yy = JY + ylo + c / wx;
            const long long t = (long long)wrap_idx(yy, A.ny) * A.nx + wrap_idx(xx, A.nx);
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int jx = JX - (xx + A.org[(long long)(N1 * i) * A.N + t].x);
                const int jy = JY - (yy + A.org[(long long)i * A.N + t].y);
                my.jx[i] = (signed char)jx;
                my.jy[i] = (signed char)jy;
                kmask |= (jx >= 0 && jx <= 3) ? 1u << i : 0u;
                lmask |= (jy >= 0 && jy <= 3) ? 1u << i : 0u;
            }
            if (kmask && lmask) {
                my.t = t;
                const double inv = A.inv_st[t];
                my.r = fma(stj, inv, -1.0);
                my.dx = (uxj - A.ux_s[t]) * inv;
                my.dy = (uyj - A.uy_s[t]) * inv;
            } else {
                kmask = lmask = 0u;
            }
        }
        // 2. the round's row jobs and hits into the warp's queues: one scan
        //    of (jobs << 16 | hits)
        const int nk = __popc(kmask), nl = __popc(lmask);
        const int mine = ((nk + nl) << 16) | (nk * nl);
        int incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += v;
        }
        const int tot = __shfl_sync(FULL, incl, 31);
        const int ex = incl - mine;
        int hoff = ex & 0xffff, joff = ex >> 16;
        const int nhit = tot & 0xffff, njob = tot >> 16;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            if (!(kmask >> k & 1u)) continue;
            jobq[joff++] = (unsigned short)((lane << 3) | k);
#pragma unroll
            for (int l = 0; l < N1; ++l)
                if (lmask >> l & 1u) hitq[hoff++] = (unsigned short)((lane << 4) | (k << 2) | l);
        }
#pragma unroll
        for (int l = 0; l < N1; ++l)
            if (lmask >> l & 1u) jobq[joff++] = (unsigned short)((lane << 3) | 4 | l);
        __syncwarp();
        // 3. the rows on full warps: G_x[k][.] or G_y[l][.] and the weight
        for (int j = lane; j < njob; j += 32) {
            const unsigned code = jobq[j];
            GatherSlot& g = s_slot[wid][code >> 3];
            const int i = (int)code & 3;
            const bool yrow = (code & 4u) != 0;
            const double base = yrow ? g.dy : g.dx, r = g.r;
            double row[N1];
#pragma unroll
            for (int a = 0; a < N1; ++a)
                row[a] = gauge_poly<N1>(L.d3[i], L.d2[i][a], L.d1[i][a], a == i ? 1.0 : 0.0,
                                        fma(L.c[a], r, base));
            if (yrow) {
                g.ly[i] = A.lw[8 * ((long long)i * A.N + g.t) + 4 + g.jy[i]];
#pragma unroll
                for (int a = 0; a < N1; ++a) g.gy[i][a] = row[a];
            } else {
                g.lx[i] = A.lw[8 * ((long long)(N1 * i) * A.N + g.t) + g.jx[i]];
#pragma unroll
                for (int a = 0; a < N1; ++a) g.gx[i][a] = row[a];
            }
        }
        __syncwarp();
        // 4. the hits on full warps: weight, then the rank-one update
        for (int h = lane; h < nhit; h += 32) {
            const unsigned code = hitq[h];
            const GatherSlot& g = s_slot[wid][code >> 4];
            const int k = (int)(code >> 2) & 3, l = (int)code & 3;
            const double coef = A.w[(long long)(N1 * k + l) * A.N + g.t] * g.lx[k] * g.ly[l];
            double gy[N1];
#pragma unroll
            for (int b = 0; b < N1; ++b) gy[b] = g.gy[l][b];
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                const double cgx = coef * g.gx[k][a];
#pragma unroll
                for (int b = 0; b < N1; ++b) fb[N1 * a + b] = fma(cgx, gy[b], fb[N1 * a + b]);
            }
        }
        __syncwarp();  // the slots and the queues are rewritten next round
    }

    // reduce over the warp: lanes 2p and 2p + 1 get population p's total
    double v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = i < Q ? fb[i] : 0.0;
    const double tot = warp_reduce_scatter16(v, lane);
    // the source-gauge cotangent from h = fb, one population per even lane:
    // dg/du_x [k][l] = sum_a d1[k][a] f[a][l] / s_j, dg/du_y [k][l] =
    // sum_b d1[l][b] f[k][b] / s_j, dg/ds the same with c_a, c_b inside
    const int p = lane >> 1;
    double pux = 0.0, puy = 0.0, pst = 0.0;
    if ((lane & 1) == 0 && p < Q) {
        const int kk = p / N1, ll = p % N1;
        double gxu = 0.0, gyu = 0.0, gsx = 0.0, gsy = 0.0;
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            // the source's populations f_j[a][ll] and f_j[kk][a]
            const double fx = A.in.f[(long long)(N1 * a + ll) * A.N + src];
            const double fy = A.in.f[(long long)(N1 * kk + a) * A.N + src];
            gxu = fma(L.d1[kk][a], fx, gxu);
            gsx = fma(L.d1[kk][a] * L.c[a], fx, gsx);
            gyu = fma(L.d1[ll][a], fy, gyu);
            gsy = fma(L.d1[ll][a] * L.c[a], fy, gsy);
        }
        pux = tot * gxu;
        puy = tot * gyu;
        pst = tot * (gsx + gsy);
        A.fbar_in[(long long)p * A.N + src] = tot;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        pux += __shfl_xor_sync(FULL, pux, o);
        puy += __shfl_xor_sync(FULL, puy, o);
        pst += __shfl_xor_sync(FULL, pst, o);
    }
    if (lane == 0) {
        const double is = 1.0 / stj;
        A.gbar_in[src] = pux * is;
        A.gbar_in[A.N + src] = puy * is;
        // s = sqrt(T / T_L): dL/dT = dL/ds / (2 s T_L)
        A.gbar_in[2 * A.N + src] = pst * is / (2.0 * stj * A.T_L);
    }
}

// Bounds {min ux, max ux, min uy, max uy, min s, max s} of a gauge field,
// exact in FP64: a grid-stride pass, warp reductions, and 64-bit integer
// atomics on an order-preserving encoding of the doubles (one per warp and
// value), decoded in place into out6.
__device__ __forceinline__ unsigned long long d2ord(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void k_minmax3_reset(unsigned long long* o) {
    const int j = threadIdx.x;
    if (j < 6) o[j] = (j & 1) ? 0ull : ~0ull;
}

__global__ void k_minmax3(const double* __restrict__ ux, const double* __restrict__ uy,
                          const double* __restrict__ st, long long N, unsigned long long* o) {
    double v[6] = {1e300, -1e300, 1e300, -1e300, 1e300, -1e300};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const double a = ux[i], b = uy[i], c = st[i];
        v[0] = fmin(v[0], a);
        v[1] = fmax(v[1], a);
        v[2] = fmin(v[2], b);
        v[3] = fmax(v[3], b);
        v[4] = fmin(v[4], c);
        v[5] = fmax(v[5], c);
    }
    // warp, then block reduction: one atomic per block and value
    __shared__ double s_b[6][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const double u = __shfl_xor_sync(0xffffffffu, v[j], off);
                v[j] = (j & 1) ? fmax(v[j], u) : fmin(v[j], u);
            }
        if (pass == 1) break;
        if (lane == 0)
#pragma unroll
            for (int j = 0; j < 6; ++j) s_b[j][warp] = v[j];
        __syncthreads();
        if (warp != 0) return;
        const bool in = lane < (int)(blockDim.x >> 5);
#pragma unroll
        for (int j = 0; j < 6; ++j) v[j] = in ? s_b[j][lane] : ((j & 1) ? -1e300 : 1e300);
    }
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            if (j & 1) atomicMax(o + j, d2ord(v[j]));
            else atomicMin(o + j, d2ord(v[j]));
        }
}

__global__ void k_minmax3_decode(unsigned long long* o) {
    const int j = threadIdx.x;
    if (j < 6) {
        const unsigned long long u = o[j];
        const unsigned long long b = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
        reinterpret_cast<double*>(o)[j] = __longlong_as_double((long long)b);
    }
}

cudaError_t launch_minmax3(const double* ux, const double* uy, const double* st, long long N,
                           double* out6, cudaStream_t s) {
    unsigned long long* o = reinterpret_cast<unsigned long long*>(out6);
    k_minmax3_reset<<<1, 32, 0, s>>>(o);
    long long nb = (N + 255) / 256;
    if (nb > 256) nb = 256;
    if (nb < 1) nb = 1;
    k_minmax3<<<(unsigned)nb, 256, 0, s>>>(ux, uy, st, N, o);
    k_minmax3_decode<<<1, 32, 0, s>>>(o);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Phase A in the staged form of the forward step (pond_staged.cuh): the
// sources are re-expressed once per tile in a reference gauge lambda_r (the
// tile's centre node of the input state), g = G(s -> r) f_s, and for each
// target population (k, l)
//   A_q(lambda) = sum_b (I + Ey)[l][b] sum_jy ly[jy] P(jy)[b],
//   P(jy)[b]    = sum_a (I + Ex)[k][a] Fi[a][b],  Fi = sum_jx lx[jx] g(x0 + jx, y0 + jy),
// with Ex, Ey the maps r -> lambda.  Its tangents at lambda* follow term by
// term: the cubic weights move with the departure point (d t / d u = -dt,
// d t / d s = -c dt) and the maps with xi_a = (s_r c_a + u_r - u) / s
// (d xi / d u = -1/s, d xi / d s = -xi / s), so one sweep of the stencil rows
// gives A and its three tangents from the interpolated rows Fi and their
// weight derivatives Fd = sum_jx lx'[jx] g.  About a third of the FP64
// arithmetic of the per-(population, source) form.

struct StagedAdj64 {
    using Real = double;
    using Real4 = Double4;
    template <int N1>
    static __device__ __forceinline__ const Lattice& lat() {
        return c_La[lattice_slot(N1)];
    }
    static __device__ __forceinline__ void load4(const Real4* p, double (&v)[4]) {
        const double2 a = reinterpret_cast<const double2*>(p)[0];
        const double2 b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x;
        v[1] = a.y;
        v[2] = b.x;
        v[3] = b.y;
    }
    static __device__ __forceinline__ void store4(Real4* p, const double (&v)[4]) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
};

// L_k(c_a + de) - [k == a] in correction form, and L_k'(c_a + de).
__device__ __forceinline__ void lag_taylor_e(const Lattice& L, int k, int a, double de, double& e,
                                            double& gd) {
    const double d1 = L.d1[k][a], d2 = L.d2[k][a], d3 = L.d3[k];
    e = fma(fma(d3, de, d2), de, d1) * de;
    gd = fma(fma(3.0 * d3, de, 2.0 * d2), de, d1);
}

// One population's A and tangents in the direct form, read from global
// memory: for a stencil that leaves the staged window.
template <int N1>
__device__ __noinline__ void adj_population_direct(const AdjArgs& A, int X, int Y, int k, int l,
                                                   double ux, double uy, double st,
                                                   double* out4) {
    const Lattice& L = c_La[lattice_slot(N1)];
    const double ck = L.c[k], cl = L.c[l];
    const double inv = 1.0 / st;
    const double vx = fma(st, ck, ux), vy = fma(st, cl, uy);
    const double depx = (double)X - vx * A.dt, depy = (double)Y - vy * A.dt;
    const double flx = floor(depx), fly = floor(depy);
    double lx[4], dlx[4], ly[4], dly[4];
    lagrange4_d(depx - flx + 1.0, lx, dlx);
    lagrange4_d(depy - fly + 1.0, ly, dly);
    const int x0 = wrap_idx((long long)flx - 1, A.nx);
    const int y0 = wrap_idx((long long)fly - 1, A.ny);
    double Aq = 0.0, dAux = 0.0, dAuy = 0.0, dAst = 0.0;
    for (int jy = 0; jy < 4; ++jy) {
        const int sy = wrap_inc(y0, jy, A.ny);
        for (int jx = 0; jx < 4; ++jx) {
            const int sx = wrap_inc(x0, jx, A.nx);
            const long long s = (long long)sy * A.nx + sx;
            const double r = fma(A.in.st[s], inv, -1.0);
            const double dx = (A.in.ux[s] - ux) * inv;
            const double dy = (A.in.uy[s] - uy) * inv;
            double gx[N1], gdx[N1], gy[N1], gdy[N1], xix[N1], xiy[N1];
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                const double ex = fma(L.c[a], r, dx), ey = fma(L.c[a], r, dy);
                xix[a] = L.c[a] + ex;
                xiy[a] = L.c[a] + ey;
                lag_taylor(L, k, a, ex, gx[a], gdx[a]);
                lag_taylor(L, l, a, ey, gy[a], gdy[a]);
            }
            double g = 0.0, gux = 0.0, guy = 0.0, gst = 0.0;
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                double h = 0.0, hp = 0.0, hq = 0.0;
#pragma unroll
                for (int b = 0; b < N1; ++b) {
                    const double fv = A.in.f[(long long)(N1 * a + b) * A.N + s];
                    h = fma(gy[b], fv, h);
                    hp = fma(gdy[b], fv, hp);
                    hq = fma(gdy[b] * xiy[b], fv, hq);
                }
                g = fma(gx[a], h, g);
                gux = fma(gdx[a], h, gux);
                guy = fma(gx[a], hp, guy);
                gst = fma(gdx[a] * xix[a], h, fma(gx[a], hq, gst));
            }
            gux *= -inv;
            guy *= -inv;
            gst *= -inv;
            const double wx = lx[jx], dwx = dlx[jx], wy = ly[jy], dwy = dly[jy];
            const double a_w = wx * wy;
            const double da_ux = -A.dt * dwx * wy;
            const double da_uy = -A.dt * wx * dwy;
            const double da_st = -A.dt * (ck * dwx * wy + cl * wx * dwy);
            Aq = fma(a_w, g, Aq);
            dAux = fma(a_w, gux, fma(da_ux, g, dAux));
            dAuy = fma(a_w, guy, fma(da_uy, g, dAuy));
            dAst = fma(a_w, gst, fma(da_st, g, dAst));
        }
    }
    out4[0] = Aq;
    out4[1] = dAux;
    out4[2] = dAuy;
    out4[3] = dAst;
}

constexpr int ADJ_TY = 8;  // staged phase A tile: 32 x 8 targets (0.8 % faster than 32 x 4)

// Phase A, staged: A*, its tangents at lambda* into jvp[4][Q][N], the
// gather's per-(population, target) stencil origin and weights, and 1 / s*.
template <int N1>
__global__ void __launch_bounds__(32 * ADJ_TY, 1)
k_adjoint_jvp_staged(AdjArgs A, int wwa, int wha, double c_max, double* __restrict__ jvp) {
    constexpr int TX = 32, NT = TX * ADJ_TY, Q = N1 * N1;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    Double4* s_f = reinterpret_cast<Double4*>(smem_raw);  // [N1][WN]
    __shared__ float s_red[4][NT / 32];
    const Lattice& L = c_La[lattice_slot(N1)];
    const int WN = wwa * wha;
    const int tid = threadIdx.x;
    const int tiles_x = (A.nx + TX - 1) / TX;
    const int tx0 = (int)(blockIdx.x % tiles_x) * TX;
    const int ty0 = (int)(blockIdx.x / tiles_x) * ADJ_TY;
    const int X = tx0 + tid % TX, Y = ty0 + tid / TX;
    const bool valid = X < A.nx && Y < A.ny;
    const long long node = (long long)Y * A.nx + X;

    // reference gauge: the tile's centre node of the input state
    const long long rnode = (long long)min(ty0 + ADJ_TY / 2, A.ny - 1) * A.nx +
                            min(tx0 + TX / 2, A.nx - 1);
    const double rux = A.in.ux[rnode], ruy = A.in.uy[rnode], rst = A.in.st[rnode];

    double ux = 0.0, uy = 0.0, st = 1.0;
    float vxlo = 3.0e38f, vxhi = -3.0e38f, vylo = 3.0e38f, vyhi = -3.0e38f;
    if (valid) {
        ux = A.ux_s[node];
        uy = A.uy_s[node];
        st = A.st_s[node];
        const float sp = (float)(c_max * st);
        vxlo = (float)ux - sp;
        vxhi = (float)ux + sp;
        vylo = (float)uy - sp;
        vyhi = (float)uy + sp;
    }
    staged_block_minmax4<StagedAdj64, NT>(vxlo, vxhi, vylo, vyhi, s_red);
    const float m = 1.0f, fdt = (float)A.dt;
    const float bxl = fminf(fmaxf(vxlo, -1.0e6f), 1.0e6f), bxh = fminf(fmaxf(vxhi, -1.0e6f), 1.0e6f);
    const float byl = fminf(fmaxf(vylo, -1.0e6f), 1.0e6f), byh = fminf(fmaxf(vyhi, -1.0e6f), 1.0e6f);
    const int wx0 = (int)floorf((float)tx0 - bxh * fdt - m) - 1;
    const int wx1 = (int)floorf((float)(tx0 + TX - 1) - bxl * fdt + m) + 2;
    const int wy0 = (int)floorf((float)ty0 - byh * fdt - m) - 1;
    const int wy1 = (int)floorf((float)(ty0 + ADJ_TY - 1) - byl * fdt + m) + 2;
    const bool fin = isfinite(vxlo) && isfinite(vxhi) && isfinite(vylo) && isfinite(vyhi) &&
                     vxlo > -1.0e6f && vxhi < 1.0e6f && vylo > -1.0e6f && vyhi < 1.0e6f;
    const int ww = fin ? max(1, min(wx1 - wx0 + 1, wwa)) : 1;
    const int wh = fin ? max(1, min(wy1 - wy0 + 1, wha)) : 1;
    GridDesc G;
    G.nx = A.nx;
    G.ny = A.ny;
    G.offset = 0;
    G.ix0 = 0;
    G.iy0 = 0;
    G.iw = A.nx;
    G.ih = A.ny;
    stage_window<StagedAdj64, N1>(A.in, A.N, G, 0, wx0, wy0, ww, wh, WN, rux, ruy, rst, s_f,
                                  nullptr, tid, NT);
    __syncthreads();
    if (!valid) return;

    const double inv = 1.0 / st;
    A.inv_st[node] = inv;
    // offsets of the maps r -> lambda*
    const double rt = (rst - st) * inv, dxt = (rux - ux) * inv, dyt = (ruy - uy) * inv;
    const double dt = A.dt;
#pragma unroll 1
    for (int k = 0; k < N1; ++k) {
        const double ck = L.c[k];
        const double depx = (double)X - fma(st, ck, ux) * dt;
        const double flx = floor(depx);
        double lx[4], dlx[4];
        lagrange4_d(depx - flx + 1.0, lx, dlx);
        const int col = (int)flx - 1 - wx0;  // flx is the absolute departure floor
        double ex[N1], gdx[N1], gdxx[N1];
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            const double de = fma(L.c[a], rt, dxt);
            lag_taylor_e(L, k, a, de, ex[a], gdx[a]);
            gdxx[a] = gdx[a] * (L.c[a] + de);
        }
        const bool colok = col >= 0 && col + 3 < ww;
        // The y-speeds in pairs (l0, l0 + 1): one sweep over the union of
        // the pair's two y-stencils, so a row both stencils hold is
        // interpolated once.  Each row is taken one component b at a time
        // (Fi, Fd of that column of the staged rows), which keeps the two
        // populations' accumulators in registers; every sum runs in the
        // order of the single-population sweep, so the results are the same.
#pragma unroll 1
        for (int l0 = 0; l0 < N1; l0 += 2) {
            const int np = l0 + 1 < N1 ? 2 : 1;
            double ly[2][4], dly[2][4];
            int top[2] = {0, 0};
            bool in[2] = {false, false};
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                if (p >= np) break;
                const int l = l0 + p;
                const double depy = (double)Y - fma(st, L.c[l], uy) * dt;
                const double fly = floor(depy);
                lagrange4_d(depy - fly + 1.0, ly[p], dly[p]);
                top[p] = (int)fly - 1 - wy0;
                in[p] = colok && top[p] >= 0 && top[p] + 3 < wh;
                const long long o = (long long)(N1 * k + l) * A.N + node;
                A.org[o] = make_int2((int)((long long)flx - 1 - X), (int)((long long)fly - 1 - Y));
                double2* pw = reinterpret_cast<double2*>(A.lw + 8 * o);
                pw[0] = make_double2(lx[0], lx[1]);
                pw[1] = make_double2(lx[2], lx[3]);
                pw[2] = make_double2(ly[p][0], ly[p][1]);
                pw[3] = make_double2(ly[p][2], ly[p][3]);
            }
            double Z[2][N1], Zux[2][N1], Zuy[2][N1], Zs[2][N1];
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int b = 0; b < N1; ++b) Z[p][b] = Zux[p][b] = Zuy[p][b] = Zs[p][b] = 0.0;
            if (in[0] || in[1]) {
                const int r0 = in[0] && in[1] ? min(top[0], top[1]) : (in[0] ? top[0] : top[1]);
                const int r1 = (in[0] && in[1] ? max(top[0], top[1]) : (in[0] ? top[0] : top[1])) + 3;
#pragma unroll 1
                for (int row = r0; row <= r1; ++row) {
                    bool cov[2];
                    double w[2], dw[2];
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        const int j = row - top[p];
                        cov[p] = in[p] && j >= 0 && j < 4;
                        w[p] = j == 0 ? ly[p][0] : j == 1 ? ly[p][1] : j == 2 ? ly[p][2] : ly[p][3];
                        dw[p] = j == 0 ? dly[p][0] : j == 1 ? dly[p][1] : j == 2 ? dly[p][2] : dly[p][3];
                    }
                    if (!cov[0] && !cov[1]) continue;  // a gap between the two stencils
                    // the row's weights in the four accumulators, per population
                    double cwux[2], cwdy[2], cwi[2], cckwux[2], cclwdy[2];
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        cwux[p] = -dt * w[p];
                        cwdy[p] = -dt * dw[p];
                        cwi[p] = -w[p] * inv;
                        cckwux[p] = ck * cwux[p];
                        cclwdy[p] = L.c[l0 + p] * cwdy[p];
                    }
                    const Double4* src = s_f + row * ww + col;
#pragma unroll
                    for (int b = 0; b < N1; ++b) {
                        double Fi[N1], Fd[N1];
#pragma unroll
                        for (int a = 0; a < N1; ++a) Fi[a] = Fd[a] = 0.0;
#pragma unroll
                        for (int jx = 0; jx < 4; ++jx) {
#pragma unroll
                            for (int a = 0; a < N1; ++a) {
                                const double v =
                                    reinterpret_cast<const double*>(src + (size_t)a * WN + jx)[b];
                                Fi[a] = fma(lx[jx], v, Fi[a]);
                                Fd[a] = fma(dlx[jx], v, Fd[a]);
                            }
                        }
                        // the row's contributions: value, and the tangents
                        // through the x-weights (Fd), the x-map (gdx) and
                        // the row weight (dw)
                        // the identity part of the x-map, Fi[k] (k is a
                        // loop variable: taken by selection, in registers)
                        double P = Fi[0], P1 = Fd[0], Pd = 0.0, Pdx = 0.0;
#pragma unroll
                        for (int a = 1; a < N1; ++a) {
                            P = k == a ? Fi[a] : P;
                            P1 = k == a ? Fd[a] : P1;
                        }
#pragma unroll
                        for (int a = 0; a < N1; ++a) {
                            P = fma(ex[a], Fi[a], P);
                            P1 = fma(ex[a], Fd[a], P1);
                            Pd = fma(gdx[a], Fi[a], Pd);
                            Pdx = fma(gdxx[a], Fi[a], Pdx);
                        }
#pragma unroll
                        for (int p = 0; p < 2; ++p) {
                            if (!cov[p]) continue;
                            Z[p][b] = fma(w[p], P, Z[p][b]);
                            Zux[p][b] = fma(cwux[p], P1, fma(cwi[p], Pd, Zux[p][b]));
                            Zuy[p][b] = fma(cwdy[p], P, Zuy[p][b]);
                            Zs[p][b] = fma(cckwux[p], P1, fma(cwi[p], Pdx, fma(cclwdy[p], P, Zs[p][b])));
                        }
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                if (p >= np) break;
                const int l = l0 + p;
                const int q = N1 * k + l;
                double R[4];
                if (in[p]) {
                    // the y-map r -> lambda* and its derivatives; its
                    // identity part exactly
                    double Al = 0.0, Axl = 0.0, Ayl = 0.0, Asl = 0.0;
#pragma unroll
                    for (int b = 0; b < N1; ++b) {
                        const bool id = b == l;
                        Al += id ? Z[p][b] : 0.0;
                        Axl += id ? Zux[p][b] : 0.0;
                        Ayl += id ? Zuy[p][b] : 0.0;
                        Asl += id ? Zs[p][b] : 0.0;
                    }
                    double Ae = 0.0, Axe = 0.0, Aye = 0.0, Ase = 0.0, Dy = 0.0, Ds = 0.0;
#pragma unroll
                    for (int b = 0; b < N1; ++b) {
                        const double de = fma(L.c[b], rt, dyt);
                        double ey, gdy;
                        lag_taylor_e(L, l, b, de, ey, gdy);
                        Ae = fma(ey, Z[p][b], Ae);
                        Axe = fma(ey, Zux[p][b], Axe);
                        Aye = fma(ey, Zuy[p][b], Aye);
                        Ase = fma(ey, Zs[p][b], Ase);
                        Dy = fma(gdy, Z[p][b], Dy);
                        Ds = fma(gdy * (L.c[b] + de), Z[p][b], Ds);
                    }
                    R[0] = Al + Ae;
                    R[1] = Axl + Axe;
                    R[2] = fma(-inv, Dy, Ayl + Aye);
                    R[3] = fma(-inv, Ds, Asl + Ase);
                } else {
                    adj_population_direct<N1>(A, X, Y, k, l, ux, uy, st, R);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) jvp[((long long)i * Q + q) * A.N + node] = R[i];
            }
        }
    }
}

// The rest of phase A from A* and its tangents: the collision cotangent,
// beta_bar, the 3 x 3 implicit solve at the fixed point and w, one thread
// per target node.  Every sum the solve needs is linear in the populations'
// values, so the node's populations are read once and folded into running
// sums (tangent d^i, i = u_x, u_y, s; e_q = |c_q|^2 - 2 T_L):
//   rho = sum A_q,  wf = sum W_q fbar_q,  af = sum A_q fbar_q,
//   sk_i = sum c_k d^i_q,  sl_i = sum c_l d^i_q,  se_i = sum e_q d^i_q,
//   sf_i = sum fbar_q d^i_q,  s1_i = sum d^i_q.
// Then J = M_A A_lambda has rows (s/rho) sk, (s/rho) sl, s/(4 rho T_L) se;
// g_i = (1 - 2 beta) sf_i + 2 beta wf s1_i + lambdabar_i (the s component
// of lambdabar taken from T: dT/ds = 2 s T_L); betabar = 2 rho wf - 2 af;
// and w_q = Abar_q + (M_A^T mu)_q.
template <int N1>
__global__ void __launch_bounds__(256) k_adjoint_epilogue(AdjArgs A, const double* __restrict__ jvp) {
    constexpr int Q = N1 * N1;
    const Lattice& L = c_La[lattice_slot(N1)];
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = node < A.N;
    double bb = 0.0;
    if (valid) {
        const long long N = A.N;
        double rho = 0.0, wf = 0.0, af = 0.0;
        double sk[3], sl[3], se[3], sf[3], s1[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) sk[i] = sl[i] = se[i] = sf[i] = s1[i] = 0.0;
        double fb[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k = q / N1, l = q % N1;
            const double ck = L.c[k], cl = L.c[l];
            const double e = fma(ck, ck, cl * cl) - 2.0 * A.T_L;
            const double a = jvp[(long long)q * N + node];
            fb[q] = A.fbar[(long long)q * N + node];
            rho += a;
            wf = fma(L.w[k] * L.w[l], fb[q], wf);
            af = fma(a, fb[q], af);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double d = jvp[((long long)(1 + i) * Q + q) * N + node];
                sk[i] = fma(ck, d, sk[i]);
                sl[i] = fma(cl, d, sl[i]);
                se[i] = fma(e, d, se[i]);
                sf[i] = fma(fb[q], d, sf[i]);
                s1[i] += d;
            }
        }
        const double st = A.st_s[node];
        const double sr = st / rho, ss = st / (4.0 * rho * A.T_L);
        bb = 2.0 * (rho * wf - af);
        // J[m][i]: moment m (u_x, u_y, s), tangent i
        double J[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            J[0][i] = sr * sk[i];
            J[1][i] = sr * sl[i];
            J[2][i] = ss * se[i];
        }
        const double b1 = 1.0 - 2.0 * A.beta, b2 = 2.0 * A.beta * wf;
        const double g0 = fma(b1, sf[0], b2 * s1[0]) + A.gbar[node];
        const double g1 = fma(b1, sf[1], b2 * s1[1]) + A.gbar[N + node];
        const double g2 = fma(b1, sf[2], b2 * s1[2]) + A.gbar[2 * N + node] * 2.0 * st * A.T_L;
        // solve J^T mu = -g by Cramer's rule (a = J^T)
        const double a00 = J[0][0], a01 = J[1][0], a02 = J[2][0];
        const double a10 = J[0][1], a11 = J[1][1], a12 = J[2][1];
        const double a20 = J[0][2], a21 = J[1][2], a22 = J[2][2];
        const double det = a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) +
                           a02 * (a10 * a21 - a11 * a20);
        const double idet = 1.0 / det;
        const double r0 = -g0, r1 = -g1, r2 = -g2;
        const double mu0 = (r0 * (a11 * a22 - a12 * a21) - a01 * (r1 * a22 - a12 * r2) +
                            a02 * (r1 * a21 - a11 * r2)) * idet;
        const double mu1 = (a00 * (r1 * a22 - a12 * r2) - r0 * (a10 * a22 - a12 * a20) +
                            a02 * (a10 * r2 - r1 * a20)) * idet;
        const double mu2 = (a00 * (a11 * r2 - r1 * a21) - a01 * (a10 * r2 - r1 * a20) +
                            r0 * (a10 * a21 - a11 * a20)) * idet;
        const double m0 = sr * mu0, m1 = sr * mu1, m2 = ss * mu2;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k = q / N1, l = q % N1;
            const double ck = L.c[k], cl = L.c[l];
            const double e = fma(ck, ck, cl * cl) - 2.0 * A.T_L;
            A.w[(long long)q * N + node] = fma(b1, fb[q], b2) + fma(ck, m0, fma(cl, m1, e * m2));
        }
    }
    // beta_bar: one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bb += __shfl_xor_sync(0xffffffffu, bb, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(A.beta_bar, bb);
}

// Shared memory and launch of the staged phase A for a window of wwa x wha
// staged nodes (FP64 rows of 32 bytes).
cudaError_t launch_adjoint_phase_a_staged(const AdjArgs& A, int n1, int wwa, int wha, double c_max,
                                          double* jvp, cudaStream_t s) {
    static int s_set[64][2] = {{0}};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const size_t smem = (size_t)n1 * wwa * wha * sizeof(Double4);
    void (*kern)(AdjArgs, int, int, double, double*) =
        n1 == 3 ? k_adjoint_jvp_staged<3> : k_adjoint_jvp_staged<4>;
    int& set = s_set[dev][n1 == 3 ? 1 : 0];
    if ((int)smem > set) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set = (int)smem;
    }
    const unsigned tiles = (unsigned)(((A.nx + 31) / 32) * ((A.ny + ADJ_TY - 1) / ADJ_TY));
    kern<<<tiles, 32 * ADJ_TY, smem, s>>>(A, wwa, wha, c_max, jvp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)((A.N + 255) / 256);
    if (n1 == 3) k_adjoint_epilogue<3><<<nb, 256, 0, s>>>(A, jvp);
    else k_adjoint_epilogue<4><<<nb, 256, 0, s>>>(A, jvp);
    return cudaGetLastError();
}

template <int N1>
__global__ void k_rho_bar(const double* __restrict__ fbar, double* __restrict__ rbar, long long N) {
    const Lattice& L = c_La[lattice_slot(N1)];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < N1 * N1; ++q) r = fma(L.w[q / N1] * L.w[q % N1], fbar[q * N + i], r);
    rbar[i] = r;
}

}  // namespace pond

using namespace pond;

void destroy_adjoint(pond_ctx* ctx) {
    AdjointScratch* a = ctx->adj;
    if (!a) return;
    cudaFree(a->fwd.f);
    cudaFree(a->fwd.ux);
    cudaFree(a->fwd.uy);
    cudaFree(a->fwd.st);
    cudaFree(a->w);
    cudaFree(a->iters);
    cudaFree(a->stats);
    cudaFree(a->beta_bar);
    cudaFree(a->minmax);
    cudaFree(a->org);
    cudaFree(a->lw);
    cudaFree(a->inv_st);
    cudaFree(a->jvp);
    cudaFree(a->nu_dev);
    delete a;
    ctx->adj = nullptr;
}

static pond_status adj_fail(pond_ctx* ctx, cudaError_t e, const char* where) {
    ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();  // clear a non-sticky error (a failed allocation) for the next call
    return e == cudaErrorMemoryAllocation ? POND_ERR_OOM : POND_ERR_CUDA;
}

#define ACK(call, where)                                           \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return adj_fail(ctx, e_, where);    \
    } while (0)

namespace pond {

// The step's output gauge (u_x, u_y, T) given by the caller, stored as the
// scratch forward gauge (u_x, u_y, sqrt(T / T_L)), the form the forward step
// itself stores.
__global__ void k_gauge_from_T(const double* __restrict__ ux, const double* __restrict__ uy,
                               const double* __restrict__ T, double* __restrict__ ux_o,
                               double* __restrict__ uy_o, double* __restrict__ st_o, long long N,
                               double T_L) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        ux_o[i] = ux[i];
        uy_o[i] = uy[i];
        st_o[i] = sqrt(T[i] / T_L);
    }
}

cudaError_t launch_gauge_from_T(const double* ux, const double* uy, const double* T,
                                double* ux_o, double* uy_o, double* st_o, long long N,
                                double T_L, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    k_gauge_from_T<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(ux, uy, T, ux_o, uy_o, st_o, N, T_L);
    return cudaGetLastError();
}

}  // namespace pond

// d(loss)/d(nu) of one adjoint step from its beta cotangent on the device:
// beta = 1 / (2 nu / (T_ref dt) + 1)  =>  d beta / d nu = -2 beta^2 / (T_ref dt).
// To the host accumulator when one is given (a copy and a synchronisation),
// else to the context's device accumulator (stream-ordered, no
// synchronisation), which pond_adjoint_nu_bar reads.
__global__ void k_nu_accum(const double* __restrict__ beta_bar, double* __restrict__ nu_dev,
                           double dbeta_dnu) {
    if (threadIdx.x == 0) *nu_dev += *beta_bar * dbeta_dnu;
}

static cudaError_t accumulate_nu_bar(pond_ctx* ctx, AdjointScratch* a, double* nu_bar_accum) {
    const double beta = ctx->P.beta;
    const double dbeta = -2.0 * beta * beta / (ctx->cfg.T_ref * ctx->cfg.dt);
    if (!nu_bar_accum) {
        k_nu_accum<<<1, 32, 0, ctx->stream>>>(a->beta_bar, a->nu_dev, dbeta);
        return cudaGetLastError();
    }
    double bb = 0.0;
    cudaError_t e = cudaMemcpyAsync(&bb, a->beta_bar, sizeof(double), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) *nu_bar_accum += bb * dbeta;
    return e;
}

// Both entry points: out_gauge = {u_x, u_y, T} of the step's output when
// the caller has it (pond_adjoint_step_given), else NULLs and the forward
// step is recomputed here.
static pond_status adjoint_step_impl(pond_ctx* ctx, const double* const out_gauge[3],
                                     const void* f_bar_in, const void* gauge_bar_in,
                                     void* f_bar_out, void* gauge_bar_out,
                                     double* nu_bar_accum) {
    if (!ctx) return POND_ERR_ARG;
    if (!f_bar_in || !gauge_bar_in || !f_bar_out || !gauge_bar_out) {
        ctx->err = "adjoint: NULL argument";
        return POND_ERR_ARG;
    }
    if (ctx->n_grids != 1 || !ctx->cfg.thermal) {
        ctx->err = "adjoint: single-grid thermal contexts only";
        return POND_ERR_ARG;
    }
    if (!ctx->grid_set[0]) {
        ctx->err = "adjoint before pond_set_state";
        return POND_ERR_STATE;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    struct Restore {
        int p, d;
        ~Restore() {
            if (p >= 0 && p != d) cudaSetDevice(p);
        }
    } restore{prev, ctx->device};

    const int64_t N = ctx->N;
    const bool fp64 = ctx->cfg.precision == POND_FP64;
    if (!ctx->adj) {
        AdjointScratch* a = new AdjointScratch();
        ctx->adj = a;
        a->N = N;
        ACK(cudaMalloc(&a->beta_bar, sizeof(double)), "adjoint alloc");
        ACK(cudaMalloc(&a->nu_dev, sizeof(double)), "adjoint alloc");
        ACK(cudaMemsetAsync(a->nu_dev, 0, sizeof(double), ctx->stream), "adjoint alloc");
        ACK(cudaMalloc(&a->minmax, sizeof(double) * 6), "adjoint alloc");
        ACK(cudaMalloc(&a->org, sizeof(int2) * 16 * N), "adjoint alloc");
        ACK(cudaMalloc(&a->lw, sizeof(double) * 8 * 16 * N), "adjoint alloc");
        ACK(cudaMalloc(&a->inv_st, sizeof(double) * N), "adjoint alloc");
        if (fp64) {
            ACK(cudaMalloc(&a->fwd.f, sizeof(double) * 16 * N), "adjoint alloc");
            ACK(cudaMalloc(&a->fwd.ux, sizeof(double) * N), "adjoint alloc");
            ACK(cudaMalloc(&a->fwd.uy, sizeof(double) * N), "adjoint alloc");
            ACK(cudaMalloc(&a->fwd.st, sizeof(double) * N), "adjoint alloc");
            ACK(cudaMalloc(&a->w, sizeof(double) * 16 * N), "adjoint alloc");
            ACK(cudaMalloc(&a->iters, sizeof(int32_t) * N), "adjoint alloc");
            ACK(cudaMalloc(&a->stats, sizeof(DevStats)), "adjoint alloc");
        }
    }
    AdjointScratch* a = ctx->adj;
    if (!fp64) {
        // FP32 populations: pond_adjoint_mixed.cu
        ACK(adjoint_step_mixed(ctx, out_gauge, static_cast<const double*>(f_bar_in),
                               static_cast<const double*>(gauge_bar_in),
                               static_cast<double*>(f_bar_out), static_cast<double*>(gauge_bar_out),
                               a->beta_bar, a->minmax),
            "adjoint (mixed)");
        ACK(accumulate_nu_bar(ctx, a, nu_bar_accum), "adjoint nu cotangent");
        return POND_OK;
    }
    const GridDesc& G = ctx->grids_host[0];
    StateBuf<double> in;
    in.f = static_cast<double*>(ctx->f[ctx->cur]);
    in.ux = ctx->ux[ctx->cur];
    in.uy = ctx->uy[ctx->cur];
    in.st = ctx->st[ctx->cur];
    cudaStream_t s = ctx->stream;

    NvtxRange nv("pond_adjoint_step (FP64)");
    // 1. the fixed point lambda*: the gauge the forward step stores, given by
    //    the caller or recomputed into scratch
    if (out_gauge[0]) {
        ACK(launch_gauge_from_T(out_gauge[0], out_gauge[1], out_gauge[2], a->fwd.ux, a->fwd.uy,
                                a->fwd.st, N, ctx->L.T_L, s),
            "adjoint given gauge");
    } else {
        ACK(launch_ctx_step_fp64(ctx, in, a->fwd, a->iters, a->stats), "adjoint forward");
    }
    // 2. velocity bounds for the transpose gather
    ACK(launch_minmax3(a->fwd.ux, a->fwd.uy, a->fwd.st, N, a->minmax, s), "adjoint bounds");
    ACK(cudaMemcpyAsync(a->host_minmax, a->minmax, sizeof(double) * 6, cudaMemcpyDeviceToHost, s),
        "adjoint bounds copy");
    ACK(cudaMemsetAsync(a->beta_bar, 0, sizeof(double), s), "adjoint reset");
    ACK(cudaStreamSynchronize(s), "adjoint sync");

    AdjArgs A{};
    A.in = in;
    A.ux_s = a->fwd.ux;
    A.uy_s = a->fwd.uy;
    A.st_s = a->fwd.st;
    A.fbar = static_cast<const double*>(f_bar_in);
    A.gbar = static_cast<const double*>(gauge_bar_in);
    A.w = a->w;
    A.fbar_in = static_cast<double*>(f_bar_out);
    A.gbar_in = static_cast<double*>(gauge_bar_out);
    A.beta_bar = a->beta_bar;
    A.org = a->org;
    A.lw = a->lw;
    A.inv_st = a->inv_st;
    A.nx = G.nx;
    A.ny = G.ny;
    A.N = N;
    A.beta = ctx->P.beta;
    A.dt = ctx->P.dt;
    A.T_L = ctx->L.T_L;
    const double* mm = a->host_minmax;
    for (int i = 0; i < 4; ++i) {
        const double c = ctx->L.c[i];
        const double slo = c >= 0 ? c * mm[4] : c * mm[5];
        const double shi = c >= 0 ? c * mm[5] : c * mm[4];
        A.vlo_x[i] = slo + mm[0];
        A.vhi_x[i] = shi + mm[1];
        A.vlo_y[i] = slo + mm[2];
        A.vhi_y[i] = shi + mm[3];
    }
    const unsigned nb = (unsigned)((N + ADJ_WARPS - 1) / ADJ_WARPS);
    nvtxRangePushA("adjoint targets + transpose gather");
    if (ctx_staged(ctx)) {
        // phase A in the staged form: a window per 32 x 4 tile of targets
        // sized from the bounds of the particle velocities at lambda*
        if (!a->jvp) ACK(cudaMalloc(&a->jvp, sizeof(double) * 4 * 16 * N), "adjoint alloc");
        const double cm = ctx->L.c_max;
        const double sx = (mm[1] - mm[0]) + 2.0 * cm * mm[5];
        const double sy = (mm[3] - mm[2]) + 2.0 * cm * mm[5];
        int wwa = 32 + window_extent(sx, A.dt, 2.0) + 5;
        int wha = ADJ_TY + window_extent(sy, A.dt, 2.0) + 5;
        const size_t cap = 200 * 1024;
        while ((size_t)ctx->L.n1 * wwa * wha * sizeof(Double4) > cap) {
            if (wwa - 32 >= wha - ADJ_TY) --wwa; else --wha;
        }
        ACK(launch_adjoint_phase_a_staged(A, ctx->L.n1, wwa, wha, cm, a->jvp, s),
            "adjoint targets (staged)");
    } else {
        if (ctx->L.n1 == 3) k_adjoint_targets<3><<<nb, ADJ_WARPS * 32, 0, s>>>(A);
        else k_adjoint_targets<4><<<nb, ADJ_WARPS * 32, 0, s>>>(A);
    }
    ACK(cudaGetLastError(), "adjoint targets");
    if (ctx_staged(ctx)) {
        const unsigned nbt = (unsigned)((N + ADJ_GATHER_WARPS - 1) / ADJ_GATHER_WARPS);
        if (ctx->L.n1 == 3) k_adjoint_sources_t<3><<<nbt, ADJ_GATHER_WARPS * 32, 0, s>>>(A);
        else k_adjoint_sources_t<4><<<nbt, ADJ_GATHER_WARPS * 32, 0, s>>>(A);
    } else {
        if (ctx->L.n1 == 3) k_adjoint_sources<3><<<nb, ADJ_WARPS * 32, 0, s>>>(A);
        else k_adjoint_sources<4><<<nb, ADJ_WARPS * 32, 0, s>>>(A);
    }
    nvtxRangePop();
    ACK(cudaGetLastError(), "adjoint sources");
    ACK(accumulate_nu_bar(ctx, a, nu_bar_accum), "adjoint nu cotangent");
    return POND_OK;
}

extern "C" pond_status pond_adjoint_nu_bar(pond_ctx* ctx, double* nu_bar) {
    if (!ctx || !nu_bar) {
        if (ctx) ctx->err = "adjoint_nu_bar: NULL argument";
        return POND_ERR_ARG;
    }
    *nu_bar = 0.0;
    AdjointScratch* a = ctx->adj;
    if (!a) return POND_OK;
    DeviceGuard dg(ctx->device);
    ACK(cudaMemcpyAsync(nu_bar, a->nu_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
        "adjoint_nu_bar copy");
    ACK(cudaMemsetAsync(a->nu_dev, 0, sizeof(double), ctx->stream), "adjoint_nu_bar reset");
    ACK(cudaStreamSynchronize(ctx->stream), "adjoint_nu_bar sync");
    return POND_OK;
}

extern "C" pond_status pond_adjoint_step(pond_ctx* ctx, const void* f_bar_in,
                                         const void* gauge_bar_in, void* f_bar_out,
                                         void* gauge_bar_out, double* nu_bar_accum) {
    const double* none[3] = {nullptr, nullptr, nullptr};
    return adjoint_step_impl(ctx, none, f_bar_in, gauge_bar_in, f_bar_out, gauge_bar_out,
                             nu_bar_accum);
}

extern "C" pond_status pond_adjoint_step_given(pond_ctx* ctx, const void* ux_out,
                                               const void* uy_out, const void* T_out,
                                               const void* f_bar_in, const void* gauge_bar_in,
                                               void* f_bar_out, void* gauge_bar_out,
                                               double* nu_bar_accum) {
    if (!ctx) return POND_ERR_ARG;
    if (!ux_out || !uy_out || !T_out) {
        ctx->err = "adjoint: NULL output gauge";
        return POND_ERR_ARG;
    }
    const double* given[3] = {static_cast<const double*>(ux_out), static_cast<const double*>(uy_out),
                              static_cast<const double*>(T_out)};
    return adjoint_step_impl(ctx, given, f_bar_in, gauge_bar_in, f_bar_out, gauge_bar_out,
                             nu_bar_accum);
}

extern "C" pond_status pond_adjoint_init(pond_ctx* ctx, const void* f_bar, void* rho_bar) {
    if (!ctx) return POND_ERR_ARG;
    if (!f_bar || !rho_bar || ctx->n_grids != 1) {
        ctx->err = "adjoint_init: NULL argument or batched context";
        return POND_ERR_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    const long long N = ctx->N;
    const unsigned nb = (unsigned)((N + 255) / 256);
    if (ctx->L.n1 == 3)
        k_rho_bar<3><<<nb, 256, 0, ctx->stream>>>(static_cast<const double*>(f_bar),
                                                   static_cast<double*>(rho_bar), N);
    else
        k_rho_bar<4><<<nb, 256, 0, ctx->stream>>>(static_cast<const double*>(f_bar),
                                                   static_cast<double*>(rho_bar), N);
    const cudaError_t e = cudaGetLastError();
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return adj_fail(ctx, e, "adjoint_init");
    return POND_OK;
}
