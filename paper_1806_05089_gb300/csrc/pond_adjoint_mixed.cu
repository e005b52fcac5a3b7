// pond_adjoint_mixed.cu -- vector-Jacobian product of one PonD step for
// mixed-precision contexts (FP32 populations, FP64 gauges).
//
// Same mathematics as pond_adjoint.cu (implicit differentiation of the
// predictor-corrector fixed point, 3 x 3 solve per node, gather-form
// transpose of the reconstruction and gauge transform, BGK collision); the
// per-pair arithmetic runs in FP32.  Gauge differences u_s - u' are formed
// from per-node (hi, lo) FP32 splits of the FP64 gauges,
// (hi_s - hi') + (lo_s - lo'), which carries FP32 precision relative to the
// difference itself.  The per-node epilogue (sums, cotangents, 3 x 3 solve)
// runs in FP32 as well; only the beta cotangent is accumulated in FP64.
// Contexts on the staged forward kernel run the staged phase A with the
// epilogue fused (k_adjoint_jvp_staged_mixed) and the target-centric gather
// (k_adjoint_sources_mixed_t); contexts on the direct kernels the per-pair
// kernels (k_adjoint_targets_mixed, k_adjoint_sources_mixed).  Templated on
// the lattice like the FP64 adjoint.
#include <cmath>

#include "pond_device.cuh"
#include "pond_staged.cuh"

namespace pond {

// FP32 lattice constants of these kernels, slot lattice_slot(n1).
__constant__ LatticeF c_Lam[2];

cudaError_t upload_lattice_adjoint_mixed() {
    const LatticeF F[2] = {to_float(make_lattice(POND_D2Q16)), to_float(make_lattice(POND_D2Q9))};
    return cudaMemcpyToSymbol(c_Lam, F, sizeof(F));
}

struct AdjMixedScratch {
    StateBuf<float> fwd{};
    float* w = nullptr;       // [Q][N] (allocated for 16)
    float4* gin = nullptr;    // [2][N]: hi / lo splits of the input gauge (s, ux, uy, 0)
    float4* gstar = nullptr;  // [2][N]: hi / lo splits of lambda*
    int32_t* iters = nullptr;
    DevStats* stats = nullptr;
    float4* f4 = nullptr;     // [4][N] the input populations as rows f[a][0..n1-1]
    int2* org = nullptr;      // [16][N] stencil origin of (q, t), relative to t
    float* lw = nullptr;      // [16][N][8] cubic weights of (q, t): x 0..3, y 0..3
    float* inv_st = nullptr;  // [N] 1 / s* at every target
    float* vb = nullptr;      // [16] per-speed velocity bounds of lambda* (k_speed_bounds)
};

// Velocity bounds of every speed index from the bounds of lambda*
// (bounds6 = {min ux*, max ux*, min uy*, max uy*, min s*, max s*}, on the
// device), each widened by a slack for the FP32 departures (their rounding
// is ~1e-6 cells): vb = {vlo_x[4], vhi_x[4], vlo_y[4], vhi_y[4]}.  One
// thread, so the gathers need no host round trip for their candidate
// windows.
struct SpeedsD {
    double c[4];
};
__global__ void k_speed_bounds(const double* __restrict__ mm, SpeedsD sp, double slack,
                               float* __restrict__ vb) {
    if (threadIdx.x != 0) return;
    for (int i = 0; i < 4; ++i) {
        const double c = sp.c[i];
        const double slo = c >= 0 ? c * mm[4] : c * mm[5];
        const double shi = c >= 0 ? c * mm[5] : c * mm[4];
        vb[i] = (float)(slo + mm[0] - slack);
        vb[4 + i] = (float)(shi + mm[1] + slack);
        vb[8 + i] = (float)(slo + mm[2] - slack);
        vb[12 + i] = (float)(shi + mm[3] + slack);
    }
}

__global__ void k_split_gauge(const double* __restrict__ ux, const double* __restrict__ uy,
                              const double* __restrict__ st, float4* __restrict__ out,
                              long long N) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double v[3] = {st[i], ux[i], uy[i]};
    float hi[3], lo[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        hi[j] = (float)v[j];
        lo[j] = (float)(v[j] - (double)hi[j]);
    }
    out[i] = make_float4(hi[0], hi[1], hi[2], 0.0f);
    out[N + i] = make_float4(lo[0], lo[1], lo[2], 0.0f);
}

// Populations as rows: f4[a][i] = (f[n1 a][i], ..., f[n1 a + n1 - 1][i]) (a
// zero fourth word on D2Q9), so that a (population, source) pair reads a
// source's populations with n1 16-byte loads.
template <int N1>
__global__ void k_rows_f4(const float* __restrict__ f, float4* __restrict__ f4, long long N) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
#pragma unroll
    for (int a = 0; a < N1; ++a)
        f4[a * N + i] = make_float4(f[(N1 * a) * N + i], f[(N1 * a + 1) * N + i],
                                    f[(N1 * a + 2) * N + i],
                                    N1 == 4 ? f[(N1 * a + 3) * N + i] : 0.0f);
}

__device__ __forceinline__ void lagrange4_df(float t, float l[4], float dl[4]) {
    const float a = t, b = t - 1.0f, c = t - 2.0f, d = t - 3.0f;
    l[0] = -(b * c * d) * (1.0f / 6.0f);
    l[1] = (a * c * d) * 0.5f;
    l[2] = -(a * b * d) * 0.5f;
    l[3] = (a * b * c) * (1.0f / 6.0f);
    dl[0] = -(c * d + b * d + b * c) * (1.0f / 6.0f);
    dl[1] = (c * d + a * d + a * c) * 0.5f;
    dl[2] = -(b * d + a * d + a * b) * 0.5f;
    dl[3] = (b * c + a * c + a * b) * (1.0f / 6.0f);
}

// difference of two split values: (hi_a - hi_b) + (lo_a - lo_b)
__device__ __forceinline__ float sdiff(float ha, float la, float hb, float lb) {
    return (ha - hb) + (la - lb);
}

struct AdjMixedArgs {
    const float* f_in;       // input populations [Q][N]
    const float4* f4;        // the same as rows [n1][N]: f4[a][s] = f[a][0..n1-1] of s
    const float4* gin;       // splits of the input gauge
    const float4* gstar;     // splits of lambda*
    const double* st_in;     // input sqrt(theta) (FP64, for the T cotangent)
    const double* st_star;
    const double* fbar;      // [Q][N]
    const double* gbar;      // [3][N]
    float* w;                // [Q][N]
    double* fbar_in;
    double* gbar_in;
    double* beta_bar;
    // per (population, target), written by the target kernel for the gather:
    // stencil origin relative to the target, cubic weights, and 1 / s*
    int2* org;
    float* lw;
    float* inv_st;
    int nx, ny;
    long long N;
    float beta, dt, T_L;
    const float* vb;  // {vlo_x[4], vhi_x[4], vlo_y[4], vhi_y[4]} (device)
};

// One thread per node, a rolled loop over the populations: a warp holds 32
// consecutive nodes of one row, all on the same population, so the source
// reads of a (population, stencil node) step are 32 neighbouring 16-byte
// records (coalesced through L1) and the lattice constants of the population
// are warp-uniform.  All per-node sums are sequential in one thread.
constexpr int ADJM_THREADS = 128;

// lattice coefficients of the 1D Lagrange-Taylor map of speed index k
template <int N1>
struct RowCoef {
    float d1[N1], d2[N1], d3;
};

template <int N1>
__device__ __forceinline__ RowCoef<N1> row_coef(const LatticeF& L, int k) {
    RowCoef<N1> r;
#pragma unroll
    for (int a = 0; a < N1; ++a) {
        r.d1[a] = L.d1[k][a];
        r.d2[a] = L.d2[k][a];
    }
    r.d3 = L.d3[k];
    return r;
}

// G[k][a] = [k == a] + d1 de + d2 de^2 + d3 de^3 and its derivative in de
template <int N1>
__device__ __forceinline__ void lag_taylor_r(const RowCoef<N1>& R, int k, int a, float de,
                                             float& g, float& gd) {
    g = fmaf(fmaf(fmaf(R.d3, de, R.d2[a]), de, R.d1[a]), de, (k == a) ? 1.0f : 0.0f);
    gd = fmaf(fmaf(3.0f * R.d3, de, 2.0f * R.d2[a]), de, R.d1[a]);
}

template <int N1>
__global__ void __launch_bounds__(ADJM_THREADS) k_adjoint_targets_mixed(AdjMixedArgs A) {
    constexpr int Q = N1 * N1;
    const LatticeF& L = c_Lam[lattice_slot(N1)];
    const long long node0 = (long long)blockIdx.x * ADJM_THREADS + threadIdx.x;
    // threads past the end compute the last node and store nothing, so that
    // the warp reduction of the beta cotangent has all its lanes
    const bool live = node0 < A.N;
    const long long node = live ? node0 : A.N - 1;
    const int X = (int)(node % A.nx), Y = (int)(node / A.nx);
    const float4 th = A.gstar[node], tl = A.gstar[A.N + node];  // (s, ux, uy)
    const float st = th.x + tl.x, ux = th.y + tl.y, uy = th.z + tl.z;
    const float inv = 1.0f / st;
    const float T_L = A.T_L;
    if (live) A.inv_st[node] = inv;

    // Per node, over the populations q with A_q and its JVPs d_q = dA_q/dlambda:
    //   rho = sum A_q, sAf = sum A_q fb_q, wf = sum W_q fb_q,
    //   P{x,y,t}_j = sum {c_k, c_l, |c|^2 - 2 T_L} d_qj   (J = M_A A_lambda),
    //   gF_j = sum fb_q d_qj, gS_j = sum d_qj              (g = A_bar^T d)
    float rho = 0.0f, sAf = 0.0f, wf = 0.0f;
    float Px[3] = {0.0f, 0.0f, 0.0f}, Py[3] = {0.0f, 0.0f, 0.0f}, Pt[3] = {0.0f, 0.0f, 0.0f};
    float gF[3] = {0.0f, 0.0f, 0.0f}, gS[3] = {0.0f, 0.0f, 0.0f};

#pragma unroll 1
    for (int q = 0; q < Q; ++q) {
        const int k = q / N1, l = q - N1 * k;
        const float ck = L.c[k], cl = L.c[l];
        const RowCoef<N1> Rk = row_coef<N1>(L, k), Rl = row_coef<N1>(L, l);
        // departure of population q at lambda*, relative to the node
        const float frx = -fmaf(st, ck, ux) * A.dt, fry = -fmaf(st, cl, uy) * A.dt;
        const float flx = floorf(frx), fly = floorf(fry);
        float lx[4], dlx[4], ly[4], dly[4];
        lagrange4_df(frx - flx + 1.0f, lx, dlx);
        lagrange4_df(fry - fly + 1.0f, ly, dly);
        const int x0 = wrap_idx((long long)X + (long long)flx - 1, A.nx);
        const int y0 = wrap_idx((long long)Y + (long long)fly - 1, A.ny);
        const long long o = (long long)q * A.N + node;
        // what the gather needs of (q, target): the stencil origin relative
        // to the target and the cubic weights
        if (live) {
            A.org[o] = make_int2((int)flx - 1, (int)fly - 1);
            float4* pw = reinterpret_cast<float4*>(A.lw + 8 * o);
            pw[0] = make_float4(lx[0], lx[1], lx[2], lx[3]);
            pw[1] = make_float4(ly[0], ly[1], ly[2], ly[3]);
        }

        float Aq = 0.0f, dAux = 0.0f, dAuy = 0.0f, dAst = 0.0f;
        // stencil rows rolled (the loop body, four (population, source)
        // pairs, stays small in the instruction cache); the row's weights by
        // selection, which keeps ly / dly in registers
#pragma unroll 1
        for (int jy = 0; jy < 4; ++jy) {
            const int sy = wrap_inc(y0, jy, A.ny);
            const float wy = jy == 0 ? ly[0] : jy == 1 ? ly[1] : jy == 2 ? ly[2] : ly[3];
            const float dwy = jy == 0 ? dly[0] : jy == 1 ? dly[1] : jy == 2 ? dly[2] : dly[3];
#pragma unroll
            for (int jx = 0; jx < 4; ++jx) {
                const int sx = wrap_inc(x0, jx, A.nx);
                const long long s = (long long)sy * A.nx + sx;
                const float4 sh = A.gin[s], sl = A.gin[A.N + s];
                const float r = sdiff(sh.x, sl.x, th.x, tl.x) * inv;
                const float dx = sdiff(sh.y, sl.y, th.y, tl.y) * inv;
                const float dy = sdiff(sh.z, sl.z, th.z, tl.z) * inv;
                float gx[N1], gdx[N1], gy[N1], gdyx[N1], gdy[N1], xix[N1];
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    const float ex = fmaf(L.c[a], r, dx), ey = fmaf(L.c[a], r, dy);
                    xix[a] = L.c[a] + ex;
                    lag_taylor_r<N1>(Rk, k, a, ex, gx[a], gdx[a]);
                    lag_taylor_r<N1>(Rl, l, a, ey, gy[a], gdy[a]);
                    gdyx[a] = gdy[a] * (L.c[a] + ey);
                }
                float g = 0.0f, gux = 0.0f, guy = 0.0f, gst = 0.0f;
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    float h = 0.0f, hp = 0.0f, hq = 0.0f;
                    const float4 r4 = A.f4[(long long)a * A.N + s];  // one 16-byte load per row
                    const float fr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                    for (int b = 0; b < N1; ++b) {
                        const float fv = fr[b];
                        h = fmaf(gy[b], fv, h);
                        hp = fmaf(gdy[b], fv, hp);
                        hq = fmaf(gdyx[b], fv, hq);
                    }
                    g = fmaf(gx[a], h, g);
                    gux = fmaf(gdx[a], h, gux);
                    guy = fmaf(gx[a], hp, guy);
                    gst = fmaf(gdx[a] * xix[a], h, fmaf(gx[a], hq, gst));
                }
                gux *= -inv;
                guy *= -inv;
                gst *= -inv;
                const float wx = lx[jx], dwx = dlx[jx];
                const float a_w = wx * wy;
                const float da_ux = -A.dt * dwx * wy;
                const float da_uy = -A.dt * wx * dwy;
                const float da_st = -A.dt * (ck * dwx * wy + cl * wx * dwy);
                Aq = fmaf(a_w, g, Aq);
                dAux = fmaf(a_w, gux, fmaf(da_ux, g, dAux));
                dAuy = fmaf(a_w, guy, fmaf(da_uy, g, dAuy));
                dAst = fmaf(a_w, gst, fmaf(da_st, g, dAst));
            }
        }
        const float fb = (float)A.fbar[o];
        const float Wq = L.w[k] * L.w[l];
        const float mt = fmaf(ck, ck, cl * cl) - 2.0f * T_L;
        const float d[3] = {dAux, dAuy, dAst};
        rho += Aq;
        sAf = fmaf(Aq, fb, sAf);
        wf = fmaf(Wq, fb, wf);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Px[j] = fmaf(ck, d[j], Px[j]);
            Py[j] = fmaf(cl, d[j], Py[j]);
            Pt[j] = fmaf(mt, d[j], Pt[j]);
            gF[j] = fmaf(fb, d[j], gF[j]);
            gS[j] += d[j];
        }
    }

    // Per-node epilogue in FP32: the inputs (A, its gauge derivatives) are
    // FP32 already, and the 3 x 3 system is J = M_A A_lambda = -(I - Phi_lambda)
    // with Phi_lambda the contraction of the fixed-point iteration, close to
    // -I and well conditioned, so FP64 here (1/64 of the FP32 rate) would buy
    // nothing; only the beta cotangent is accumulated in FP64.
    // With A_bar_q = (1 - 2 beta) fb_q + 2 beta wf and the moment maps
    // mu_q = s* (c_k, c_l, (|c|^2 - 2 T_L) / (4 T_L)) / rho:
    const float sd = (float)A.st_star[node];
    const float beta = A.beta;
    const float irho = 1.0f / rho;
    const float sx = sd * irho, stt = sd * irho / (4.0f * T_L);
    float J[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        J[0][j] = sx * Px[j];
        J[1][j] = sx * Py[j];
        J[2][j] = stt * Pt[j];
    }
    const float c1 = 1.0f - 2.0f * beta, c2b = 2.0f * beta * wf;
    const float g0 = fmaf(c1, gF[0], c2b * gS[0]) + (float)A.gbar[node];
    const float g1 = fmaf(c1, gF[1], c2b * gS[1]) + (float)A.gbar[A.N + node];
    const float g2 = fmaf(c1, gF[2], c2b * gS[2]) + (float)A.gbar[2 * A.N + node] * 2.0f * sd * T_L;
    const float a00 = J[0][0], a01 = J[1][0], a02 = J[2][0];
    const float a10 = J[0][1], a11 = J[1][1], a12 = J[2][1];
    const float a20 = J[0][2], a21 = J[1][2], a22 = J[2][2];
    const float det = a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) +
                      a02 * (a10 * a21 - a11 * a20);
    const float idet = 1.0f / det;
    const float r0 = -g0, r1 = -g1, r2 = -g2;
    const float mu0 = (r0 * (a11 * a22 - a12 * a21) - a01 * (r1 * a22 - a12 * r2) +
                       a02 * (r1 * a21 - a11 * r2)) * idet;
    const float mu1 = (a00 * (r1 * a22 - a12 * r2) - r0 * (a10 * a22 - a12 * a20) +
                       a02 * (a10 * r2 - r1 * a20)) * idet;
    const float mu2 = (a00 * (a11 * r2 - r1 * a21) - a01 * (a10 * r2 - r1 * a20) +
                       r0 * (a10 * a21 - a11 * a20)) * idet;
    if (live) {
        const float m0 = sx * mu0, m1 = sx * mu1, m2 = stt * mu2;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k = q / N1, l = q % N1;
            const float ck = L.c[k], cl = L.c[l];
            const float mt = fmaf(ck, ck, cl * cl) - 2.0f * T_L;
            const long long o = (long long)q * A.N + node;
            const float Abar = fmaf(c1, (float)A.fbar[o], c2b);
            A.w[o] = fmaf(ck, m0, fmaf(cl, m1, fmaf(mt, m2, Abar)));
        }
    }
    // beta cotangent sum 2 (rho W_q - A_q) fb_q, reduced over the warp in FP64
    double bb = live ? 2.0 * ((double)rho * (double)wf - (double)sAf) : 0.0;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) bb += __shfl_xor_sync(0xffffffffu, bb, m);
    if ((threadIdx.x & 31) == 0) atomicAdd(A.beta_bar, bb);
}

template <int N1>
__global__ void __launch_bounds__(ADJM_THREADS) k_adjoint_sources_mixed(AdjMixedArgs A) {
    constexpr int Q = N1 * N1;
    const LatticeF& L = c_Lam[lattice_slot(N1)];
    const long long src0 = (long long)blockIdx.x * ADJM_THREADS + threadIdx.x;
    if (src0 >= A.N) return;  // no warp-wide operation follows
    const long long src = src0;
    const int JX = (int)(src % A.nx), JY = (int)(src / A.nx);
    float fj[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fj[i] = A.f_in[(long long)i * A.N + src];
    const float4 jh = A.gin[src], jl = A.gin[A.N + src];

    float fb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fb[i] = 0.0f;
    float bux = 0.0f, buy = 0.0f, bst = 0.0f;
#pragma unroll 1
    for (int q = 0; q < Q; ++q) {
        const int k = q / N1, l = q - N1 * k;
        const RowCoef<N1> Rk = row_coef<N1>(L, k), Rl = row_coef<N1>(L, l);
        // candidate targets: J is in the stencil of the target at x when
        // floor(x - v dt) is in [J - 2, J + 1], i.e. x in [J - 2 + v dt, J + 2 + v dt);
        // over v in [vlo, vhi] (the bounds carry a 1e-3-cell margin for the
        // FP32 departures) the integers x from ceil(J - 2 + vlo dt) to
        // ceil(J + 2 + vhi dt) - 1; the exact test below decides.
        // ceil(J + a) = J + ceil(a) for integer J, so the bounds are free of
        // the rounding of large coordinates, and the window's offsets from J
        // are the same for every thread.
        const int xlo = JX + (int)ceilf(-2.0f + A.vb[k] * A.dt);
        const int xhi = JX + (int)ceilf(2.0f + A.vb[4 + k] * A.dt) - 1;
        const int ylo = JY + (int)ceilf(-2.0f + A.vb[8 + l] * A.dt);
        const int yhi = JY + (int)ceilf(2.0f + A.vb[12 + l] * A.dt) - 1;
        // wrapped coordinates advance with the loop counters (one modulo
        // per population, not per candidate)
        const int tx0 = wrap_idx(xlo, A.nx);
        int ty = wrap_idx(ylo, A.ny);
        for (int yy = ylo; yy <= yhi; ++yy, ty = (ty + 1 == A.ny) ? 0 : ty + 1) {
            const long long row = (long long)ty * A.nx;
            int tx = tx0;
            for (int xx = xlo; xx <= xhi; ++xx, tx = (tx + 1 == A.nx) ? 0 : tx + 1) {
                const long long t = row + tx;
                // the target's stencil origin for population q, as the
                // target kernel found it
                const long long o = (long long)q * A.N + t;
                const int2 og = A.org[o];
                const int jx = JX - (xx + og.x), jy = JY - (yy + og.y);
                if (jx < 0 || jx > 3 || jy < 0 || jy > 3) continue;
                const float4 th = A.gstar[t], tl = A.gstar[A.N + t];
                const float wgt = A.lw[8 * o + jx] * A.lw[8 * o + 4 + jy];
                const float coef = A.w[o] * wgt;
                const float inv = A.inv_st[t];
                const float r = sdiff(jh.x, jl.x, th.x, tl.x) * inv;
                const float dx = sdiff(jh.y, jl.y, th.y, tl.y) * inv;
                const float dy = sdiff(jh.z, jl.z, th.z, tl.z) * inv;
                float gx[N1], gdx[N1], gy[N1], gdy[N1];
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    lag_taylor_r<N1>(Rk, k, a, fmaf(L.c[a], r, dx), gx[a], gdx[a]);
                    lag_taylor_r<N1>(Rl, l, a, fmaf(L.c[a], r, dy), gy[a], gdy[a]);
                }
                float sux = 0.0f, suy = 0.0f, sst = 0.0f;
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    const float cgx = coef * gx[a];
                    float h = 0.0f, hp = 0.0f, hq = 0.0f;
#pragma unroll
                    for (int b = 0; b < N1; ++b) {
                        fb[N1 * a + b] = fmaf(cgx, gy[b], fb[N1 * a + b]);
                        const float fv = fj[N1 * a + b];
                        h = fmaf(gy[b], fv, h);
                        hp = fmaf(gdy[b], fv, hp);
                        hq = fmaf(gdy[b] * L.c[b], fv, hq);
                    }
                    sux = fmaf(gdx[a], h, sux);
                    suy = fmaf(gx[a], hp, suy);
                    sst = fmaf(gdx[a] * L.c[a], h, fmaf(gx[a], hq, sst));
                }
                const float ci = coef * inv;
                bux = fmaf(ci, sux, bux);
                buy = fmaf(ci, suy, buy);
                bst = fmaf(ci, sst, bst);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) A.fbar_in[(long long)i * A.N + src] = (double)fb[i];
    A.gbar_in[src] = (double)bux;
    A.gbar_in[A.N + src] = (double)buy;
    A.gbar_in[2 * A.N + src] = (double)bst / (2.0 * A.st_in[src] * (double)A.T_L);
}

// The gather of the staged contexts (see k_adjoint_sources_t in
// pond_adjoint.cu): the source-gauge derivatives are taken out of the hit
// loop (G(j -> t) = G(r -> t) G(j -> r) with r held at the source's gauge),
// and the gather is organised by target: the hits of a (source, target)
// pair are a product set K x L, since the x-stencil's origin depends on the
// x-speed alone and the y-stencil's on the y-speed alone.  Each thread walks the union of its
// source's candidate windows once, evaluates a hit target's rows G_x[k][.]
// (k in K) and G_y[l][.] (l in L) once, then does each hit's weight and
// rank-one update.
template <int N1>
__global__ void __launch_bounds__(ADJM_THREADS, 5)  // 5 CTAs per SM: measured 2 % faster than 4
k_adjoint_sources_mixed_t(AdjMixedArgs A) {
    constexpr int Q = N1 * N1;
    const LatticeF& L = c_Lam[lattice_slot(N1)];
    const long long src0 = (long long)blockIdx.x * ADJM_THREADS + threadIdx.x;
    if (src0 >= A.N) return;  // no warp-wide operation follows
    const long long src = src0;
    const int JX = (int)(src % A.nx), JY = (int)(src / A.nx);
    float fj[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fj[i] = A.f_in[(long long)i * A.N + src];
    const float4 jh = A.gin[src], jl = A.gin[A.N + src];

    float fb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fb[i] = 0.0f;
    float bux = 0.0f, buy = 0.0f, bst = 0.0f;
    // the union over the speeds of the candidate windows of
    // k_adjoint_sources_mixed (bounds with the FP32 departures' margin)
    int wxl = 0x7fffffff, wxh = -0x7fffffff, wyl = 0x7fffffff, wyh = -0x7fffffff;
#pragma unroll
    for (int i = 0; i < N1; ++i) {
        wxl = min(wxl, (int)ceilf(-2.0f + A.vb[i] * A.dt));
        wxh = max(wxh, (int)ceilf(2.0f + A.vb[4 + i] * A.dt) - 1);
        wyl = min(wyl, (int)ceilf(-2.0f + A.vb[8 + i] * A.dt));
        wyh = max(wyh, (int)ceilf(2.0f + A.vb[12 + i] * A.dt) - 1);
    }
    const int xlo = JX + wxl, xhi = JX + wxh, ylo = JY + wyl, yhi = JY + wyh;
    const int tx0 = wrap_idx(xlo, A.nx);
    int ty = wrap_idx(ylo, A.ny);
    for (int yy = ylo; yy <= yhi; ++yy, ty = (ty + 1 == A.ny) ? 0 : ty + 1) {
        const long long row = (long long)ty * A.nx;
        int tx = tx0;
        for (int xx = xlo; xx <= xhi; ++xx, tx = (tx + 1 == A.nx) ? 0 : tx + 1) {
            const long long t = row + tx;
            int jx[N1], jy[N1];
            unsigned kmask = 0u, lmask = 0u;
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                jx[i] = JX - (xx + A.org[(long long)(N1 * i) * A.N + t].x);
                jy[i] = JY - (yy + A.org[(long long)i * A.N + t].y);
                kmask |= (jx[i] >= 0 && jx[i] <= 3) ? 1u << i : 0u;
                lmask |= (jy[i] >= 0 && jy[i] <= 3) ? 1u << i : 0u;
            }
            if (!kmask || !lmask) continue;
            const float4 th = A.gstar[t], tl = A.gstar[A.N + t];
            const float inv = A.inv_st[t];
            const float r = sdiff(jh.x, jl.x, th.x, tl.x) * inv;
            const float dx = sdiff(jh.y, jl.y, th.y, tl.y) * inv;
            const float dy = sdiff(jh.z, jl.z, th.z, tl.z) * inv;
            float gx[N1][N1], gy[N1][N1], lxs[N1], lys[N1];
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                lxs[k] = 0.0f;
                if (!(kmask >> k & 1u)) continue;
                lxs[k] = A.lw[8 * ((long long)(N1 * k) * A.N + t) + jx[k]];
#pragma unroll
                for (int a = 0; a < N1; ++a)
                    gx[k][a] = gauge_poly<N1>(L.d3[k], L.d2[k][a], L.d1[k][a], a == k ? 1.0f : 0.0f,
                                              fmaf(L.c[a], r, dx));
            }
#pragma unroll
            for (int l = 0; l < N1; ++l) {
                lys[l] = 0.0f;
                if (!(lmask >> l & 1u)) continue;
                lys[l] = A.lw[8 * ((long long)l * A.N + t) + 4 + jy[l]];
#pragma unroll
                for (int b = 0; b < N1; ++b)
                    gy[l][b] = gauge_poly<N1>(L.d3[l], L.d2[l][b], L.d1[l][b], b == l ? 1.0f : 0.0f,
                                              fmaf(L.c[b], r, dy));
            }
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                if (!(kmask >> k & 1u)) continue;
#pragma unroll
                for (int l = 0; l < N1; ++l) {
                    if (!(lmask >> l & 1u)) continue;
                    const float coef = A.w[(long long)(N1 * k + l) * A.N + t] * (lxs[k] * lys[l]);
#pragma unroll
                    for (int a = 0; a < N1; ++a) {
                        const float cgx = coef * gx[k][a];
#pragma unroll
                        for (int b = 0; b < N1; ++b) fb[N1 * a + b] = fmaf(cgx, gy[l][b], fb[N1 * a + b]);
                    }
                }
            }
        }
    }
    // the source-gauge cotangent from fb (= h, the populations' cotangent in
    // the frame r = lambda_j): dg/du_x [k][l] = sum_a d1[k][a] f[a][l] / s_j,
    // dg/du_y [k][l] = sum_b d1[l][b] f[k][b] / s_j, dg/ds with c_a, c_b inside
    {
        const float is = (float)(1.0 / A.st_in[src]);
#pragma unroll
        for (int kk = 0; kk < N1; ++kk)
#pragma unroll
            for (int ll = 0; ll < N1; ++ll) {
                float gxu = 0.0f, gyu = 0.0f, gsx = 0.0f, gsy = 0.0f;
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    gxu = fmaf(L.d1[kk][a], fj[N1 * a + ll], gxu);
                    gsx = fmaf(L.d1[kk][a] * L.c[a], fj[N1 * a + ll], gsx);
                    gyu = fmaf(L.d1[ll][a], fj[N1 * kk + a], gyu);
                    gsy = fmaf(L.d1[ll][a] * L.c[a], fj[N1 * kk + a], gsy);
                }
                const float h = fb[N1 * kk + ll];
                bux = fmaf(h, gxu * is, bux);
                buy = fmaf(h, gyu * is, buy);
                bst = fmaf(h, (gsx + gsy) * is, bst);
            }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) A.fbar_in[(long long)i * A.N + src] = (double)fb[i];
    A.gbar_in[src] = (double)bux;
    A.gbar_in[A.N + src] = (double)buy;
    A.gbar_in[2 * A.N + src] = (double)bst / (2.0 * A.st_in[src] * (double)A.T_L);
}

// ---------------------------------------------------------------------------
// Phase A in the staged form (the FP64 counterpart is k_adjoint_jvp_staged in
// pond_adjoint.cu): the window of sources a 32 x 4 tile of targets can reach
// is staged once in the tile's reference gauge lambda_r (FP32 rows, the
// forward step's own staging), and each population's A* and its three
// tangents come from one pass over its four stencil rows: the rows
// interpolated with the cubic weights (Fi) and with their derivatives (Fd),
// the x-map r -> lambda* applied, the y-map after.  The per-node epilogue of
// k_adjoint_targets_mixed follows in the same thread (running sums over the
// populations, the 3 x 3 solve, w, the beta cotangent), so A* and its
// tangents never leave registers.

struct StagedAdj32 {
    using Real = float;
    using Real4 = float4;
    template <int N1>
    static __device__ __forceinline__ const LatticeF& lat() {
        return c_Lam[lattice_slot(N1)];
    }
    static __device__ __forceinline__ void store4(float4* p, const float (&v)[4]) {
        *p = make_float4(v[0], v[1], v[2], v[3]);
    }
};

constexpr int ADJM_TY = 4;  // staged phase A tile: 32 x 4 targets

// L_k(c_a + de) - [k == a] in correction form, and L_k'(c_a + de)
__device__ __forceinline__ void lag_taylor_ef(const LatticeF& L, int k, int a, float de, float& e,
                                              float& gd) {
    const float d1 = L.d1[k][a], d2 = L.d2[k][a], d3 = L.d3[k];
    e = fmaf(fmaf(d3, de, d2), de, d1) * de;
    gd = fmaf(fmaf(3.0f * d3, de, 2.0f * d2), de, d1);
}

// One population's A and tangents in the per-pair form, read from global
// memory (the pair loop of k_adjoint_targets_mixed): for a stencil that
// leaves the staged window.  th, tl: splits of lambda* at the target.
template <int N1>
__device__ __noinline__ void adj_population_direct_mixed(const AdjMixedArgs& A, int X, int Y, int k,
                                                         int l, float4 th, float4 tl, float st,
                                                         float ux, float uy, float inv,
                                                         float* out4) {
    const LatticeF& L = c_Lam[lattice_slot(N1)];
    const float ck = L.c[k], cl = L.c[l];
    const RowCoef<N1> Rk = row_coef<N1>(L, k), Rl = row_coef<N1>(L, l);
    const float frx = -fmaf(st, ck, ux) * A.dt, fry = -fmaf(st, cl, uy) * A.dt;
    const float flx = floorf(frx), fly = floorf(fry);
    float lx[4], dlx[4], ly[4], dly[4];
    lagrange4_df(frx - flx + 1.0f, lx, dlx);
    lagrange4_df(fry - fly + 1.0f, ly, dly);
    const int x0 = wrap_idx((long long)X + (long long)flx - 1, A.nx);
    const int y0 = wrap_idx((long long)Y + (long long)fly - 1, A.ny);
    float Aq = 0.0f, dAux = 0.0f, dAuy = 0.0f, dAst = 0.0f;
    for (int jy = 0; jy < 4; ++jy) {
        const int sy = wrap_inc(y0, jy, A.ny);
        for (int jx = 0; jx < 4; ++jx) {
            const int sx = wrap_inc(x0, jx, A.nx);
            const long long s = (long long)sy * A.nx + sx;
            const float4 sh = A.gin[s], sl = A.gin[A.N + s];
            const float r = sdiff(sh.x, sl.x, th.x, tl.x) * inv;
            const float dx = sdiff(sh.y, sl.y, th.y, tl.y) * inv;
            const float dy = sdiff(sh.z, sl.z, th.z, tl.z) * inv;
            float gx[N1], gdx[N1], gy[N1], gdyx[N1], gdy[N1], xix[N1];
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                const float ex = fmaf(L.c[a], r, dx), ey = fmaf(L.c[a], r, dy);
                xix[a] = L.c[a] + ex;
                lag_taylor_r<N1>(Rk, k, a, ex, gx[a], gdx[a]);
                lag_taylor_r<N1>(Rl, l, a, ey, gy[a], gdy[a]);
                gdyx[a] = gdy[a] * (L.c[a] + ey);
            }
            float g = 0.0f, gux = 0.0f, guy = 0.0f, gst = 0.0f;
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                float h = 0.0f, hp = 0.0f, hq = 0.0f;
                const float4 r4 = A.f4[(long long)a * A.N + s];
                const float fr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                for (int b = 0; b < N1; ++b) {
                    h = fmaf(gy[b], fr[b], h);
                    hp = fmaf(gdy[b], fr[b], hp);
                    hq = fmaf(gdyx[b], fr[b], hq);
                }
                g = fmaf(gx[a], h, g);
                gux = fmaf(gdx[a], h, gux);
                guy = fmaf(gx[a], hp, guy);
                gst = fmaf(gdx[a] * xix[a], h, fmaf(gx[a], hq, gst));
            }
            gux *= -inv;
            guy *= -inv;
            gst *= -inv;
            const float wx = lx[jx], dwx = dlx[jx], wy = ly[jy], dwy = dly[jy];
            const float a_w = wx * wy;
            Aq = fmaf(a_w, g, Aq);
            dAux = fmaf(a_w, gux, fmaf(-A.dt * dwx * wy, g, dAux));
            dAuy = fmaf(a_w, guy, fmaf(-A.dt * wx * dwy, g, dAuy));
            dAst = fmaf(a_w, gst, fmaf(-A.dt * (ck * dwx * wy + cl * wx * dwy), g, dAst));
        }
    }
    out4[0] = Aq;
    out4[1] = dAux;
    out4[2] = dAuy;
    out4[3] = dAst;
}

// Phase A, staged, with the per-node epilogue: writes w, the gather's
// per-(population, target) stencil origin and weights, 1 / s*, and adds the
// beta cotangent.  in: the step's input state; ux_star / uy_star (and
// A.st_star): lambda* in FP64; wwa x wha: the window capacity.
template <int N1>
__global__ void __launch_bounds__(32 * ADJM_TY, 3)  // 3 CTAs per SM: measured 2 % faster than 2
k_adjoint_jvp_staged_mixed(AdjMixedArgs A, StateBuf<float> in, const double* __restrict__ ux_star,
                           const double* __restrict__ uy_star, int wwa, int wha, float c_max) {
    constexpr int TX = 32, NT = TX * ADJM_TY, Q = N1 * N1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* s_f = reinterpret_cast<float4*>(smem_raw);  // [N1][WN]
    __shared__ float s_red[4][NT / 32];
    const LatticeF& L = c_Lam[lattice_slot(N1)];
    const int WN = wwa * wha;
    const int tid = threadIdx.x;
    const int tiles_x = (A.nx + TX - 1) / TX;
    const int tx0 = (int)(blockIdx.x % tiles_x) * TX;
    const int ty0 = (int)(blockIdx.x / tiles_x) * ADJM_TY;
    const int X = tx0 + tid % TX, Y = ty0 + tid / TX;
    const bool valid = X < A.nx && Y < A.ny;
    const long long node = (long long)Y * A.nx + X;

    // reference gauge: the tile's centre node of the input state
    const long long rnode = (long long)min(ty0 + ADJM_TY / 2, A.ny - 1) * A.nx +
                            min(tx0 + TX / 2, A.nx - 1);
    const double rux = in.ux[rnode], ruy = in.uy[rnode], rst = in.st[rnode];

    double uxd = 0.0, uyd = 0.0, sdd = 1.0;
    float vxlo = 3.0e38f, vxhi = -3.0e38f, vylo = 3.0e38f, vyhi = -3.0e38f;
    if (valid) {
        uxd = ux_star[node];
        uyd = uy_star[node];
        sdd = A.st_star[node];
        const float sp = c_max * (float)sdd;
        vxlo = (float)uxd - sp;
        vxhi = (float)uxd + sp;
        vylo = (float)uyd - sp;
        vyhi = (float)uyd + sp;
    }
    staged_block_minmax4<StagedAdj32, NT>(vxlo, vxhi, vylo, vyhi, s_red);
    const float m = 1.0f, fdt = A.dt;
    const float bxl = fminf(fmaxf(vxlo, -1.0e6f), 1.0e6f), bxh = fminf(fmaxf(vxhi, -1.0e6f), 1.0e6f);
    const float byl = fminf(fmaxf(vylo, -1.0e6f), 1.0e6f), byh = fminf(fmaxf(vyhi, -1.0e6f), 1.0e6f);
    const int wx0 = (int)floorf((float)tx0 - bxh * fdt - m) - 1;
    const int wx1 = (int)floorf((float)(tx0 + TX - 1) - bxl * fdt + m) + 2;
    const int wy0 = (int)floorf((float)ty0 - byh * fdt - m) - 1;
    const int wy1 = (int)floorf((float)(ty0 + ADJM_TY - 1) - byl * fdt + m) + 2;
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
    stage_window<StagedAdj32, N1>(in, A.N, G, 0, wx0, wy0, ww, wh, WN, rux, ruy, rst, s_f, nullptr,
                                  tid, NT);
    __syncthreads();

    double bb = 0.0;
    if (valid) {
        const float st = (float)sdd, ux = (float)uxd, uy = (float)uyd;
        const float inv = 1.0f / st;
        A.inv_st[node] = inv;
        // offsets of the maps r -> lambda*, formed in FP64 and rounded once
        const double invd = 1.0 / sdd;
        const float rt = (float)((rst - sdd) * invd);
        const float dxt = (float)((rux - uxd) * invd);
        const float dyt = (float)((ruy - uyd) * invd);
        const float4 th = A.gstar[node], tl = A.gstar[A.N + node];
        const float dt = A.dt, T_L = A.T_L;
        // running sums of the epilogue (k_adjoint_targets_mixed)
        float rho = 0.0f, sAf = 0.0f, wf = 0.0f;
        float Px[3] = {0.0f, 0.0f, 0.0f}, Py[3] = {0.0f, 0.0f, 0.0f}, Pt[3] = {0.0f, 0.0f, 0.0f};
        float gF[3] = {0.0f, 0.0f, 0.0f}, gS[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const float ck = L.c[k];
            const float frx = -fmaf(st, ck, ux) * dt;
            const float flx = floorf(frx);
            float lx[4], dlx[4];
            lagrange4_df(frx - flx + 1.0f, lx, dlx);
            const int col = X + (int)flx - 1 - wx0;
            float ex[N1], gdx[N1], gdxx[N1];
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                const float de = fmaf(L.c[a], rt, dxt);
                lag_taylor_ef(L, k, a, de, ex[a], gdx[a]);
                gdxx[a] = gdx[a] * (L.c[a] + de);
            }
#pragma unroll 1
            for (int l = 0; l < N1; ++l) {
                const float cl = L.c[l];
                const float fry = -fmaf(st, cl, uy) * dt;
                const float fly = floorf(fry);
                float ly[4], dly[4];
                lagrange4_df(fry - fly + 1.0f, ly, dly);
                const int top = Y + (int)fly - 1 - wy0;
                const int q = N1 * k + l;
                const long long o = (long long)q * A.N + node;
                A.org[o] = make_int2((int)flx - 1, (int)fly - 1);
                float4* pw = reinterpret_cast<float4*>(A.lw + 8 * o);
                pw[0] = make_float4(lx[0], lx[1], lx[2], lx[3]);
                pw[1] = make_float4(ly[0], ly[1], ly[2], ly[3]);
                float R[4];
                if (col >= 0 && col + 3 < ww && top >= 0 && top + 3 < wh) {
                    float Z[N1], Zux[N1], Zuy[N1], Zs[N1];
#pragma unroll
                    for (int b = 0; b < N1; ++b) Z[b] = Zux[b] = Zuy[b] = Zs[b] = 0.0f;
#pragma unroll 1
                    for (int jy = 0; jy < 4; ++jy) {
                        const float w = jy == 0 ? ly[0] : jy == 1 ? ly[1] : jy == 2 ? ly[2] : ly[3];
                        const float dw = jy == 0 ? dly[0] : jy == 1 ? dly[1] : jy == 2 ? dly[2] : dly[3];
                        const float4* src = s_f + (top + jy) * ww + col;
                        float Fi[N1][N1], Fd[N1][N1];
#pragma unroll
                        for (int a = 0; a < N1; ++a)
#pragma unroll
                            for (int b = 0; b < N1; ++b) Fi[a][b] = Fd[a][b] = 0.0f;
#pragma unroll
                        for (int jx = 0; jx < 4; ++jx) {
#pragma unroll
                            for (int a = 0; a < N1; ++a) {
                                const float4 v = src[(size_t)a * WN + jx];
                                const float fr[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                                for (int b = 0; b < N1; ++b) {
                                    Fi[a][b] = fmaf(lx[jx], fr[b], Fi[a][b]);
                                    Fd[a][b] = fmaf(dlx[jx], fr[b], Fd[a][b]);
                                }
                            }
                        }
                        // the row's contributions: value, and the tangents
                        // through the x-weights (Fd), the x-map (gdx) and
                        // the row weight (dw)
                        const float wux = -dt * w, wdy = -dt * dw, wi = -w * inv;
#pragma unroll
                        for (int b = 0; b < N1; ++b) {
                            float P = Fi[k][b], P1 = Fd[k][b], Pd = 0.0f, Pdx = 0.0f;
#pragma unroll
                            for (int a = 0; a < N1; ++a) {
                                P = fmaf(ex[a], Fi[a][b], P);
                                P1 = fmaf(ex[a], Fd[a][b], P1);
                                Pd = fmaf(gdx[a], Fi[a][b], Pd);
                                Pdx = fmaf(gdxx[a], Fi[a][b], Pdx);
                            }
                            Z[b] = fmaf(w, P, Z[b]);
                            Zux[b] = fmaf(wux, P1, fmaf(wi, Pd, Zux[b]));
                            Zuy[b] = fmaf(wdy, P, Zuy[b]);
                            Zs[b] = fmaf(ck * wux, P1, fmaf(wi, Pdx, fmaf(cl * wdy, P, Zs[b])));
                        }
                    }
                    // the y-map r -> lambda* and its derivatives; its
                    // identity part exactly
                    float Al = 0.0f, Axl = 0.0f, Ayl = 0.0f, Asl = 0.0f;
#pragma unroll
                    for (int b = 0; b < N1; ++b) {
                        const bool id = b == l;
                        Al += id ? Z[b] : 0.0f;
                        Axl += id ? Zux[b] : 0.0f;
                        Ayl += id ? Zuy[b] : 0.0f;
                        Asl += id ? Zs[b] : 0.0f;
                    }
                    float Ae = 0.0f, Axe = 0.0f, Aye = 0.0f, Ase = 0.0f, Dy = 0.0f, Ds = 0.0f;
#pragma unroll
                    for (int b = 0; b < N1; ++b) {
                        const float de = fmaf(L.c[b], rt, dyt);
                        float ey, gdy;
                        lag_taylor_ef(L, l, b, de, ey, gdy);
                        Ae = fmaf(ey, Z[b], Ae);
                        Axe = fmaf(ey, Zux[b], Axe);
                        Aye = fmaf(ey, Zuy[b], Aye);
                        Ase = fmaf(ey, Zs[b], Ase);
                        Dy = fmaf(gdy, Z[b], Dy);
                        Ds = fmaf(gdy * (L.c[b] + de), Z[b], Ds);
                    }
                    R[0] = Al + Ae;
                    R[1] = Axl + Axe;
                    R[2] = fmaf(-inv, Dy, Ayl + Aye);
                    R[3] = fmaf(-inv, Ds, Asl + Ase);
                } else {
                    adj_population_direct_mixed<N1>(A, X, Y, k, l, th, tl, st, ux, uy, inv, R);
                }
                const float fb = (float)A.fbar[o];
                const float mt = fmaf(ck, ck, cl * cl) - 2.0f * T_L;
                rho += R[0];
                sAf = fmaf(R[0], fb, sAf);
                wf = fmaf(L.w[k] * L.w[l], fb, wf);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    Px[j] = fmaf(ck, R[1 + j], Px[j]);
                    Py[j] = fmaf(cl, R[1 + j], Py[j]);
                    Pt[j] = fmaf(mt, R[1 + j], Pt[j]);
                    gF[j] = fmaf(fb, R[1 + j], gF[j]);
                    gS[j] += R[1 + j];
                }
            }
        }
        // the epilogue of k_adjoint_targets_mixed: J = M_A A_lambda, g, the
        // 3 x 3 solve by Cramer's rule, w
        const float beta = A.beta;
        const float irho = 1.0f / rho;
        const float sx = st * irho, stt = st * irho / (4.0f * T_L);
        float J[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            J[0][j] = sx * Px[j];
            J[1][j] = sx * Py[j];
            J[2][j] = stt * Pt[j];
        }
        const float c1 = 1.0f - 2.0f * beta, c2b = 2.0f * beta * wf;
        const float g0 = fmaf(c1, gF[0], c2b * gS[0]) + (float)A.gbar[node];
        const float g1 = fmaf(c1, gF[1], c2b * gS[1]) + (float)A.gbar[A.N + node];
        const float g2 = fmaf(c1, gF[2], c2b * gS[2]) + (float)A.gbar[2 * A.N + node] * 2.0f * st * T_L;
        const float a00 = J[0][0], a01 = J[1][0], a02 = J[2][0];
        const float a10 = J[0][1], a11 = J[1][1], a12 = J[2][1];
        const float a20 = J[0][2], a21 = J[1][2], a22 = J[2][2];
        const float det = a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) +
                          a02 * (a10 * a21 - a11 * a20);
        const float idet = 1.0f / det;
        const float r0 = -g0, r1 = -g1, r2 = -g2;
        const float mu0 = (r0 * (a11 * a22 - a12 * a21) - a01 * (r1 * a22 - a12 * r2) +
                           a02 * (r1 * a21 - a11 * r2)) * idet;
        const float mu1 = (a00 * (r1 * a22 - a12 * r2) - r0 * (a10 * a22 - a12 * a20) +
                           a02 * (a10 * r2 - r1 * a20)) * idet;
        const float mu2 = (a00 * (a11 * r2 - r1 * a21) - a01 * (a10 * r2 - r1 * a20) +
                           r0 * (a10 * a21 - a11 * a20)) * idet;
        const float m0 = sx * mu0, m1 = sx * mu1, m2 = stt * mu2;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k = q / N1, l = q % N1;
            const float ck = L.c[k], cl = L.c[l];
            const float mt = fmaf(ck, ck, cl * cl) - 2.0f * T_L;
            const long long o = (long long)q * A.N + node;
            const float Abar = fmaf(c1, (float)A.fbar[o], c2b);
            A.w[o] = fmaf(ck, m0, fmaf(cl, m1, fmaf(mt, m2, Abar)));
        }
        bb = 2.0 * ((double)rho * (double)wf - (double)sAf);
    }
    // beta cotangent sum 2 (rho W_q - A_q) fb_q, reduced over the warp in FP64
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bb += __shfl_xor_sync(0xffffffffu, bb, o);
    if ((tid & 31) == 0) atomicAdd(A.beta_bar, bb);
}
// Shared memory and launch of the staged phase A for a window capacity of
// wwa x wha staged nodes (FP32 rows of 16 bytes).
static cudaError_t launch_adjoint_phase_a_staged_mixed(const AdjMixedArgs& A,
                                                       const StateBuf<float>& in,
                                                       const double* ux_star,
                                                       const double* uy_star, int n1, int wwa,
                                                       int wha, float c_max, cudaStream_t s) {
    static int s_set[64][2] = {{0}};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const size_t smem = (size_t)n1 * wwa * wha * sizeof(float4);
    void (*kern)(AdjMixedArgs, StateBuf<float>, const double*, const double*, int, int, float) =
        n1 == 3 ? k_adjoint_jvp_staged_mixed<3> : k_adjoint_jvp_staged_mixed<4>;
    int& set = s_set[dev][n1 == 3 ? 1 : 0];
    if ((int)smem > set) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set = (int)smem;
    }
    const unsigned tiles = (unsigned)(((A.nx + 31) / 32) * ((A.ny + ADJM_TY - 1) / ADJM_TY));
    kern<<<tiles, 32 * ADJM_TY, smem, s>>>(A, in, ux_star, uy_star, wwa, wha, c_max);
    return cudaGetLastError();
}

}  // namespace pond

using namespace pond;

void destroy_adjoint_mixed(pond_ctx* ctx) {
    AdjMixedScratch* a = ctx->adjm;
    if (!a) return;
    cudaFree(a->fwd.f);
    cudaFree(a->fwd.ux);
    cudaFree(a->fwd.uy);
    cudaFree(a->fwd.st);
    cudaFree(a->w);
    cudaFree(a->gin);
    cudaFree(a->gstar);
    cudaFree(a->iters);
    cudaFree(a->stats);
    cudaFree(a->f4);
    cudaFree(a->org);
    cudaFree(a->lw);
    cudaFree(a->inv_st);
    cudaFree(a->vb);
    delete a;
    ctx->adjm = nullptr;
}

// Mixed-precision adjoint step; arguments already validated by
// pond_adjoint_step.  minmax_dev receives the bounds {min ux*, max ux*,
// min uy*, max uy*, min s*, max s*} of the forward gauge; everything stays on
// the stream (no host synchronisation).
cudaError_t adjoint_step_mixed(pond_ctx* ctx, const double* const out_gauge[3],
                               const double* fbar, const double* gbar, double* fbar_out,
                               double* gbar_out, double* beta_bar_dev, double* minmax_dev) {
    NvtxRange nv("pond_adjoint_step (FP32)");
    const int64_t N = ctx->N;
    cudaStream_t s = ctx->stream;
    cudaError_t e;
    if (!ctx->adjm) {
        AdjMixedScratch* a = new AdjMixedScratch();
        ctx->adjm = a;
        if ((e = cudaMalloc(&a->fwd.f, sizeof(float) * 16 * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->fwd.ux, sizeof(double) * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->fwd.uy, sizeof(double) * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->fwd.st, sizeof(double) * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->w, sizeof(float) * 16 * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->gin, sizeof(float4) * 2 * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->gstar, sizeof(float4) * 2 * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->iters, sizeof(int32_t) * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->stats, sizeof(DevStats))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->f4, sizeof(float4) * 4 * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->org, sizeof(int2) * 16 * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->lw, sizeof(float) * 8 * 16 * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->inv_st, sizeof(float) * N)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a->vb, sizeof(float) * 16)) != cudaSuccess) return e;
    }
    AdjMixedScratch* a = ctx->adjm;
    StateBuf<float> in;
    in.f = static_cast<float*>(ctx->f[ctx->cur]);
    in.ux = ctx->ux[ctx->cur];
    in.uy = ctx->uy[ctx->cur];
    in.st = ctx->st[ctx->cur];
    // 1. the fixed point lambda*: the gauge the forward step stores, given by
    //    the caller or recomputed into scratch
    if (out_gauge[0])
        e = launch_gauge_from_T(out_gauge[0], out_gauge[1], out_gauge[2], a->fwd.ux, a->fwd.uy,
                                a->fwd.st, N, ctx->L.T_L, s);
    else
        e = launch_ctx_step_mixed(ctx, in, a->fwd, a->iters, a->stats);
    if (e != cudaSuccess) return e;
    const unsigned nb256 = (unsigned)((N + 255) / 256);
    k_split_gauge<<<nb256, 256, 0, s>>>(in.ux, in.uy, in.st, a->gin, N);
    if (ctx->L.n1 == 3) k_rows_f4<3><<<nb256, 256, 0, s>>>(in.f, a->f4, N);
    else k_rows_f4<4><<<nb256, 256, 0, s>>>(in.f, a->f4, N);
    k_split_gauge<<<nb256, 256, 0, s>>>(a->fwd.ux, a->fwd.uy, a->fwd.st, a->gstar, N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_minmax3(a->fwd.ux, a->fwd.uy, a->fwd.st, N, minmax_dev, s)) != cudaSuccess)
        return e;
    {
        SpeedsD sp;
        for (int i = 0; i < 4; ++i) sp.c[i] = ctx->L.c[i];
        k_speed_bounds<<<1, 32, 0, s>>>(minmax_dev, sp, 1e-3 / ctx->P.dt, a->vb);
    }
    if ((e = cudaMemsetAsync(beta_bar_dev, 0, sizeof(double), s)) != cudaSuccess) return e;

    const GridDesc& G = ctx->grids_host[0];
    AdjMixedArgs A{};
    A.f_in = in.f;
    A.f4 = a->f4;
    A.gin = a->gin;
    A.gstar = a->gstar;
    A.st_in = in.st;
    A.st_star = a->fwd.st;
    A.fbar = fbar;
    A.gbar = gbar;
    A.w = a->w;
    A.fbar_in = fbar_out;
    A.gbar_in = gbar_out;
    A.beta_bar = beta_bar_dev;
    A.org = a->org;
    A.lw = a->lw;
    A.inv_st = a->inv_st;
    A.nx = G.nx;
    A.ny = G.ny;
    A.N = N;
    A.beta = (float)ctx->P.beta;
    A.dt = (float)ctx->P.dt;
    A.T_L = (float)ctx->L.T_L;
    A.vb = a->vb;
    const unsigned nb = (unsigned)((N + ADJM_THREADS - 1) / ADJM_THREADS);
    if (ctx_staged(ctx)) {
        // phase A in the staged form.  Its window capacity comes from the
        // input state's particle-velocity spans (on the host since
        // pond_set_state, so no synchronisation), widened by two cells for
        // lambda*'s departure from the input gauge; the kernel sizes each
        // tile's window from lambda* itself, and a stencil beyond the
        // capacity takes the per-pair path from global memory.
        const float* sp = &ctx->spans[0];
        const double sx = (double)sp[1] - sp[0], sy = (double)sp[3] - sp[2];
        const double dt = ctx->P.dt;
        int wwa = 32 + window_extent(sx, dt, 2.0) + 7;
        int wha = ADJM_TY + window_extent(sy, dt, 2.0) + 7;
        if (!std::isfinite(sx) || !std::isfinite(sy) || wwa > 4096 || wha > 4096)
            wwa = wha = 1;  // absurd or non-finite spans
        const size_t cap = 160 * 1024;
        while ((size_t)ctx->L.n1 * wwa * wha * sizeof(float4) > cap) {
            if (wwa - 32 >= wha - ADJM_TY) --wwa; else --wha;
        }
        e = launch_adjoint_phase_a_staged_mixed(A, in, a->fwd.ux, a->fwd.uy, ctx->L.n1, wwa, wha,
                                                (float)ctx->L.c_max, s);
        if (e != cudaSuccess) return e;
    } else {
        if (ctx->L.n1 == 3) k_adjoint_targets_mixed<3><<<nb, ADJM_THREADS, 0, s>>>(A);
        else k_adjoint_targets_mixed<4><<<nb, ADJM_THREADS, 0, s>>>(A);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (ctx_staged(ctx)) {
        if (ctx->L.n1 == 3) k_adjoint_sources_mixed_t<3><<<nb, ADJM_THREADS, 0, s>>>(A);
        else k_adjoint_sources_mixed_t<4><<<nb, ADJM_THREADS, 0, s>>>(A);
    } else {
        if (ctx->L.n1 == 3) k_adjoint_sources_mixed<3><<<nb, ADJM_THREADS, 0, s>>>(A);
        else k_adjoint_sources_mixed<4><<<nb, ADJM_THREADS, 0, s>>>(A);
    }
    return cudaGetLastError();
}
