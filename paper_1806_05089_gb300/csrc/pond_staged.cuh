// pond_staged.cuh -- the reference-gauge staged PonD step kernel, for the FP64
// form (Real = double) and the mixed form (Real = float).
//
// The gauge transform of Eq. transform is a composition: for any reference
// gauge lambda_r, M_t^-1 M_s = (M_t^-1 M_r)(M_r^-1 M_s), because the Q
// matched moments (m, n < n1 in each dimension) determine the Q populations
// uniquely.  The reconstruction of Eq. interpolation is linear in the
// transformed sources, and the transform from lambda_r to the target gauge
// lambda_t does not depend on the source.  So for population q = (k, l) of a
// node with gauge lambda_t,
//
//   f_q = sum_s a_s [G(s -> t) f_s]_q
//       = [G(r -> t) sum_s a_s G(s -> r) f_s]_q,
//
// and with G = G_x (x) G_y on the tensor lattice and a_s = lx_k(x_s) ly_l(y_s)
// (App. C), the sum splits into a sweep over the stencil rows:
//
//   P_k(y)[b] = sum_a Gx(r->t)[k][a] sum_jx lx_k[jx] g(x0_k + jx, y)[a][b]
//   f_(k,l)   = sum_jy ly_l[jy] sum_b Gy(r->t)[l][b] P_k(y0_l + jy)[b]
//
// where g = G(s -> r) f_s is each source's populations re-expressed in the
// tile's reference gauge (the gauge of the tile's centre node).  A CTA stages
// the window of sources its tile's stencils can reach once per step, already
// transformed into lambda_r; every predictor-corrector pass then needs only
// the 1D maps G(r -> t) of each target node, and for each x-speed index k one
// sweep over the union of the n1 y-stencils' rows, 4 sources per row.  In
// exact arithmetic this is the paper's f_q; it takes a quarter (mixed form)
// to a fifth (FP64 form) of the arithmetic of the per-(population, source)
// form, since the transform is paid per staged source and per target
// instead of per pair.
//
// Both 1D maps are written around the identity, G = I + E with E[k][a] =
// de (d1 + de (d2 + de d3)) (de = xi_a - c_a).  The staging and the mixed
// form apply them in correction form f + E f, so rounding never touches the
// identity part; the FP64 form folds Gx(r->t)[k][a] into the x-weights
// (lx_k[jx] Gx[k][a], once per x-speed and pass), takes the pass's Ey
// entries from a per-thread shared-memory table, and accumulates each
// population once over its four stencil rows from a four-row buffer of P.
//
// One CTA per TX x TY tile (TX = 32: a warp is one tile row of 32 nodes);
// batched ensembles take (grid, tile) items from an atomic counter.  The pass
// loop is warp-synchronous: the row sweep's bounds are the union over the
// warp's active lanes (__reduce_min/max_sync), lanes whose node has converged
// idle, and a lane's populations take only the rows of their own stencils.
// A stencil that leaves the staged window is computed from global memory by
// staged_fallback and counted.
//
// Tr (the including translation unit's traits) provides:
//   Real, Real4 (16 or 32 bytes), kUnrollK, kPacked (the packed FP32 sweep),
//   kEyTable (the Ey table in shared memory), min_blocks<threads>(),
//   lat<N1>() (lattice constants of that unit's constant bank), departure
//   (the floor of a displacement and the cubic weights at its fraction),
//   load4 / store4, update(...) (the moments -> gauge update and the App. E
//   test of that form) and finish<N1>(...) (re-gauge into the co-moving
//   frame, BGK, store).
#pragma once

#include "pond_device.cuh"

namespace pond {

// Four FP64 values in 32 bytes: one row of a staged FP64 source.
struct __align__(32) Double4 {
    double x, y, z, w;
};

template <typename Real>
struct StagedArgs {
    StateBuf<Real> in, out;
    int32_t* iters;
    DevStats* stats;
    const GridDesc* grids;
    const int64_t* tile_prefix;
    int n_grids;
    long long n_tiles;
    long long plane;  // plane stride of the packed state
    unsigned int* work_counter;
    int ww, wh;       // allocated window
    double c_max;
    float margin;
    StepParams P;
};

// Per-node state of the pass loop shared by the traits' update/finish.
struct PassGauge {
    double ux, uy, st;      // gauge of the current pass (FP64)
    double nux, nuy, nst;   // gauge the last pass's moments define
    double rho;             // density of the last pass
    int pass;
    unsigned int flag;      // 1: not converged at max_iter, 2: non-physical
};

template <class Tr, int NT>
__device__ __forceinline__ void staged_block_minmax4(float& a, float& b, float& c, float& d,
                                                     float (*red)[NT / 32]) {
    for (int o = 16; o > 0; o >>= 1) {
        a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        c = fminf(c, __shfl_xor_sync(0xffffffffu, c, o));
        d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = a;
        red[1][w] = b;
        red[2][w] = c;
        red[3][w] = d;
    }
    __syncthreads();
    a = red[0][0];
    b = red[1][0];
    c = red[2][0];
    d = red[3][0];
#pragma unroll
    for (int i = 1; i < NT / 32; ++i) {
        a = fminf(a, red[0][i]);
        b = fmaxf(b, red[1][i]);
        c = fminf(c, red[2][i]);
        d = fmaxf(d, red[3][i]);
    }
    __syncthreads();
}


// One population's reconstruction read straight from global memory, for a
// stencil that leaves the staged window (a displacement beyond the planned
// halo): the direct form f_q = sum_s a_s [G(s -> t) f_s]_q with the source
// offsets formed in FP64.
template <class Tr, int N1>
__device__ __noinline__ typename Tr::Real staged_fallback(const StagedArgs<typename Tr::Real>& A,
                                                          const GridDesc& G, long long base,
                                                          int X, int Y, int k, int l,
                                                          double ux, double uy, double st) {
    using Real = typename Tr::Real;
    const auto& L = Tr::template lat<N1>();
    const Real stf = (Real)st, dt = (Real)A.P.dt;
    Real fx, fy;
    Real lx[4], ly[4];
    Tr::departure(-fma(stf, (Real)L.c[k], (Real)ux) * dt, fx, lx);
    Tr::departure(-fma(stf, (Real)L.c[l], (Real)uy) * dt, fy, ly);
    const int x0 = wrap_idx((long long)X + (long long)fx - 1, G.nx);
    const int y0 = wrap_idx((long long)Y + (long long)fy - 1, G.ny);
    const double inv = 1.0 / st;
    Real acc = (Real)0;
#pragma unroll 1
    for (int jy = 0; jy < 4; ++jy) {
        const int sy = wrap_inc(y0, jy, G.ny);
        Real rowacc = (Real)0;
#pragma unroll
        for (int jx = 0; jx < 4; ++jx) {
            const int sx = wrap_inc(x0, jx, G.nx);
            const long long s = base + (long long)sy * G.nx + sx;
            if (!POND_INDEX_OK(sx >= 0 && sx < G.nx && sy >= 0 && sy < G.ny, A.stats)) continue;
            const Real r = (Real)((A.in.st[s] - st) * inv);
            const Real dx = (Real)((A.in.ux[s] - ux) * inv);
            const Real dy = (Real)((A.in.uy[s] - uy) * inv);
            Real gx[N1], gy[N1];
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                gx[a] = gauge_poly<N1>((Real)L.d3[k], (Real)L.d2[k][a], (Real)L.d1[k][a],
                                       a == k ? (Real)1 : (Real)0, fma((Real)L.c[a], r, dx));
                gy[a] = gauge_poly<N1>((Real)L.d3[l], (Real)L.d2[l][a], (Real)L.d1[l][a],
                                       a == l ? (Real)1 : (Real)0, fma((Real)L.c[a], r, dy));
            }
            Real g = (Real)0;
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                Real h = (Real)0;
#pragma unroll
                for (int b = 0; b < N1; ++b) h = fma(gy[b], A.in.f[(N1 * a + b) * A.plane + s], h);
                g = fma(gx[a], h, g);
            }
            rowacc = fma(lx[jx], g, rowacc);
        }
        acc = fma(ly[jy], rowacc, acc);
    }
    return acc;
}

// Stage the window [wx0, wx0 + ww) x [wy0, wy0 + wh) of grid G (periodic
// wrap; state planes of stride `plane`) into s_f, each source re-expressed in
// the reference gauge lambda_r = (rux, ruy, rst):
//   g = f_s + Ex (f_s + Ey f_s) + Ey f_s   (G(s -> r) = (I + Ex) (x) (I + Ey)),
// with xi_a = c_a + c_a (st_s/st_r - 1) + (u_s - u_r)/st_r formed in FP64.
// Rows a = 0..n1-1 of g at s_f[a * WN + i], i = the window-relative node.
// All threads of the block take part (a block-stride loop); the caller
// synchronises afterwards.
template <class Tr, int N1>
__device__ __forceinline__ void stage_window(const StateBuf<typename Tr::Real>& in, long long plane,
                                             const GridDesc& G, long long base, int wx0, int wy0,
                                             int ww, int wh, int WN, double rux, double ruy,
                                             double rst, typename Tr::Real4* s_f,
                                             DevStats* stats, int tid, int nt) {
    using Real = typename Tr::Real;
    constexpr int Q = N1 * N1;
    const auto& L = Tr::template lat<N1>();
    const double inv_rst = 1.0 / rst;
    (void)stats;
    for (int i = tid; i < ww * wh; i += nt) {
        const int cx = i % ww, cy = i / ww;
        const int gx = wrap_idx((long long)wx0 + cx, G.nx);
        const int gy = wrap_idx((long long)wy0 + cy, G.ny);
        const long long gi = base + (long long)gy * G.nx + gx;
        if (!POND_INDEX_OK(gx >= 0 && gx < G.nx && gy >= 0 && gy < G.ny && i < WN, stats))
            continue;
        const Real r = (Real)((__ldg(in.st + gi) - rst) * inv_rst);
        const Real dx = (Real)((__ldg(in.ux + gi) - rux) * inv_rst);
        const Real dy = (Real)((__ldg(in.uy + gi) - ruy) * inv_rst);
        Real f[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) f[q] = __ldg(in.f + gi + (long long)q * plane);
        Real ex[N1][N1], ey[N1][N1];  // [k][a]
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            const Real dex = fma((Real)L.c[a], r, dx), dey = fma((Real)L.c[a], r, dy);
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                ex[k][a] = gauge_tail<N1>((Real)L.d3[k], (Real)L.d2[k][a], (Real)L.d1[k][a], dex) * dex;
                ey[k][a] = gauge_tail<N1>((Real)L.d3[k], (Real)L.d2[k][a], (Real)L.d1[k][a], dey) * dey;
            }
        }
        Real H[Q];
#pragma unroll
        for (int a = 0; a < N1; ++a)
#pragma unroll
            for (int l = 0; l < N1; ++l) {
                Real v = (Real)0;
#pragma unroll
                for (int b = 0; b < N1; ++b) v = fma(ey[l][b], f[N1 * a + b], v);
                H[N1 * a + l] = v;
            }
        Real out[4][4];
#pragma unroll
        for (int k = 0; k < N1; ++k) {
#pragma unroll
            for (int l = 0; l < N1; ++l) {
                Real c = H[N1 * k + l];
#pragma unroll
                for (int a = 0; a < N1; ++a) c = fma(ex[k][a], f[N1 * a + l] + H[N1 * a + l], c);
                out[k][l] = f[N1 * k + l] + c;
            }
            if constexpr (N1 == 3) out[k][3] = (Real)0;
            Tr::store4(s_f + (size_t)k * WN + i, out[k]);
        }
    }
}

template <class Tr, int TX, int TY, int N1>
__global__ void __launch_bounds__(TX* TY, Tr::template min_blocks<TX * TY>())
k_step_staged(StagedArgs<typename Tr::Real> A) {
    using Real = typename Tr::Real;
    using Real4 = typename Tr::Real4;
    constexpr int NT = TX * TY;
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(TX == 32, "a warp is one tile row");
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int WN = A.ww * A.wh;
    Real4* s_f = reinterpret_cast<Real4*>(smem_raw);              // [N1][WN]: row a of g
    Real* s_acc = reinterpret_cast<Real*>(s_f + (size_t)N1 * WN);  // [Q][NT]
    Real* s_ey = s_acc + (size_t)N1 * N1 * NT;  // [Q][NT] Ey[l][b] of the pass (kEyTable)
    __shared__ float s_red[4][NT / 32];
    __shared__ long long s_item;
    __shared__ unsigned long long s_passes, s_nc, s_np, s_fb;
    __shared__ unsigned int s_max;
    const auto& L = Tr::template lat<N1>();
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_passes = 0ull;
        s_nc = 0ull;
        s_np = 0ull;
        s_fb = 0ull;
        s_max = 0u;
    }
    const int lxi = tid % TX, lyi = tid / TX;
    const Real dt = (Real)A.P.dt;
    const unsigned long long t_begin = (A.work_counter && tid == 0) ? pond_globaltimer() : 0ull;

    long long item = blockIdx.x;
    for (;;) {
        if (A.work_counter) {
            __syncthreads();
            if (tid == 0) s_item = (long long)atomicAdd(A.work_counter, 1u);
            __syncthreads();
            item = s_item;
        }
        if (item >= A.n_tiles) break;

        int g = 0;
        if (A.n_grids > 1) {
            int lo = 0, hi = A.n_grids - 1;  // largest g with prefix[g] <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (A.tile_prefix[mid] <= item) lo = mid; else hi = mid - 1;
            }
            g = lo;
        }
        const GridDesc G = A.grids[g];
        const long long t = item - A.tile_prefix[g];
        // tiles cover the grid's interior rectangle (the whole grid unless a
        // domain decomposition narrowed it to the part inside its halo)
        const int tiles_x = (G.iw + TX - 1) / TX;
        const int tx0 = G.ix0 + (int)(t % tiles_x) * TX;
        const int ty0 = G.iy0 + (int)(t / tiles_x) * TY;
        const int X = tx0 + lxi, Y = ty0 + lyi;
        const bool valid = X < G.ix0 + G.iw && Y < G.iy0 + G.ih;
        const long long base = G.offset;
        const long long node = base + (long long)Y * G.nx + X;

        // reference gauge lambda_r of the tile: its centre node (clamped to
        // the interior), so the staged sources' gauges differ from lambda_r by
        // at most about half the window
        const long long rnode = base + (long long)min(ty0 + TY / 2, G.iy0 + G.ih - 1) * G.nx +
                                min(tx0 + TX / 2, G.ix0 + G.iw - 1);
        const double rux = A.in.ux[rnode], ruy = A.in.uy[rnode], rst = A.in.st[rnode];

        PassGauge pg;
        pg.ux = 0.0;
        pg.uy = 0.0;
        pg.st = 1.0;
        float vxlo = 3.0e38f, vxhi = -3.0e38f, vylo = 3.0e38f, vyhi = -3.0e38f;
        if (valid) {
            pg.ux = A.in.ux[node];
            pg.uy = A.in.uy[node];
            pg.st = A.in.st[node];
            if (A.P.seed_mode == 1) {
                pg.ux = 0.0;
                pg.uy = 0.0;
                pg.st = 1.0;
            } else if (A.P.seed_mode == 2) {
                pg.ux = -pg.ux;
                pg.uy = -pg.uy;
            }
            const float sp = (float)(A.c_max * pg.st);
            vxlo = (float)pg.ux - sp;
            vxhi = (float)pg.ux + sp;
            vylo = (float)pg.uy - sp;
            vyhi = (float)pg.uy + sp;
        }
        staged_block_minmax4<Tr, NT>(vxlo, vxhi, vylo, vyhi, s_red);

        // staged window in unwrapped grid coordinates (departure = x - v dt)
        const float m = A.margin;
        const float fdt = (float)A.P.dt;
        const float bxl = fminf(fmaxf(vxlo, -1.0e6f), 1.0e6f), bxh = fminf(fmaxf(vxhi, -1.0e6f), 1.0e6f);
        const float byl = fminf(fmaxf(vylo, -1.0e6f), 1.0e6f), byh = fminf(fmaxf(vyhi, -1.0e6f), 1.0e6f);
        const int wx0 = (int)floorf((float)tx0 - bxh * fdt - m) - 1;
        const int wx1 = (int)floorf((float)(tx0 + TX - 1) - bxl * fdt + m) + 2;
        const int wy0 = (int)floorf((float)ty0 - byh * fdt - m) - 1;
        const int wy1 = (int)floorf((float)(ty0 + TY - 1) - byl * fdt + m) + 2;
        // a tile whose bounds are not finite (NaN gauge) stages a 1 x 1 window
        // and reads every stencil through the global-memory path
        const bool fin = isfinite(vxlo) && isfinite(vxhi) && isfinite(vylo) && isfinite(vyhi) &&
                         vxlo > -1.0e6f && vxhi < 1.0e6f && vylo > -1.0e6f && vyhi < 1.0e6f;
        const int ww = fin ? max(1, min(wx1 - wx0 + 1, A.ww)) : 1;
        const int wh = fin ? max(1, min(wy1 - wy0 + 1, A.wh)) : 1;

        // stage the window, each source re-expressed in lambda_r
        stage_window<Tr, N1>(A.in, A.plane, G, base, wx0, wy0, ww, wh, WN, rux, ruy, rst, s_f,
                             A.stats, tid, NT);
        __syncthreads();

        // ---------------------------------------------------- pass loop
        pg.nux = pg.ux;
        pg.nuy = pg.uy;
        pg.nst = pg.st;
        pg.rho = 0.0;
        pg.pass = 0;
        pg.flag = 0u;
        unsigned int fallbacks = 0u;
        bool done = !valid;
        while (__any_sync(FULL, !done)) {
            const bool work = !done;
            // target gauge of this pass, and its offsets from lambda_r:
            // xi_a(r -> t) = c_a + c_a (st_r/st_t - 1) + (u_r - u_t)/st_t
            const Real stf = (Real)pg.st, uxf = (Real)pg.ux, uyf = (Real)pg.uy;
            const Real invf = (Real)1 / stf;
            const Real rt = (Real)(rst - pg.st) * invf;
            const Real dxt = (Real)(rux - pg.ux) * invf;
            const Real dyt = (Real)(ruy - pg.uy) * invf;
            if constexpr (Tr::kEyTable) {
                // the y-map r -> lambda of this pass, Ey[l][b] in correction
                // form, for every x-speed
                if (work) {
#pragma unroll
                    for (int l = 0; l < N1; ++l)
#pragma unroll
                        for (int b = 0; b < N1; ++b) {
                            const Real de = fma((Real)L.c[b], rt, dyt);
                            s_ey[(N1 * l + b) * NT + tid] =
                                gauge_tail<N1>((Real)L.d3[l], (Real)L.d2[l][b], (Real)L.d1[l][b], de) * de;
                        }
                }
            }
            // y-stencils of the n1 y-speeds: top row in the window and weights
            int top[N1];
            bool ynear[N1];
            Real ly[N1][4];
#pragma unroll
            for (int l = 0; l < N1; ++l) {
                Real fy;
                Tr::departure(-fma(stf, (Real)L.c[l], uyf) * dt, fy, ly[l]);
                ynear[l] = fabs(fy) < (Real)1.0e6;
                top[l] = ynear[l] ? Y - wy0 + (int)fy - 1 : -1;
            }
            Real m0 = 0, m1 = 0, m2 = 0, m3 = 0;
            unsigned int offwin = 0u;
            // The x-speed loop is unrolled where the register budget allows
            // (the identity term of the x-map is then a register, Fi[k][b]);
            // rolled, that term is formed exactly as sum_a [a == k] Fi[a][b]
            constexpr int KU = Tr::kUnrollK ? N1 : 1;
#pragma unroll KU
            for (int k = 0; k < N1; ++k) {
                const Real ck = (Real)L.c[k];
                Real fx;
                Real lx[4];
                Tr::departure(-fma(stf, ck, uxf) * dt, fx, lx);
                const bool xnear = fabs(fx) < (Real)1.0e6;
                const int col = xnear ? X - wx0 + (int)fx - 1 : -1;
                const bool colok = work && xnear && col >= 0 && col + 3 < ww;
                Real ext[N1], ik[N1];
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    ik[a] = a == k ? (Real)1 : (Real)0;
                    const Real de = fma((Real)L.c[a], rt, dxt);
                    ext[a] = gauge_tail<N1>((Real)L.d3[k], (Real)L.d2[k][a], (Real)L.d1[k][a], de) * de;
                }
                bool on[N1];
                int lo = 0x7fffffff, hi = -0x7fffffff;
#pragma unroll
                for (int l = 0; l < N1; ++l) {
                    on[l] = colok && ynear[l] && top[l] >= 0 && top[l] + 3 < wh;
                    if (on[l]) {
                        lo = min(lo, top[l]);
                        hi = max(hi, top[l] + 3);
                    }
                }
                lo = __reduce_min_sync(FULL, lo);
                hi = __reduce_max_sync(FULL, hi);
                // Z_l[b] = sum_y ly_l(y) P(y)[b] over population l's four
                // stencil rows; the y-map is applied after the sweep:
                // f_(k,l) = Z_l[l] + sum_b Ey[l][b] Z_l[b].
                // Scalar form: the sweep keeps the P of its last four rows
                // (Pb[3] the newest), and population l takes its four rows
                // when the sweep reaches its last one, y = top[l] + 3, with
                // the fused multiply-adds in row order -- the same result as
                // adding ly_l(y) P(y) on every row with zero weights outside
                // the stencil, without those zero-weight FMAs.
                // Packed form (at its 128-register budget the four-row
                // buffer costs more than it saves: measured 45 % slower):
                // every row adds w_l(y) P(y) to the n1 populations, with the
                // row's weights selected per population.
                Real Z[N1][N1];
#pragma unroll
                for (int l = 0; l < N1; ++l)
#pragma unroll
                    for (int b = 0; b < N1; ++b) Z[l][b] = (Real)0;
                int last[N1];   // the row that completes population l's stencil
                int ontop[N1];  // top row of an on-window stencil, else out of reach
                bool anyon = false;
#pragma unroll
                for (int l = 0; l < N1; ++l) {
                    last[l] = on[l] ? top[l] + 3 : -1;
                    ontop[l] = on[l] ? top[l] : -0x40000000;
                    anyon = anyon || on[l];
                }
                float2 Z2[N1][2];  // the packed form's accumulators (pairs of b)
                Real Pb[4][N1];    // the scalar form's row buffer
                // The scalar (FP64) form folds the x-map into the x-weights,
                // cxa[jx][a] = lx[jx] (I + Ex)[k][a], once per x-speed and
                // pass: a row then costs the interpolation alone.  (The packed
                // FP32 form keeps the correction form P = Fi[k] + Ex Fi, whose
                // identity term is exact: there 1 + Ex would round in FP32.)
                Real cxa[4][N1];
                if constexpr (!Tr::kPacked) {
#pragma unroll
                    for (int jx = 0; jx < 4; ++jx)
#pragma unroll
                        for (int a = 0; a < N1; ++a) cxa[jx][a] = lx[jx] * (ik[a] + ext[a]);
                }
#pragma unroll
                for (int l = 0; l < N1; ++l) Z2[l][0] = Z2[l][1] = make_float2(0.f, 0.f);
                // the rows of the warp's union [lo, hi] lie in the window for
                // every thread with a population on it; a thread with none
                // skips the sweep
#pragma unroll 1
                for (int y = anyon ? lo : hi + 1; y <= hi; ++y) {
                    const Real4* src = s_f + y * ww + col;
                    const bool rowok = POND_INDEX_OK(y >= 0 && col >= 0 && y < wh && col + 3 < ww &&
                                                         y * ww + col + 3 < WN,
                                                     A.stats);
                    if constexpr (Tr::kPacked) {
                        // pairs of b on fma.rn.f32x2: two FP32 FMAs per
                        // instruction, each rounded as the scalar one
                        // the row's weight in population l's stencil: j = y - top
                        // in 0..3 picks ly[l][j] by its two bits; off-window
                        // stencils have their top far out of reach (ontop)
                        Real wl[N1];
                        bool any = false;
#pragma unroll
                        for (int l = 0; l < N1; ++l) {
                            const unsigned j = (unsigned)(y - ontop[l]);
                            const bool in = j < 4u;
                            const Real lo = (j & 1u) ? ly[l][1] : ly[l][0];
                            const Real hi = (j & 1u) ? ly[l][3] : ly[l][2];
                            wl[l] = in ? ((j & 2u) ? hi : lo) : (Real)0;
                            any = any || in;
                        }
                        if (!any) continue;
                        float2 Fi2[N1][2];
#pragma unroll
                        for (int a = 0; a < N1; ++a) Fi2[a][0] = Fi2[a][1] = make_float2(0.f, 0.f);
#pragma unroll
                        for (int jx = 0; jx < 4; ++jx) {
                            const float2 w2 = make_float2(lx[jx], lx[jx]);
#pragma unroll
                            for (int a = 0; a < N1; ++a) {
                                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                                if (rowok) v = src[(size_t)a * WN + jx];
                                Fi2[a][0] = __ffma2_rn(w2, make_float2(v.x, v.y), Fi2[a][0]);
                                Fi2[a][1] = __ffma2_rn(w2, make_float2(v.z, v.w), Fi2[a][1]);
                            }
                        }
                        float2 P2[2] = {Fi2[k][0], Fi2[k][1]};
#pragma unroll
                        for (int a = 0; a < N1; ++a) {
                            const float2 e2 = make_float2(ext[a], ext[a]);
                            P2[0] = __ffma2_rn(e2, Fi2[a][0], P2[0]);
                            P2[1] = __ffma2_rn(e2, Fi2[a][1], P2[1]);
                        }
#pragma unroll
                        for (int l = 0; l < N1; ++l) {
                            const float2 w2 = make_float2(wl[l], wl[l]);
                            Z2[l][0] = __ffma2_rn(w2, P2[0], Z2[l][0]);
                            Z2[l][1] = __ffma2_rn(w2, P2[1], Z2[l][1]);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 3; ++i)
#pragma unroll
                            for (int b = 0; b < N1; ++b) Pb[i][b] = Pb[i + 1][b];
                        // P[b] = sum_{jx, a} cxa[jx][a] g(col + jx, y)[a][b]:
                        // the row's four sources interpolated in x and mapped
                        // r -> lambda in one contraction (n1^2 FMAs per source)
                        Real P[N1];
#pragma unroll
                        for (int b = 0; b < N1; ++b) P[b] = (Real)0;
#pragma unroll
                        for (int jx = 0; jx < 4; ++jx) {
                            Real fr[N1][4];
#pragma unroll
                            for (int a = 0; a < N1; ++a) {
                                if (rowok) {
                                    Tr::load4(src + (size_t)a * WN + jx, fr[a]);
                                } else {
#pragma unroll
                                    for (int b = 0; b < 4; ++b) fr[a][b] = (Real)0;
                                }
                            }
#pragma unroll
                            for (int a = 0; a < N1; ++a)
#pragma unroll
                                for (int b = 0; b < N1; ++b) P[b] = fma(cxa[jx][a], fr[a][b], P[b]);
                        }
#pragma unroll
                        for (int b = 0; b < N1; ++b) Pb[3][b] = P[b];
#pragma unroll
                        for (int l = 0; l < N1; ++l) {
                            if (y != last[l]) continue;
#pragma unroll
                            for (int j = 0; j < 4; ++j)
#pragma unroll
                                for (int b = 0; b < N1; ++b) Z[l][b] = fma(ly[l][j], Pb[j][b], Z[l][b]);
                        }
                    }
                }
                if constexpr (Tr::kPacked) {
#pragma unroll
                    for (int l = 0; l < N1; ++l) {
                        const float z4[4] = {Z2[l][0].x, Z2[l][0].y, Z2[l][1].x, Z2[l][1].y};
#pragma unroll
                        for (int b = 0; b < N1; ++b) Z[l][b] = z4[b];
                    }
                }
                if (work) {
#pragma unroll
                    for (int l = 0; l < N1; ++l) {
                        Real acc = (Real)0;  // stencils off the window: below
                        if (on[l]) {
                            acc = Z[l][l];
#pragma unroll
                            for (int b = 0; b < N1; ++b) {
                                Real ey;
                                if constexpr (Tr::kEyTable) {
                                    ey = s_ey[(N1 * l + b) * NT + tid];
                                } else {
                                    const Real de = fma((Real)L.c[b], rt, dyt);
                                    ey = gauge_tail<N1>((Real)L.d3[l], (Real)L.d2[l][b],
                                                        (Real)L.d1[l][b], de) * de;
                                }
                                acc = fma(ey, Z[l][b], acc);
                            }
                        } else {
                            offwin |= 1u << (N1 * k + l);
                        }
                        s_acc[(N1 * k + l) * NT + tid] = acc;
                        const Real cl = (Real)L.c[l];
                        m0 += acc;
                        m1 = fma(ck, acc, m1);
                        m2 = fma(cl, acc, m2);
                        m3 = fma(fma(ck, ck, cl * cl), acc, m3);
                    }
                }
            }
            // populations whose stencil leaves the staged window, from
            // global memory (outside the sweep, so the sweep keeps its
            // registers)
            while (offwin) {
                const int q = __ffs(offwin) - 1;
                offwin &= offwin - 1;
                const int k = q / N1, l = q - N1 * k;
                const Real acc = staged_fallback<Tr, N1>(A, G, base, X, Y, k, l, pg.ux, pg.uy, pg.st);
                ++fallbacks;
                s_acc[q * NT + tid] = acc;
                const Real ck = (Real)L.c[k], cl = (Real)L.c[l];
                m0 += acc;
                m1 = fma(ck, acc, m1);
                m2 = fma(cl, acc, m2);
                m3 = fma(fma(ck, ck, cl * cl), acc, m3);
            }
            if (work) done = Tr::update(A.P, pg, m0, m1, m2, m3);
        }
        if (valid && POND_INDEX_OK(node >= base && node < base + (long long)G.nx * G.ny, A.stats)) {
            Tr::template finish<N1>(A, s_acc, NT, tid, node, pg);
            if (A.iters) A.iters[node] = pg.pass;
            atomicAdd(&s_passes, (unsigned long long)pg.pass);
            atomicMax(&s_max, (unsigned int)pg.pass);
            if (pg.flag & 1u) atomicAdd(&s_nc, 1ull);
            if (pg.flag & 2u) atomicAdd(&s_np, 1ull);
            if (fallbacks) atomicAdd(&s_fb, (unsigned long long)fallbacks);
        }
        if (!A.work_counter) break;
        __syncthreads();  // the next item restages the window
    }
    __syncthreads();
    if (tid == 0 && A.stats) {
        atomicAdd(&A.stats->passes, s_passes);
        atomicMax(&A.stats->max_passes, s_max);
        if (s_nc) atomicAdd(&A.stats->nonconverged, s_nc);
        if (s_np) atomicAdd(&A.stats->nonphysical, s_np);
        if (s_fb) atomicAdd(&A.stats->halo_fallback, s_fb);
        if (A.work_counter) persistent_exit(A.stats, t_begin);
    }
}

// Dynamic shared memory of the staged kernel for a window: the staged rows,
// the pass's populations and, in the FP64 form (8-byte reals), the y-map
// table.
inline size_t staged_smem_bytes(int n1, int ww, int wh, int nt, size_t real_bytes) {
    const size_t per_node = real_bytes == 8 ? 2 : 1;
    return (size_t)n1 * ww * wh * 4 * real_bytes + per_node * n1 * n1 * nt * real_bytes;
}

}  // namespace pond
