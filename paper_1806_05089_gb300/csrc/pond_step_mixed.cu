// pond_step_mixed.cu -- mixed-precision PonD time step (FP32 populations and
// bulk arithmetic, FP64 gauges), for one grid or a batched ensemble.
//
// This file holds the direct mixed kernel (k2_step_mixed, described here;
// contexts with kernel = POND_KERNEL_DIRECT) and, in its last section, the
// FP32 traits of the reference-gauge staged kernel of pond_staged.cuh
// (StagedFP32), which mixed contexts run by default.
//
// Direct kernel: one CTA per tile of TX x TY target nodes, one thread per node.  The CTA
// first bounds the particle velocities of its tile (u -+ c_max sqrt(theta)),
// stages the whole window of source nodes that the departure stencils can
// reach (tile + halo, periodic wrap applied while staging) in shared memory:
// the Q FP32 populations as n1 float4 rows f[a][0..n1-1] (one 16-byte load
// per row of the n1 x n1 contraction; the fourth word is unused on D2Q9)
// and the gauge as FP32 offsets from the
// tile's reference gauge, formed in FP64.  Gauge differences u_s - u' are then
// differences of those offsets, so they carry FP32 precision RELATIVE TO THE
// TILE'S GAUGE SPREAD, which is what FP64 differences rounded to FP32 give
// (the FP64 part of the "Vandermonde solve" inputs).  The moments and the
// gauge increments of a pass are formed in FP32 and accumulated into the FP64
// gauge; the convergence test of App. E runs in FP64.
//
// Threads of a warp are 32 consecutive nodes of a tile row and process the
// same population at the same time, so their stencil reads hit consecutive
// shared-memory words (conflict-free up to the one-column jitter of floor()).
// A stencil that leaves the staged window (displacement beyond the planned
// halo) is read from global memory instead and counted.
//
// Batched ensembles (many grids of uneven sizes) run as a persistent kernel:
// CTAs take (grid, tile) work items from an atomic counter; the item -> grid
// map is a prefix sum over the grids' tile counts.
#include "pond_device.cuh"
#include "pond_staged.cuh"

namespace pond {

// FP32 lattice constants, slot lattice_slot(n1) (D2Q16, D2Q9).
__constant__ LatticeF c_Lf[2];

cudaError_t upload_lattice_mixed() {
    const LatticeF F[2] = {to_float(make_lattice(POND_D2Q16)), to_float(make_lattice(POND_D2Q9))};
    return cudaMemcpyToSymbol(c_Lf, F, sizeof(F));
}

// Row a of the n1 x n1 contraction: sum_b gy[b] f[a][b] from one float4.
template <int N1>
__device__ __forceinline__ float row_dot(const float (&gy)[N1], const float4 f4) {
    float h = gy[0] * f4.x;
    h = fmaf(gy[1], f4.y, h);
    h = fmaf(gy[2], f4.z, h);
    if constexpr (N1 == 4) h = fmaf(gy[3], f4.w, h);
    return h;
}

struct MixedArgs {
    StateBuf<float> in, out;
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

// One stencil contraction read straight from global memory (window miss).
template <int N1>
__device__ __noinline__ float stencil_global(const MixedArgs& A, const GridDesc& G, long long base,
                                             int X, int Y, float fx, float fy,
                                             const float* lxw, const float* lyw, int k, int l,
                                             double ux, double uy, double st) {
    const LatticeF& L = c_Lf[lattice_slot(N1)];
    const int x0 = wrap_idx((long long)X + (long long)fx - 1, G.nx);
    const int y0 = wrap_idx((long long)Y + (long long)fy - 1, G.ny);
    const double inv = 1.0 / st;
    float gv[4][4];
    for (int jy = 0; jy < 4; ++jy) {
        const int sy = wrap_inc(y0, jy, G.ny);
        for (int jx = 0; jx < 4; ++jx) {
            const int sx = wrap_inc(x0, jx, G.nx);
            const long long s = base + (long long)sy * G.nx + sx;
            const float r = (float)((A.in.st[s] - st) * inv);
            const float dx = (float)((A.in.ux[s] - ux) * inv);
            const float dy = (float)((A.in.uy[s] - uy) * inv);
            float gx[N1], gy[N1];
            for (int a = 0; a < N1; ++a) {
                const float de = fmaf(L.c[a], r, dx);
                gx[a] = gauge_poly<N1>(L.d3[k], L.d2[k][a], L.d1[k][a], a == k ? 1.0f : 0.0f, de);
                const float de2 = fmaf(L.c[a], r, dy);
                gy[a] = gauge_poly<N1>(L.d3[l], L.d2[l][a], L.d1[l][a], a == l ? 1.0f : 0.0f, de2);
            }
            float g = 0.0f;
            for (int a = 0; a < N1; ++a) {
                float h = 0.0f;
                for (int b = 0; b < N1; ++b) h = fmaf(gy[b], A.in.f[(N1 * a + b) * A.plane + s], h);
                g = fmaf(gx[a], h, g);
            }
            gv[jy][jx] = g;
        }
    }
    // reconstruction relative to the node nearest the departure point
    const float gref = gv[1][1];
    float acc = 0.0f;
    for (int jy = 0; jy < 4; ++jy) {
        float rowacc = 0.0f;
        for (int jx = 0; jx < 4; ++jx) rowacc = fmaf(lxw[jx], gv[jy][jx] - gref, rowacc);
        acc = fmaf(lyw[jy], rowacc, acc);
    }
    return acc + gref;
}

// Final part of a node update: re-express the last pass's populations (in
// this thread's s_acc column) in the gauge lambda_{n+1} their moments define
// (Eq. transform at the node itself), then BGK relaxation toward rho W in
// that co-moving gauge (Eq. postcollision) and the store.  (r, dx, dy) are
// the Taylor offsets of that transform: xi_a = c_a + c_a r + d.  Kept out of
// line so the pass loop keeps its register budget.
template <int N1, class Args>
__device__ __noinline__ void finish_node(const Args& A, float* s_acc, int NT, int tid,
                                         long long node, bool regauge, float r, float dx,
                                         float dy, double ux, double uy, double st, float rho) {
    constexpr int Q = N1 * N1;
    const LatticeF& L = c_Lf[lattice_slot(N1)];
    if (regauge) {
        // In correction form, f + (G - I) f: at convergence G - I is of the
        // size of the last gauge increment (~1e-7 to 1e-6), so writing the
        // diagonal as fl(1 + e) would round e away while the off-diagonal
        // terms survive -- the columns of G would no longer sum to one and
        // each parcel would lose or gain mass the same way every step.
        //   (G f)_kl - f_kl = sum_b ey_lb f_kb + sum_a ex_ka (f_al + sum_b ey_lb f_ab)
        // with ex, ey the Taylor polynomials without their identity term.
        float ex[N1][N1], ey[N1][N1];  // [k][a]
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            const float dex = fmaf(L.c[a], r, dx), dey = fmaf(L.c[a], r, dy);
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                ex[k][a] = gauge_tail<N1>(L.d3[k], L.d2[k][a], L.d1[k][a], dex) * dex;
                ey[k][a] = gauge_tail<N1>(L.d3[k], L.d2[k][a], L.d1[k][a], dey) * dey;
            }
        }
        float f[Q], H[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) f[q] = s_acc[q * NT + tid];
#pragma unroll
        for (int a = 0; a < N1; ++a)
#pragma unroll
            for (int l = 0; l < N1; ++l) {
                float v = 0.0f;
#pragma unroll
                for (int b = 0; b < N1; ++b) v = fmaf(ey[l][b], f[N1 * a + b], v);
                H[N1 * a + l] = v;  // y-correction of row a
            }
#pragma unroll
        for (int k = 0; k < N1; ++k)
#pragma unroll
            for (int l = 0; l < N1; ++l) {
                float c = H[N1 * k + l];
#pragma unroll
                for (int a = 0; a < N1; ++a) c = fmaf(ex[k][a], f[N1 * a + l] + H[N1 * a + l], c);
                s_acc[(N1 * k + l) * NT + tid] = f[N1 * k + l] + c;
            }
    }
    // BGK in FP32, kept exactly conservative: the relaxed non-equilibrium
    // part n = f - rho W is first stripped of its mass, momentum and energy
    // moments (W-weighted projection onto the dual basis of {1, c_x, c_y,
    // |c|^2}: on D2Q16 the W-Gram matrix is [[1,0,0,2],[0,1,0,0],[0,0,1,0],
    // [2,0,0,8]] and the duals W(2 - |c|^2/2), W c_x, W c_y, W(|c|^2/4 -
    // 1/2); on D2Q9 (T_L = 1/3) W(2 - 3|c|^2/2), 3 W c_x, 3 W c_y,
    // W(9|c|^2/4 - 3/2)).  In exact arithmetic at the fixed point those
    // moments are zero and this is the plain f + 2 beta (rho W - f) of
    // Eq. postcollision; in FP32 their rounding would otherwise act on each
    // advected parcel the same way step after step and drift its mass and
    // temperature.  (Isothermal runs keep T fixed and do not conserve energy:
    // there only mass and momentum are projected out, with dual basis W,
    // W c_x / T_L, W c_y / T_L.)
    float M0 = 0.0f, M1 = 0.0f, M2 = 0.0f, M3 = 0.0f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k = q / N1, l = q % N1;
        const float n = fmaf(-rho, L.w[k] * L.w[l], s_acc[q * NT + tid]);
        M0 += n;
        M1 = fmaf(L.c[k], n, M1);
        M2 = fmaf(L.c[l], n, M2);
        M3 = fmaf(fmaf(L.c[k], L.c[k], L.c[l] * L.c[l]), n, M3);
    }
    float e0 = L.pe0, e2 = L.pe2, t0 = L.pt0, t2 = L.pt2;  // thermal dual basis
    if (!A.P.thermal) {
        e0 = 1.0f;
        e2 = 0.0f;
        M3 = 0.0f;
    }
    M1 *= L.inv_TL;
    M2 *= L.inv_TL;
    const float two_beta = (float)(2.0 * A.P.beta);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k = q / N1, l = q % N1;
        const float Wq = L.w[k] * L.w[l];
        const float c2 = fmaf(L.c[k], L.c[k], L.c[l] * L.c[l]);
        const float a = s_acc[q * NT + tid];
        float n = fmaf(-rho, Wq, a);
        const float proj = fmaf(M0, fmaf(e2, c2, e0),
                                fmaf(M1, L.c[k], fmaf(M2, L.c[l], M3 * fmaf(t2, c2, t0))));
        n = fmaf(-Wq, proj, n);
        A.out.f[q * A.plane + node] = fmaf(-two_beta, n, a);
    }
    A.out.ux[node] = ux;
    A.out.uy[node] = uy;
    A.out.st[node] = st;
}

template <int NT>
__device__ __forceinline__ void block_minmax4(float& a, float& b, float& c, float& d,
                                              float (*red)[NT / 32]) {
    // a, c: min; b, d: max
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

// Every tile shape is compiled for 128 registers per thread (512 threads of
// resident CTAs per SM: 4 x 128, 2 x 256 or 1 x 512).
template <int TX, int TY, int N1>
__global__ void __launch_bounds__(TX* TY, 512 / (TX * TY)) k2_step_mixed(MixedArgs A) {
    constexpr int NT = TX * TY;
    constexpr int Q = N1 * N1;
    extern __shared__ __align__(16) float4 smem4[];
    const int WN = A.ww * A.wh;
    // staged window, one float4 per (x-speed index a, node): f[a][0..n1-1],
    // so one 16-byte load feeds one row of the n1 x n1 contraction; and the
    // tile-relative gauge (s - s_ref, u_x - u_x,ref, u_y - u_y,ref): on D2Q16
    // a float4 of its own per node, on D2Q9 the spare fourth words of the
    // three rows (one 16-byte load fewer per pair)
    constexpr int GROWS = N1 == 4 ? 1 : 0;
    float4* s_f4 = smem4;           // [N1][WN]
    float4* s_g4 = s_f4 + N1 * WN;  // [GROWS][WN]
    float* s_acc = reinterpret_cast<float*>(s_g4 + GROWS * WN);  // [Q][NT]
    __shared__ float s_red[4][NT / 32];
    __shared__ long long s_item;
    __shared__ unsigned long long s_passes, s_nc, s_np, s_fb;
    __shared__ unsigned int s_max;
    const LatticeF& L = c_Lf[lattice_slot(N1)];
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_passes = 0ull;
        s_nc = 0ull;
        s_np = 0ull;
        s_fb = 0ull;
        s_max = 0u;
    }
    const int lxi = tid % TX, lyi = tid / TX;
    const float dt = (float)A.P.dt;
    const float half_over_TL = (float)(0.5 / A.P.T_L);

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
        const int tiles_x = (G.nx + TX - 1) / TX;
        const int tx0 = (int)(t % tiles_x) * TX;
        const int ty0 = (int)(t / tiles_x) * TY;
        const int X = tx0 + lxi, Y = ty0 + lyi;
        const bool valid = X < G.nx && Y < G.ny;
        const long long base = G.offset;
        const long long node = base + (long long)Y * G.nx + X;

        // reference gauge of the tile (its origin node always exists)
        const long long rnode = base + (long long)ty0 * G.nx + tx0;
        const double rux = A.in.ux[rnode], ruy = A.in.uy[rnode], rst = A.in.st[rnode];

        double ux = 0.0, uy = 0.0, st = 1.0;
        float vxlo = 3.0e38f, vxhi = -3.0e38f, vylo = 3.0e38f, vyhi = -3.0e38f;
        if (valid) {
            ux = A.in.ux[node];
            uy = A.in.uy[node];
            st = A.in.st[node];
            if (A.P.seed_mode == 1) {
                ux = 0.0;
                uy = 0.0;
                st = 1.0;
            } else if (A.P.seed_mode == 2) {
                ux = -ux;
                uy = -uy;
            }
            const float sp = (float)(A.c_max * st);
            vxlo = (float)ux - sp;
            vxhi = (float)ux + sp;
            vylo = (float)uy - sp;
            vyhi = (float)uy + sp;
        }
        block_minmax4<NT>(vxlo, vxhi, vylo, vyhi, s_red);

        // staged window in unwrapped grid coordinates (departure = x - v dt)
        const float m = A.margin;
        const float bxl = fminf(fmaxf(vxlo, -1.0e6f), 1.0e6f), bxh = fminf(fmaxf(vxhi, -1.0e6f), 1.0e6f);
        const float byl = fminf(fmaxf(vylo, -1.0e6f), 1.0e6f), byh = fminf(fmaxf(vyhi, -1.0e6f), 1.0e6f);
        const int wx0 = (int)floorf((float)tx0 - bxh * dt - m) - 1;
        const int wx1 = (int)floorf((float)(tx0 + TX - 1) - bxl * dt + m) + 2;
        const int wy0 = (int)floorf((float)ty0 - byh * dt - m) - 1;
        const int wy1 = (int)floorf((float)(ty0 + TY - 1) - byl * dt + m) + 2;
        // a tile whose bounds are not finite (NaN gauge) stages a 1 x 1 window
        // and reads every stencil through the global-memory path
        const bool fin = isfinite(vxlo) && isfinite(vxhi) && isfinite(vylo) && isfinite(vyhi) &&
                         vxlo > -1.0e6f && vxhi < 1.0e6f && vylo > -1.0e6f && vyhi < 1.0e6f;
        const int ww = fin ? max(1, min(wx1 - wx0 + 1, A.ww)) : 1;
        const int wh = fin ? max(1, min(wy1 - wy0 + 1, A.wh)) : 1;

        for (int i = tid; i < ww * wh; i += NT) {
            const int cx = i % ww, cy = i / ww;
            const int gx = wrap_idx((long long)wx0 + cx, G.nx);
            const int gy = wrap_idx((long long)wy0 + cy, G.ny);
            const long long gi = base + (long long)gy * G.nx + gx;
            const float* fp = A.in.f + gi;
            const float go[3] = {(float)(__ldg(A.in.st + gi) - rst), (float)(__ldg(A.in.ux + gi) - rux),
                                 (float)(__ldg(A.in.uy + gi) - ruy)};
#pragma unroll
            for (int a = 0; a < N1; ++a)
                s_f4[a * WN + i] = make_float4(__ldg(fp + (N1 * a + 0) * A.plane), __ldg(fp + (N1 * a + 1) * A.plane),
                                               __ldg(fp + (N1 * a + 2) * A.plane),
                                               N1 == 4 ? __ldg(fp + (N1 * a + 3) * A.plane) : go[a]);
            if constexpr (GROWS == 1) s_g4[i] = make_float4(go[0], go[1], go[2], 0.0f);
        }
        __syncthreads();

        int pass = 0;
        unsigned int flag = 0u;
        unsigned int fallbacks = 0u;
        if (valid) {
            // the pass gauge in FP64 (accumulated) and its FP32 working copies:
            // absolute (departures) and tile-relative (gauge differences)
            float stf = (float)st, uxf = (float)ux, uyf = (float)uy;
            float tdst = (float)(st - rst), tdux = (float)(ux - rux), tduy = (float)(uy - ruy);
            double nux = ux, nuy = uy, nst = st;  // gauge the last pass's moments define
            float lr = 0.0f, ldx = 0.0f, ldy = 0.0f, rhof = 0.0f;
            for (;;) {
                ++pass;
                const float invf = 1.0f / stf;
                const float bst = -tdst * invf, bux = -tdux * invf, buy = -tduy * invf;
                float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f, m3 = 0.0f;
#pragma unroll 1
                for (int q = 0; q < Q; ++q) {
                    const int k = q / N1, l = q % N1;
                    const float ck = L.c[k], cl = L.c[l];
                    const float dxp = -fmaf(stf, ck, uxf) * dt;
                    const float dyp = -fmaf(stf, cl, uyf) * dt;
                    const float fx = floorf(dxp), fy = floorf(dyp);
                    float lxw[4], lyw[4];
                    lagrange4f(dxp - fx + 1.0f, lxw);
                    lagrange4f(dyp - fy + 1.0f, lyw);
                    const bool near = fabsf(dxp) < 1.0e6f && fabsf(dyp) < 1.0e6f;
                    const int col = near ? X - wx0 + (int)fx - 1 : -1;
                    const int row = near ? Y - wy0 + (int)fy - 1 : -1;
                    float acc;
                    if (col >= 0 && col + 3 < ww && row >= 0 && row + 3 < wh) {
                        float d1k[N1], d2k[N1], d1l[N1], d2l[N1], ik[N1], il[N1];
#pragma unroll
                        for (int a = 0; a < N1; ++a) {
                            d1k[a] = L.d1[k][a];
                            d2k[a] = L.d2[k][a];
                            d1l[a] = L.d1[l][a];
                            d2l[a] = L.d2[l][a];
                            ik[a] = (a == k) ? 1.0f : 0.0f;
                            il[a] = (a == l) ? 1.0f : 0.0f;
                        }
                        const float d3k = L.d3[k], d3l = L.d3[l];
                        // one (population, source) pair: (G f_s)_q with the
                        // source's tile-relative gauge offset
                        auto pair = [&](int jx, int jy) -> float {
                            const int si = (row + jy) * ww + col + jx;
                            float4 g4;       // gauge offsets of the source
                            float4 fr[N1];   // D2Q9: rows read up front (they hold the gauge)
                            if constexpr (GROWS == 1) {
                                g4 = s_g4[si];
                            } else {
#pragma unroll
                                for (int a = 0; a < N1; ++a) fr[a] = s_f4[a * WN + si];
                                g4 = make_float4(fr[0].w, fr[1].w, fr[2].w, 0.0f);
                            }
                            const float r = fmaf(g4.x, invf, bst);   // s_s/s' - 1
                            const float dx = fmaf(g4.y, invf, bux);  // (u_s,x - u'_x)/s'
                            const float dy = fmaf(g4.z, invf, buy);
                            float gx[N1], gy[N1];
#pragma unroll
                            for (int a = 0; a < N1; ++a) {
                                const float de = fmaf(L.c[a], r, dx);
                                gx[a] = gauge_poly<N1>(d3k, d2k[a], d1k[a], ik[a], de);
                            }
#pragma unroll
                            for (int b = 0; b < N1; ++b) {
                                const float de = fmaf(L.c[b], r, dy);
                                gy[b] = gauge_poly<N1>(d3l, d2l[b], d1l[b], il[b], de);
                            }
                            float gsum = 0.0f;
#pragma unroll
                            for (int a = 0; a < N1; ++a) {
                                // D2Q16: each row read where it is used
                                const float4 f4 = GROWS == 1 ? s_f4[a * WN + si] : fr[a];
                                gsum = fmaf(gx[a], row_dot<N1>(gy, f4), gsum);
                            }
                            return gsum;
                        };
                        // reconstruction relative to the stencil node nearest
                        // the departure point: the weights sum to one exactly,
                        // so their FP32 rounding multiplies only differences
                        // (otherwise it acts coherently on each advected parcel
                        // step after step)
                        const float gref = pair(1, 1);
                        acc = 0.0f;
#pragma unroll
                        for (int jy = 0; jy < 4; ++jy) {
                            float rowacc = 0.0f;
#pragma unroll
                            for (int jx = 0; jx < 4; ++jx) {
                                if (jx == 1 && jy == 1) continue;
                                rowacc = fmaf(lxw[jx], pair(jx, jy) - gref, rowacc);
                            }
                            acc = fmaf(lyw[jy], rowacc, acc);
                        }
                        acc += gref;
                    } else {
                        acc = stencil_global<N1>(A, G, base, X, Y, fx, fy, lxw, lyw, k, l, ux, uy, st);
                        ++fallbacks;
                    }
                    s_acc[q * NT + tid] = acc;
                    m0 += acc;
                    m1 = fmaf(ck, acc, m1);
                    m2 = fmaf(cl, acc, m2);
                    m3 = fmaf(fmaf(ck, ck, cl * cl), acc, m3);
                }
                // gauge update (central form of Eqs. conservation_*) in FP32,
                // accumulated into the FP64 gauge; convergence test in FP64
                const float irf = 1.0f / m0;
                const float dux = stf * m1 * irf, duy = stf * m2 * irf;
                float dst = 0.0f;
                bool ok = (m0 > 0.0f) && isfinite(dux) && isfinite(duy);
                if (A.P.thermal) {
                    // theta_{n+1} / theta_n - 1
                    const float rm1 = (m3 * irf - (dux * dux + duy * duy) * invf * invf) * half_over_TL - 1.0f;
                    ok = ok && (rm1 > -1.0f) && isfinite(rm1);
                    dst = stf * rm1 / (sqrtf(1.0f + rm1) + 1.0f);
                }
                if (!ok) {
                    flag |= 2u;
                    break;
                }
                rhof = m0;
                const double ux1 = ux + (double)dux, uy1 = uy + (double)duy, st1 = st + (double)dst;
                nux = ux1;
                nuy = uy1;
                nst = st1;
                const float nstf = (float)st1;
                lr = -dst / nstf;
                ldx = -dux / nstf;
                ldy = -duy / nstf;
                const bool conv = fabs((double)dux) < A.P.eps_abs + A.P.eps_rel * fabs(ux1) &&
                                  fabs((double)duy) < A.P.eps_abs + A.P.eps_rel * fabs(uy1) &&
                                  fabs((double)dst) < A.P.eps_abs + A.P.eps_rel * fabs(st1);
                bool stop;
                if (A.P.fixed_iter > 0) {
                    stop = pass >= A.P.fixed_iter;
                } else {
                    stop = conv || pass >= A.P.max_iter;
                    if (!conv && pass >= A.P.max_iter) flag |= 1u;
                }
                if (stop) break;
                ux = ux1;
                uy = uy1;
                st = st1;
                stf = nstf;
                uxf = (float)ux1;
                uyf = (float)uy1;
                tdst += dst;
                tdux += dux;
                tduy += duy;
            }
            if (flag & 2u) {
                // non-physical moments: keep the pass's populations and gauge
                float r0 = 0.0f;
#pragma unroll
                for (int q = 0; q < Q; ++q) r0 += s_acc[q * NT + tid];
                finish_node<N1>(A, s_acc, NT, tid, node, false, 0.0f, 0.0f, 0.0f, ux, uy, st, r0);
            } else {
                finish_node<N1>(A, s_acc, NT, tid, node, true, lr, ldx, ldy, nux, nuy, nst, rhof);
            }
            if (A.iters) A.iters[node] = pass;
            atomicAdd(&s_passes, (unsigned long long)pass);
            atomicMax(&s_max, (unsigned int)pass);
            if (flag & 1u) atomicAdd(&s_nc, 1ull);
            if (flag & 2u) atomicAdd(&s_np, 1ull);
            if (fallbacks) atomicAdd(&s_fb, (unsigned long long)fallbacks);
        }
        if (!A.work_counter) break;
    }
    __syncthreads();
    if (tid == 0 && A.stats) {
        atomicAdd(&A.stats->passes, s_passes);
        atomicMax(&A.stats->max_passes, s_max);
        if (s_nc) atomicAdd(&A.stats->nonconverged, s_nc);
        if (s_np) atomicAdd(&A.stats->nonphysical, s_np);
        if (s_fb) atomicAdd(&A.stats->halo_fallback, s_fb);
    }
}

// ---------------------------------------------------------------------------
// Paired variant: each thread owns two vertically adjacent nodes.  For one
// population their 4 x 4 stencils usually share three rows (same column
// origin, row origins one apart), so the 5 x 4 union of sources is read from
// shared memory once for both nodes -- 20 instead of 32 staged-node reads per
// population, the kernel's binding resource.  When the two origins do not
// line up, or only one of the two nodes is still iterating, each node takes
// the single-node sweep.

struct NodeOff {
    float invf, bst, bux, buy;
};

struct QCoef {
    float d1k[4], d2k[4], d1l[4], d2l[4], ik[4], il[4], d3k, d3l;
};

__device__ __forceinline__ float pair_g(const float4 g4, const float4 (&fr)[4], const NodeOff& o,
                                        const QCoef& C) {
    const LatticeF& L = c_Lf[lattice_slot(4)];
    const float r = fmaf(g4.x, o.invf, o.bst);
    const float dx = fmaf(g4.y, o.invf, o.bux);
    const float dy = fmaf(g4.z, o.invf, o.buy);
    float gx[4], gy[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const float de = fmaf(L.c[a], r, dx);
        gx[a] = fmaf(fmaf(fmaf(C.d3k, de, C.d2k[a]), de, C.d1k[a]), de, C.ik[a]);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const float de = fmaf(L.c[b], r, dy);
        gy[b] = fmaf(fmaf(fmaf(C.d3l, de, C.d2l[b]), de, C.d1l[b]), de, C.il[b]);
    }
    float gsum = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        float h = gy[0] * fr[a].x;
        h = fmaf(gy[1], fr[a].y, h);
        h = fmaf(gy[2], fr[a].z, h);
        h = fmaf(gy[3], fr[a].w, h);
        gsum = fmaf(gx[a], h, gsum);
    }
    return gsum;
}

// one node's 16-source sweep inside the staged window (relative to the
// stencil node nearest the departure point, as in the single-node kernel)
__device__ __forceinline__ float sweep_one(const float4* s_f4, const float4* s_g4, int WN, int ww,
                                           int row, int col, const float (&lxw)[4],
                                           const float (&lyw)[4], const NodeOff& o,
                                           const QCoef& C) {
    auto load = [&](int si, float4 (&fr)[4]) {
#pragma unroll
        for (int a = 0; a < 4; ++a) fr[a] = s_f4[a * WN + si];
    };
    float4 fr[4];
    int si = (row + 1) * ww + col + 1;
    load(si, fr);
    const float gref = pair_g(s_g4[si], fr, o, C);
    float acc = 0.0f;
#pragma unroll
    for (int jy = 0; jy < 4; ++jy) {
        float rowacc = 0.0f;
#pragma unroll
        for (int jx = 0; jx < 4; ++jx) {
            if (jx == 1 && jy == 1) continue;
            si = (row + jy) * ww + col + jx;
            load(si, fr);
            rowacc = fmaf(lxw[jx], pair_g(s_g4[si], fr, o, C) - gref, rowacc);
        }
        acc = fmaf(lyw[jy], rowacc, acc);
    }
    return acc + gref;
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX* TY, 1) k2_step_mixed_pair(MixedArgs A) {
    constexpr int NT = TX * TY;  // threads
    constexpr int RY = 2 * TY;   // node rows of the tile
    extern __shared__ __align__(16) float4 smem4[];
    const int WN = A.ww * A.wh;
    float4* s_f4 = smem4;          // [4][WN]
    float4* s_g4 = s_f4 + 4 * WN;  // [WN]
    float* s_acc = reinterpret_cast<float*>(s_g4 + WN);  // [16][2 NT], column 2 tid + slot
    __shared__ float s_red[4][NT / 32];
    __shared__ long long s_item;
    __shared__ unsigned long long s_passes, s_nc, s_np, s_fb;
    __shared__ unsigned int s_max;
    const LatticeF& L = c_Lf[lattice_slot(4)];
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_passes = 0ull;
        s_nc = 0ull;
        s_np = 0ull;
        s_fb = 0ull;
        s_max = 0u;
    }
    const int lxi = tid % TX, lyi = tid / TX;
    const float dt = (float)A.P.dt;
    const float half_over_TL = (float)(0.5 / A.P.T_L);

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
            int lo = 0, hi = A.n_grids - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (A.tile_prefix[mid] <= item) lo = mid; else hi = mid - 1;
            }
            g = lo;
        }
        const GridDesc G = A.grids[g];
        const long long t = item - A.tile_prefix[g];
        const int tiles_x = (G.nx + TX - 1) / TX;
        const int tx0 = (int)(t % tiles_x) * TX;
        const int ty0 = (int)(t / tiles_x) * RY;
        const int X = tx0 + lxi;
        const int Yn[2] = {ty0 + 2 * lyi, ty0 + 2 * lyi + 1};
        const long long base = G.offset;
        const long long rnode = base + (long long)ty0 * G.nx + tx0;
        const double rux = A.in.ux[rnode], ruy = A.in.uy[rnode], rst = A.in.st[rnode];

        bool act[2];
        long long node[2];
        double ux[2], uy[2], st[2];
        float vxlo = 3.0e38f, vxhi = -3.0e38f, vylo = 3.0e38f, vyhi = -3.0e38f;
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
            act[sl] = X < G.nx && Yn[sl] < G.ny;
            node[sl] = base + (long long)Yn[sl] * G.nx + X;
            ux[sl] = 0.0;
            uy[sl] = 0.0;
            st[sl] = 1.0;
            if (act[sl]) {
                ux[sl] = A.in.ux[node[sl]];
                uy[sl] = A.in.uy[node[sl]];
                st[sl] = A.in.st[node[sl]];
                if (A.P.seed_mode == 1) {
                    ux[sl] = 0.0;
                    uy[sl] = 0.0;
                    st[sl] = 1.0;
                } else if (A.P.seed_mode == 2) {
                    ux[sl] = -ux[sl];
                    uy[sl] = -uy[sl];
                }
                const float sp = (float)(A.c_max * st[sl]);
                vxlo = fminf(vxlo, (float)ux[sl] - sp);
                vxhi = fmaxf(vxhi, (float)ux[sl] + sp);
                vylo = fminf(vylo, (float)uy[sl] - sp);
                vyhi = fmaxf(vyhi, (float)uy[sl] + sp);
            }
        }
        block_minmax4<NT>(vxlo, vxhi, vylo, vyhi, s_red);

        const float m = A.margin;
        const float bxl = fminf(fmaxf(vxlo, -1.0e6f), 1.0e6f), bxh = fminf(fmaxf(vxhi, -1.0e6f), 1.0e6f);
        const float byl = fminf(fmaxf(vylo, -1.0e6f), 1.0e6f), byh = fminf(fmaxf(vyhi, -1.0e6f), 1.0e6f);
        const int wx0 = (int)floorf((float)tx0 - bxh * dt - m) - 1;
        const int wx1 = (int)floorf((float)(tx0 + TX - 1) - bxl * dt + m) + 2;
        const int wy0 = (int)floorf((float)ty0 - byh * dt - m) - 1;
        const int wy1 = (int)floorf((float)(ty0 + RY - 1) - byl * dt + m) + 2;
        const bool fin = isfinite(vxlo) && isfinite(vxhi) && isfinite(vylo) && isfinite(vyhi) &&
                         vxlo > -1.0e6f && vxhi < 1.0e6f && vylo > -1.0e6f && vyhi < 1.0e6f;
        const int ww = fin ? max(1, min(wx1 - wx0 + 1, A.ww)) : 1;
        const int wh = fin ? max(1, min(wy1 - wy0 + 1, A.wh)) : 1;

        for (int i = tid; i < ww * wh; i += NT) {
            const int cx = i % ww, cy = i / ww;
            const int gx = wrap_idx((long long)wx0 + cx, G.nx);
            const int gy = wrap_idx((long long)wy0 + cy, G.ny);
            const long long gi = base + (long long)gy * G.nx + gx;
            const float* fp = A.in.f + gi;
#pragma unroll
            for (int a = 0; a < 4; ++a)
                s_f4[a * WN + i] = make_float4(__ldg(fp + (4 * a + 0) * A.plane), __ldg(fp + (4 * a + 1) * A.plane),
                                               __ldg(fp + (4 * a + 2) * A.plane), __ldg(fp + (4 * a + 3) * A.plane));
            s_g4[i] = make_float4((float)(__ldg(A.in.st + gi) - rst), (float)(__ldg(A.in.ux + gi) - rux),
                                  (float)(__ldg(A.in.uy + gi) - ruy), 0.0f);
        }
        __syncthreads();

        int pass[2] = {0, 0};
        unsigned int flag[2] = {0u, 0u}, fallbacks[2] = {0u, 0u};
        float stf[2], uxf[2], uyf[2], tdst[2], tdux[2], tduy[2];
        double nux[2], nuy[2], nst[2];
        float lr[2] = {0.f, 0.f}, ldx[2] = {0.f, 0.f}, ldy[2] = {0.f, 0.f}, rhof[2] = {0.f, 0.f};
        const bool valid[2] = {act[0], act[1]};
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
            stf[sl] = (float)st[sl];
            uxf[sl] = (float)ux[sl];
            uyf[sl] = (float)uy[sl];
            tdst[sl] = (float)(st[sl] - rst);
            tdux[sl] = (float)(ux[sl] - rux);
            tduy[sl] = (float)(uy[sl] - ruy);
            nux[sl] = ux[sl];
            nuy[sl] = uy[sl];
            nst[sl] = st[sl];
        }
        while (act[0] || act[1]) {
            NodeOff o[2];
            float m0[2] = {0.f, 0.f}, m1[2] = {0.f, 0.f}, m2[2] = {0.f, 0.f}, m3[2] = {0.f, 0.f};
#pragma unroll
            for (int sl = 0; sl < 2; ++sl) {
                if (act[sl]) ++pass[sl];
                o[sl].invf = 1.0f / stf[sl];
                o[sl].bst = -tdst[sl] * o[sl].invf;
                o[sl].bux = -tdux[sl] * o[sl].invf;
                o[sl].buy = -tduy[sl] * o[sl].invf;
            }
#pragma unroll 1
            for (int q = 0; q < 16; ++q) {
                const int k = q >> 2, l = q & 3;
                const float ck = L.c[k], cl = L.c[l];
                QCoef C;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    C.d1k[a] = L.d1[k][a];
                    C.d2k[a] = L.d2[k][a];
                    C.d1l[a] = L.d1[l][a];
                    C.d2l[a] = L.d2[l][a];
                    C.ik[a] = (a == k) ? 1.0f : 0.0f;
                    C.il[a] = (a == l) ? 1.0f : 0.0f;
                }
                C.d3k = L.d3[k];
                C.d3l = L.d3[l];
                float lxw[2][4], lyw[2][4], fxs[2], fys[2];
                int col[2], row[2];
                bool inw[2];
#pragma unroll
                for (int sl = 0; sl < 2; ++sl) {
                    const float dxp = -fmaf(stf[sl], ck, uxf[sl]) * dt;
                    const float dyp = -fmaf(stf[sl], cl, uyf[sl]) * dt;
                    fxs[sl] = floorf(dxp);
                    fys[sl] = floorf(dyp);
                    lagrange4f(dxp - fxs[sl] + 1.0f, lxw[sl]);
                    lagrange4f(dyp - fys[sl] + 1.0f, lyw[sl]);
                    const bool near = fabsf(dxp) < 1.0e6f && fabsf(dyp) < 1.0e6f;
                    col[sl] = near ? X - wx0 + (int)fxs[sl] - 1 : -1;
                    row[sl] = near ? Yn[sl] - wy0 + (int)fys[sl] - 1 : -1;
                    inw[sl] = col[sl] >= 0 && col[sl] + 3 < ww && row[sl] >= 0 && row[sl] + 3 < wh;
                }
                float acc[2] = {0.f, 0.f};
                if (act[0] && act[1] && inw[0] && inw[1] && col[0] == col[1] &&
                    row[1] == row[0] + 1) {
                    // shared sweep over the 5 x 4 union of the two stencils
                    float4 fr[4];
                    int si = (row[0] + 1) * ww + col[0] + 1;
#pragma unroll
                    for (int a = 0; a < 4; ++a) fr[a] = s_f4[a * WN + si];
                    float4 g4 = s_g4[si];
                    const float gra = pair_g(g4, fr, o[0], C);  // node a at (1, 1)
                    const float grb = pair_g(g4, fr, o[1], C);  // node b at (1, 0)
                    float ra[4] = {0.f, 0.f, 0.f, 0.f}, rb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int R = 0; R < 5; ++R) {
#pragma unroll
                        for (int jx = 0; jx < 4; ++jx) {
                            if (R == 1 && jx == 1) continue;
                            si = (row[0] + R) * ww + col[0] + jx;
#pragma unroll
                            for (int a = 0; a < 4; ++a) fr[a] = s_f4[a * WN + si];
                            g4 = s_g4[si];
                            if (R <= 3) ra[R] = fmaf(lxw[0][jx], pair_g(g4, fr, o[0], C) - gra, ra[R]);
                            if (R >= 1) rb[R - 1] = fmaf(lxw[1][jx], pair_g(g4, fr, o[1], C) - grb, rb[R - 1]);
                        }
                    }
                    // node b's reference is its (jx, jy) = (1, 0) source
                    float aa = 0.f, ab = 0.f;
#pragma unroll
                    for (int jy = 0; jy < 4; ++jy) {
                        aa = fmaf(lyw[0][jy], ra[jy], aa);
                        ab = fmaf(lyw[1][jy], rb[jy], ab);
                    }
                    acc[0] = aa + gra;
                    acc[1] = ab + grb;
                } else {
#pragma unroll
                    for (int sl = 0; sl < 2; ++sl) {
                        if (!act[sl]) continue;
                        if (inw[sl]) {
                            acc[sl] = sweep_one(s_f4, s_g4, WN, ww, row[sl], col[sl], lxw[sl],
                                                lyw[sl], o[sl], C);
                        } else {
                            acc[sl] = stencil_global<4>(A, G, base, X, Yn[sl], fxs[sl], fys[sl],
                                                     lxw[sl], lyw[sl], k, l, nux[sl] - 0.0,
                                                     nuy[sl] - 0.0, nst[sl] - 0.0);
                            ++fallbacks[sl];
                        }
                    }
                }
#pragma unroll
                for (int sl = 0; sl < 2; ++sl) {
                    if (!act[sl]) continue;
                    s_acc[q * 2 * NT + 2 * tid + sl] = acc[sl];
                    m0[sl] += acc[sl];
                    m1[sl] = fmaf(ck, acc[sl], m1[sl]);
                    m2[sl] = fmaf(cl, acc[sl], m2[sl]);
                    m3[sl] = fmaf(fmaf(ck, ck, cl * cl), acc[sl], m3[sl]);
                }
            }
#pragma unroll
            for (int sl = 0; sl < 2; ++sl) {
                if (!act[sl]) continue;
                const float irf = 1.0f / m0[sl];
                const float dux = stf[sl] * m1[sl] * irf, duy = stf[sl] * m2[sl] * irf;
                float dst = 0.0f;
                bool ok = (m0[sl] > 0.0f) && isfinite(dux) && isfinite(duy);
                if (A.P.thermal) {
                    const float inv = o[sl].invf;
                    const float rm1 = (m3[sl] * irf - (dux * dux + duy * duy) * inv * inv) * half_over_TL - 1.0f;
                    ok = ok && (rm1 > -1.0f) && isfinite(rm1);
                    dst = stf[sl] * rm1 / (sqrtf(1.0f + rm1) + 1.0f);
                }
                bool stop = false;
                if (!ok) {
                    flag[sl] |= 2u;
                    stop = true;
                } else {
                    rhof[sl] = m0[sl];
                    const double ux1 = nux[sl] + (double)dux, uy1 = nuy[sl] + (double)duy;
                    const double st1 = nst[sl] + (double)dst;
                    const float nstf = (float)st1;
                    lr[sl] = -dst / nstf;
                    ldx[sl] = -dux / nstf;
                    ldy[sl] = -duy / nstf;
                    const bool conv = fabs((double)dux) < A.P.eps_abs + A.P.eps_rel * fabs(ux1) &&
                                      fabs((double)duy) < A.P.eps_abs + A.P.eps_rel * fabs(uy1) &&
                                      fabs((double)dst) < A.P.eps_abs + A.P.eps_rel * fabs(st1);
                    if (A.P.fixed_iter > 0) {
                        stop = pass[sl] >= A.P.fixed_iter;
                    } else {
                        stop = conv || pass[sl] >= A.P.max_iter;
                        if (!conv && pass[sl] >= A.P.max_iter) flag[sl] |= 1u;
                    }
                    // keep the pass gauge (nux..) as lambda_n until it is
                    // replaced by lambda_{n+1} for the next pass
                    if (stop) {
                        ux[sl] = nux[sl];
                        uy[sl] = nuy[sl];
                        st[sl] = nst[sl];
                    }
                    nux[sl] = ux1;
                    nuy[sl] = uy1;
                    nst[sl] = st1;
                    if (!stop) {
                        stf[sl] = nstf;
                        uxf[sl] = (float)ux1;
                        uyf[sl] = (float)uy1;
                        tdst[sl] += dst;
                        tdux[sl] += dux;
                        tduy[sl] += duy;
                    }
                }
                if (stop) {
                    if (flag[sl] & 2u) {
                        float r0 = 0.0f;
#pragma unroll
                        for (int q = 0; q < 16; ++q) r0 += s_acc[q * 2 * NT + 2 * tid + sl];
                        finish_node<4>(A, s_acc, 2 * NT, 2 * tid + sl, node[sl], false, 0.f, 0.f, 0.f,
                                    nux[sl], nuy[sl], nst[sl], r0);
                    } else {
                        finish_node<4>(A, s_acc, 2 * NT, 2 * tid + sl, node[sl], true, lr[sl], ldx[sl],
                                    ldy[sl], nux[sl], nuy[sl], nst[sl], rhof[sl]);
                    }
                    act[sl] = false;
                }
            }
        }
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
            if (!valid[sl]) continue;
            if (A.iters) A.iters[node[sl]] = pass[sl];
            atomicAdd(&s_passes, (unsigned long long)pass[sl]);
            atomicMax(&s_max, (unsigned int)pass[sl]);
            if (flag[sl] & 1u) atomicAdd(&s_nc, 1ull);
            if (flag[sl] & 2u) atomicAdd(&s_np, 1ull);
            if (fallbacks[sl]) atomicAdd(&s_fb, (unsigned long long)fallbacks[sl]);
        }
        if (!A.work_counter) break;
    }
    __syncthreads();
    if (tid == 0 && A.stats) {
        atomicAdd(&A.stats->passes, s_passes);
        atomicMax(&A.stats->max_passes, s_max);
        if (s_nc) atomicAdd(&A.stats->nonconverged, s_nc);
        if (s_np) atomicAdd(&A.stats->nonphysical, s_np);
        if (s_fb) atomicAdd(&A.stats->halo_fallback, s_fb);
    }
}

// ---------------------------------------------------------------------------
// The reference-gauge staged kernel (pond_staged.cuh) in the mixed form: FP32
// populations, staged sources and sweep; the gauge offsets of every map
// formed from the FP64 gauges and rounded once; the moments and gauge
// increments of a pass in FP32, accumulated into the FP64 gauge; the App. E
// test in FP64; the exactly conservative FP32 collision of finish_node.
// The gauge-transform maps themselves (their Lagrange-Taylor polynomials in
// those offsets, and the contractions) are FP32, a deliberate choice: only
// their inputs are formed in FP64.  FP64 polynomials would put this kernel
// on the FP64 pipe (1/64 of the FP32 rate), at the FP64 form's speed; written
// around the identity, the FP32 maps round only their correction terms.

struct StagedFP32 {
    using Real = float;
    using Real4 = float4;
    static constexpr bool kUnrollK = true;
    static constexpr bool kPacked = true;  // the sweep on packed FP32 pairs
    static constexpr bool kEyTable = false;  // no room: 4 CTAs of 128 threads per SM
    template <int NT>
    static constexpr int min_blocks() {
        return 512 / NT;
    }
    template <int N1>
    static __device__ __forceinline__ const LatticeF& lat() {
        return c_Lf[lattice_slot(N1)];
    }
    static __device__ __forceinline__ void lagrange(float t, float (&l)[4]) { lagrange4f(t, l); }
    // floor of the displacement d and the cubic weights at its fraction,
    // from the centred coordinate d - floor - 1/2, with the weight of the
    // node nearest the departure point set to 1 minus the other three: the
    // FP32 weights then sum to one to within one rounding, where each
    // weight's own rounding would otherwise leave a sum off by a few units
    // -- an error that an advected parcel, meeting the same departure
    // fraction every step, would take on as a growth of its populations
    // step after step.
    static __device__ __forceinline__ void departure(float d, float& fl, float (&l)[4]) {
        fl = floorf(d);
        const float s = (d - fl) - 0.5f;
        lagrange4f_centred(s, l);
        if (s < 0.0f) l[1] = 1.0f - ((l[0] + l[2]) + l[3]);
        else l[2] = 1.0f - ((l[0] + l[1]) + l[3]);
    }
    static __device__ __forceinline__ void load4(const float4* p, float (&v)[4]) {
        const float4 a = *p;
        v[0] = a.x;
        v[1] = a.y;
        v[2] = a.z;
        v[3] = a.w;
    }
    static __device__ __forceinline__ void store4(float4* p, const float (&v)[4]) {
        *p = make_float4(v[0], v[1], v[2], v[3]);
    }
    // FP32 moments -> FP32 increments of (u_x, u_y, sqrt(theta)) (central
    // form of Eqs. conservation_*), added to the FP64 gauge; App. E test on
    // the increments in FP64.
    static __device__ __forceinline__ bool update(const StepParams& P, PassGauge& g, float m0,
                                                  float m1, float m2, float m3) {
        ++g.pass;
        const float stf = (float)g.st;
        const float invf = 1.0f / stf;
        const float irf = 1.0f / m0;
        const float dux = stf * m1 * irf, duy = stf * m2 * irf;
        float dst = 0.0f;
        bool ok = (m0 > 0.0f) && isfinite(dux) && isfinite(duy);
        if (P.thermal) {
            // theta_{n+1} / theta_n - 1
            const float rm1 = (m3 * irf - (dux * dux + duy * duy) * invf * invf) *
                                  (float)(0.5 / P.T_L) - 1.0f;
            ok = ok && (rm1 > -1.0f) && isfinite(rm1);
            dst = stf * rm1 / (sqrtf(1.0f + rm1) + 1.0f);
        }
        if (!ok) {
            g.flag |= 2u;
            g.rho = m0;
            return true;
        }
        g.rho = m0;
        const double ux1 = g.ux + (double)dux, uy1 = g.uy + (double)duy, st1 = g.st + (double)dst;
        g.nux = ux1;
        g.nuy = uy1;
        g.nst = st1;
        const bool conv = fabs((double)dux) < P.eps_abs + P.eps_rel * fabs(ux1) &&
                          fabs((double)duy) < P.eps_abs + P.eps_rel * fabs(uy1) &&
                          fabs((double)dst) < P.eps_abs + P.eps_rel * fabs(st1);
        bool stop;
        if (P.fixed_iter > 0) {
            stop = g.pass >= P.fixed_iter;
        } else {
            stop = conv || g.pass >= P.max_iter;
            if (!conv && g.pass >= P.max_iter) g.flag |= 1u;
        }
        if (!stop) {
            g.ux = ux1;
            g.uy = uy1;
            g.st = st1;
        }
        return stop;
    }
    template <int N1>
    static __device__ void finish(const StagedArgs<float>& A, float* s_acc, int NT, int tid,
                                  long long node, const PassGauge& g) {
        if (g.flag & 2u) {
            // non-physical moments: keep the pass's populations and gauge
            float r0 = 0.0f;
#pragma unroll
            for (int q = 0; q < N1 * N1; ++q) r0 += s_acc[q * NT + tid];
            finish_node<N1>(A, s_acc, NT, tid, node, false, 0.0f, 0.0f, 0.0f, g.ux, g.uy, g.st, r0);
        } else {
            // re-gauge lambda_n -> lambda_{n+1}: xi_a = c_a + c_a r + d with
            // r = st_n / st_{n+1} - 1, d = (u_n - u_{n+1}) / st_{n+1}
            const double inv1 = 1.0 / g.nst;
            finish_node<N1>(A, s_acc, NT, tid, node, true, (float)((g.st - g.nst) * inv1),
                            (float)((g.ux - g.nux) * inv1), (float)((g.uy - g.nuy) * inv1), g.nux,
                            g.nuy, g.nst, (float)g.rho);
        }
    }
};

template <int TY, int N1>
static cudaError_t staged32_shape(size_t smem, int* per_sm, int* s_set) {
    void (*kern)(StagedArgs<float>) = k_step_staged<StagedFP32, 32, TY, N1>;
    if ((int)smem > *s_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        *s_set = (int)smem;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, 32 * TY, smem);
}

cudaError_t staged_prepare_mixed(int ty, int n1, size_t smem, int* ctas_per_sm) {
    static int s_set[64][6] = {{0}};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int t = ty == 4 ? 0 : ty == 8 ? 1 : ty == 16 ? 2 : -1;
    if (t < 0) return cudaErrorInvalidValue;
    int* set = &s_set[dev][(n1 == 3 ? 3 : 0) + t];
    if (n1 == 3) {
        if (ty == 4) return staged32_shape<4, 3>(smem, ctas_per_sm, set);
        if (ty == 8) return staged32_shape<8, 3>(smem, ctas_per_sm, set);
        return staged32_shape<16, 3>(smem, ctas_per_sm, set);
    }
    if (ty == 4) return staged32_shape<4, 4>(smem, ctas_per_sm, set);
    if (ty == 8) return staged32_shape<8, 4>(smem, ctas_per_sm, set);
    return staged32_shape<16, 4>(smem, ctas_per_sm, set);
}

cudaError_t launch_step_staged_mixed(const StateBuf<float>& in, const StateBuf<float>& out,
                                     int32_t* iters, DevStats* stats, const GridDesc* grids_dev,
                                     const int64_t* tile_prefix_dev, int n_grids, int64_t n_tiles,
                                     int64_t plane, unsigned int* work_counter,
                                     const TileWindow& win, int persistent_ctas, const Lattice& L,
                                     const StepParams& P, cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    if (win.n1 != L.n1 || win.tx != 32 || (win.ty != 4 && win.ty != 8 && win.ty != 16))
        return cudaErrorInvalidValue;
    StagedArgs<float> A{};
    A.in = in;
    A.out = out;
    A.iters = iters;
    A.stats = stats;
    A.grids = grids_dev;
    A.tile_prefix = tile_prefix_dev;
    A.n_grids = n_grids;
    A.n_tiles = n_tiles;
    A.plane = plane;
    A.work_counter = work_counter;
    A.ww = win.ww;
    A.wh = win.wh;
    A.c_max = L.c_max;
    A.margin = 1.0f;
    A.P = P;
    const size_t smem = staged_smem_bytes(L.n1, win.ww, win.wh, 32 * win.ty, sizeof(float));
    unsigned int nb;
    if (work_counter) {
        cudaError_t e = cudaMemsetAsync(work_counter, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
        nb = (unsigned int)(persistent_ctas < n_tiles ? persistent_ctas : n_tiles);
    } else {
        nb = (unsigned int)n_tiles;
    }
    if (L.n1 == 3) {
        switch (win.ty) {
            case 4: k_step_staged<StagedFP32, 32, 4, 3><<<nb, 128, smem, s>>>(A); break;
            case 8: k_step_staged<StagedFP32, 32, 8, 3><<<nb, 256, smem, s>>>(A); break;
            default: k_step_staged<StagedFP32, 32, 16, 3><<<nb, 512, smem, s>>>(A); break;
        }
    } else {
        switch (win.ty) {
            case 4: k_step_staged<StagedFP32, 32, 4, 4><<<nb, 128, smem, s>>>(A); break;
            case 8: k_step_staged<StagedFP32, 32, 8, 4><<<nb, 256, smem, s>>>(A); break;
            default: k_step_staged<StagedFP32, 32, 16, 4><<<nb, 512, smem, s>>>(A); break;
        }
    }
    return cudaGetLastError();
}

size_t mixed_smem_bytes(const TileWindow& w) {
    // n1 float4 population rows per staged node, plus a float4 gauge on
    // D2Q16 (D2Q9 keeps it in the rows' spare words); Q floats of pass
    // populations per target node
    const size_t n1 = (size_t)w.n1;
    const size_t rows = n1 + (n1 == 4 ? 1 : 0);
    return sizeof(float) * (4 * rows * w.ww * w.wh + n1 * n1 * w.tx * w.ty);
}

template <int TY, bool PAIR, int N1>
static cudaError_t prepare_shape(size_t smem_bytes, int* ctas_per_sm, int* s_set) {
    void (*kern)(MixedArgs);
    if constexpr (PAIR) kern = k2_step_mixed_pair<MIXED_TX, TY / 2>;
    else kern = k2_step_mixed<MIXED_TX, TY, N1>;
    const int threads = PAIR ? MIXED_TX * TY / 2 : MIXED_TX * TY;
    cudaError_t e;
    if ((int)smem_bytes > *s_set) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        if (e != cudaSuccess) return e;
        *s_set = (int)smem_bytes;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, kern, threads, smem_bytes);
}

cudaError_t mixed_prepare(int ty, bool pair, int n1, size_t smem_bytes, int* ctas_per_sm) {
    // the attribute is per function and device: only ever raise it, so that
    // every live context's window stays launchable
    static int s_set[64][7] = {{0}};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (pair) {
        if (ty != 16 || n1 != 4) return cudaErrorInvalidValue;
        return prepare_shape<16, true, 4>(smem_bytes, ctas_per_sm, &s_set[dev][3]);
    }
    if (n1 == 3) {
        switch (ty) {
            case 4: return prepare_shape<4, false, 3>(smem_bytes, ctas_per_sm, &s_set[dev][4]);
            case 8: return prepare_shape<8, false, 3>(smem_bytes, ctas_per_sm, &s_set[dev][5]);
            case 16: return prepare_shape<16, false, 3>(smem_bytes, ctas_per_sm, &s_set[dev][6]);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (ty) {
        case 4: return prepare_shape<4, false, 4>(smem_bytes, ctas_per_sm, &s_set[dev][0]);
        case 8: return prepare_shape<8, false, 4>(smem_bytes, ctas_per_sm, &s_set[dev][1]);
        case 16: return prepare_shape<16, false, 4>(smem_bytes, ctas_per_sm, &s_set[dev][2]);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_mixed(const StateBuf<float>& in, const StateBuf<float>& out,
                              int32_t* iters, DevStats* stats, const GridDesc* grids_dev,
                              const int64_t* tile_prefix_dev, int n_grids, int64_t n_tiles,
                              int64_t plane, unsigned int* work_counter, const TileWindow& win,
                              int persistent_ctas, const Lattice& L, const StepParams& P,
                              cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    if (win.n1 != L.n1) return cudaErrorInvalidValue;
    MixedArgs A{};
    A.in = in;
    A.out = out;
    A.iters = iters;
    A.stats = stats;
    A.grids = grids_dev;
    A.tile_prefix = tile_prefix_dev;
    A.n_grids = n_grids;
    A.n_tiles = n_tiles;
    A.plane = plane;
    A.work_counter = work_counter;
    A.ww = win.ww;
    A.wh = win.wh;
    A.c_max = L.c_max;
    A.margin = 1.0f;
    A.P = P;
    const size_t smem = mixed_smem_bytes(win);
    unsigned int nb;
    if (work_counter) {
        cudaError_t e = cudaMemsetAsync(work_counter, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
        nb = (unsigned int)(persistent_ctas < n_tiles ? persistent_ctas : n_tiles);
    } else {
        nb = (unsigned int)n_tiles;
    }
    if (win.pair) {
        if (win.ty != 16 || L.n1 != 4) return cudaErrorInvalidValue;
        k2_step_mixed_pair<MIXED_TX, 8><<<nb, MIXED_TX * 8, smem, s>>>(A);
        return cudaGetLastError();
    }
    if (L.n1 == 3) {
        switch (win.ty) {
            case 4: k2_step_mixed<MIXED_TX, 4, 3><<<nb, MIXED_TX * 4, smem, s>>>(A); break;
            case 8: k2_step_mixed<MIXED_TX, 8, 3><<<nb, MIXED_TX * 8, smem, s>>>(A); break;
            case 16: k2_step_mixed<MIXED_TX, 16, 3><<<nb, MIXED_TX * 16, smem, s>>>(A); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (win.ty) {
        case 4: k2_step_mixed<MIXED_TX, 4, 4><<<nb, MIXED_TX * 4, smem, s>>>(A); break;
        case 8: k2_step_mixed<MIXED_TX, 8, 4><<<nb, MIXED_TX * 8, smem, s>>>(A); break;
        case 16: k2_step_mixed<MIXED_TX, 16, 4><<<nb, MIXED_TX * 16, smem, s>>>(A); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pond
