// pond_step_fp64.cu -- FP64 PonD time step of one periodic grid.
//
// This file holds the direct FP64 kernels (described here; contexts with
// kernel = POND_KERNEL_DIRECT, and the allocation-free entry point at the
// end of the file), the FP64 traits of the reference-gauge staged kernel of
// pond_staged.cuh (StagedFP64, which FP64 contexts run by default), and that
// entry point.
//
// The direct kernels, both bound by the FP64 pipe, all source reads through
// the read-only L1 path, templated on the lattice (D2Q16, N1 = 4, or D2Q9,
// N1 = 3):
//  * k1_step_fp64_node (the direct form's default): one node per thread, a
//    rolled loop over the populations; the per-node scalar work of a pass
//    runs once per node.
//  * k1_step_fp64<N1, NPW>: one, two or (D2Q9) three target nodes per warp,
//    16 (D2Q9 with three nodes: 10) lanes per node, lane = population q.
//    With one node, the lane's other index (lane >> 4) halves the four
//    stencil rows and one shuffle sums the halves; with two, it picks the
//    node and each lane sweeps all four rows.  The moments of the Q
//    populations are reduced by shuffles within the node's lanes, so every
//    lane of a node holds rho, u, T and takes the same convergence decision;
//    on D2Q9 with 16 lanes per node, lanes with q >= 9 only join the
//    shuffles.
//
// Per predictor-corrector pass (Eqs. advection, vi, interpolation, transform):
//   departure  y_q = x - (sqrt(theta) c_q + u) dt, origin floor(y_q) - 1
//   for each of the 16 stencil nodes s:
//     delta_a = xi_a - c_a = c_a (st_s/st' - 1) + (u_s - u')/st'
//     G[k][a] = [k==a] + delta (d1[k][a] + delta (d2[k][a] + delta d3[k]))
//     (G f_s)_q = sum_a Gx[k][a] sum_b Gy[l][b] f_s[N1 a + b]
//   f_q = sum_s a_s(y_q - x_s) (G f_s)_q
// then the moments in central form (algebraically equal to Eqs.
// conservation_rho/rhou/T):  rho = sum f,  u_{n+1} = u_n + st sum c f / rho,
// 2 T_{n+1} = st^2 sum |c|^2 f / rho - |u_{n+1} - u_n|^2,
// the convergence test of App. E on (u_x, u_y, sqrt(theta)), then the last
// pass's populations re-expressed in the gauge their moments define (so the
// stored gauge is exactly their co-moving frame), and finally the BGK
// relaxation f + 2 beta (rho W - f) (Eq. postcollision).
#include <cuda.h>

#include <mutex>

#include "pond_device.cuh"
#include "pond_staged.cuh"

namespace pond {

constexpr int K1_WARPS = 4;

// Lattice constants of this translation unit (uploaded once per device),
// slot lattice_slot(N1).
__constant__ Lattice c_L[2];

cudaError_t upload_lattice_fp64() {
    const Lattice L[2] = {make_lattice(POND_D2Q16), make_lattice(POND_D2Q9)};
    return cudaMemcpyToSymbol(c_L, L, sizeof(L));
}

// NPW nodes per warp.  NPW = 1: lane = (q, half of the stencil rows), the
// halves summed by one shuffle; the warp never diverges on the pass count.
// NPW = 2: lane = (q, node of the pair), each lane sweeps all four stencil
// rows; the per-node scalar work of a pass (reciprocals, square root, cubic
// weights, moment butterflies, convergence test) is then issued once per
// two nodes, at the price of the two nodes' pass counts diverging (the pair
// runs the larger count, the finished node's lanes idle).  NPW = 3 (D2Q9
// only): three nodes in 10-lane groups (lanes 0-8, 10-18, 20-28 hold the
// nine populations), 27 busy lanes instead of 18; the moments are summed by
// nine indexed shuffles instead of the xor butterflies.
template <int N1, int NPW>
__global__ void __launch_bounds__(K1_WARPS * 32, 3)
k1_step_fp64(StateBuf<double> in, StateBuf<double> out, int32_t* __restrict__ iters,
             DevStats* __restrict__ stats, int nx, int ny, long long N, StepParams P) {
    constexpr int Q = N1 * N1;
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(NPW != 3 || N1 == 3, "three nodes per warp: D2Q9 only");
    const Lattice& L = c_L[lattice_slot(N1)];
    __shared__ unsigned long long s_passes, s_nc, s_np;
    __shared__ unsigned int s_max;
    if (threadIdx.x == 0) {
        s_passes = 0ull;
        s_nc = 0ull;
        s_np = 0ull;
        s_max = 0u;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    // sub: node of the warp (NPW 2, 3) or half of the stencil rows (NPW 1)
    const int sub = NPW == 3 ? lane / 10 : lane >> 4;
    const int q = NPW == 3 ? lane - 10 * sub : lane & 15;
    const long long warp = (long long)blockIdx.x * K1_WARPS + (threadIdx.x >> 5);
    const long long node = NPW == 1 ? warp : warp * NPW + sub;
    // warp-uniform when NPW == 1 (both halves hold the same node)
    const bool valid = node < N && (NPW == 1 || sub < NPW);
    const int half = NPW == 1 ? sub : 0;
    // first lane of this node (lanes 30, 31 of NPW 3 hold no node)
    const int qbase = NPW == 1 ? 0 : (NPW == 2 ? (lane & 16) : 10 * min(sub, 2));
    if (__any_sync(FULL, valid)) {
        const long long nd = valid ? node : 0;
        const int X = (int)(nd % nx);
        const int Y = (int)(nd / nx);
        const bool act = q < Q;  // lane holds a population (all on D2Q16)
        const int qa = act ? q : 0, k = qa / N1, l = qa % N1;
        const double ck = act ? L.c[k] : 0.0, cl = act ? L.c[l] : 0.0;
        double d1k[N1], d2k[N1], d1l[N1], d2l[N1], ik[N1], il[N1];
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            d1k[a] = L.d1[k][a];
            d2k[a] = L.d2[k][a];
            d1l[a] = L.d1[l][a];
            d2l[a] = L.d2[l][a];
            ik[a] = (a == k) ? 1.0 : 0.0;
            il[a] = (a == l) ? 1.0 : 0.0;
        }
        const double d3k = L.d3[k], d3l = L.d3[l];

        // seed gauge (Eqs. seed_gauge, seed_gauge_T)
        double ux = in.ux[nd], uy = in.uy[nd], st = in.st[nd];
        if (P.seed_mode == 1) {
            ux = 0.0;
            uy = 0.0;
            st = 1.0;
        } else if (P.seed_mode == 2) {
            ux = -ux;
            uy = -uy;
        }

        int pass = 0;
        unsigned int flag = 0u;
        double total = 0.0, rho = 0.0;
        double nux = ux, nuy = uy, nst = st;  // gauge the last pass's moments define
        bool done = !valid;
        while (__any_sync(FULL, !done)) {
            const bool work = !done;
            double acc = 0.0;
            if (work) {
                ++pass;
                const double inv = 1.0 / st;
                const double vx = fma(st, ck, ux), vy = fma(st, cl, uy);
                const double depx = (double)X - vx * P.dt;
                const double depy = (double)Y - vy * P.dt;
                const double flx = floor(depx), fly = floor(depy);
                double lx[4], ly[4];
                lagrange4(depx - flx + 1.0, lx);
                lagrange4(depy - fly + 1.0, ly);
                const int x0 = wrap_idx((long long)flx - 1, nx);
                const int y0 = wrap_idx((long long)fly - 1, ny);
                const double bx = -ux * inv, by = -uy * inv;
                if (act) {
                    constexpr int ROWS = NPW == 1 ? 2 : 4;
#pragma unroll
                    for (int jj = 0; jj < ROWS; ++jj) {
                        const int jy = NPW == 1 ? 2 * half + jj : jj;
                        const double wy = NPW == 1 ? (half ? ly[2 + jj] : ly[jj]) : ly[jj];
                        const int sy = wrap_inc(y0, jy, ny);
                        double rowacc = 0.0;
#pragma unroll
                        for (int jx = 0; jx < 4; ++jx) {
                            const int sx = wrap_inc(x0, jx, nx);
                            const long long s = (long long)sy * nx + sx;
                            const double sts = __ldg(in.st + s);
                            const double uxs = __ldg(in.ux + s);
                            const double uys = __ldg(in.uy + s);
                            const double r = fma(sts, inv, -1.0);  // st_s/st' - 1
                            const double dx = fma(uxs, inv, bx);   // (u_s,x - u'_x)/st'
                            const double dy = fma(uys, inv, by);
                            double gx[N1], gy[N1];
#pragma unroll
                            for (int a = 0; a < N1; ++a) {
                                const double de = fma(L.c[a], r, dx);
                                gx[a] = gauge_poly<N1>(d3k, d2k[a], d1k[a], ik[a], de);
                            }
#pragma unroll
                            for (int b = 0; b < N1; ++b) {
                                const double de = fma(L.c[b], r, dy);
                                gy[b] = gauge_poly<N1>(d3l, d2l[b], d1l[b], il[b], de);
                            }
                            double g = 0.0;
#pragma unroll
                            for (int a = 0; a < N1; ++a) {
                                double h = 0.0;
#pragma unroll
                                for (int b = 0; b < N1; ++b)
                                    h = fma(gy[b], __ldg(in.f + (long long)(N1 * a + b) * N + s), h);
                                g = fma(gx[a], h, g);
                            }
                            rowacc = fma(lx[jx], g, rowacc);
                        }
                        acc = fma(wy, rowacc, acc);
                    }
                }
            }
            double tp = acc;
            if (NPW == 1) tp = acc + __shfl_xor_sync(FULL, acc, 16);

            // moments of the pass (central form), summed over the node's lanes
            double m0 = tp, m1 = ck * tp, m2 = cl * tp, m3 = (ck * ck + cl * cl) * tp;
            if constexpr (NPW == 3) {
                const double v0 = m0, v1 = m1, v2 = m2, v3 = m3;
                m0 = m1 = m2 = m3 = 0.0;
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    m0 += __shfl_sync(FULL, v0, qbase + j);
                    m1 += __shfl_sync(FULL, v1, qbase + j);
                    m2 += __shfl_sync(FULL, v2, qbase + j);
                    m3 += __shfl_sync(FULL, v3, qbase + j);
                }
            } else {
#pragma unroll
                for (int o = 1; o < 16; o <<= 1) {
                    m0 += __shfl_xor_sync(FULL, m0, o);
                    m1 += __shfl_xor_sync(FULL, m1, o);
                    m2 += __shfl_xor_sync(FULL, m2, o);
                    m3 += __shfl_xor_sync(FULL, m3, o);
                }
            }
            if (work) {
                total = tp;
                rho = m0;
                const double ir = 1.0 / rho;
                const double dux = st * m1 * ir, duy = st * m2 * ir;
                const double ux1 = ux + dux, uy1 = uy + duy;
                double st1 = st;
                bool ok = (rho > 0.0) && isfinite(ux1) && isfinite(uy1);
                if (P.thermal) {
                    const double T1 = 0.5 * (st * st * m3 * ir - (dux * dux + duy * duy));
                    ok = ok && (T1 > 0.0) && isfinite(T1);
                    st1 = sqrt(T1 / P.T_L);
                }
                if (!ok) {
                    flag |= 2u;
                    done = true;
                } else {
                    nux = ux1;
                    nuy = uy1;
                    nst = st1;
                    const bool conv = fabs(ux1 - ux) < P.eps_abs + P.eps_rel * fabs(ux1) &&
                                      fabs(uy1 - uy) < P.eps_abs + P.eps_rel * fabs(uy1) &&
                                      fabs(st1 - st) < P.eps_abs + P.eps_rel * fabs(st1);
                    bool stop;
                    if (P.fixed_iter > 0) {
                        stop = pass >= P.fixed_iter;
                    } else {
                        stop = conv || pass >= P.max_iter;
                        if (!conv && pass >= P.max_iter) flag |= 1u;
                    }
                    if (stop) {
                        done = true;
                    } else {
                        ux = ux1;
                        uy = uy1;
                        st = st1;
                    }
                }
            }
        }

        // Re-express f^{lambda_n} in the gauge lambda_{n+1} its moments define
        // (Eq. transform at the node itself): that gauge is then exactly the
        // co-moving frame of the stored populations.  The shuffles run on
        // every lane; a node with non-physical moments keeps its populations.
        {
            const double inv1 = 1.0 / nst;
            const double r = fma(st, inv1, -1.0);
            const double dx = (ux - nux) * inv1, dy = (uy - nuy) * inv1;
            double gx[N1], gy[N1];
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                const double de = fma(L.c[a], r, dx);
                gx[a] = gauge_poly<N1>(d3k, d2k[a], d1k[a], ik[a], de);
                const double de2 = fma(L.c[a], r, dy);
                gy[a] = gauge_poly<N1>(d3l, d2l[a], d1l[a], il[a], de2);
            }
            double g = 0.0;
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                double h = 0.0;
#pragma unroll
                for (int b = 0; b < N1; ++b)
                    h = fma(gy[b], __shfl_sync(FULL, total, qbase + N1 * a + b), h);
                g = fma(gx[a], h, g);
            }
            if (!(flag & 2u)) {
                total = g;
                ux = nux;
                uy = nuy;
                st = nst;
            }
        }

        // BGK relaxation toward rho W in the co-moving gauge (Eq. postcollision)
        if (valid && half == 0 && act) {
            const double feq = rho * L.w[k] * L.w[l];
            out.f[(long long)q * N + node] = total + 2.0 * P.beta * (feq - total);
        }
        if (valid && q == 0 && half == 0) {
            out.ux[node] = ux;
            out.uy[node] = uy;
            out.st[node] = st;
            if (iters) iters[node] = pass;
            atomicAdd(&s_passes, (unsigned long long)pass);
            atomicMax(&s_max, (unsigned int)pass);
            if (flag & 1u) atomicAdd(&s_nc, 1ull);
            if (flag & 2u) atomicAdd(&s_np, 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && stats) {
        atomicAdd(&stats->passes, s_passes);
        atomicMax(&stats->max_passes, s_max);
        if (s_nc) atomicAdd(&stats->nonconverged, s_nc);
        if (s_np) atomicAdd(&stats->nonphysical, s_np);
    }
}

// One node per thread (nodes_per_warp = 32): a rolled loop over the
// populations, each sweeping its 4 x 4 stencil, so the per-node scalar work
// of a pass (the reciprocal, the moment sums, the square root and the
// convergence test) is issued once per node instead of once per population
// lane, and every lane of the FP64 pipe does pair work.  A warp holds 32
// consecutive nodes on the same population (warp-uniform lattice constants);
// it runs the largest pass count of its nodes, the finished ones idle.  The
// pass's populations sit in shared memory for the closing re-gauge, one
// column per thread (conflict-free).
constexpr int K1N_THREADS = 128;

template <int N1>
__global__ void __launch_bounds__(K1N_THREADS, 3)
k1_step_fp64_node(StateBuf<double> in, StateBuf<double> out, int32_t* __restrict__ iters,
                  DevStats* __restrict__ stats, int nx, int ny, long long N, StepParams P) {
    constexpr int Q = N1 * N1;
    const Lattice& L = c_L[lattice_slot(N1)];
    __shared__ double s_f[Q][K1N_THREADS];
    __shared__ unsigned long long s_passes, s_nc, s_np;
    __shared__ unsigned int s_max;
    if (threadIdx.x == 0) {
        s_passes = 0ull;
        s_nc = 0ull;
        s_np = 0ull;
        s_max = 0u;
    }
    __syncthreads();

    const int tid = threadIdx.x;
    const long long node = (long long)blockIdx.x * K1N_THREADS + tid;
    if (node < N) {
        const int X = (int)(node % nx);
        const int Y = (int)(node / nx);

        // seed gauge (Eqs. seed_gauge, seed_gauge_T)
        double ux = in.ux[node], uy = in.uy[node], st = in.st[node];
        if (P.seed_mode == 1) {
            ux = 0.0;
            uy = 0.0;
            st = 1.0;
        } else if (P.seed_mode == 2) {
            ux = -ux;
            uy = -uy;
        }

        int pass = 0;
        unsigned int flag = 0u;
        double rho = 0.0;
        double nux = ux, nuy = uy, nst = st;  // gauge the last pass's moments define
        bool done = false;
        while (!done) {
            ++pass;
            const double inv = 1.0 / st;
            const double bx = -ux * inv, by = -uy * inv;
            double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
#pragma unroll 1
            for (int q = 0; q < Q; ++q) {
                const int k = q / N1, l = q - N1 * k;
                const double ck = L.c[k], cl = L.c[l];
                double d1k[N1], d2k[N1], d1l[N1], d2l[N1];
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    d1k[a] = L.d1[k][a];
                    d2k[a] = L.d2[k][a];
                    d1l[a] = L.d1[l][a];
                    d2l[a] = L.d2[l][a];
                }
                const double d3k = L.d3[k], d3l = L.d3[l];
                const double vx = fma(st, ck, ux), vy = fma(st, cl, uy);
                const double depx = (double)X - vx * P.dt;
                const double depy = (double)Y - vy * P.dt;
                const double flx = floor(depx), fly = floor(depy);
                double lx[4], ly[4];
                lagrange4(depx - flx + 1.0, lx);
                lagrange4(depy - fly + 1.0, ly);
                const int x0 = wrap_idx((long long)flx - 1, nx);
                const int y0 = wrap_idx((long long)fly - 1, ny);
                double acc = 0.0;
#pragma unroll
                for (int jy = 0; jy < 4; ++jy) {
                    const int sy = wrap_inc(y0, jy, ny);
                    double rowacc = 0.0;
#pragma unroll
                    for (int jx = 0; jx < 4; ++jx) {
                        const int sx = wrap_inc(x0, jx, nx);
                        const long long s = (long long)sy * nx + sx;
                        const double sts = __ldg(in.st + s);
                        const double uxs = __ldg(in.ux + s);
                        const double uys = __ldg(in.uy + s);
                        const double r = fma(sts, inv, -1.0);  // st_s/st' - 1
                        const double dx = fma(uxs, inv, bx);   // (u_s,x - u'_x)/st'
                        const double dy = fma(uys, inv, by);
                        double gx[N1], gy[N1];
#pragma unroll
                        for (int a = 0; a < N1; ++a) {
                            const double de = fma(L.c[a], r, dx);
                            gx[a] = gauge_poly<N1>(d3k, d2k[a], d1k[a], a == k ? 1.0 : 0.0, de);
                        }
#pragma unroll
                        for (int b = 0; b < N1; ++b) {
                            const double de = fma(L.c[b], r, dy);
                            gy[b] = gauge_poly<N1>(d3l, d2l[b], d1l[b], b == l ? 1.0 : 0.0, de);
                        }
                        double g = 0.0;
#pragma unroll
                        for (int a = 0; a < N1; ++a) {
                            double h = 0.0;
#pragma unroll
                            for (int b = 0; b < N1; ++b)
                                h = fma(gy[b], __ldg(in.f + (long long)(N1 * a + b) * N + s), h);
                            g = fma(gx[a], h, g);
                        }
                        rowacc = fma(lx[jx], g, rowacc);
                    }
                    acc = fma(ly[jy], rowacc, acc);
                }
                s_f[q][tid] = acc;
                // moments of the pass (central form)
                m0 += acc;
                m1 = fma(ck, acc, m1);
                m2 = fma(cl, acc, m2);
                m3 = fma(ck * ck + cl * cl, acc, m3);
            }

            rho = m0;
            const double ir = 1.0 / rho;
            const double dux = st * m1 * ir, duy = st * m2 * ir;
            const double ux1 = ux + dux, uy1 = uy + duy;
            double st1 = st;
            bool ok = (rho > 0.0) && isfinite(ux1) && isfinite(uy1);
            if (P.thermal) {
                const double T1 = 0.5 * (st * st * m3 * ir - (dux * dux + duy * duy));
                ok = ok && (T1 > 0.0) && isfinite(T1);
                st1 = sqrt(T1 / P.T_L);
            }
            if (!ok) {
                flag |= 2u;
                done = true;
            } else {
                nux = ux1;
                nuy = uy1;
                nst = st1;
                const bool conv = fabs(ux1 - ux) < P.eps_abs + P.eps_rel * fabs(ux1) &&
                                  fabs(uy1 - uy) < P.eps_abs + P.eps_rel * fabs(uy1) &&
                                  fabs(st1 - st) < P.eps_abs + P.eps_rel * fabs(st1);
                bool stop;
                if (P.fixed_iter > 0) {
                    stop = pass >= P.fixed_iter;
                } else {
                    stop = conv || pass >= P.max_iter;
                    if (!conv && pass >= P.max_iter) flag |= 1u;
                }
                if (stop) {
                    done = true;
                } else {
                    ux = ux1;
                    uy = uy1;
                    st = st1;
                }
            }
        }

        // Re-express f^{lambda_n} in the gauge lambda_{n+1} its moments define
        // (Eq. transform at the node itself), then BGK toward rho W in that
        // co-moving gauge (Eq. postcollision).  A node with non-physical
        // moments keeps its populations and the gauge of its last pass.
        const bool regauge = !(flag & 2u);
        const double inv1 = 1.0 / nst;
        const double r = fma(st, inv1, -1.0);
        const double dx = (ux - nux) * inv1, dy = (uy - nuy) * inv1;
#pragma unroll 1
        for (int q = 0; q < Q; ++q) {
            const int k = q / N1, l = q - N1 * k;
            double total = s_f[q][tid];
            if (regauge) {
                double gx[N1], gy[N1];
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    gx[a] = gauge_poly<N1>(L.d3[k], L.d2[k][a], L.d1[k][a], a == k ? 1.0 : 0.0,
                                           fma(L.c[a], r, dx));
                    gy[a] = gauge_poly<N1>(L.d3[l], L.d2[l][a], L.d1[l][a], a == l ? 1.0 : 0.0,
                                           fma(L.c[a], r, dy));
                }
                double g = 0.0;
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    double h = 0.0;
#pragma unroll
                    for (int b = 0; b < N1; ++b) h = fma(gy[b], s_f[N1 * a + b][tid], h);
                    g = fma(gx[a], h, g);
                }
                total = g;
            }
            const double feq = rho * L.w[k] * L.w[l];
            out.f[(long long)q * N + node] = total + 2.0 * P.beta * (feq - total);
        }
        if (regauge) {
            ux = nux;
            uy = nuy;
            st = nst;
        }
        out.ux[node] = ux;
        out.uy[node] = uy;
        out.st[node] = st;
        if (iters) iters[node] = pass;
        atomicAdd(&s_passes, (unsigned long long)pass);
        atomicMax(&s_max, (unsigned int)pass);
        if (flag & 1u) atomicAdd(&s_nc, 1ull);
        if (flag & 2u) atomicAdd(&s_np, 1ull);
    }
    __syncthreads();
    if (threadIdx.x == 0 && stats) {
        atomicAdd(&stats->passes, s_passes);
        atomicMax(&stats->max_passes, s_max);
        if (s_nc) atomicAdd(&stats->nonconverged, s_nc);
        if (s_np) atomicAdd(&stats->nonphysical, s_np);
    }
}

cudaError_t launch_step_fp64(const StateBuf<double>& in, const StateBuf<double>& out,
                             int32_t* iters, DevStats* stats, int nx, int ny, const Lattice& L,
                             const StepParams& P, int nodes_per_warp, cudaStream_t s) {
    const long long N = (long long)nx * ny;
    if (N == 0) return cudaSuccess;
    if (nodes_per_warp == FP64_NODE_PER_THREAD) {
        const unsigned nbn = (unsigned)((N + K1N_THREADS - 1) / K1N_THREADS);
        if (L.n1 == 3)
            k1_step_fp64_node<3><<<nbn, K1N_THREADS, 0, s>>>(in, out, iters, stats, nx, ny, N, P);
        else
            k1_step_fp64_node<4><<<nbn, K1N_THREADS, 0, s>>>(in, out, iters, stats, nx, ny, N, P);
        return cudaGetLastError();
    }
    const int npw = (nodes_per_warp == 3 && L.n1 == 3) ? 3 : (nodes_per_warp == 1 ? 1 : 2);
    const long long per_cta = (long long)K1_WARPS * npw;
    const unsigned nb = (unsigned)((N + per_cta - 1) / per_cta);
    const int T = K1_WARPS * 32;
    if (L.n1 == 3) {
        if (npw == 3) k1_step_fp64<3, 3><<<nb, T, 0, s>>>(in, out, iters, stats, nx, ny, N, P);
        else if (npw == 2) k1_step_fp64<3, 2><<<nb, T, 0, s>>>(in, out, iters, stats, nx, ny, N, P);
        else k1_step_fp64<3, 1><<<nb, T, 0, s>>>(in, out, iters, stats, nx, ny, N, P);
    } else {
        if (npw == 2) k1_step_fp64<4, 2><<<nb, T, 0, s>>>(in, out, iters, stats, nx, ny, N, P);
        else k1_step_fp64<4, 1><<<nb, T, 0, s>>>(in, out, iters, stats, nx, ny, N, P);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The reference-gauge staged kernel (pond_staged.cuh) in FP64: gauges,
// populations and every product in FP64; the moments of a pass in central
// form, as k1_step_fp64_node; plain BGK (Eq. postcollision).

struct StagedFP64 {
    using Real = double;
    using Real4 = Double4;
    static constexpr bool kUnrollK = true;
    static constexpr bool kPacked = false;  // the sweep on packed FP32 pairs
    // the y-map entries Ey[l][b] of a pass in a shared-memory table (they do
    // not depend on the x-speed; computing them once per pass instead of once
    // per (k, l) saves ~190 FP64 operations per node-pass)
    static constexpr bool kEyTable = true;
    template <int NT>
    static constexpr int min_blocks() {
        return NT >= 256 ? 1 : 2;
    }
    template <int N1>
    static __device__ __forceinline__ const Lattice& lat() {
        return c_L[lattice_slot(N1)];
    }
    static __device__ __forceinline__ void lagrange(double t, double (&l)[4]) { lagrange4(t, l); }
    // floor of the displacement d and the cubic weights at t = d - floor + 1
    static __device__ __forceinline__ void departure(double d, double& fl, double (&l)[4]) {
        fl = floor(d);
        lagrange4(d - fl + 1.0, l);
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
    // Moments of the pass -> the next gauge (Eqs. conservation_*, central
    // form: u_{n+1} = u_n + st sum c f / rho, 2 T_{n+1} = st^2 sum |c|^2 f /
    // rho - |u_{n+1} - u_n|^2) and the App. E test.  Returns true when the
    // node stops.
    static __device__ __forceinline__ bool update(const StepParams& P, PassGauge& g, double m0,
                                                  double m1, double m2, double m3) {
        ++g.pass;
        g.rho = m0;
        const double ir = 1.0 / m0;
        const double dux = g.st * m1 * ir, duy = g.st * m2 * ir;
        const double ux1 = g.ux + dux, uy1 = g.uy + duy;
        double st1 = g.st;
        bool ok = (m0 > 0.0) && isfinite(ux1) && isfinite(uy1);
        if (P.thermal) {
            const double T1 = 0.5 * (g.st * g.st * m3 * ir - (dux * dux + duy * duy));
            ok = ok && (T1 > 0.0) && isfinite(T1);
            st1 = sqrt(T1 / P.T_L);
        }
        if (!ok) {
            g.flag |= 2u;
            return true;
        }
        g.nux = ux1;
        g.nuy = uy1;
        g.nst = st1;
        const bool conv = fabs(ux1 - g.ux) < P.eps_abs + P.eps_rel * fabs(ux1) &&
                          fabs(uy1 - g.uy) < P.eps_abs + P.eps_rel * fabs(uy1) &&
                          fabs(st1 - g.st) < P.eps_abs + P.eps_rel * fabs(st1);
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
    // The last pass's populations (this thread's s_acc column) re-expressed
    // in the gauge their moments define (Eq. transform at the node, in
    // correction form f + (G - I) f), then BGK toward rho W in that co-moving
    // gauge (Eq. postcollision) and the store.  A node with non-physical
    // moments keeps its populations and the gauge of its last pass.
    template <int N1>
    static __device__ void finish(const StagedArgs<double>& A, double* s_acc, int NT, int tid,
                                  long long node, const PassGauge& g) {
        constexpr int Q = N1 * N1;
        const Lattice& L = lat<N1>();
        double f[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) f[q] = s_acc[q * NT + tid];
        double ux = g.ux, uy = g.uy, st = g.st;
        if (!(g.flag & 2u)) {
            // xi_a = c_a + c_a (st_n / st_{n+1} - 1) + (u_n - u_{n+1}) / st_{n+1}
            const double inv1 = 1.0 / g.nst;
            const double r = (g.st - g.nst) * inv1;
            const double dx = (g.ux - g.nux) * inv1, dy = (g.uy - g.nuy) * inv1;
            double ex[N1][N1], ey[N1][N1];
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                const double dex = fma(L.c[a], r, dx), dey = fma(L.c[a], r, dy);
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    ex[k][a] = gauge_tail<N1>(L.d3[k], L.d2[k][a], L.d1[k][a], dex) * dex;
                    ey[k][a] = gauge_tail<N1>(L.d3[k], L.d2[k][a], L.d1[k][a], dey) * dey;
                }
            }
            double H[Q];
#pragma unroll
            for (int a = 0; a < N1; ++a)
#pragma unroll
                for (int l = 0; l < N1; ++l) {
                    double v = 0.0;
#pragma unroll
                    for (int b = 0; b < N1; ++b) v = fma(ey[l][b], f[N1 * a + b], v);
                    H[N1 * a + l] = v;
                }
            double o[Q];
#pragma unroll
            for (int k = 0; k < N1; ++k)
#pragma unroll
                for (int l = 0; l < N1; ++l) {
                    double c = H[N1 * k + l];
#pragma unroll
                    for (int a = 0; a < N1; ++a) c = fma(ex[k][a], f[N1 * a + l] + H[N1 * a + l], c);
                    o[N1 * k + l] = f[N1 * k + l] + c;
                }
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = o[q];
            ux = g.nux;
            uy = g.nuy;
            st = g.nst;
        }
        const double two_beta = 2.0 * A.P.beta;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const double feq = g.rho * L.w[q / N1] * L.w[q % N1];
            A.out.f[q * A.plane + node] = f[q] + two_beta * (feq - f[q]);
        }
        A.out.ux[node] = ux;
        A.out.uy[node] = uy;
        A.out.st[node] = st;
    }
};

template <int TY, int N1>
static cudaError_t staged64_shape(size_t smem, int* per_sm, int* s_set) {
    void (*kern)(StagedArgs<double>) = k_step_staged<StagedFP64, 32, TY, N1>;
    if ((int)smem > *s_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        *s_set = (int)smem;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, 32 * TY, smem);
}

cudaError_t staged_prepare_fp64(int ty, int n1, size_t smem, int* ctas_per_sm) {
    static int s_set[64][4] = {{0}};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int slot = (n1 == 3 ? 2 : 0) + (ty == 8 ? 1 : 0);
    if (ty != 4 && ty != 8) return cudaErrorInvalidValue;
    if (n1 == 3)
        return ty == 4 ? staged64_shape<4, 3>(smem, ctas_per_sm, &s_set[dev][slot])
                       : staged64_shape<8, 3>(smem, ctas_per_sm, &s_set[dev][slot]);
    return ty == 4 ? staged64_shape<4, 4>(smem, ctas_per_sm, &s_set[dev][slot])
                   : staged64_shape<8, 4>(smem, ctas_per_sm, &s_set[dev][slot]);
}

cudaError_t launch_step_staged_fp64(const StateBuf<double>& in, const StateBuf<double>& out,
                                    int32_t* iters, DevStats* stats, const GridDesc* grids_dev,
                                    const int64_t* tile_prefix_dev, int n_grids, int64_t n_tiles,
                                    int64_t plane, unsigned int* work_counter,
                                    const TileWindow& win, int persistent_ctas, const Lattice& L,
                                    const StepParams& P, cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    if (win.n1 != L.n1 || (win.ty != 4 && win.ty != 8) || win.tx != 32) return cudaErrorInvalidValue;
    StagedArgs<double> A{};
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
    const size_t smem = staged_smem_bytes(L.n1, win.ww, win.wh, 32 * win.ty, sizeof(double));
    unsigned int nb;
    if (work_counter) {
        cudaError_t e = cudaMemsetAsync(work_counter, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
        nb = (unsigned int)(persistent_ctas < n_tiles ? persistent_ctas : n_tiles);
    } else {
        nb = (unsigned int)n_tiles;
    }
    if (L.n1 == 3) {
        if (win.ty == 4) k_step_staged<StagedFP64, 32, 4, 3><<<nb, 128, smem, s>>>(A);
        else k_step_staged<StagedFP64, 32, 8, 3><<<nb, 256, smem, s>>>(A);
    } else {
        if (win.ty == 4) k_step_staged<StagedFP64, 32, 4, 4><<<nb, 128, smem, s>>>(A);
        else k_step_staged<StagedFP64, 32, 8, 4><<<nb, 256, smem, s>>>(A);
    }
    return cudaGetLastError();
}

}  // namespace pond

// ----------------------------------------------------------------------------
// FP64 step without a context and without any allocation.
//
// For callers that cannot allocate device memory: code running where
// cudaMalloc is not allowed or not wanted (inside a host callback, a custom
// allocator or memory pool, a process whose device memory is fully reserved
// by its framework, a real-time loop that must not enter the allocator).
// They pass their own input and output arrays; the only extra device memory
// the step needs -- sqrt(T / T_L) of the input and output gauges and the step
// counters -- lives in the file-scope array below, which every GPU that loads
// this library holds until the process exits (2 x 8 x 262144 + 256 bytes).
namespace pond {

constexpr int64_t kNoAllocMaxNodes = POND_NOALLOC_MAX_NODES;
constexpr size_t kNoAllocStatsOffset = 2 * sizeof(double) * (size_t)kNoAllocMaxNodes;
constexpr size_t kNoAllocBytes = kNoAllocStatsOffset + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__global__ void k_noalloc_t_to_st(const double* __restrict__ T, double* __restrict__ st,
                                  long long N, double T_L) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) st[i] = sqrt(T[i] / T_L);
}

__global__ void k_noalloc_st_to_t(const double* __restrict__ st, double* __restrict__ T,
                                  long long N, double T_L) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const double s = st[i];
        T[i] = s * s * T_L;
    }
}

static_assert(sizeof(DevStats) <= 256 && alignof(DevStats) <= 256,
              "the step counters must fit the 256-byte tail of the scratch array");
static_assert(kNoAllocStatsOffset % 256 == 0, "the counters' tail must stay 256-byte aligned");

namespace {
std::mutex g_noalloc_mu;
// per device: id of the context whose constant bank holds the lattice
unsigned long long g_noalloc_ctx[256] = {0};

// Unique id of the calling thread's current context (0 if it cannot be
// read).  A device reset or a released and re-created primary context gives
// a new id, which tells the set-up below to upload the constants again.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             nullptr) == cudaSuccess)
            get_current = reinterpret_cast<GetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault,
                                             nullptr) == cudaSuccess)
            get_id = reinterpret_cast<GetId>(p);
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c ||
        get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}
}  // namespace

// Every call, with the device current: the device address of the scratch
// array (its name in host code is only a host-side stand-in; the lookup
// allocates nothing, but on the first call in a context it may make the
// driver load this module, which places the array), and, once per context,
// the lattice constants of this translation unit (a synchronous copy).
static cudaError_t noalloc_setup(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (id == 0 || g_noalloc_ctx[dev] != id) {
        e = upload_lattice_fp64();
        if (e != cudaSuccess) return e;
        g_noalloc_ctx[dev] = id;
    }
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

}  // namespace pond

extern "C" pond_status pond_step_fp64_noalloc(const pond_config* cfg, int32_t nx, int32_t ny,
                                              const double* f_in, const double* ux_in,
                                              const double* uy_in, const double* T_in,
                                              double* f_out, double* ux_out, double* uy_out,
                                              double* T_out, int32_t* iters, pond_stats* stats,
                                              void* cuda_stream) {
    using namespace pond;
    if (!cfg || !f_in || !ux_in || !uy_in || !T_in || !f_out || !ux_out || !uy_out || !T_out)
        return POND_ERR_ARG;
    if (cfg->precision != POND_FP64 || !(cfg->nu > 0.0) || !(cfg->T_ref > 0.0) ||
        !(cfg->dt > 0.0) || cfg->max_iter < 1 || cfg->fixed_iter < 0 || cfg->seed_mode < 0 ||
        cfg->seed_mode > 2 || (cfg->lattice != POND_D2Q16 && cfg->lattice != POND_D2Q9) ||
        !fp64_npw_valid(cfg->nodes_per_warp, cfg->lattice))
        return POND_ERR_ARG;
    if (nx < 1 || ny < 1 || (int64_t)nx * ny > kNoAllocMaxNodes) return POND_ERR_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return POND_ERR_CUDA;
    unsigned char* scratch = nullptr;
    e = noalloc_setup(dev, &scratch);
    if (e != cudaSuccess) return POND_ERR_CUDA;

    const Lattice L = make_lattice(cfg->lattice);
    StepParams P;
    P.beta = 1.0 / (2.0 * cfg->nu / (cfg->T_ref * cfg->dt) + 1.0);
    P.dt = cfg->dt;
    P.eps_abs = cfg->eps_abs;
    P.eps_rel = cfg->eps_rel;
    P.T_L = L.T_L;
    P.max_iter = cfg->max_iter;
    P.fixed_iter = cfg->fixed_iter;
    P.thermal = cfg->thermal;
    P.seed_mode = cfg->seed_mode;

    const long long N = (long long)nx * ny;
    double* st_in = reinterpret_cast<double*>(scratch);
    double* st_out = st_in + kNoAllocMaxNodes;
    DevStats* dstats = reinterpret_cast<DevStats*>(scratch + kNoAllocStatsOffset);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    // the counters keep the previous call's values: they must start at zero
    e = cudaMemsetAsync(dstats, 0, sizeof(DevStats), s);
    if (e != cudaSuccess) return POND_ERR_CUDA;
    const unsigned nb = (unsigned)((N + 255) / 256);
    k_noalloc_t_to_st<<<nb, 256, 0, s>>>(T_in, st_in, N, L.T_L);
    StateBuf<double> in, out;
    in.f = const_cast<double*>(f_in);
    in.ux = const_cast<double*>(ux_in);
    in.uy = const_cast<double*>(uy_in);
    in.st = st_in;
    out.f = f_out;
    out.ux = ux_out;
    out.uy = uy_out;
    out.st = st_out;
    e = launch_step_fp64(in, out, iters, dstats, nx, ny, L, P,
                         cfg->nodes_per_warp ? cfg->nodes_per_warp : fp64_default_npw(L.n1), s);
    if (e != cudaSuccess) return POND_ERR_CUDA;
    k_noalloc_st_to_t<<<nb, 256, 0, s>>>(st_out, T_out, N, L.T_L);
    e = cudaGetLastError();
    if (e != cudaSuccess) return POND_ERR_CUDA;
    if (stats) {
        DevStats h;
        e = cudaMemcpyAsync(&h, dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return POND_ERR_CUDA;
        stats->node_updates = N;
        stats->passes = (int64_t)h.passes;
        stats->max_passes = (int32_t)h.max_passes;
        stats->tile_rows = 0;
        stats->nonconverged = (int64_t)h.nonconverged;
        stats->nonphysical = (int64_t)h.nonphysical;
        stats->halo_fallback = 0;
        stats->index_faults = (int64_t)h.index_faults;
        if (h.nonphysical) return POND_ERR_NONPHYSICAL;
        if (cfg->strict && h.nonconverged) return POND_ERR_NOT_CONVERGED;
    }
    return POND_OK;
}
