// pond_common.cu -- lattice constants, state initialisation / read-out and
// displacement bounds for the PonD library.
#include <cmath>

#include "pond_device.cuh"

namespace pond {

// Lattice constants from their closed forms -- D2Q16: He4 roots and their
// Gauss-Hermite weights; D2Q9: c = -1, 0, 1, W = 1/6, 2/3, 1/6, T_L = 1/3
// (App. A) -- and the Taylor coefficients of the Lagrange basis polynomials
// L_k(x) = prod_{j != k} (x - c_j)/(c_k - c_j) around each speed c_a.
Lattice make_lattice(int kind) {
    Lattice L{};
    if (kind == POND_D2Q9) {
        L.n1 = 3;
        L.c[0] = -1.0;
        L.c[1] = 0.0;
        L.c[2] = 1.0;
        L.w[0] = L.w[2] = 1.0 / 6.0;
        L.w[1] = 2.0 / 3.0;
        L.T_L = 1.0 / 3.0;
    } else {
        const double s6 = std::sqrt(6.0);
        L.n1 = 4;
        L.c[0] = -std::sqrt(3.0 + s6);
        L.c[1] = -std::sqrt(3.0 - s6);
        L.c[2] = std::sqrt(3.0 - s6);
        L.c[3] = std::sqrt(3.0 + s6);
        L.w[0] = L.w[3] = (3.0 - s6) / 12.0;
        L.w[1] = L.w[2] = (3.0 + s6) / 12.0;
        L.T_L = 1.0;
    }
    const int n1 = L.n1;
    L.q = n1 * n1;
    L.c_max = L.c[n1 - 1];
    for (int k = 0; k < n1; ++k) {
        double p[4] = {1.0, 0.0, 0.0, 0.0};  // coefficients of x^0..x^3
        double den = 1.0;
        for (int j = 0; j < n1; ++j) {
            if (j == k) continue;
            double np[4] = {0.0, 0.0, 0.0, 0.0};
            for (int i = 0; i < 4; ++i) {
                if (i + 1 < 4) np[i + 1] += p[i];
                np[i] -= L.c[j] * p[i];
            }
            for (int i = 0; i < 4; ++i) p[i] = np[i];
            den *= (L.c[k] - L.c[j]);
        }
        for (int i = 0; i < 4; ++i) p[i] /= den;
        for (int a = 0; a < n1; ++a) {
            const double x = L.c[a];
            L.d1[k][a] = p[1] + 2.0 * p[2] * x + 3.0 * p[3] * x * x;
            L.d2[k][a] = p[2] + 3.0 * p[3] * x;
        }
        L.d3[k] = p[3];
    }
    // W-dual basis of {1, |c|^2}: inverse of [[1, 2 T_L], [2 T_L, g]]
    double K4 = 0.0;
    for (int a = 0; a < n1; ++a) K4 += L.w[a] * L.c[a] * L.c[a] * L.c[a] * L.c[a];
    const double g = 2.0 * K4 + 2.0 * L.T_L * L.T_L;
    const double det = g - 4.0 * L.T_L * L.T_L;
    L.pe0 = g / det;
    L.pe2 = -2.0 * L.T_L / det;
    L.pt0 = -2.0 * L.T_L / det;
    L.pt2 = 1.0 / det;
    L.inv_TL = 1.0 / L.T_L;
    return L;
}

LatticeF to_float(const Lattice& L) {
    LatticeF F{};
    for (int i = 0; i < 4; ++i) {
        F.c[i] = (float)L.c[i];
        F.w[i] = (float)L.w[i];
        F.d3[i] = (float)L.d3[i];
        for (int j = 0; j < 4; ++j) {
            F.d1[i][j] = (float)L.d1[i][j];
            F.d2[i][j] = (float)L.d2[i][j];
        }
    }
    F.pe0 = (float)L.pe0;
    F.pe2 = (float)L.pe2;
    F.pt0 = (float)L.pt0;
    F.pt2 = (float)L.pt2;
    F.inv_TL = (float)L.inv_TL;
    return F;
}

// f_q = rho W_q in the node's own gauge (Eq. equilibrium), or a copy of the
// given FP64 populations; T -> sqrt(theta).
template <typename Real>
__global__ void k_init_state(const double* __restrict__ rho, const double* __restrict__ ux,
                             const double* __restrict__ uy, const double* __restrict__ T,
                             const double* __restrict__ f_given, StateBuf<Real> st, int64_t N,
                             int64_t plane, Lattice L) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    st.ux[i] = ux[i];
    st.uy[i] = uy[i];
    st.st[i] = sqrt(T[i] / L.T_L);
    if (f_given) {
        for (int q = 0; q < L.q; ++q) st.f[q * plane + i] = (Real)f_given[q * N + i];
    } else {
        const double r = rho[i];
        for (int q = 0; q < L.q; ++q)
            st.f[q * plane + i] = (Real)(r * L.w[q / L.n1] * L.w[q % L.n1]);
    }
}

template <typename Real>
cudaError_t launch_init_state(const double* rho, const double* ux, const double* uy,
                              const double* T, const double* f_given, StateBuf<Real> st,
                              int64_t N, int64_t plane, const Lattice& L, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const int bs = 256;
    const unsigned nb = (unsigned)((N + bs - 1) / bs);
    k_init_state<Real><<<nb, bs, 0, s>>>(rho, ux, uy, T, f_given, st, N, plane, L);
    return cudaGetLastError();
}

template <typename Real>
__global__ void k_read_state(StateBuf<Real> st, int64_t N, int64_t plane, double* rho,
                             double* ux, double* uy, double* T, double* f, Lattice L) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double r = 0.0;
    for (int q = 0; q < L.q; ++q) {
        const double v = (double)st.f[q * plane + i];
        r += v;
        if (f) f[q * N + i] = v;
    }
    if (rho) rho[i] = r;
    if (ux) ux[i] = st.ux[i];
    if (uy) uy[i] = st.uy[i];
    if (T) {
        const double s = st.st[i];
        T[i] = s * s * L.T_L;
    }
}

template <typename Real>
cudaError_t launch_read_state(StateBuf<Real> st, int64_t N, int64_t plane, double* rho,
                              double* ux, double* uy, double* T, double* f, const Lattice& L,
                              cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const int bs = 256;
    const unsigned nb = (unsigned)((N + bs - 1) / bs);
    k_read_state<Real><<<nb, bs, 0, s>>>(st, N, plane, rho, ux, uy, T, f, L);
    return cudaGetLastError();
}

template cudaError_t launch_init_state<double>(const double*, const double*, const double*,
                                               const double*, const double*, StateBuf<double>,
                                               int64_t, int64_t, const Lattice&, cudaStream_t);
template cudaError_t launch_init_state<float>(const double*, const double*, const double*,
                                              const double*, const double*, StateBuf<float>,
                                              int64_t, int64_t, const Lattice&, cudaStream_t);
template cudaError_t launch_read_state<double>(StateBuf<double>, int64_t, int64_t, double*,
                                               double*, double*, double*, double*,
                                               const Lattice&, cudaStream_t);
template cudaError_t launch_read_state<float>(StateBuf<float>, int64_t, int64_t, double*,
                                              double*, double*, double*, double*,
                                              const Lattice&, cudaStream_t);

// Bounds of the particle velocities over a grid: out4 = {min(u_x - c_max st),
// max(u_x + c_max st), min(u_y - c_max st), max(u_y + c_max st)} (as floats,
// combined by integer atomics on an order-preserving encoding).
__device__ __forceinline__ unsigned int f2ord(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_disp_bounds(const double* __restrict__ ux, const double* __restrict__ uy,
                              const double* __restrict__ st, int64_t N, double cmax,
                              unsigned int* out5) {
    float lo_x = 3.0e38f, hi_x = -3.0e38f, lo_y = 3.0e38f, hi_y = -3.0e38f;
    unsigned int bad = 0u;  // nodes with s <= 0 or a non-finite gauge
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = ux[i], y = uy[i], t = st[i];
        bad += (t > 0.0 && isfinite(t) && isfinite(x) && isfinite(y)) ? 0u : 1u;
        const double s = cmax * t;
        lo_x = fminf(lo_x, (float)(x - s));
        hi_x = fmaxf(hi_x, (float)(x + s));
        lo_y = fminf(lo_y, (float)(y - s));
        hi_y = fmaxf(hi_y, (float)(y + s));
    }
    // warp, then block reduction: one atomic per block and value (atomics on
    // one address serialise, so one per warp would dominate the pass)
    __shared__ float s_b[4][32];
    __shared__ unsigned int s_bad[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int pass = 0; pass < 2; ++pass) {
        for (int o = 16; o > 0; o >>= 1) {
            lo_x = fminf(lo_x, __shfl_xor_sync(0xffffffffu, lo_x, o));
            hi_x = fmaxf(hi_x, __shfl_xor_sync(0xffffffffu, hi_x, o));
            lo_y = fminf(lo_y, __shfl_xor_sync(0xffffffffu, lo_y, o));
            hi_y = fmaxf(hi_y, __shfl_xor_sync(0xffffffffu, hi_y, o));
        }
        bad = __reduce_add_sync(0xffffffffu, bad);
        if (pass == 1) break;
        if (lane == 0) {
            s_b[0][warp] = lo_x;
            s_b[1][warp] = hi_x;
            s_b[2][warp] = lo_y;
            s_b[3][warp] = hi_y;
            s_bad[warp] = bad;
        }
        __syncthreads();
        if (warp != 0) return;
        const bool in = lane < (int)(blockDim.x >> 5);
        lo_x = in ? s_b[0][lane] : 3.0e38f;
        hi_x = in ? s_b[1][lane] : -3.0e38f;
        lo_y = in ? s_b[2][lane] : 3.0e38f;
        hi_y = in ? s_b[3][lane] : -3.0e38f;
        bad = in ? s_bad[lane] : 0u;
    }
    if (lane == 0) {
        atomicMin(out5 + 0, f2ord(lo_x));
        atomicMax(out5 + 1, f2ord(hi_x));
        atomicMin(out5 + 2, f2ord(lo_y));
        atomicMax(out5 + 3, f2ord(hi_y));
        if (bad) atomicAdd(out5 + 4, bad);
    }
}

__global__ void k_ord_to_float(unsigned int* v) {
    const int i = threadIdx.x;
    if (i < 4) {
        const unsigned int u = v[i];
        const unsigned int b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
        v[i] = b;  // now the float bit pattern
    }
}

__global__ void k_bounds_reset(unsigned int* v) {
    const int i = threadIdx.x;
    if (i < 4) v[i] = (i & 1) ? 0u : 0xffffffffu;
    if (i == 4) v[4] = 0u;
}

// Halo strips of a domain decomposition: a rectangle of the state to or from
// a contiguous device buffer.  The stored representation moves unchanged
// (populations widened to FP64 exactly, the gauge as stored), so a state
// split over sub-domains and reassembled is bit-identical.
template <typename Real>
__global__ void k_pack_rect(StateBuf<Real> st, int nx, int x0, int y0, int w, int h, int q,
                            long long plane, double* __restrict__ buf) {
    const long long n = (long long)w * h;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long node = (long long)(y0 + i / w) * nx + x0 + i % w;
    for (int c = 0; c < q; ++c) buf[c * n + i] = (double)st.f[c * plane + node];
    buf[q * n + i] = st.ux[node];
    buf[(q + 1) * n + i] = st.uy[node];
    buf[(q + 2) * n + i] = st.st[node];
}

template <typename Real>
__global__ void k_unpack_rect(StateBuf<Real> st, int nx, int x0, int y0, int w, int h, int q,
                              long long plane, const double* __restrict__ buf) {
    const long long n = (long long)w * h;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long node = (long long)(y0 + i / w) * nx + x0 + i % w;
    for (int c = 0; c < q; ++c) st.f[c * plane + node] = (Real)buf[c * n + i];
    st.ux[node] = buf[q * n + i];
    st.uy[node] = buf[(q + 1) * n + i];
    st.st[node] = buf[(q + 2) * n + i];
}

template <typename Real>
cudaError_t launch_pack_rect(StateBuf<Real> st, int nx, int x0, int y0, int w, int h, int q,
                             int64_t plane, double* buf, cudaStream_t s) {
    const long long n = (long long)w * h;
    if (n == 0) return cudaSuccess;
    k_pack_rect<Real><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(st, nx, x0, y0, w, h, q, plane, buf);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_unpack_rect(StateBuf<Real> st, int nx, int x0, int y0, int w, int h, int q,
                               int64_t plane, const double* buf, cudaStream_t s) {
    const long long n = (long long)w * h;
    if (n == 0) return cudaSuccess;
    k_unpack_rect<Real><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(st, nx, x0, y0, w, h, q, plane, buf);
    return cudaGetLastError();
}

template cudaError_t launch_pack_rect<double>(StateBuf<double>, int, int, int, int, int, int,
                                              int64_t, double*, cudaStream_t);
template cudaError_t launch_pack_rect<float>(StateBuf<float>, int, int, int, int, int, int,
                                             int64_t, double*, cudaStream_t);
template cudaError_t launch_unpack_rect<double>(StateBuf<double>, int, int, int, int, int, int,
                                                int64_t, const double*, cudaStream_t);
template cudaError_t launch_unpack_rect<float>(StateBuf<float>, int, int, int, int, int, int,
                                               int64_t, const double*, cudaStream_t);

cudaError_t launch_disp_bounds(const double* ux, const double* uy, const double* st, int64_t N,
                               double c_max, float* out5, cudaStream_t s) {
    unsigned int* o = reinterpret_cast<unsigned int*>(out5);
    k_bounds_reset<<<1, 32, 0, s>>>(o);
    const int bs = 256;
    int64_t nb = (N + bs - 1) / bs;
    if (nb > 256) nb = 256;
    if (nb < 1) nb = 1;
    k_disp_bounds<<<(unsigned)nb, bs, 0, s>>>(ux, uy, st, N, c_max, o);
    k_ord_to_float<<<1, 32, 0, s>>>(o);
    return cudaGetLastError();
}

}  // namespace pond
