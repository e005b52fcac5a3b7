// pond_device.cuh -- small device helpers shared by the PonD kernels.
#pragma once

#include "pond_internal.cuh"

namespace pond {

// Debug builds (-DPOND_DEBUG, build.build(debug=True)): index checks on the
// staged kernel's global and shared-memory accesses.  A failed check adds
// one to the step counters' index_faults and the access is skipped (a
// zero is read, nothing is written); nothing traps.  Release builds compile
// the checks away.
#ifdef POND_DEBUG
__device__ __forceinline__ bool pond_index_ok(bool ok, DevStats* st) {
    if (!ok && st) atomicAdd(&st->index_faults, 1ull);
    return ok;
}
#define POND_INDEX_OK(cond, stats) ::pond::pond_index_ok((cond), (stats))
#else
#define POND_INDEX_OK(cond, stats) true
#endif

// The GPU's global nanosecond timer (PTX %globaltimer).
__device__ __forceinline__ unsigned long long pond_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Exit of one CTA of a persistent launch (one thread per CTA): adds its busy
// time and widens the launch's span; the launch's last CTA to exit folds the
// launch into busy_ns and slot_ns (gridDim.x x span) and zeroes the scratch
// for the next launch.  1 - busy/slot is the share of the launch's CTA slots
// left idle, by the start skew and the tail after the work list ran dry.
// No CTA waits on another.
__device__ __forceinline__ void persistent_exit(DevStats* st, unsigned long long t_begin) {
    const unsigned long long t_end = pond_globaltimer();
    atomicAdd(&st->l_busy, t_end - t_begin);
    atomicMax(&st->l_begin_inv, ~t_begin);
    atomicMax(&st->l_end, t_end);
    __threadfence();
    if (atomicAdd(&st->l_done, 1u) == gridDim.x - 1) {
        __threadfence();
        const unsigned long long busy = atomicAdd(&st->l_busy, 0ull);
        const unsigned long long b = ~atomicAdd(&st->l_begin_inv, 0ull);
        const unsigned long long e = atomicAdd(&st->l_end, 0ull);
        st->busy_ns += busy;
        st->slot_ns += (unsigned long long)gridDim.x * (e > b ? e - b : 0ull);
        st->l_busy = 0ull;
        st->l_begin_inv = 0ull;
        st->l_end = 0ull;
        st->l_done = 0u;
    }
}

// Cubic Lagrange weights on the nodes 0, 1, 2, 3 at local coordinate t
// (App. C: a_n(t) = prod_{k != n} (t - k)/(n - k)).
__device__ __forceinline__ void lagrange4(double t, double l[4]) {
    const double a = t, b = t - 1.0, c = t - 2.0, d = t - 3.0;
    const double cd = c * d, ab = a * b;
    l[0] = -(b * cd) * (1.0 / 6.0);
    l[1] = (a * cd) * 0.5;
    l[2] = -(ab * d) * 0.5;
    l[3] = (ab * c) * (1.0 / 6.0);
}

__device__ __forceinline__ void lagrange4f(float t, float l[4]) {
    const float a = t, b = t - 1.0f, c = t - 2.0f, d = t - 3.0f;
    const float cd = c * d, ab = a * b;
    l[0] = -(b * cd) * (1.0f / 6.0f);
    l[1] = (a * cd) * 0.5f;
    l[2] = -(ab * d) * 0.5f;
    l[3] = (ab * c) * (1.0f / 6.0f);
}

// The same weights at t = s + 3/2, from the centred coordinate s in
// [-1/2, 1/2): the factors t - j are then s + 3/2, s + 1/2, s - 1/2, s - 3/2,
// each within half an FP32 unit of [1/2, 2) of its exact value, instead of
// carrying the rounding of t in [1, 2).
__device__ __forceinline__ void lagrange4f_centred(float s, float l[4]) {
    const float a = s + 1.5f, b = s + 0.5f, c = s - 0.5f, d = s - 1.5f;
    const float cd = c * d, ab = a * b;
    l[0] = -(b * cd) * (1.0f / 6.0f);
    l[1] = (a * cd) * 0.5f;
    l[2] = -(ab * d) * 0.5f;
    l[3] = (ab * c) * (1.0f / 6.0f);
}

// One entry of the 1D gauge transform in Taylor form around the identity,
// G[k][a] = id + de (d1 + d2 de (+ d3 de^2 on D2Q16, where L_k is cubic; on
// D2Q9 L_k is quadratic and d3 = 0)).  gauge_tail is the bracket, G - I
// divided by de.
template <int N1, typename T>
__device__ __forceinline__ T gauge_tail(T d3, T d2, T d1, T de) {
    if constexpr (N1 == 4)
        return fma(fma(d3, de, d2), de, d1);
    else
        return fma(d2, de, d1);
}

template <int N1, typename T>
__device__ __forceinline__ T gauge_poly(T d3, T d2, T d1, T id, T de) {
    return fma(gauge_tail<N1>(d3, d2, d1, de), de, id);
}

// Periodic wrap of a possibly far out-of-range index.
__device__ __forceinline__ int wrap_idx(long long v, int n) {
    long long r = v % n;
    return (int)(r < 0 ? r + n : r);
}

// Index + small offset (0..3) wrapped, for an already wrapped base.
__device__ __forceinline__ int wrap_inc(int base, int off, int n) {
    int v = base + off;
    while (v >= n) v -= n;
    return v;
}

}  // namespace pond
