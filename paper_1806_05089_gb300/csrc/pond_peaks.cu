// pond_peaks.cu -- arithmetic-pipe peak probes (measurement utility).
//
// The PonD step is bound by plain ALU arithmetic (the FP64 pipe for the FP64
// form, the FP32 FMA pipe for the mixed form), so its roofline denominators
// are FMA rates, not HBM bandwidth or tensor throughput.  These kernels
// measure them on the device in use: every thread runs eight independent
// fused multiply-add chains (enough independent work per warp to hide the
// pipe latency at full occupancy), the grid is a multiple of the SM count,
// and the host times one launch with CUDA events after a warm-up launch.
// The chains compute a = a b + c with |b| < 1, so values stay bounded; one
// store guarded by an impossible comparison keeps the compiler from
// removing them.
#include <cuda_runtime.h>

#include "../../include/pond.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_fma_chains(T* __restrict__ sink, int iters, T b, T c) {
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == (T)-12345.0) sink[0] = s;
}

// Packed FP32: fma.rn.f32x2 issues two FP32 FMAs per thread instruction.
__global__ void __launch_bounds__(kThreads)
k_fma_chains_f32x2(float* __restrict__ sink, int iters, float b, float c) {
    unsigned long long a[kChains];
    const unsigned long long bb =
        ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
    const unsigned long long cc =
        ((unsigned long long)__float_as_uint(c) << 32) | __float_as_uint(c);
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        const unsigned v = __float_as_uint((float)(threadIdx.x + j) * 1e-3f);
        a[j] = ((unsigned long long)v << 32) | v;
    }
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int j = 0; j < kChains; ++j)
                asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(a[j]) : "l"(a[j]), "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        s += __uint_as_float((unsigned)(a[j] & 0xffffffffu)) + __uint_as_float((unsigned)(a[j] >> 32));
    if (s == -12345.f) sink[0] = s;
}

}  // namespace

extern "C" pond_status pond_measure_peak(int32_t pipe, int32_t iters, void* sink,
                                         void* cuda_stream, double* tflops, double* seconds) {
    if (!tflops || !sink || iters < 1 || pipe < POND_PIPE_FP64 || pipe > POND_PIPE_FP32X2)
        return POND_ERR_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return POND_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return POND_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    if (pipe == POND_PIPE_FP64)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<double>, kThreads, 0);
    else if (pipe == POND_PIPE_FP32)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<float>, kThreads, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains_f32x2, kThreads, 0);
    if (e != cudaSuccess || per_sm < 1) return POND_ERR_CUDA;
    const unsigned grid = (unsigned)(sms * per_sm);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return POND_ERR_CUDA;
    }
    auto launch = [&]() {
        if (pipe == POND_PIPE_FP64)
            k_fma_chains<double><<<grid, kThreads, 0, s>>>(static_cast<double*>(sink), iters,
                                                          0.999999, 1e-7);
        else if (pipe == POND_PIPE_FP32)
            k_fma_chains<float><<<grid, kThreads, 0, s>>>(static_cast<float*>(sink), iters,
                                                         0.9999f, 1e-4f);
        else
            k_fma_chains_f32x2<<<grid, kThreads, 0, s>>>(static_cast<float*>(sink), iters,
                                                         0.9999f, 1e-4f);
    };
    launch();  // warm-up (module load, clocks)
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || !(ms > 0.f)) return POND_ERR_CUDA;
    const double fmas_per_thread = (double)iters * 16 * kChains * (pipe == POND_PIPE_FP32X2 ? 2 : 1);
    const double flops = 2.0 * fmas_per_thread * (double)grid * kThreads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    if (seconds) *seconds = ms * 1e-3;
    return POND_OK;
}
