// Measurement utility: the device's FP64 and FP32 fused multiply-add rates.
//
// The FP64 product is bound by FP64 arithmetic (its FFT passes), not by
// memory, so its roofline needs an FP64 peak; none is supplied with the
// device, so it is measured here: every thread runs independent FMA chains
// (enough of them to hide the pipeline latency), timed with CUDA events.
#include <cuda_runtime.h>

#include "gofd_internal.cuh"

namespace gofd {

constexpr int FMA_CHAINS = 8;
constexpr int FMA_STEPS = 4096;

template <class T>
__global__ void __launch_bounds__(256) fma_rate_kernel(T* out, T a, T b) {
    T x[FMA_CHAINS];
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
    for (int s = 0; s < FMA_STEPS; ++s) {
#pragma unroll
        for (int c = 0; c < FMA_CHAINS; ++c) x[c] = x[c] * a + b;
    }
    T sum = 0;
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) sum += x[c];
    if (sum == (T)-1.2345) out[0] = sum;   // keeps the chains live; never true for these inputs
}

// FLOP/s (2 per FMA) of fma_rate_kernel<T> on the current device, in GFLOP/s
template <class T>
double fma_rate(cudaStream_t st) {
    int dev = 0, sms = 0;
    GOFD_CUDA_TRY(cudaGetDevice(&dev));
    GOFD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DevBuf out;
    out.alloc(sizeof(T));
    const unsigned blocks = (unsigned)sms * 8;
    cudaEvent_t a, b;
    GOFD_CUDA_TRY(cudaEventCreate(&a));
    GOFD_CUDA_TRY(cudaEventCreate(&b));
    fma_rate_kernel<T><<<blocks, 256, 0, st>>>(out.as<T>(), (T)0.999999, (T)1e-7);   // warm-up
    GOFD_CHECK_LAUNCH();
    GOFD_CUDA_TRY(cudaEventRecord(a, st));
    constexpr int reps = 5;
    for (int r = 0; r < reps; ++r) fma_rate_kernel<T><<<blocks, 256, 0, st>>>(out.as<T>(), (T)0.999999, (T)1e-7);
    GOFD_CHECK_LAUNCH();
    GOFD_CUDA_TRY(cudaEventRecord(b, st));
    GOFD_CUDA_TRY(cudaEventSynchronize(b));
    float ms = 0;
    GOFD_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double flops = 2.0 * FMA_CHAINS * FMA_STEPS * 256.0 * blocks * reps;
    return flops / (ms * 1e-3) / 1e9;
}

}  // namespace gofd

extern "C" gofd_status gofd_fma_rates(void* stream, double* fp64_gflops, double* fp32_gflops) {
    try {
        if (fp64_gflops) *fp64_gflops = gofd::fma_rate<double>((cudaStream_t)stream);
        if (fp32_gflops) *fp32_gflops = gofd::fma_rate<float>((cudaStream_t)stream);
        return GOFD_OK;
    } catch (const gofd::Error& e) {
        return e.code;
    }
}
