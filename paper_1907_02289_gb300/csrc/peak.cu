// peak.cu -- bh_measure_peak: the arithmetic peak of the device, measured
// with independent fused multiply-add chains (no memory traffic in the timed
// loop), for the roofline denominators of the FP32 and FP64 force kernels.
#include "bh_internal.cuh"

namespace bh {
namespace {

constexpr int kChains = 8;    // independent FMA chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(T* out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll 16
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int measure(int iters, double* tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
        cudaGetLastError();
        return BH_E_CUDA;
    }
    const unsigned blocks = (unsigned)(sms * kBlocksPerSm);
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * kThreads) != cudaSuccess) {
        cudaGetLastError();
        return BH_E_NOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const T a = (T)0.999999, b = (T)1e-3;
    if (e == cudaSuccess) {
        k_fma_peak<T><<<blocks, kThreads>>>(out, iters, a, b);  // warm-up
        e = cudaGetLastError();
    }
    float best = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0);
        if (e == cudaSuccess) k_fma_peak<T><<<blocks, kThreads>>>(out, iters, a, b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return BH_E_CUDA;
    }
    const double flops = 2.0 * kChains * 16.0 * (double)iters * (double)blocks * kThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return BH_OK;
}

}  // namespace
}  // namespace bh

extern "C" int bh_measure_peak(int kind, double* tflops) {
    if (!tflops) return BH_E_INVAL;
    // about 2.6e12 FP32 flops (~35 ms at peak) and 8e10 FP64 flops per timed launch
    if (kind == BH_PEAK_FP32) return bh::measure<float>(32768, tflops);
    if (kind == BH_PEAK_FP64) return bh::measure<double>(1024, tflops);
    return BH_E_INVAL;
}
