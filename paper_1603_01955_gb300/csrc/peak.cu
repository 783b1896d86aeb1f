// Fused multiply-add throughput of the GPU in FP32 or FP64: the compute peak
// that the measured FLOP rate of a sweep is set against.  Every thread runs
// kChains independent dependency chains of fused multiply-adds, enough to
// hide the pipe latency; the grid fills every SM several times over.  The
// chains converge to a fixed point near 1, so no value overflows or becomes
// subnormal, and a store that never happens keeps them live.
#include <cuda_runtime.h>

#include "../../include/clb.h"
#include "clb_internal.h"

namespace {

constexpr int kChains = 8;

// Where a result would go if the chains ever summed to -1 (they do not).
__device__ float g_sink_f;
__device__ double g_sink_d;
__device__ __forceinline__ float* sink(float) { return &g_sink_f; }
__device__ __forceinline__ double* sink(double) { return &g_sink_d; }
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

template <class R>
__global__ void __launch_bounds__(kThreads) peak_fma_kernel(int iters, R b, R c) {
    R acc[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = R(1) + R(j) * R(1e-3) + R(threadIdx.x) * R(1e-6);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) acc[j] = fma(acc[j], b, c);
    }
    R s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += acc[j];
    if (s == R(-1)) *sink(s) = s;  // never true: keeps the chains from being removed
}

template <class R>
cudaError_t time_peak(cudaStream_t st, int iters, double* tflops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const dim3 grid(sms * kBlocksPerSm), block(kThreads);
    const R b = R(0.999), c = R(0.001);  // fixed point c / (1 - b) = 1
    peak_fma_kernel<R><<<grid, block, 0, st>>>(iters / 8, b, c);  // warm-up
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    cudaEventRecord(e0, st);
    peak_fma_kernel<R><<<grid, block, 0, st>>>(iters, b, c);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * kChains * (double)iters * grid.x * block.x;
    *tflops = ms > 0 ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return cudaSuccess;
}

}  // namespace

extern "C" clb_status clb_peak_fma(int storage, void* stream, double* tflops) {
    clb::TraceRange trace_("clb_peak_fma");
    if (!tflops) return (clb_status)clb::set_error(CLB_EINVAL, "clb_peak_fma: tflops is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (storage == CLB_FP64)
        e = time_peak<double>(st, 1 << 12, tflops);
    else if (storage == CLB_FP32_SHIFTED)
        e = time_peak<float>(st, 1 << 16, tflops);
    else
        return (clb_status)clb::set_error(CLB_EINVAL, "clb_peak_fma: storage must be CLB_FP64 or CLB_FP32_SHIFTED");
    if (e != cudaSuccess) return (clb_status)clb::set_error(CLB_ECUDA, "clb_peak_fma: %s", cudaGetErrorString(e));
    return CLB_OK;
}
