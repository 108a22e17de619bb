// peak.cu -- measurement utility (not part of the paper's method): the FP64 FMA throughput of
// the current GPU, the denominator of the FP64 rooflines reported for the binary64 stages.
#include <cuda_runtime.h>

#include "internal.h"

namespace mpj {

// Each thread runs kChains independent FMA chains of kIters steps (enough independent work to
// cover the FP64 pipe's latency on every sub-partition). The result is stored only if it is
// impossible (never in practice), so the compiler keeps every FMA.
constexpr int kChains = 8;
constexpr int kIters = 16384;  // about 0.1 s per launch: long enough for the clocks to settle

static __global__ void __launch_bounds__(256) k_fp64_fma(double seed, double* sink)
{
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (double)(threadIdx.x * kChains + c) * 1e-9;
    const double x = 1.0 - 1e-12, y = 1e-13;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.0) *sink = s;
}

static int measure_fp64(cudaStream_t stream, double* tflops)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail("peak: device", e);
    cudaEvent_t ev[2];
    if ((e = cudaEventCreate(&ev[0])) != cudaSuccess) return cuda_fail("peak: event", e);
    if ((e = cudaEventCreate(&ev[1])) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return cuda_fail("peak: event", e);
    }
    const int blocks = sms * 8;  // 2048 threads per SM
    double best = 0.0;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(ev[0], stream);
        k_fp64_fma<<<blocks, 256, 0, stream>>>(1.0 + rep, nullptr);
        cudaEventRecord(ev[1], stream);
        e = cudaEventSynchronize(ev[1]);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e == cudaSuccess && ms > 0.0f && rep > 0) {  // the first launch is a warm-up
            const double flops = 2.0 * (double)blocks * 256.0 * kChains * kIters;
            const double t = flops / (ms * 1e-3) / 1e12;
            if (t > best) best = t;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) return cuda_fail("peak: run", e);
    *tflops = best;
    return 0;
}

}  // namespace mpj

extern "C" int mpjsvd_measure_fp64_peak(void* cuda_stream, double* tflops)
{
    if (!tflops) return -2;
    return mpj::measure_fp64((cudaStream_t)cuda_stream, tflops);
}
