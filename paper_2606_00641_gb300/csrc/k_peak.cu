// k_peak.cu -- FP64 fused multiply-add throughput of the device's CUDA cores.
//
// The FP64 forms of the fused step (and the dissipative model's FP64 form)
// are bound by the FP64 arithmetic pipe on GB300, not by HBM; their roofline
// needs the rate that pipe sustains.  One kernel: every thread runs eight
// independent FMA chains (enough independent work per warp to cover the
// pipe's latency at four 256-thread CTAs per SM), no memory traffic but one
// guarded store that keeps the chains live.
#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 4;
constexpr int kSink = 4096;

// where the guarded store would go (device code names it directly)
__device__ double g_fp64_sink[kSink];

__global__ void __launch_bounds__(kPeakThreads) k_fp64_fma(int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * (threadIdx.x + 1) + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    // never true (every chain stays positive for a, b > 0); keeps the chains live
    if (s == -1.0 && blockIdx.x < kSink) g_fp64_sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace vlbm

extern "C" vlbm_status vlbm_measure_fp64_rate(int iters, void *stream, double *tflops)
{
    using namespace vlbm;
    if (!tflops || iters < 1 || iters > (1 << 20)) return fail(nullptr, VLBM_ERR_ARG, "fp64 rate: bad arguments");
    int dev = 0, sms = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "fp64 rate: device query");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_check(nullptr, e, "fp64 rate: events");
    }
    const unsigned grid = (unsigned)(sms * kPeakCtasPerSm);
    // 0 < a < 1, b > 0: every chain stays positive and bounded (x -> b / (1 - a))
    const double a = 0.999999, b = 1e-6;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
        cudaEventRecord(e0, st);
        k_fp64_fma<<<grid, kPeakThreads, 0, st>>>(iters, a, b);
        e = cudaGetLastError();
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "fp64 rate: launch");
    const double flop = 2.0 * kChains * (double)iters * grid * kPeakThreads;
    *tflops = flop / (best * 1e-3) / 1e12;
    return VLBM_OK;
}
