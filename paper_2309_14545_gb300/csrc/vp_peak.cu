// Measured FP32 FMA throughput of the device: the denominator the validation
// kernels' FLOP rate is also reported against (beside the one derived from
// lane counts and the clock).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/vp.h"

namespace {

// Eight independent FMA chains per thread: enough to cover the FMA latency at
// full occupancy, so the pipe, not dependencies, sets the rate.
__global__ void __launch_bounds__(256) ffma_chains_kernel(float x, float y, int iters, float *sink) {
    float a0 = threadIdx.x * 1e-7f, a1 = a0 + 1.f, a2 = a0 + 2.f, a3 = a0 + 3.f;
    float a4 = a0 + 4.f, a5 = a0 + 5.f, a6 = a0 + 6.f, a7 = a0 + 7.f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            a0 = fmaf(a0, x, y); a1 = fmaf(a1, x, y); a2 = fmaf(a2, x, y); a3 = fmaf(a3, x, y);
            a4 = fmaf(a4, x, y); a5 = fmaf(a5, x, y); a6 = fmaf(a6, x, y); a7 = fmaf(a7, x, y);
        }
    }
    const float s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == 12345.678f) *sink = s;  // keeps the chains alive; never true for these inputs
}

}  // namespace

extern "C" vp_status vp_measure_fp32_peak(int device, double seconds, double *tflops) {
    if (!tflops || !(seconds > 0.0) || seconds > 60.0) return VP_ERR_ARG;
    *tflops = 0.0;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return VP_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return VP_ERR_ARG;
    int sms = 0, bps = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, ffma_chains_kernel, 256, 0);
    float *sink = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    double best = 0.0;
    if (e == cudaSuccess) {
        const int grid = sms * std::max(bps, 1);
        const double flops_per_iter = static_cast<double>(grid) * 256 * 16 * 8 * 2;
        int iters = 256;
        auto run = [&](float *ms) {
            cudaEventRecord(t0);
            ffma_chains_kernel<<<grid, 256>>>(1.0000001f, -1e-7f, iters, sink);
            cudaEventRecord(t1);
            e = cudaEventSynchronize(t1);
            if (e == cudaSuccess) e = cudaGetLastError();
            *ms = 0.f;
            if (e == cudaSuccess) cudaEventElapsedTime(ms, t0, t1);
        };
        // grow one launch to about a quarter of `seconds`, then keep the best of three
        float ms = 0.f;
        run(&ms);
        while (e == cudaSuccess && ms < 250.0 * seconds && iters < (1 << 24)) {
            iters *= 2;
            run(&ms);
        }
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            run(&ms);
            if (e == cudaSuccess && ms > 0.f) best = std::max(best, flops_per_iter * iters / (ms * 1e-3) / 1e12);
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (sink) cudaFree(sink);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return VP_ERR_CUDA;
    *tflops = best;
    return best > 0.0 ? VP_OK : VP_ERR_CUDA;
}
