// FP64 pipe rate of the GPU, measured: the roofline of the FP64 kernels here (integrals, FP64 J and K,
// FP64 whitening and SCF algebra) is the FP64 pipe, not HBM, so its denominator is taken on the same
// device by two loops, timed with CUDA events:
//   - DFMA: every thread runs 8 independent fused multiply-add chains, 4 CTAs of 256 threads per SM;
//   - DMMA: every warp runs 4 independent mma.sync m8n8k4 FP64 accumulations (256 multiply-adds each).
// Both count 2 flops per multiply-add. The values stay bounded (multipliers below 1 in magnitude) and
// are folded into a sink that is written only if the loop result were NaN, so nothing is optimised out.
#include "common.cuh"

namespace dfhf {
namespace {

constexpr int THREADS = 256;
constexpr int CHAINS = 8;

__global__ void __launch_bounds__(THREADS) dfma_loop_kernel(long long iters, double a, double c, double* sink) {
    double x[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) x[j] = 1e-3 * (double)(threadIdx.x + j);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < CHAINS; ++j) x[j] = fma(x[j], a, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += x[j];
    if (s != s) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(THREADS) dmma_loop_kernel(long long iters, double a, double b, double* sink) {
    double d[4][2];
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j][0] = d[j][1] = 0.0;
    const double av = a * (1.0 + 1e-3 * (threadIdx.x & 31));
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                         : "+d"(d[j][0]), "+d"(d[j][1])
                         : "d"(av), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) s += d[j][0] + d[j][1];
    if (s != s) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace dfhf

extern "C" int df_fp64_rate(int kind, long long iters, double* tflops, double* ms) {
    using namespace dfhf;
    if ((kind != 0 && kind != 1) || iters < 1 || !tflops) return DF_E_ARG;
    double* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DF_OK;
    try {
        int dev = 0, sms = 0;
        DF_CUDA(cudaGetDevice(&dev));
        DF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int grid = 4 * sms;
        DF_CUDA(cudaMalloc((void**)&sink, sizeof(double) * grid));
        DF_CUDA(cudaEventCreate(&e0));
        DF_CUDA(cudaEventCreate(&e1));
        auto launch = [&](long long it) {
            if (kind == 0) dfma_loop_kernel<<<grid, THREADS>>>(it, 0.9999999, 1e-7, sink);
            else dmma_loop_kernel<<<grid, THREADS>>>(it, 0.5, 1e-7, sink);
            DF_CHECK_LAUNCH();
        };
        launch(iters / 16 + 1);   // warm-up: module load, clocks up
        DF_CUDA(cudaEventRecord(e0));
        launch(iters);
        DF_CUDA(cudaEventRecord(e1));
        DF_CUDA(cudaEventSynchronize(e1));
        float t = 0.f;
        DF_CUDA(cudaEventElapsedTime(&t, e0, e1));
        const double fma_count = kind == 0 ? (double)grid * THREADS * CHAINS * (double)iters
                                           : (double)grid * (THREADS / 32) * 4 * 256.0 * (double)iters;
        *tflops = 2.0 * fma_count / (t * 1e-3) / 1e12;
        if (ms) *ms = t;
    } catch (const Error& e) {
        rc = e.code;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}
