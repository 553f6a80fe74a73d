// fp64_probe.cu -- FP64 throughput probe (include/fp64_probe.h): independent DFMA chains and
// FP64 mma.sync (DMMA m8n8k4) tiles, timed with CUDA events.  Each kernel runs a fixed
// number of iterations and stores one value per thread, nothing else.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fp64_probe.h"

namespace {

constexpr int kThreads = 256;
constexpr int kSink = 1 << 17;  // doubles in the sink buffer (1 MB)

// 8 independent chains per thread: x_k <- x_k * a + b, 16 flops per iteration.
__global__ void k_dfma(int iters, double a, double b, double* sink) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    sink[(blockIdx.x * blockDim.x + threadIdx.x) & (kSink - 1)] = s;
}

// 4 independent m8n8k4 accumulators per warp: D <- A B + D, each 8 x 8 x 4 FMAs per warp.
__global__ void k_dmma(int iters, double a, double b, double* sink) {
    double acc[4][2];
#pragma unroll
    for (int k = 0; k < 4; ++k) { acc[k][0] = 1e-3 * k; acc[k][1] = 2e-3 * k; }
    const double fa = a + 1e-6 * (threadIdx.x & 31), fb = b;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(acc[k][0]), "+d"(acc[k][1]) : "d"(fa), "d"(fb));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += acc[k][0] + acc[k][1];
    sink[(blockIdx.x * blockDim.x + threadIdx.x) & (kSink - 1)] = s;
}

// half the blocks run DFMA chains, half DMMA tiles
__global__ void k_mixed(int iters, double a, double b, double* sink) {
    if (blockIdx.x & 1) {
        double acc[4][2];
#pragma unroll
        for (int k = 0; k < 4; ++k) { acc[k][0] = 1e-3 * k; acc[k][1] = 2e-3 * k; }
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                             : "+d"(acc[k][0]), "+d"(acc[k][1]) : "d"(a), "d"(b));
        }
        sink[(blockIdx.x * blockDim.x + threadIdx.x) & (kSink - 1)] = acc[0][0] + acc[3][1];
    } else {
        double x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
        }
        sink[(blockIdx.x * blockDim.x + threadIdx.x) & (kSink - 1)] = x[0] + x[7];
    }
}

std::mutex g_mu;
double* g_sink[64] = {};

}  // namespace

extern "C" int fp64_probe_run(int kind, int iters, void* stream, double* tflops, float* ms) {
    if (kind < 0 || kind > 2 || iters < 1 || !tflops || !ms) return -1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -6;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -6;
    double* sink = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_sink[dev] && cudaMalloc(&g_sink[dev], kSink * sizeof(double)) != cudaSuccess)
            return -6;
        sink = g_sink[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = sms * 8;  // 8 blocks of 8 warps per SM
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -6;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -6; }
    cudaEventRecord(e0, s);
    if (kind == 0) k_dfma<<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-7, sink);
    else if (kind == 1) k_dmma<<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-7, sink);
    else k_mixed<<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-7, sink);
    cudaEventRecord(e1, s);
    int rc = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess ? 0 : -6;
    float t = 0.f;
    if (!rc && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = -6;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const double threads = (double)blocks * kThreads, warps = threads / 32.0;
    const double dfma_flops = threads * iters * 8 * 2.0;
    const double dmma_flops = warps * iters * 4 * (8.0 * 8 * 4 * 2);
    const double flops = kind == 0 ? dfma_flops : kind == 1 ? dmma_flops
                                                            : 0.5 * (dfma_flops + dmma_flops);
    *ms = t;
    *tflops = flops / (t * 1e-3) / 1e12;
    return 0;
}
