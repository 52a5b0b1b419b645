// Measured peak of the pipe that bounds the direct SFU form: the throughput
// of the hardware sine (__sinf: one MUFU operation) when nothing else limits
// it -- eight independent chains per thread, every SM full.  The direct
// kernel's roofline fraction is stated against this as well as against the
// nominal 16 results per clock per SM.
#include <cuda_runtime.h>

#include "kernels.h"

namespace cgh {

namespace {

constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(256) mufu_probe_kernel(float *out, int iters, float seed)
{
    float x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = seed * (float)(threadIdx.x + 1 + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = __sinf(x[k]);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += x[k];
    if (s == 12345.0f) out[blockIdx.x] = s;   // keeps the chains alive; never true for |s| <= 8
}

}  // namespace

double measure_mufu_rate(int num_sms, cudaStream_t s)
{
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double rate = -1.0;
    const int blocks = num_sms * 8, threads = 256, iters = 4096;
    if (cudaMalloc(&sink, blocks * sizeof(float)) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        mufu_probe_kernel<<<blocks, threads, 0, s>>>(sink, 64, 0.001f);   // warm-up
        cudaEventRecord(e0, s);
        mufu_probe_kernel<<<blocks, threads, 0, s>>>(sink, iters, 0.001f);
        cudaEventRecord(e1, s);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f)
            rate = (double)blocks * threads * iters * kProbeChains / (ms * 1e-3);
    }
    cudaGetLastError();
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rate;
}

}  // namespace cgh
