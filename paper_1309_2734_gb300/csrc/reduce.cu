// a5: deterministic reduction of partial holograms.  The direct kernel's
// point chunks and the GEMM's K splits each write one plane of partial sums;
// this kernel adds the planes in a fixed order (0, 1, ..., S-1), so repeated
// runs give bit-identical output.  HBM-bound: (S + 1) * 4 bytes per pixel.
#include "kernels.h"

namespace cgh {

namespace {

__global__ void reduce_slices_vec4(const float4 *__restrict__ parts, int slices, long long n4, long long stride4,
                                   float4 *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        float4 acc = parts[i];
        for (int s = 1; s < slices; ++s) {
            const float4 v = parts[(long long)s * stride4 + i];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        out[i] = acc;
    }
}

__global__ void reduce_slices_scalar(const float *__restrict__ parts, int slices, long long n, long long stride,
                                     float *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float acc = parts[i];
        for (int s = 1; s < slices; ++s) acc += parts[(long long)s * stride + i];
        out[i] = acc;
    }
}

int grid_for(long long work, int threads)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (work + threads - 1) / threads;
    long long cap = (long long)sms * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_reduce_slices(const float *parts, int slices, int64_t n, int64_t slice_stride, float *out,
                                 cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const bool vec = (n % 4 == 0) && (slice_stride % 4 == 0) && ((uintptr_t)parts % 16 == 0) &&
                     ((uintptr_t)out % 16 == 0);
    if (vec) {
        reduce_slices_vec4<<<grid_for(n / 4, threads), threads, 0, s>>>(
            reinterpret_cast<const float4 *>(parts), slices, n / 4, slice_stride / 4, reinterpret_cast<float4 *>(out));
    } else {
        reduce_slices_scalar<<<grid_for(n, threads), threads, 0, s>>>(parts, slices, n, slice_stride, out);
    }
    return cudaGetLastError();
}

}  // namespace cgh
