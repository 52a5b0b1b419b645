// f3: Fresnel diffraction, Eq. 10, on the pixel grid -- the path for grids
// beyond the library's own FFT (fft.cu: padded sides up to 16384).
//
//   O(m, n) = pre * sum_{m', n'} u(m', n') h(m - m', n - n'),
//   h(k, l) = exp(i pi p^2 (k^2 + l^2) / (lambda z)),  pre = exp(i 2 pi z / lambda) / (i lambda z) * p^2,
//
// the linear convolution of the H x W input with the chirp, cropped to H x W,
// by zero-padding both to 2H x 2W (offsets k in (-H, H) at k mod 2H), FFT,
// pointwise product, inverse FFT and crop, so that the circular convolution
// wraps nothing into the kept window.  Here the FFTs are cuFFT's
// single-precision C2C transforms; the kernels expand the input planes into
// the padded buffer, build the chirp (64-bit fixed-point turns c k^2 + c l^2,
// accurate sine and cosine; the prefactor and the inverse transform's
// 1/(4 H W) folded in), multiply by its cached spectrum, and crop back into
// planes.
#include <cufft.h>

#include "kernels.h"

namespace cgh {

namespace {

constexpr int kThreads = 256;

int grid_for(long long n)
{
    long long b = (n + kThreads - 1) / kThreads;
    return (int)(b > 1048576 ? 1048576 : (b > 0 ? b : 1));
}

// The chirp on the 2H x 2W grid, h(k, l) = pre exp(i 2 pi C (k'^2 + l'^2) / 2^64) with the signed offsets k', l',
// as pre a(k) a(l), a(k) = exp(i 2 pi C k'^2 / 2^64): a thread takes its kChirpCols column factors once and, for each
// of its block's kChirpRows rows, one row factor and a complex product per entry (each factor an accurate
// single-precision sine and cosine of its fixed-point turn; the two turns sum to the joint turn within 2^-31).
constexpr int kChirpCols = 8, kChirpRows = 64;

__device__ __forceinline__ float2 chirp_factor(unsigned long long C, int k, int half)
{
    const long long kk = k < half ? k : k - 2 * half;
    const uint32_t t = (uint32_t)((C * (unsigned long long)(kk * kk)) >> 32);   // turn, 2^-32 units
    float s, c;
    sincospif((float)(int)t * (1.0f / 2147483648.0f), &s, &c);   // [-1, 1): twice the signed turn
    return make_float2(c, s);
}

__global__ void chirp_kernel(float2 *__restrict__ h, int H, int W, unsigned long long C, float pre_re, float pre_im)
{
    const int W2 = 2 * W, l0 = blockIdx.x * kThreads * kChirpCols + threadIdx.x;
    float2 a[kChirpCols];
#pragma unroll
    for (int j = 0; j < kChirpCols; ++j) {
        const int l = l0 + j * kThreads;
        a[j] = l < W2 ? chirp_factor(C, l, W) : make_float2(0.0f, 0.0f);
    }
    const int k1 = min(2 * H, (int)(blockIdx.y + 1) * kChirpRows);
    for (int k = blockIdx.y * kChirpRows; k < k1; ++k) {
        const float2 r = chirp_factor(C, k, H);
        const float2 b = make_float2(pre_re * r.x - pre_im * r.y, pre_re * r.y + pre_im * r.x);
#pragma unroll
        for (int j = 0; j < kChirpCols; ++j) {
            const int l = l0 + j * kThreads;
            if (l < W2)
                h[(long long)k * W2 + l] = make_float2(b.x * a[j].x - b.y * a[j].y, b.x * a[j].y + b.y * a[j].x);
        }
    }
}

// One row of the padded plane per blockIdx.y, two complex words per thread.
__global__ void expand_kernel(const float *__restrict__ in, int H, int W, float2 *__restrict__ pad)
{
    const int k = blockIdx.y;
    const int l = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (l >= 2 * W) return;
    const long long plane = (long long)H * W;
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (k < H) {
        const float *re = in + (long long)k * W, *im = re + plane;
        if (l < W) v.x = re[l], v.y = im[l];
        if (l + 1 < W) v.z = re[l + 1], v.w = im[l + 1];
    }
    *reinterpret_cast<float4 *>(pad + (long long)k * 2 * W + l) = v;   // 2W is even: 16-byte aligned
}

// n is even (4 H W): two complex words per 16-byte access.
__global__ void multiply_kernel(float2 *__restrict__ a, const float2 *__restrict__ b, long long n)
{
    float4 *a4 = reinterpret_cast<float4 *>(a);
    const float4 *b4 = reinterpret_cast<const float4 *>(b);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n / 2;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 x = a4[i], y = b4[i];
        a4[i] = make_float4(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x, x.z * y.z - x.w * y.w,
                            x.z * y.w + x.w * y.z);
    }
}

__global__ void crop_kernel(const float2 *__restrict__ pad, int H, int W, float *__restrict__ out)
{
    const int k = blockIdx.y;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= W) return;
    const float2 v = pad[(long long)k * 2 * W + l];
    const long long j = (long long)k * W + l;
    out[j] = v.x;
    out[(long long)H * W + j] = v.y;
}

}  // namespace

bool fft_plan_2d(int rows, int cols, void **plan, cudaStream_t s)
{
    cufftHandle h = 0;
    if (cufftPlan2d(&h, rows, cols, CUFFT_C2C) != CUFFT_SUCCESS) return false;
    if (cufftSetStream(h, s) != CUFFT_SUCCESS) {
        cufftDestroy(h);
        return false;
    }
    *plan = reinterpret_cast<void *>(static_cast<uintptr_t>(h));
    return true;
}

void fft_plan_destroy(void *plan)
{
    if (plan) cufftDestroy(static_cast<cufftHandle>(reinterpret_cast<uintptr_t>(plan)));
}

bool fft_exec(void *plan, float2 *data, bool inverse, cudaStream_t s)
{
    const cufftHandle h = static_cast<cufftHandle>(reinterpret_cast<uintptr_t>(plan));
    if (cufftSetStream(h, s) != CUFFT_SUCCESS) return false;
    return cufftExecC2C(h, reinterpret_cast<cufftComplex *>(data), reinterpret_cast<cufftComplex *>(data),
                        inverse ? CUFFT_INVERSE : CUFFT_FORWARD) == CUFFT_SUCCESS;
}

cudaError_t launch_chirp(float2 *h, int H, int W, unsigned long long C, double pre_re, double pre_im, cudaStream_t s)
{
    chirp_kernel<<<dim3((2 * W + kThreads * kChirpCols - 1) / (kThreads * kChirpCols), (2 * H + kChirpRows - 1) / kChirpRows),
                   kThreads, 0, s>>>(h, H, W, C, (float)pre_re, (float)pre_im);
    return cudaGetLastError();
}

cudaError_t launch_expand(const float *in, int H, int W, float2 *pad, cudaStream_t s)
{
    const dim3 grid((W + kThreads - 1) / kThreads, 2 * H);   // 2W columns, two per thread
    expand_kernel<<<grid, kThreads, 0, s>>>(in, H, W, pad);
    return cudaGetLastError();
}

cudaError_t launch_cmul(float2 *a, const float2 *b, int64_t n, cudaStream_t s)
{
    multiply_kernel<<<grid_for(n / 2), kThreads, 0, s>>>(a, b, (long long)n);
    return cudaGetLastError();
}

cudaError_t launch_crop(const float2 *pad, int H, int W, float *out, cudaStream_t s)
{
    const dim3 grid((W + kThreads - 1) / kThreads, H);
    crop_kernel<<<grid, kThreads, 0, s>>>(pad, H, W, out);
    return cudaGetLastError();
}

}  // namespace cgh
