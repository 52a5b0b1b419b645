// a6: 8-bit quantisation of an amplitude hologram (min/max rule).
//
// The paper stores its phase-only holograms as unsigned char with
// 255/(2 pi) per radian (Section 4.1).  For the amplitude hologram of Eq. 5
// the range is not known in advance, so it is measured:
//   pass 1: lo = min, hi = max over the field (order independent: atomic
//           min/max on an order-preserving integer encoding; NaN skipped);
//   pass 2: s = the smallest float >= 255 / ((double)hi - (double)lo),
//           q = floor(fl(fl(v - lo) * s)) clamped to [0, 255], NaN -> 0.
// Each single-precision operation is rounded on its own (no FMA contraction),
// so the output is reproducible bit for bit by any IEEE implementation.
#include <cfloat>

#include "kernels.h"

namespace cgh {

namespace {

__device__ __forceinline__ uint32_t order_key(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float from_key(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void minmax_init(uint32_t *scratch)
{
    scratch[0] = 0xffffffffu;   // running minimum key
    scratch[1] = 0u;            // running maximum key
}

__global__ void minmax_kernel(const float *__restrict__ f, long long n, uint32_t *scratch)
{
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = f[i];
        if (v == v) {
            const uint32_t k = order_key(v);
            lo = min(lo, k);
            hi = max(hi, k);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ uint32_t s_lo[32], s_hi[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        lo = lane < nw ? s_lo[lane] : 0xffffffffu;
        hi = lane < nw ? s_hi[lane] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            atomicMin(&scratch[0], lo);
            atomicMax(&scratch[1], hi);
        }
    }
}

__device__ __forceinline__ uint8_t quantize_one(float v, float lo, float s)
{
    const float q = floorf(__fmul_rn(__fsub_rn(v, lo), s));
    return (q >= 255.0f) ? (uint8_t)255 : ((q >= 0.0f) ? (uint8_t)q : (uint8_t)0);
}

__global__ void map_kernel(const float *__restrict__ f, long long n, const uint32_t *scratch,
                           uint8_t *__restrict__ out, bool vec)
{
    const float lo = from_key(scratch[0]);
    const float hi = from_key(scratch[1]);
    const bool degenerate = !(hi > lo);
    float s = 0.0f;
    if (!degenerate) {
        const double sd = 255.0 / ((double)hi - (double)lo);
        if (sd > (double)FLT_MAX) {
            s = FLT_MAX;
        } else {
            s = __double2float_ru(sd);
            if (isinf(s)) s = FLT_MAX;
        }
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long done = 0;
    if (vec) {
        const long long n16 = n / 16;
        const float4 *f4 = reinterpret_cast<const float4 *>(f);
        uint4 *o16 = reinterpret_cast<uint4 *>(out);
        for (long long i = first; i < n16; i += stride) {
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 v = f4[4 * i + k];
                uint32_t b0, b1, b2, b3;
                if (degenerate) {
                    b0 = b1 = b2 = b3 = 0;
                } else {
                    b0 = quantize_one(v.x, lo, s);
                    b1 = quantize_one(v.y, lo, s);
                    b2 = quantize_one(v.z, lo, s);
                    b3 = quantize_one(v.w, lo, s);
                }
                w[k] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
            }
            o16[i] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        done = n16 * 16;
    }
    for (long long i = done + first; i < n; i += stride) out[i] = degenerate ? (uint8_t)0 : quantize_one(f[i], lo, s);
}

int quant_grid(long long work)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (work + 255) / 256;
    const long long cap = (long long)sms * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

// Phase of the complex wave in [0, 2 pi) (Eq. 3; the listings add 2 pi to
// negative phases), scaled by 255 / (2 pi) and floored, as the listings of
// Section 4.1 store their phase-only holograms (clamped to 255: psi + 2 pi may
// round up to 2 pi in single precision; NaN -> 0).
__global__ void kinoform_kernel(const float *__restrict__ re, const float *__restrict__ im, long long n,
                                uint8_t *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float psi = atan2f(im[i], re[i]);
        if (psi < 0.0f) psi = __fadd_rn(psi, 6.28318530717958648f);
        const float x = floorf(__fmul_rn(psi, 40.58451048843331f));   // 255 / (2 pi)
        out[i] = (x >= 255.0f) ? (uint8_t)255 : ((x >= 0.0f) ? (uint8_t)x : (uint8_t)0);
    }
}

}  // namespace

cudaError_t launch_kinoform8(const float *re, const float *im, int64_t n, uint8_t *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    kinoform_kernel<<<quant_grid(n), 256, 0, s>>>(re, im, n, out);
    return cudaGetLastError();
}

cudaError_t launch_quantize8(const float *field, int64_t n, uint8_t *out, uint32_t *scratch, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    minmax_init<<<1, 1, 0, s>>>(scratch);
    minmax_kernel<<<quant_grid(n), 256, 0, s>>>(field, n, scratch);
    const bool vec = ((uintptr_t)field % 16 == 0) && ((uintptr_t)out % 16 == 0);
    map_kernel<<<quant_grid(vec ? n / 16 : n), 256, 0, s>>>(field, n, scratch, out, vec);
    return cudaGetLastError();
}

}  // namespace cgh
