// f2: the exact spherical wave of Eq. 1 (and the amplitude hologram of the
// middle line of Eq. 5), direct form, hardware sine.
//
// The phase of point j at pixel (m, n) in turns is t = sqrt(r^2 + z^2) / lambda
// (r in metres).  With Z = z / lambda and u = r^2 / z^2,
//   t = Z + Z u / 2 + delta,   delta = Z (sqrt(1 + u) - 1 - u / 2),
// where Z + Z u / 2 = z / lambda + r^2 / (2 lambda z) is the Fresnel phase of
// Eq. 2 with its piston: that part is exact in 64-bit fixed point (C_j and the
// piston from the point preparation), walked over the thread's pixels with the
// recurrence of Eqs. 6-8 like the direct kernel.  The remainder is small
// (|delta| <= Z u^2 / 8: a fraction of a turn to a few turns at display sizes)
// and is evaluated in single precision without cancellation:
//   sqrt(1 + u) - 1 = u / (1 + s),  s = sqrt(1 + u),
//   delta = Z (u / (1 + s) - u / 2) = -(Z / 2) (u / (1 + s))^2.
// Per term: one reciprocal square root, one reciprocal (MUFU) and the sine
// (MUFU); relative error of delta a few 1e-7, i.e. ~1e-7 turn per turn of delta.
// When u < 0.05 at every pixel for a point (flagged by the point preparation:
// the sign of (p / z)^2), delta comes from the binomial series instead,
//   sqrt(1 + u) - 1 - u / 2 = -u^2/8 + u^3/16 - 5 u^4/128 + 7 u^5/256 - 21 u^6/1024 + ...,
// five FMA-pipe terms whose remainder is below 0.13 u^5 of the first
// (4e-8 at u = 0.05): the sine is then the only MUFU operation of the term.
//
// Point tiles are staged in shared memory with plain cooperative loads (the
// kernel is bound by the MUFU pipe -- three operations per term in the closed
// form, one with the series -- so the loads need no asynchronous pipeline and
// the kernel has no waits to bound).
#include "device_util.cuh"
#include "kernels.h"

namespace cgh {

namespace {

constexpr int kSphTL = 4, kSphTR = 4, kSphBX = 32, kSphBY = 8;   // 128 x 32 pixels per CTA of 256 threads
constexpr float kSphK1 = 6.28318595886230469f;                   // 2 pi rounded so that 1.5 K1 is a float
constexpr float kSphK0 = 9.42477893829345703f;                   // 1.5 K1
constexpr uint32_t kSphBias = (1u << 30) + 256u;                 // a quarter turn, and rounding to 23 bits
constexpr float kRoundMagic = 12582912.0f;                       // 1.5 2^23: x + M - M rounds x to an integer

static_assert(kSphBX * kSphBY == kPointTile, "one point per thread in each tile load");

template <int PLANES, bool SERIES>
__device__ __forceinline__ void sph_point_terms(const int4 q, const uint2 w, const float2 x, int m0, int n0,
                                                uint32_t rg, uint32_t rdx, uint32_t rdy,
                                                float (&acc)[PLANES][kSphTR][kSphTL])
{
    const uint32_t chi = (uint32_t)q.z, clo = (uint32_t)q.w;
    const int dxi = m0 - q.x, dyi = n0 - q.y;
    const uint32_t dx = (uint32_t)dxi, dy = (uint32_t)dyi;
    const uint32_t r2 = dx * dx + dy * dy;
    const uint32_t r2x = r2 + 2u * dx + 1u;
    const uint32_t r2y = r2 + 2u * dy + 1u;
    const uint32_t c0 = chi * r2 + __umulhi(clo, r2);
    uint32_t d = chi * r2x + __umulhi(clo, r2x) - c0 + rdx;
    uint32_t e = chi * r2y + __umulhi(clo, r2y) - c0 + rdy;
    const uint32_t D = __funnelshift_l(clo, chi, 1);
    const float a = __uint_as_float(w.y);
    const float qz = fabsf(x.x), zh = x.y;   // (p / z)^2, z / (2 lambda)
    // squared column and row offsets of the thread's pixels, in pixels^2
    float xs[kSphTL], ys[kSphTR];
#pragma unroll
    for (int i = 0; i < kSphTL; ++i) {
        const float t = (float)(dxi + i);
        xs[i] = t * t;
    }
#pragma unroll
    for (int r = 0; r < kSphTR; ++r) {
        const float t = (float)(dyi + r);
        ys[r] = t * t;
    }
    uint32_t g[kSphTL];
    g[0] = c0 + w.x + rg + kSphBias;
#pragma unroll
    for (int i = 1; i < kSphTL; ++i) {
        g[i] = g[i - 1] + d;
        d += D;
    }
#pragma unroll
    for (int r = 0; r < kSphTR; ++r) {
#pragma unroll
        for (int i = 0; i < kSphTL; ++i) {
            const float u = (xs[i] + ys[r]) * qz;
            float delta;   // turns, <= 0
            if constexpr (SERIES) {
                float c = -0.0205078125f;                      // -21/1024
                c = fmaf(c, u, 0.02734375f);                   // 7/256
                c = fmaf(c, u, -0.0390625f);                   // -5/128
                c = fmaf(c, u, 0.0625f);                       // 1/16
                c = fmaf(c, u, -0.125f);                       // -1/8
                delta = (2.0f * zh) * (u * u) * c;             // Z u^2 (...)
            } else {
                const float rs = rsqrtf(1.0f + u);
                const float s = (1.0f + u) * rs;
                const float v = __fdividef(u, 1.0f + s);
                delta = -zh * v * v;
            }
            const float df = delta - ((delta + kRoundMagic) - kRoundMagic);  // its fractional part, [-1/2, 1/2]
            const float f = __uint_as_float(__funnelshift_r(g[i], 0x7fu, 9));
            const float ang = fmaf(df, kSphK1, fmaf(f, kSphK1, -kSphK0));   // 2 pi (t - 1/4), |ang| <= 2 pi
            if constexpr (PLANES == 1) {
                acc[0][r][i] = fmaf(-a, __sinf(ang), acc[0][r][i]);          // A cos(2 pi t)
            } else {
                float sn, cs;
                __sincosf(ang, &sn, &cs);
                acc[0][r][i] = fmaf(-a, sn, acc[0][r][i]);                   // A cos(2 pi t)
                acc[1][r][i] = fmaf(a, cs, acc[1][r][i]);                    // A sin(2 pi t)
            }
        }
        if (r + 1 < kSphTR) {
#pragma unroll
            for (int i = 0; i < kSphTL; ++i) g[i] += e;
            e += D;
        }
    }
}

// blockIdx.x = pixel tile, blockIdx.y = point chunk (its own output plane).
template <int PLANES>
__global__ void __launch_bounds__(kSphBX *kSphBY, 2)
    spherical_kernel(const int4 *__restrict__ geo, const uint2 *__restrict__ aux, const float2 *__restrict__ ext,
                     int n_ptiles, int width, int height, int tiles_x, int split, float *__restrict__ out,
                     long long slice_stride, long long im_offset, const PhaseRef ref)
{
    __shared__ int4 s_geo[kPointTile];
    __shared__ uint2 s_aux[kPointTile];
    __shared__ float2 s_ext[kPointTile];
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int m0 = (tile % tiles_x) * (kSphBX * kSphTL) + (tid % kSphBX) * kSphTL;
    const int n0 = (tile / tiles_x) * (kSphBY * kSphTR) + (tid / kSphBX) * kSphTR;
    const int t_begin = (int)((long long)blockIdx.y * n_ptiles / split);
    const int t_end = (int)((long long)(blockIdx.y + 1) * n_ptiles / split);
    const uint32_t rg = ref_turn(ref, m0, n0), rdx = ref_step(ref.kx), rdy = ref_step(ref.ky);

    float tot[PLANES][kSphTR][kSphTL];
#pragma unroll
    for (int c = 0; c < PLANES; ++c)
#pragma unroll
        for (int r = 0; r < kSphTR; ++r)
#pragma unroll
            for (int i = 0; i < kSphTL; ++i) tot[c][r][i] = 0.0f;

    for (int t = t_begin; t < t_end; ++t) {
        const long long j = (long long)t * kPointTile + tid;
        __syncthreads();   // the previous tile is consumed
        s_geo[tid] = geo[j];
        s_aux[tid] = aux[j];
        s_ext[tid] = ext[j];
        __syncthreads();
        float part[PLANES][kSphTR][kSphTL];
#pragma unroll
        for (int c = 0; c < PLANES; ++c)
#pragma unroll
            for (int r = 0; r < kSphTR; ++r)
#pragma unroll
                for (int i = 0; i < kSphTL; ++i) part[c][r][i] = 0.0f;
#pragma unroll 1
        for (int p = 0; p < kPointTile; ++p) {
            if (s_ext[p].x >= 0.0f)   // the same point, so the same branch, in every thread
                sph_point_terms<PLANES, true>(s_geo[p], s_aux[p], s_ext[p], m0, n0, rg, rdx, rdy, part);
            else
                sph_point_terms<PLANES, false>(s_geo[p], s_aux[p], s_ext[p], m0, n0, rg, rdx, rdy, part);
        }
#pragma unroll
        for (int c = 0; c < PLANES; ++c)
#pragma unroll
            for (int r = 0; r < kSphTR; ++r)
#pragma unroll
                for (int i = 0; i < kSphTL; ++i) tot[c][r][i] += part[c][r][i];
    }

    float *dst = out + (long long)blockIdx.y * slice_stride;
#pragma unroll
    for (int c = 0; c < PLANES; ++c)
#pragma unroll
        for (int r = 0; r < kSphTR; ++r) {
            const int n = n0 + r;
            if (n >= height) continue;
#pragma unroll
            for (int i = 0; i < kSphTL; ++i)
                if (m0 + i < width) dst[(long long)c * im_offset + (long long)n * width + m0 + i] = tot[c][r][i];
        }
}

}  // namespace

DirectShape spherical_shape()
{
    return DirectShape{kSphBX * kSphTL, kSphBY * kSphTR, kSphBX * kSphBY};
}

cudaError_t launch_spherical(const int4 *geo, const uint2 *aux, const float2 *ext, int n_pad, int width, int height,
                             int split, int planes, float *out, int64_t slice_stride, int64_t im_offset,
                             const PhaseRef &ref, cudaStream_t s)
{
    const DirectShape sh = spherical_shape();
    const int tiles_x = (width + sh.tile_w - 1) / sh.tile_w;
    const int tiles_y = (height + sh.tile_h - 1) / sh.tile_h;
    const int n_ptiles = n_pad / kPointTile;
    if (split < 1) split = 1;
    dim3 grid(tiles_x * tiles_y, split);
    if (planes == 2)
        spherical_kernel<2><<<grid, sh.threads, 0, s>>>(geo, aux, ext, n_ptiles, width, height, tiles_x, split, out,
                                                        (long long)slice_stride, (long long)im_offset, ref);
    else
        spherical_kernel<1><<<grid, sh.threads, 0, s>>>(geo, aux, ext, n_ptiles, width, height, tiles_x, split, out,
                                                        (long long)slice_stride, 0, ref);
    return cudaGetLastError();
}

}  // namespace cgh
