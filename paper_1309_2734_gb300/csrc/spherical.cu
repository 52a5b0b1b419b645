// f2: the exact spherical wave of Eq. 1 (and the amplitude hologram of the
// middle line of Eq. 5), direct form, hardware sine.
//
// The phase of point j at pixel (m, n) in turns is t = sqrt(r^2 + z^2) / lambda
// (r in metres).  With Z = z / lambda and u = r^2 / z^2,
//   t = Z + Z u / 2 + delta,   delta = Z h(u),   h(u) = sqrt(1 + u) - 1 - u / 2,
// where Z + Z u / 2 = z / lambda + r^2 / (2 lambda z) is the Fresnel phase of
// Eq. 2 with its piston: that part is exact in 64-bit fixed point (C_j and the
// piston from the point preparation), walked over the thread's pixels with the
// recurrence of Eqs. 6-8 like the direct kernel.  The remainder delta is split
// at the centre of each thread's pixel tile, delta = d0 + (delta - d0):
//  - d0 = Z h(U0) can reach hundreds of turns for close points on wide
//    holograms; its fraction is taken in double-float arithmetic (float pairs)
//    once per point and tile, or from the float series while |d0| <= 1/2;
//  - the variation over the tile is a quadratic in w = u - U0 (two FP32
//    operations per term, added to the fixed-point phase through a
//    magic-number conversion) where the point preparation's bounds allow, and
//    otherwise a closed form without cancellation (two MUFU operations).
// In the quadratic form -- every point at display distances -- the sine is the
// term's only MUFU operation and the kernel is bound by instruction issue.
//
// Point tiles are staged in shared memory with plain cooperative loads (the
// kernel is compute-bound, so the loads need no asynchronous pipeline and the
// kernel has no waits to bound).
#include "device_util.cuh"
#include "host_util.h"
#include "kernels.h"

namespace cgh {

namespace {

constexpr int kSphBX = 32, kSphBY = 8;                             // threads per CTA, the wide shape: 32 x 8
constexpr int kSphTallBX = 16, kSphTallBY = 16;                    // the tall shape: 16 x 16
constexpr int kSphShortBX = 16, kSphShortBY = 8;                   // the short shape: 16 x 8, four CTAs per SM
constexpr float kSphK1 = 6.28318595886230469f;                   // 2 pi rounded so that 1.5 K1 is a float
constexpr float kSphK0 = 9.42477893829345703f;                   // 1.5 K1
constexpr uint32_t kSphBias = (1u << 30) + 256u;                 // a quarter turn, and rounding to 23 bits
constexpr float kRoundMagic = 12582912.0f;                       // 1.5 2^23: x + M - M rounds x to an integer
constexpr float kQuadScale = 4194304.0f;                         // 2^22: turns to the quadratic's units
constexpr float kSeriesD0Max = 0.5f;                             // |d0| (turns) the float series may carry

static_assert(kPointTile % (kSphShortBX * kSphShortBY) == 0, "whole points per thread in each tile load");

// Exact small integer to float without a conversion instruction (|v| < 2^22).
__device__ __forceinline__ float small_int_to_float(int v)
{
    return __int_as_float(v + 0x4B400000) - kRoundMagic;
}

// Error-free transformations on float pairs (hi + lo): Knuth's two-sum, Dekker's fast two-sum (|a| >= |b|).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}

// The remainder at the thread tile's centre, d0 = Z h(U0) = -(Z / 2) v0^2 with v0 = sqrt(1 + U0) - 1 and
// U0 = (cx^2 + cy^2) (p / z)^2, in double-float arithmetic (float pairs, about 44 significant bits) from the
// point's (p / z)^2 and Z / 2 as pairs: a float alone would carry d0 only to ~1e-7 of itself, and d0 reaches
// hundreds of turns for close points on wide holograms.  Returns d0 - round(d0) (turns); v0, s0 = sqrt(1 + U0)
// and rs0 = 1 / s0 as floats.
__device__ __forceinline__ float sph_d0_frac(float cx, float cy, const float4 x, float &v0, float &s0, float &rs0)
{
    const float qh = fabsf(x.x), zh = fabsf(x.y), ql = x.z, zl = x.w;
    // R0 = cx^2 + cy^2, exact as a pair (half-integers below 2^17)
    const float px = cx * cx, ex = fmaf(cx, cx, -px);
    const float py = cy * cy, ey = fmaf(cy, cy, -py);
    float rh, rl;
    two_sum(px, py, rh, rl);
    fast_two_sum(rh, rl + (ex + ey), rh, rl);
    // U0 = R0 (p / z)^2 and 1 + U0
    float uh = rh * qh;
    float ul = fmaf(rh, qh, -uh) + fmaf(rh, ql, rl * qh);
    fast_two_sum(uh, ul, uh, ul);
    float oh, ol;
    two_sum(1.0f, uh, oh, ol);
    fast_two_sum(oh, ol + ul, oh, ol);
    // s0: one Newton step from the float estimate doubles its ~22 correct bits
    const float rs = rsqrtf(oh);
    const float y = oh * rs;
    float sh, sl;
    fast_two_sum(y, (fmaf(-y, y, oh) + ol) * (0.5f * rs), sh, sl);
    // v0 = s0 - 1 (exact subtraction), then d0 = -(Z / 2) v0^2
    float vh, vl;
    two_sum(sh, -1.0f, vh, vl);
    fast_two_sum(vh, vl + sl, vh, vl);
    const float wh = vh * vh, wl = fmaf(vh, vh, -wh) + 2.0f * vh * vl;
    float dh = zh * wh;
    float dl = fmaf(zh, wh, -dh) + fmaf(zh, wl, zl * wh);
    fast_two_sum(dh, dl, dh, dl);
    v0 = vh;
    s0 = sh;
    rs0 = rs;
    return -((dh - rintf(dh)) + dl);
}

// The Fresnel part of the phase (exact, 32-bit fixed-point turns) at the thread's first column of each row:
// g[i] for its columns, the row step e and second difference D, as in the direct kernel (Eqs. 6-8).
template <int TL>
struct SphFresnel {
    uint32_t g[TL];
    uint32_t e, D;
};

template <int TL>
__device__ __forceinline__ SphFresnel<TL> sph_fresnel(const int4 q, uint32_t piston, int dxi, int dyi, uint32_t rg,
                                                  uint32_t rdx, uint32_t rdy)
{
    const uint32_t chi = (uint32_t)q.z, clo = (uint32_t)q.w;
    const uint32_t dx = (uint32_t)dxi, dy = (uint32_t)dyi;
    const uint32_t r2 = dx * dx + dy * dy;
    const uint32_t r2x = r2 + 2u * dx + 1u;
    const uint32_t r2y = r2 + 2u * dy + 1u;
    const uint32_t c0 = chi * r2 + __umulhi(clo, r2);
    SphFresnel<TL> F;
    uint32_t d = chi * r2x + __umulhi(clo, r2x) - c0 + rdx;
    F.e = chi * r2y + __umulhi(clo, r2y) - c0 + rdy;
    F.D = __funnelshift_l(clo, chi, 1);
    F.g[0] = c0 + piston + rg + kSphBias;
#pragma unroll
    for (int i = 1; i < TL; ++i) {
        F.g[i] = F.g[i - 1] + d;
        d += F.D;
    }
    return F;
}

// Adds A cos(2 pi t) (and A sin(2 pi t)) for the phase t whose fixed-point turns are gi.
template <int PLANES>
__device__ __forceinline__ void sph_accumulate(uint32_t gi, float a, float &re, float &im)
{
    const float f = __uint_as_float(__funnelshift_r(gi, 0x7fu, 9));
    const float ang = fmaf(f, kSphK1, -kSphK0);   // 2 pi (t - 1/4), |ang| <= pi
    if constexpr (PLANES == 1) {
        re = fmaf(-a, __sinf(ang), re);
    } else {
        float sn, cs;
        __sincosf(ang, &sn, &cs);
        re = fmaf(-a, sn, re);
        im = fmaf(a, cs, im);
    }
}

// One point over the thread's TR x TL pixels, the remainder as a quadratic about the tile's centre.
// With cx, cy the centre's offsets from the point (pixels; integer + 1/2 for the 4 x 4 tile), U0 its u and a
// pixel at offsets (t, s) from the centre,
//   u = U0 + a + b,  a = t (2 cx + t) (p / z)^2,  b = s (2 cy + s) (p / z)^2,  w = a + b,
//   delta ~ d0 + d1 w + d2 w^2,  d0 = Z h(U0),  d1 = Z h'(U0),  d2 = Z h''(U0) / 2,
// with truncation error at most Z max|h'''| |w|^3 / 6 = (Z / 16) |w|^3 (h''' = (3/8)(1 + u)^(-5/2)).  d1 and
// d2 come from the closed forms d1 = -(Z / 2) v0 / s0, d2 = -(Z / 8) / s0^3 or, with SERIES (u < kSeriesU),
// from the binomial series of sqrt(1 + u) and its derivatives, which also give d0 while |d0| <= kSeriesD0Max;
// otherwise d0 comes from sph_d0_frac.  With d0 reduced to [-1/2, 1/2] turn and the quadratic's variation over
// the tile below kSphRangeTurns (the point preparation checks both bounds), M + 2^22 delta with M = 1.5 2^23 is
// a float in [2^23, 2^24) whose low 22 mantissa bits hold round(2^22 delta) in two's complement: shifted up by
// ten they add delta to the 32-bit fixed-point phase (resolution 2^-22 turn).  The column constant d2 a^2 is
// converted so once per point and column and joins the column's phase; the rest, d0 + d1 w + d2 (b^2 + 2 a b),
// stays below 1 turn in magnitude since |b^2 + 2 a b| <= (|a| + |b|)^2 (each part rounded to 2^-22 turn).  Per
// term: one FMA for the quadratic, one shift-add into the phase, and the sine as the term's only MUFU operation.
template <int PLANES, int TL, int TR, bool SERIES>
__device__ __forceinline__ void sph_point_quad(const int4 q, const uint2 w, const float4 x, int m0, int n0,
                                               uint32_t rg, uint32_t rdx, uint32_t rdy,
                                               float (&acc)[PLANES][TR][TL])
{
    const int dxi = m0 - q.x, dyi = n0 - q.y;
    SphFresnel<TL> F = sph_fresnel<TL>(q, w.x, dxi, dyi, rg, rdx, rdy);
    const float a = __uint_as_float(w.y);
    const float qz = x.x, zh = fabsf(x.y);   // (p / z)^2, z / (2 lambda)
    const float hx = 0.5f * (TL - 1), hy = 0.5f * (TR - 1);
    const float cx = small_int_to_float(dxi) + hx, cy = small_int_to_float(dyi) + hy;
    float d0f, d1, d2;
    if constexpr (SERIES) {
        const float U0 = fmaf(cx, cx, cy * cy) * qz;
        float p0 = -0.0205078125f;   // binom(1/2, k), k = 6 .. 2
        p0 = fmaf(p0, U0, 0.02734375f);
        p0 = fmaf(p0, U0, -0.0390625f);
        p0 = fmaf(p0, U0, 0.0625f);
        p0 = fmaf(p0, U0, -0.125f);
        float p1 = -0.123046875f;    // k binom(1/2, k)
        p1 = fmaf(p1, U0, 0.13671875f);
        p1 = fmaf(p1, U0, -0.15625f);
        p1 = fmaf(p1, U0, 0.1875f);
        p1 = fmaf(p1, U0, -0.25f);
        float p2 = -0.3076171875f;   // k (k - 1) / 2 binom(1/2, k)
        p2 = fmaf(p2, U0, 0.2734375f);
        p2 = fmaf(p2, U0, -0.234375f);
        p2 = fmaf(p2, U0, 0.1875f);
        p2 = fmaf(p2, U0, -0.125f);
        const float Z = 2.0f * zh;
        const float d0 = (Z * (U0 * U0)) * p0;
        d1 = (Z * U0) * p1;
        d2 = Z * p2;
        if (fabsf(d0) <= kSeriesD0Max) {
            d0f = d0 - ((d0 + kRoundMagic) - kRoundMagic);
        } else {
            float v0, s0, rs0;
            d0f = sph_d0_frac(cx, cy, x, v0, s0, rs0);
        }
    } else {
        float v0, s0, rs0;
        d0f = sph_d0_frac(cx, cy, x, v0, s0, rs0);
        d1 = -zh * v0 * rs0;
        d2 = (-0.25f * zh) * (rs0 * rs0 * rs0);
    }
    const float sd1 = kQuadScale * d1, sd2 = kQuadScale * d2;
    const float X = cx * qz, Y = cy * qz;
    float av[TL];   // a per column; d2 a^2, a column constant, joins the column's fixed-point phase
#pragma unroll
    for (int i = 0; i < TL; ++i) {
        const float t = (float)i - hx;
        av[i] = fmaf(2.0f * t, X, (t * t) * qz);
        F.g[i] += __float_as_uint(fmaf(sd2 * av[i], av[i], kRoundMagic)) << 10;
    }
    // Per row: M + 2^22 (row part) and 2^22 (d1 + 2 d2 b), the row part being d0 + d1 b + d2 b^2.  On tiles
    // eight columns wide the row part also takes the row's Fresnel phase relative to the first row (fixed
    // point, erow; the sum reduced to [-1/2, 1/2) turn), which saves the columns' phases a step per row;
    // narrower tiles step the columns' phases.
    constexpr bool kRowFold = TL >= 8;
    float pm[TR], qr[TR];
    uint32_t erow = 0u;
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        const float s = (float)r - hy;
        const float b = fmaf(2.0f * s, Y, (s * s) * qz);
        pm[r] = fmaf(fmaf(fmaf(d2, b, d1), b, d0f), kQuadScale, kRoundMagic);
        qr[r] = fmaf(2.0f * sd2, b, sd1);
        if constexpr (kRowFold) {
            const uint32_t row = erow + (__float_as_uint(pm[r]) << 10);   // mod 1 turn, 2^-32 units
            pm[r] = fmaf((float)(int)row, 1.0f / 1024.0f, kRoundMagic);
            erow += F.e;
            F.e += F.D;
        }
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) {
#pragma unroll
        for (int i = 0; i < TL; ++i) {
            // M + 2^22 (row part + d1 a + 2 d2 a b): the quadratic but its column constant d2 a^2, which the
            // column's phase holds
            const float y = fmaf(av[i], qr[r], pm[r]);
            sph_accumulate<PLANES>(F.g[i] + (__float_as_uint(y) << 10), a, acc[0][r][i],
                                   acc[PLANES - 1][r][i]);
        }
        if (!kRowFold && r + 1 < TR) {
#pragma unroll
            for (int i = 0; i < TL; ++i) F.g[i] += F.e;
            F.e += F.D;
        }
    }
}

// One point over the thread's pixels, the remainder term by term where the quadratic's bounds fail (points
// close to a wide hologram): delta = d0 + Delta with d0 at the tile centre (sph_d0_frac) and the variation
//   Delta = Z ((s - s0) - w / 2) = -(Z / 2) w (v + v0) / (s + s0) = -(Z / 2) w (u + v0 (1 + s)) / ((1 + s)(s + s0)),
// s = sqrt(1 + u), v = s - 1 = u / (1 + s): no cancellation, so Delta carries ~1e-7 of itself, and d0's
// fraction ~2^-40 turn.  Per term: a reciprocal square root, a reciprocal and the sine (three MUFU operations).
template <int PLANES, int TL, int TR>
__device__ __forceinline__ void sph_point_terms(const int4 q, const uint2 w, const float4 x, int m0, int n0,
                                                uint32_t rg, uint32_t rdx, uint32_t rdy,
                                                float (&acc)[PLANES][TR][TL])
{
    const int dxi = m0 - q.x, dyi = n0 - q.y;
    SphFresnel<TL> F = sph_fresnel<TL>(q, w.x, dxi, dyi, rg, rdx, rdy);
    const float a = __uint_as_float(w.y);
    const float qz = fabsf(x.x), zh = fabsf(x.y);
    const float hx = 0.5f * (TL - 1), hy = 0.5f * (TR - 1);
    const float cx = small_int_to_float(dxi) + hx, cy = small_int_to_float(dyi) + hy;
    float v0, s0, rs0;
    const float d0f = sph_d0_frac(cx, cy, x, v0, s0, rs0);
    const float U0 = fmaf(cx, cx, cy * cy) * qz;
    const float X = cx * qz, Y = cy * qz;
    float av[TL], bv[TR];
#pragma unroll
    for (int i = 0; i < TL; ++i) {
        const float t = (float)i - hx;
        av[i] = fmaf(2.0f * t, X, (t * t) * qz);
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        const float s = (float)r - hy;
        bv[r] = fmaf(2.0f * s, Y, (s * s) * qz);
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) {
#pragma unroll
        for (int i = 0; i < TL; ++i) {
            const float wv = av[i] + bv[r];
            const float u = U0 + wv;
            const float ou = 1.0f + u;
            const float s = ou * rsqrtf(ou);
            const float s1 = 1.0f + s;
            const float delta = fmaf(-zh * wv, __fdividef(fmaf(v0, s1, u), s1 * (s + s0)), d0f);   // turns
            const float df = delta - ((delta + kRoundMagic) - kRoundMagic);   // its fraction, [-1/2, 1/2]
            const float y = fmaf(df, kQuadScale, kRoundMagic);                 // into the phase as above
            sph_accumulate<PLANES>(F.g[i] + (__float_as_uint(y) << 10), a, acc[0][r][i], acc[PLANES - 1][r][i]);
        }
        if (r + 1 < TR) {
#pragma unroll
            for (int i = 0; i < TL; ++i) F.g[i] += F.e;
            F.e += F.D;
        }
    }
}

// blockIdx.x = pixel tile, blockIdx.y = point chunk (its own output plane).  A thread owns
// sph_tile_rows(PLANES) rows of sph_tile_cols(PLANES) pixels: 8 x 8 for the amplitude hologram, 4 x 4 for the
// complex wave.  Each point tile's partial sums stay in registers; the running totals live in shared memory
// (index-major, so a warp's accesses are consecutive words), which leaves the registers of two CTAs per SM to the
// partial sums.
template <int PLANES, int BX, int BY>
__global__ void __launch_bounds__(BX *BY, 512 / (BX * BY))
    spherical_kernel(const int4 *__restrict__ geo, const uint2 *__restrict__ aux, const float4 *__restrict__ ext,
                     int n_ptiles, int width, int height, int tiles_x, int split, float *__restrict__ out,
                     long long slice_stride, long long im_offset, const PhaseRef ref)
{
    constexpr int TL = sph_tile_cols(PLANES), TR = sph_tile_rows(PLANES), T = BX * BY;
    __shared__ int4 s_geo[kPointTile];
    __shared__ uint2 s_aux[kPointTile];
    __shared__ float4 s_ext[kPointTile];
    extern __shared__ float s_tot[];   // [PLANES * TR * TL][T]
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int m0 = (tile % tiles_x) * (BX * TL) + (tid % BX) * TL;
    const int n0 = (tile / tiles_x) * (BY * TR) + (tid / BX) * TR;
    const int t_begin = (int)((long long)blockIdx.y * n_ptiles / split);
    const int t_end = (int)((long long)(blockIdx.y + 1) * n_ptiles / split);
    const uint32_t rg = ref_turn(ref, m0, n0), rdx = ref_step(ref.kx), rdy = ref_step(ref.ky);

#pragma unroll
    for (int k = 0; k < PLANES * TR * TL; ++k) s_tot[k * T + tid] = 0.0f;

    for (int t = t_begin; t < t_end; ++t) {
        __syncthreads();   // the previous tile is consumed
        for (int k = tid; k < kPointTile; k += T) {
            const long long j = (long long)t * kPointTile + k;
            s_geo[k] = geo[j];
            s_aux[k] = aux[j];
            s_ext[k] = ext[j];
        }
        __syncthreads();
        float part[PLANES][TR][TL];
#pragma unroll
        for (int c = 0; c < PLANES; ++c)
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int i = 0; i < TL; ++i) part[c][r][i] = 0.0f;
#pragma unroll 1
        for (int p = 0; p < kPointTile; ++p) {
            const float4 x = s_ext[p];   // the same point, so the same branch, in every thread
            if (x.x < 0.0f)
                sph_point_terms<PLANES, TL, TR>(s_geo[p], s_aux[p], x, m0, n0, rg, rdx, rdy, part);
            else if (x.y >= 0.0f)
                sph_point_quad<PLANES, TL, TR, true>(s_geo[p], s_aux[p], x, m0, n0, rg, rdx, rdy, part);
            else
                sph_point_quad<PLANES, TL, TR, false>(s_geo[p], s_aux[p], x, m0, n0, rg, rdx, rdy, part);
        }
#pragma unroll
        for (int c = 0; c < PLANES; ++c)
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int i = 0; i < TL; ++i) s_tot[((c * TR + r) * TL + i) * T + tid] += part[c][r][i];
    }

    float *dst = out + (long long)blockIdx.y * slice_stride;
#pragma unroll
    for (int c = 0; c < PLANES; ++c)
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const int n = n0 + r;
            if (n >= height) continue;
#pragma unroll
            for (int i = 0; i < TL; ++i)
                if (m0 + i < width)
                    dst[(long long)c * im_offset + (long long)n * width + m0 + i] = s_tot[((c * TR + r) * TL + i) * T + tid];
        }
}

}  // namespace

DirectShape spherical_shape(int planes, int variant)
{
    const int tl = sph_tile_cols(planes), tr = sph_tile_rows(planes);
    if (variant == 1) return DirectShape{kSphTallBX * tl, kSphTallBY * tr, kSphTallBX * kSphTallBY, kSphTallBX, 2};
    if (variant == 2) return DirectShape{kSphShortBX * tl, kSphShortBY * tr, kSphShortBX * kSphShortBY, kSphShortBX, 4};
    return DirectShape{kSphBX * tl, kSphBY * tr, kSphBX * kSphBY, kSphBX, 2};
}

namespace {
template <int PLANES, int BX, int BY>
void spherical_as(dim3 grid, cudaStream_t s, const int4 *geo, const uint2 *aux, const float4 *ext, int n_ptiles,
                  int width, int height, int tiles_x, int split, float *out, long long ss, long long im,
                  const PhaseRef &ref)
{
    constexpr size_t tot_bytes = (size_t)PLANES * sph_tile_rows(PLANES) * sph_tile_cols(PLANES) * BX * BY * sizeof(float);
    static PerDeviceOnce configured;   // the running totals exceed the default 48 KB of dynamic shared memory
    if (configured.run([&] {
            return cudaFuncSetAttribute(spherical_kernel<PLANES, BX, BY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)tot_bytes);
        }) != cudaSuccess)
        return;
    spherical_kernel<PLANES, BX, BY><<<grid, BX * BY, tot_bytes, s>>>(geo, aux, ext, n_ptiles, width, height, tiles_x,
                                                                      split, out, ss, im, ref);
}
}  // namespace

cudaError_t launch_spherical(const DirectShape &sh, const int4 *geo, const uint2 *aux, const float4 *ext, int n_pad,
                             int width, int height, int split, int planes, float *out, int64_t slice_stride,
                             int64_t im_offset, const PhaseRef &ref, cudaStream_t s)
{
    const int tiles_x = (width + sh.tile_w - 1) / sh.tile_w;
    const int tiles_y = (height + sh.tile_h - 1) / sh.tile_h;
    const int n_ptiles = n_pad / kPointTile;
    if (split < 1) split = 1;
    dim3 grid(tiles_x * tiles_y, split);
    const long long ss = (long long)slice_stride;
    const long long im = planes == 2 ? (long long)im_offset : 0;
    const int variant = sh.bx == kSphBX ? 0 : (sh.threads == kSphTallBX * kSphTallBY ? 1 : 2);
#define CGH_SPH(P, BXV, BYV)                                                                                     \
    spherical_as<P, BXV, BYV>(grid, s, geo, aux, ext, n_ptiles, width, height, tiles_x, split, out, ss, im, ref)
    if (planes == 2) {
        if (variant == 1) CGH_SPH(2, kSphTallBX, kSphTallBY);
        else if (variant == 2) CGH_SPH(2, kSphShortBX, kSphShortBY);
        else CGH_SPH(2, kSphBX, kSphBY);
    } else {
        if (variant == 1) CGH_SPH(1, kSphTallBX, kSphTallBY);
        else if (variant == 2) CGH_SPH(1, kSphShortBX, kSphShortBY);
        else CGH_SPH(1, kSphBX, kSphBY);
    }
#undef CGH_SPH
    return cudaGetLastError();
}

}  // namespace cgh
