// Device-side code of the separable factors (a3), shared by the factor kernel
// (factors.cu) and by the persistent batch kernel (persist.cu).  The method and
// its numerics are described at the top of factors.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace cgh {
namespace dev {

constexpr int kRowsPerBlock = 32;
constexpr int kFactorThreads = 128;

// (cos 2 pi t, sin 2 pi t) for t in [-1/2, 1/2), hardware sine and cosine
__device__ __forceinline__ void sincos_turn(float t, float &s, float &c)
{
    __sincosf(t * 6.28318530717958648f, &s, &c);
}

__device__ __forceinline__ uint32_t pack(float lo_col, float hi_col, int mode, bool second)
{
    if (mode == kFactorBF16) {
        const __nv_bfloat162 v = __floats2bfloat162_rn(lo_col, hi_col);
        return *reinterpret_cast<const uint32_t *>(&v);
    }
    const __half2 h = __floats2half2_rn(lo_col, hi_col);
    if (!second) return *reinterpret_cast<const uint32_t *>(&h);
    const __half2 l = __floats2half2_rn(lo_col - __low2float(h), hi_col - __high2float(h));
    return *reinterpret_cast<const uint32_t *>(&l);
}

// K1 is 2 pi rounded to a float whose 1.5 multiple K0 is exact, so that the argument grid (f - 1.5) K1 of the
// fixed-point turn conversions below is symmetric about zero and the hardware sine's odd error cancels in sums.
constexpr float kTurnK1 = 6.28318595886230469f;   // 0x40c90fdc
constexpr float kTurnK0 = 9.42477893829345703f;   // 1.5 * kTurnK1, exact

// One point's entry of a row: P (cos b, sin b); Q, the amplitude times (cos a, -sin a), or with IMAG
// (sin a, cos a) -- the imaginary part's factor.
template <bool IS_P, bool IMAG>
__device__ __forceinline__ void factor_entry(float s, float c, float a, float &re, float &im)
{
    if (IS_P) {
        re = c;
        im = s;
    } else {
        re = IMAG ? a * s : a * c;
        im = IMAG ? a * c : -a * s;
    }
}

// FP16 / BF16 factors of rows [line0, line1) of P (IS_P) or Q for the thread's four points: the turn walked down the
// rows by the second-order recurrence of Eqs. 6-8 in 32-bit fixed point from its exact value and first difference at
// line0 (drift below 32^2 / 2 units of 2^-32 turn over a block's 32 rows, far below the factors' 2^-11), converted
// by its top 23 bits as a float mantissa with a half turn added (so (f - 1.5) K1 is the angle itself in [-pi, pi)):
// no 64-bit product and no conversion instruction per entry.
template <int MODE, bool IS_P, bool IMAG>
__device__ __forceinline__ void factor_rows_walk(int line0, int line1, const int (&coord)[4], const uint32_t (&chi)[4],
                                                 const uint32_t (&clo)[4], const uint32_t (&pist)[4],
                                                 const float (&a)[4], const bool (&live)[4], uint16_t *base,
                                                 long long ld, int j0, const PhaseRef &ref)
{
    if (line0 >= line1) return;
    uint32_t g[4], e[4], D[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t d = (uint32_t)(line0 - coord[q]), d1 = d + 1u;
        const uint32_t G0 = chi[q] * (d * d) + __umulhi(clo[q], d * d);
        const uint32_t G1 = chi[q] * (d1 * d1) + __umulhi(clo[q], d1 * d1);
        g[q] = G0 + (IS_P ? 0u : pist[q]) + 0x80000100u;   // a half turn, and rounding to 23 bits
        e[q] = G1 - G0;
        D[q] = __funnelshift_l(clo[q], chi[q], 1);          // 2 C, top 32 bits
    }
    for (int line = line0; line < line1; ++line) {
        // reference phase of this row (P: ky n) or column (Q: kx m + phi0)
        const uint32_t radd = IS_P ? ref_turn(ref, 0, line) - ref.phi0 : ref_turn(ref, line, 0);
        float v[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float f = __uint_as_float(__funnelshift_r(g[q] + radd, 0x7fu, 9));
            float s, c;
            __sincosf(fmaf(f, kTurnK1, -kTurnK0), &s, &c);
            float re, im;
            factor_entry<IS_P, IMAG>(s, c, a[q], re, im);
            v[2 * q] = live[q] ? re : 0.0f;
            v[2 * q + 1] = live[q] ? im : 0.0f;
            g[q] += e[q];
            e[q] += D[q];
        }
        uint16_t *dst = base + (long long)line * ld + 2 * j0;
        *reinterpret_cast<uint4 *>(dst) = make_uint4(pack(v[0], v[1], MODE, false), pack(v[2], v[3], MODE, false),
                                                     pack(v[4], v[5], MODE, false), pack(v[6], v[7], MODE, false));
    }
}

// The factors of one thread's four points j0 .. j0 + 3 (those below n_points; the rest of the slots are zero
// columns) on rows [r_begin, r_end) of the stacked rows (P's rows below height, then Q's rows), Q scaled by
// scale (1 / max|A|).
template <int MODE, bool IMAG>
__device__ __forceinline__ void factor_thread(int j0, int r_begin, int r_end, const int4 *__restrict__ geo,
                                              const uint2 *__restrict__ aux, int n_points, int height, int width,
                                              uint16_t *__restrict__ P, uint16_t *__restrict__ Q, long long ld,
                                              long long plane_p, long long plane_q, float scale, const PhaseRef &ref)
{
    int px[4], py[4];
    uint32_t chi[4], clo[4], pist[4];
    float a[4];
    bool live[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + q;
        live[q] = j < n_points;
        if (live[q]) {
            const int4 g = geo[j];
            px[q] = g.x;
            py[q] = g.y;
            chi[q] = (uint32_t)g.z;
            clo[q] = (uint32_t)g.w;
            const uint2 w = aux[j];
            pist[q] = ref.piston ? w.x : 0u;
            a[q] = __uint_as_float(w.y) * scale;
        } else {
            px[q] = py[q] = 0;
            chi[q] = clo[q] = pist[q] = 0u;
            a[q] = 0.0f;
        }
    }
    if constexpr (MODE != kFactorSplit16) {
        // P rows below height, Q rows (columns) above
        factor_rows_walk<MODE, true, IMAG>(r_begin, min(r_end, height), py, chi, clo, pist, a, live, P, ld, j0, ref);
        factor_rows_walk<MODE, false, IMAG>(max(r_begin, height) - height, r_end - height, px, chi, clo, pist, a, live,
                                            Q, ld, j0, ref);
        return;
    }
    // split FP16: the exact turn of every entry (its hi + lo pair carries 2^-22 of it)
    for (int r = r_begin; r < r_end; ++r) {
        const bool is_p = r < height;
        const int line = is_p ? r : r - height;
        // reference phase of this row (P: ky n) or column (Q: kx m + phi0)
        const uint32_t radd = is_p ? ref_turn(ref, 0, line) - ref.phi0 : ref_turn(ref, line, 0);
        float v[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float c = 0.0f, s = 0.0f;
            if (live[q]) {
                const uint32_t d = (uint32_t)(line - (is_p ? py[q] : px[q]));
                const uint32_t d2 = d * d;                                   // < 2^30
                const uint32_t g = chi[q] * d2 + __umulhi(clo[q], d2) + radd + (is_p ? 0u : pist[q]);   // turn
                const float t = (float)(int)g * 2.3283064365386963e-10f;     // [-1/2, 1/2)
                sincos_turn(t, s, c);
                if (!is_p) {
                    const float cc = c;
                    c = IMAG ? a[q] * s : a[q] * c;
                    s = IMAG ? a[q] * cc : -a[q] * s;
                }
            }
            v[2 * q] = c;
            v[2 * q + 1] = s;
        }
        uint16_t *dst = (is_p ? P + (long long)line * ld : Q + (long long)line * ld) + 2 * j0;
        const uint4 hi = make_uint4(pack(v[0], v[1], MODE, false), pack(v[2], v[3], MODE, false),
                                    pack(v[4], v[5], MODE, false), pack(v[6], v[7], MODE, false));
        *reinterpret_cast<uint4 *>(dst) = hi;
        const uint4 lo = make_uint4(pack(v[0], v[1], MODE, true), pack(v[2], v[3], MODE, true),
                                    pack(v[4], v[5], MODE, true), pack(v[6], v[7], MODE, true));
        *reinterpret_cast<uint4 *>(dst + (is_p ? plane_p : plane_q)) = lo;
    }
}

}  // namespace dev
}  // namespace cgh
