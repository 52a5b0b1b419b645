// Device-side code of the direct form, shared by its kernels (direct.cu) and by the persistent batch kernel
// (persist.cu): the terms of one point in a thread's block of pixels and the unit of work that sums the points of a
// range into a tile of pixels.
//
// a2, the direct form.  Every thread owns a TL x TR block of hologram pixels
// (TL consecutive columns of TR consecutive rows) and sums every point of the
// cloud into it, I(m, n) = sum_j A_j cos(2 pi c_j r^2) (Eq. 5, restricted form).
//
// Point tiles of kPointTile prepared points are staged in shared memory by
// 1-D bulk copies (TMA engine, no multicast), double buffered behind two
// mbarriers, and read back as warp-wide broadcasts.
//
// Phase.  For one point the squared distance splits into a column part and a
// row part, r^2 = (m - x)^2 + (n - y)^2.  The thread forms the turns of its
// first column and first row, C d^2 mod 2^64 (top 32 bits, exact to one unit
// of 2^-32 turn), their first differences, and walks its TL columns and its TR
// rows with the recurrence of Eqs. 6-8 (Section 2.2): Gamma_{k+1} = Gamma_k +
// delta_k, delta_{k+1} = delta_k + Delta, Delta = 2 c_j, in 32-bit fixed-point
// turns, where wrap-around is the reduction modulo one turn (drift below
// 1 + TL + TL^2/2 units of 2^-32 turn along the columns, the same with TR down
// the rows).  The point's piston and the reference phase join the column
// turns (its row step the row turns).
//
// Sine and cosine.  The term is A cos 2 pi (a_i + b_r), taken by the cosine
// addition formula from the sine and cosine of the TL + TR turns
// (point_terms_sep).  A turn's top 23 bits become the mantissa of a float f in
// [1, 2) (one funnel shift, rounded to nearest by a bias) and u = K1 f - K0 is
// the angle in [-pi, pi) (one FFMA):
//  - SFU form: the hardware sine and cosine of u (__sincosf, MUFU).  The MUFU
//    sine is exactly odd, but its error is not zero on average over an
//    arbitrary argument grid: on the grid of the plain fl(2 pi) f - fl(3 pi),
//    which sits a third of a step off symmetric, it averaged +1.35e-8 (a bias
//    that grew linearly with N when each term took one hardware sine).  K1 is
//    therefore 2 pi rounded to a float whose 1.5 multiple K0 is exact, so the
//    FFMA returns exactly RN((f - 1.5) K1): the argument grid is symmetric
//    about zero.  K1 is 1.04e-7 above 2 pi (a zero-mean phase-scale error below
//    3.3e-7 rad).  The hardware cosine's error is even; every other point is
//    shifted by half a turn so that its mean cancels (point_terms_sep).
//  - accurate form: the turn, read as a signed 32-bit integer, converts to
//    t in [-1/2, 1/2) and cos(2 pi t) is a degree-12 even polynomial
//    (cospoly.h), all on the FMA pipe; the sine is the cosine a quarter turn
//    back.
//
// Accumulation is two-level: each point tile is summed into fresh partials
// that are then added into the running totals, which keeps single-precision
// rounding error at N = 10^6 well below 1e-5 relative.
#pragma once

#include <type_traits>

#include "cospoly.h"
#include "device_util.cuh"
#include "kernels.h"

namespace cgh {
namespace dev {

// 2 pi rounded up to the nearest float whose mantissa is a multiple of 4,
// so that 1.5 K1 is a float too (0x40c90fdc and 0x4116cbe5)
constexpr float kK1 = 6.28318595886230469f;
constexpr float kK0 = 9.42477893829345703f;   // exactly 1.5 * kK1
// a half turn (so (f - 1.5) K1 is the angle itself in [-pi, pi)) and rounding of the 23-bit truncation
constexpr uint32_t kHalfBias = (1u << 31) + 256u;
// cos(2 pi t) of a signed fixed-point turn t in [-1/2, 1/2) (2^-32 turn) by the polynomial of cospoly.h.
__device__ __forceinline__ float cos_turn_poly(uint32_t g)
{
    const float t = (float)(int)g * 2.3283064365386963e-10f;   // signed turn, [-1/2, 1/2)
    const float u = t * t;
    float c = CGH_COSPOLY_6;
    c = fmaf(c, u, CGH_COSPOLY_5);
    c = fmaf(c, u, CGH_COSPOLY_4);
    c = fmaf(c, u, CGH_COSPOLY_3);
    c = fmaf(c, u, CGH_COSPOLY_2);
    c = fmaf(c, u, CGH_COSPOLY_1);
    c = fmaf(c, u, CGH_COSPOLY_0);
    return c;
}

// The reference phase seen by one thread: its value at the thread's corner
// pixel and its change per column and per row (all 2^-32 turn).  Added to a
// point's corner phase and first differences, it costs three additions per
// point, none per term; the kernels without piston and reference (EXTRA =
// false) skip even those (measured 3 % on the SFU form).
struct PixelRef {
    uint32_t g, dx, dy;
};

__device__ __forceinline__ PixelRef pixel_ref(const PhaseRef &r, int m0, int n0)
{
    return PixelRef{ref_turn(r, m0, n0), ref_step(r.kx), ref_step(r.ky)};
}

// Adds one point's terms to a thread's TL x TR block by the separability of the squared distance inside the block:
// with a_i the turn of column m0 + i and b_r that of row n0 + r (each walked by Eqs. 6-8 in exact fixed point, the
// piston and the reference phase's corner and column steps in a_i, its row step in b_r),
//     A cos 2 pi (a_i + b_r) = cos 2 pi a_i (A cos 2 pi b_r) - sin 2 pi a_i (A sin 2 pi b_r),
// so the hardware sine and cosine (one __sincosf, two MUFU operations) of TL + TR turns serve TL x TR terms at two
// FFMAs each: TL TR / (2 (TL + TR)) times fewer MUFU operations than one cosine per term (2x at 8 x 8).  Each turn
// is rounded to 2^-23 and taken on the symmetric argument grid of kK1 and kK0.  The hardware cosine's error is even in
// its argument and does not average to zero over the grid, which made the field's error grow with the number of
// points (NRMS 9.0e-7 at 10^4 points, 3.1e-6 at 2 10^5, 1920x1080); flip = a half turn on every other point
// shifts both of its turns by pi, which leaves the term as it is (cos((a + pi) + (b + pi)) = cos(a + b)) and
// turns the sign of that mean, so it cancels over pairs of points (5.8e-7 and 6.9e-7).
// ACC: the accurate form -- cos 2 pi t from the polynomial of cos_turn_poly and sin 2 pi t = cos 2 pi (t - 1/4) from the
// same polynomial, on the FMA pipe (no flip needed: the polynomial's mean error over the turns is about zero).
// PLANES = 2: the complex object wave (Eq. 2, restricted form), A e^{i 2 pi (a_i + b_r)}: the real part to part,
// the imaginary part, sin 2 pi a_i (A cos 2 pi b_r) + cos 2 pi a_i (A sin 2 pi b_r), to part_im.
template <int TL, int TR, bool EXTRA, bool ACC = false, int PLANES = 1>
__device__ __forceinline__ void point_terms_sep(const int4 q, const uint2 w, int m0, int n0, const PixelRef &pr,
                                                uint32_t flip, float (&part)[TR][TL], float (&part_im)[TR][TL])
{
    const uint32_t chi = (uint32_t)q.z, clo = (uint32_t)q.w;
    const uint32_t dx = (uint32_t)(m0 - q.x);
    const uint32_t dy = (uint32_t)(n0 - q.y);
    const uint32_t x2 = dx * dx, x2n = x2 + 2u * dx + 1u;   // dx^2, (dx + 1)^2: below 2^32, exact
    const uint32_t y2 = dy * dy, y2n = y2 + 2u * dy + 1u;
    uint32_t a = chi * x2 + __umulhi(clo, x2) + kHalfBias + flip;
    uint32_t da = chi * x2n + __umulhi(clo, x2n) - (a - kHalfBias - flip);
    uint32_t b = chi * y2 + __umulhi(clo, y2) + kHalfBias + flip;
    uint32_t db = chi * y2n + __umulhi(clo, y2n) - (b - kHalfBias - flip);
    uint32_t D = w.x;
    if constexpr (EXTRA) {   // piston (aux.x) and reference; 2 C formed from C
        da += pr.dx;
        db += pr.dy;
        a += w.x + pr.g;
        D = __funnelshift_l(clo, chi, 1);
    }
    const float amp = __uint_as_float(w.y);
    // (cos, sin) of 2 pi times a turn held with the bias above
    auto cis = [](uint32_t t, float &s, float &c) {
        if constexpr (ACC) {
            const uint32_t u = t - kHalfBias;            // the turn itself (the flip is a whole half turn)
            c = cos_turn_poly(u);
            s = cos_turn_poly(u - (1u << 30));   // cos 2 pi (t - 1/4)
        } else {
            const float f = __uint_as_float(__funnelshift_r(t, 0x7fu, 9));
            __sincosf(fmaf(f, kK1, -kK0), &s, &c);
        }
    };
    float ca[TL], sa[TL];
#pragma unroll
    for (int i = 0; i < TL; ++i) {
        cis(a, sa[i], ca[i]);
        a += da;
        da += D;
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        float sb, cb;
        cis(b, sb, cb);
        cb *= amp;
        sb *= amp;
#pragma unroll
        for (int i = 0; i < TL; ++i) {
            part[r][i] = fmaf(-sa[i], sb, fmaf(ca[i], cb, part[r][i]));
            if constexpr (PLANES == 2) part_im[r][i] = fmaf(ca[i], sb, fmaf(sa[i], cb, part_im[r][i]));
        }
        b += db;
        db += D;
    }
}

// Tables of the tile (TABLES): the sine and cosine of a column's turn depend on the point and the column only, a
// row's on the point and the row only, so per group of points the CTA takes them once for its whole pixel tile --
// TILE_W column pairs and TILE_H row pairs (the amplitude folded into the rows) per point, spread over the threads
// -- and every thread reads its 8 columns and TR rows from shared memory: 2 FMAs a term, and per point and
// thread (TILE_W + TILE_H) / threads sine-cosine pairs instead of TL + TR.  A group of 8 columns is stored as
// four 16-byte quads (cos c, cos c+1, sin c, sin c+1), the operands of packed FMAs over two columns, and padded
// to five quads (80 bytes), so the 8 threads of a quarter warp that read their quads fall on distinct banks.  A
// row is stored as (A cos b, -A sin b).
template <int TILE_W, int TILE_H>
struct SepTable {
    static_assert(TILE_W % 8 == 0, "whole groups of 8 columns");
    static constexpr int kColStride = TILE_W / 8 * 10;   // float2s of one point's columns
    static constexpr int kPerPoint = kColStride + TILE_H;
    // float index of column k's cosine (its sine two floats on)
    __device__ static int col_cos(int k) { return (k >> 3) * 20 + ((k & 7) >> 1) * 4 + (k & 1); }
};
// points per table fill (double buffered: one CTA barrier per group; 8 measured 2.69 ms, 32 3.04 -- two CTAs no
// longer fit an SM -- against 2.51 at 16, 1920x1080, 10^4 points); the complex wave, whose two planes of totals
// take twice the shared memory, fills 8
constexpr int kSepGroup = 16;
template <int PLANES>
__host__ __device__ constexpr int sep_group()
{
    return PLANES == 2 ? 8 : kSepGroup;
}

// The tables of np <= GROUP points p0, p0 + 1, ... for a tile: NTHREADS / GROUP threads a point (a half warp or a
// warp), each taking its point's turn constants once and then its share of the columns and rows, one entry at a
// time (entry(e), e < kEntries: its columns, then its rows), so that a caller can spread them over other work.  A
// half warp's column stores cover groups q and q + 4 of 8 columns, whose cosines (and sines) fall on disjoint banks.
template <int TILE_W, int TILE_H, int NTHREADS, int GROUP, bool EXTRA, bool ACC>
struct SepFiller {
    using S = SepTable<TILE_W, TILE_H>;
    static constexpr int TPP = NTHREADS / GROUP;   // threads a point
    static_assert(NTHREADS % GROUP == 0 && (TPP == 16 || TPP == 32), "a half warp or a warp a point");
    static_assert(TILE_W % TPP == 0 && TILE_W % 64 == 0 && TILE_H % TPP == 0,
                  "whole pairs of column groups, whole rows a thread");
    static constexpr int kCols = TILE_W / TPP, kEntries = TILE_W / TPP + TILE_H / TPP;

    int4 q;
    uint2 w;
    float2 *dst;
    int j, tile_m0, tile_n0;
    uint32_t flip;
    bool active;

    __device__ __forceinline__ SepFiller(const int4 *sg, const uint2 *sa, int p0, int np, int m0, int n0,
                                         float2 *tab, int tid)
    {
        const int g = tid / TPP;
        j = tid % TPP;
        tile_m0 = m0;
        tile_n0 = n0;
        active = g < np;
        const int p = p0 + g;
        flip = ACC ? 0u : (uint32_t)(p & 1) << 31;   // the flip of every other point (point_terms_sep)
        dst = tab + g * S::kPerPoint;
        if (active) {
            q = sg[p];
            w = sa[p];
        }
    }

    // the point's turn at a column (row) coordinate, exact: C d^2 mod 2^64, top 32 bits (d^2 below 2^31)
    __device__ __forceinline__ uint32_t turn(int coord, int center) const
    {
        const uint32_t d = (uint32_t)(coord - center);
        const uint32_t d2 = d * d;
        return (uint32_t)q.z * d2 + __umulhi((uint32_t)q.w, d2);
    }

    __device__ __forceinline__ void sincos_turn(uint32_t t, float &sn, float &cs) const
    {
        if constexpr (ACC) {
            cs = cos_turn_poly(t);
            sn = cos_turn_poly(t - (1u << 30));   // cos 2 pi (t - 1/4)
        } else {
            t += kHalfBias + flip;
            const float f = __uint_as_float(__funnelshift_r(t, 0x7fu, 9));
            __sincosf(fmaf(f, kK1, -kK0), &sn, &cs);
        }
    }

    // entry e of the thread (a constant once the caller's loop is unrolled)
    __device__ __forceinline__ void entry(int e, const PhaseRef &ref) const
    {
        if (!active) return;
        if (e < kCols) {
            const int x = e * (TPP / 8) + (j >> 3);                 // the thread's group of 8 columns, in order ...
            const int grp = (x & 1) * 4 + ((x >> 1) & 3) + (x & ~7);   // ... taken as 0, 4, 1, 5, 2, 6, 3, 7, 8, ...
            const int k = grp * 8 + (j & 7);
            const int coord = tile_m0 + k;
            uint32_t t = turn(coord, q.x);
            if constexpr (EXTRA) t += w.x + ref_turn(ref, coord, 0);   // piston, the reference's column part
            float sn, cs;
            sincos_turn(t, sn, cs);
            float *c = reinterpret_cast<float *>(dst) + S::col_cos(k);
            c[0] = cs;
            c[2] = sn;
        } else {
            const int k = j + TPP * (e - kCols);
            const int coord = tile_n0 + k;
            uint32_t t = turn(coord, q.y);
            if constexpr (EXTRA) t += ref_turn(ref, 0, coord) - ref.phi0;   // the reference phase's row part
            float sn, cs;
            sincos_turn(t, sn, cs);
            const float a = __uint_as_float(w.y);
            dst[S::kColStride + k] = make_float2(a * cs, -(a * sn));
        }
    }

    __device__ __forceinline__ void all(const PhaseRef &ref) const
    {
#pragma unroll
        for (int e = 0; e < kEntries; ++e) entry(e, ref);
    }
};

// One point's tables for a thread: its 8 column pairs (from column cx) and TR row pairs (from row ry) as float4s.
template <int TR, int TILE_W, int TILE_H>
struct SepQuads {
    float4 c[4], r[TR / 2];
    __device__ __forceinline__ void load(const float2 *tab, int cx, int ry)
    {
        using S = SepTable<TILE_W, TILE_H>;
        const float4 *c4 = reinterpret_cast<const float4 *>(tab + (cx >> 3) * 10);
        const float4 *r4 = reinterpret_cast<const float4 *>(tab + S::kColStride + ry);
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = c4[j];
#pragma unroll
        for (int h = 0; h < TR / 2; ++h) r[h] = r4[h];
    }
};

// One point's terms from its quads, two columns a packed FMA (the two lanes' FMAs in one instruction):
// acc[0][r][j] += (cos a_2j, cos a_2j+1) (A cos b_r) + (sin a_2j, sin a_2j+1) (-A sin b_r), the same two roundings
// per term as two scalar FMAs; with PLANES = 2 also the imaginary part, acc[1][r][j] += (sin a) (A cos b_r) +
// (cos a) (A sin b_r).
template <int TR, int TILE_W, int TILE_H, int PLANES>
__device__ __forceinline__ void point_terms_table(const SepQuads<TR, TILE_W, TILE_H> &q,
                                                  float2 (&acc)[PLANES][TR][4])
{
    static_assert(TR % 2 == 0, "row pairs in 16-byte quads");
#pragma unroll
    for (int h = 0; h < TR / 2; ++h) {
        const float4 v = q.r[h];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 c = make_float2(q.c[j].x, q.c[j].y), s = make_float2(q.c[j].z, q.c[j].w);
            acc[0][2 * h][j] =
                __ffma2_rn(s, make_float2(v.y, v.y), __ffma2_rn(c, make_float2(v.x, v.x), acc[0][2 * h][j]));
            acc[0][2 * h + 1][j] =
                __ffma2_rn(s, make_float2(v.w, v.w), __ffma2_rn(c, make_float2(v.z, v.z), acc[0][2 * h + 1][j]));
            if constexpr (PLANES == 2) {
                acc[1][2 * h][j] = __ffma2_rn(c, make_float2(-v.y, -v.y),
                                              __ffma2_rn(s, make_float2(v.x, v.x), acc[1][2 * h][j]));
                acc[1][2 * h + 1][j] = __ffma2_rn(c, make_float2(-v.w, -v.w),
                                                  __ffma2_rn(s, make_float2(v.z, v.z), acc[1][2 * h + 1][j]));
            }
        }
    }
}

// The points of the unit are those of tiles [t_begin, t_end), less the first p_first points of the first tile
// and the points from p_last_end on of the last one.  Sink: PlainStore writes the totals to dst; any other sink
// is called as sink(tot) with the thread's TR x TL totals of plane 0 (the amplitude hologram only).
// Sync: the threads that share the unit and their barrier -- CtaSync (the whole CTA) or GroupSync (a named
// barrier over a group of warps of a larger CTA).  T: points per shared-memory tile (the prepared points are
// padded to a multiple of kPointTile, which T divides).
struct PlainStore {};

struct CtaSync {
    __device__ static int tid() { return threadIdx.x; }
    __device__ static void sync() { __syncthreads(); }
    __device__ static bool sync_or(bool p) { return __syncthreads_or(p) != 0; }
};

template <int ID, int NTHREADS, int BASE>
struct GroupSync {
    __device__ static int tid() { return (int)threadIdx.x - BASE; }
    __device__ static void sync() { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(NTHREADS) : "memory"); }
    __device__ static bool sync_or(bool p)
    {
        uint32_t r;
        asm volatile(
            "{\n\t.reg .pred a, b;\n\t"
            "setp.ne.u32 a, %1, 0;\n\t"
            "bar.red.or.pred b, %2, %3, a;\n\t"
            "selp.u32 %0, 1, 0, b;\n\t}"
            : "=r"(r)
            : "r"((uint32_t)p), "n"(ID), "n"(NTHREADS)
            : "memory");
        return r != 0;
    }
};

template <int TL, int TR, int BX, int BY, bool SFU, int PLANES = 1, bool EXTRA = false, bool SMEM_TOT = false,
          class Sink = PlainStore, class Sync = CtaSync, int T = kPointTile, bool TABLES = false>
__device__ __forceinline__ bool direct_unit(const int4 *__restrict__ geo, const uint2 *__restrict__ aux,
                                            int t_begin, int t_end, int tile_m0, int tile_n0, int width,
                                            int height, float *__restrict__ dst, bool vec, int4 (*s_geo)[T],
                                            uint2 (*s_aux)[T], uint64_t *s_bar, uint32_t &kg, int *status,
                                            unsigned long long timeout_ns, int drop = -1, long long im_offset = 0,
                                            const PhaseRef &ref = PhaseRef(), float *s_tot = nullptr,
                                            int p_first = 0, int p_last_end = T, Sink sink = Sink(),
                                            float2 *s_tab = nullptr)
{
    static_assert(kPointTile % T == 0 && T % 16 == 0, "point tiles divide the padding");
    constexpr uint32_t kTileBytes = T * (sizeof(int4) + sizeof(uint2));
    const int tid = Sync::tid();
    const int lx = tid % BX, ly = tid / BX;
    const int m0 = tile_m0 + lx * TL;
    const int n0 = tile_n0 + ly * TR;
    const int nt = t_end - t_begin;
    const PixelRef pr = pixel_ref(ref, m0, n0);

    auto issue = [&](int k) {
        if (k == drop) return;   // test hook: this tile's barrier is never completed
        const int st = (int)((kg + (uint32_t)k) & 1u);
        const long long first = (long long)(t_begin + k) * T;
        mbar_arrive_expect_tx(&s_bar[st], kTileBytes);
        bulk_copy_g2s(&s_geo[st][0], geo + first, T * sizeof(int4), &s_bar[st]);
        bulk_copy_g2s(&s_aux[st][0], aux + first, T * sizeof(uint2), &s_bar[st]);
    };
    if (tid == 0) {
        if (nt > 0) issue(0);
        if (nt > 1) issue(1);
    }

    constexpr int NT = BX * BY;
    auto tidx = [&](int c, int r, int i) { return ((c * TR + r) * TL + i) * NT + tid; };
    float tot[PLANES][TR][TL];
#pragma unroll
    for (int c = 0; c < PLANES; ++c)
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int i = 0; i < TL; ++i) {
                if constexpr (SMEM_TOT) s_tot[tidx(c, r, i)] = 0.0f;
                else tot[c][r][i] = 0.0f;
            }

    bool ok = true;
    for (int k = 0; k < nt; ++k) {
        const uint32_t kk = kg + (uint32_t)k;
        const int st = (int)(kk & 1u);
        const bool arrived = mbar_wait(&s_bar[st], (kk >> 1) & 1u, timeout_ns);
        if (Sync::sync_or(!arrived)) {
            if (tid == 0) {
                atomicOr(status, kStatusTimeout);
                // wait (bounded) for the other tile copy this unit may still have in flight
                if (k + 1 < nt && k + 1 != drop) {
                    const uint32_t kn = kk + 1u;
                    mbar_wait(&s_bar[kn & 1u], (kn >> 1) & 1u, timeout_ns);
                }
            }
            Sync::sync();
            ok = false;
            break;
        }
        float part[PLANES][TR][TL];
#pragma unroll
        for (int c = 0; c < PLANES; ++c)
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int i = 0; i < TL; ++i) part[c][r][i] = 0.0f;

        const int4 *sg = s_geo[st];
        const uint2 *sa = s_aux[st];
        const int p_lo = k == 0 ? p_first : 0;
        const int p_hi = k == nt - 1 ? p_last_end : T;
        if constexpr (TABLES) {
            static_assert(TL == 8, "tables serve 8-column blocks");
            static_assert(PLANES == 1 || SFU, "the complex wave takes the hardware sine and cosine");
            constexpr int TW = BX * TL, TH = BY * TR, GROUP = sep_group<PLANES>();
            using ST = SepTable<TW, TH>;
            float2 acc[PLANES][TR][TL / 2];   // columns 2 j and 2 j + 1
#pragma unroll
            for (int c = 0; c < PLANES; ++c)
#pragma unroll
                for (int r = 0; r < TR; ++r)
#pragma unroll
                    for (int j = 0; j < TL / 2; ++j) acc[c][r][j] = make_float2(0.0f, 0.0f);
            // The next group's tables are filled while this group's are read: for the amplitude hologram the
            // fill's entries (integer products, hardware or polynomial sines) are spread over the point loop's
            // packed FMAs (1920x1080, 10^4 points: 1.77 against 1.79 ms filled before the loop; the complex wave,
            // short of registers, measured 3.26 against 3.21 and fills first); one barrier a group hands the
            // buffers over.
            using Filler = SepFiller<TW, TH, BX * BY, GROUP, EXTRA, !SFU>;
            constexpr int U = PLANES == 1 ? 4 : 2;   // points a step (the loop was measured fastest unrolled by
                                                     // four, 2.30 ms against 2.32 by two at 1920x1080, 10^4 points;
                                                     // the complex wave's two planes leave the registers for two)
            constexpr int kSteps = GROUP / U;
            constexpr int kPerStep = (Filler::kEntries + kSteps - 1) / kSteps;
            const int n_grp = (p_hi - p_lo + GROUP - 1) / GROUP;
            int gi = 0;
            if (n_grp > 0) {
                Filler(sg, sa, p_lo, min(GROUP, p_hi - p_lo), tile_m0, tile_n0, s_tab, tid).all(ref);
                Sync::sync();
            }
#pragma unroll 1
            for (int gg = 0; gg < n_grp; ++gg, ++gi) {
                const int p0 = p_lo + gg * GROUP;
                const int np = min(GROUP, p_hi - p0);
                const float2 *cur = s_tab + (gi & 1) * (GROUP * ST::kPerPoint);
                const int pn = p0 + GROUP;
                const int npn = gg + 1 < n_grp ? min(GROUP, p_hi - pn) : 0;
                const Filler next(sg, sa, pn, npn, tile_m0, tile_n0, s_tab + ((gi + 1) & 1) * (GROUP * ST::kPerPoint),
                                  tid);
                if constexpr (PLANES == 2) next.all(ref);
                if (PLANES == 1 && np == GROUP) {
#pragma unroll
                    for (int st = 0; st < kSteps; ++st) {
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            SepQuads<TR, TW, TH> qd;
                            qd.load(cur + (st * U + u) * ST::kPerPoint, lx * TL, ly * TR);
                            point_terms_table<TR, TW, TH, PLANES>(qd, acc);
                        }
#pragma unroll
                        for (int e = st * kPerStep; e < (st + 1) * kPerStep && e < Filler::kEntries; ++e)
                            next.entry(e, ref);
                    }
                } else {   // the complex wave (filled above), or a short last group (nothing to fill after it)
#pragma unroll U
                    for (int g = 0; g < np; ++g) {
                        SepQuads<TR, TW, TH> qd;
                        qd.load(cur + g * ST::kPerPoint, lx * TL, ly * TR);
                        point_terms_table<TR, TW, TH, PLANES>(qd, acc);
                    }
                }
                Sync::sync();   // the next group's tables are written, this group's are no longer read
            }
#pragma unroll
            for (int c = 0; c < PLANES; ++c)
#pragma unroll
                for (int r = 0; r < TR; ++r)
#pragma unroll
                    for (int j = 0; j < TL / 2; ++j) {
                        part[c][r][2 * j] = acc[c][r][j].x;
                        part[c][r][2 * j + 1] = acc[c][r][j].y;
                    }
        } else {
            static_assert(PLANES == 1 || SFU, "the complex wave takes the hardware sine and cosine");
#pragma unroll 1
            for (int p = p_lo; p < p_hi; ++p)   // p has the parity of the point's index (tiles start even)
                point_terms_sep<TL, TR, EXTRA, !SFU, PLANES>(sg[p], sa[p], m0, n0, pr,
                                                             SFU ? (uint32_t)(p & 1) << 31 : 0u, part[0],
                                                             part[PLANES - 1]);
        }
#pragma unroll
        for (int c = 0; c < PLANES; ++c)
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int i = 0; i < TL; ++i) {
                    if constexpr (SMEM_TOT) s_tot[tidx(c, r, i)] += part[c][r][i];
                    else tot[c][r][i] += part[c][r][i];
                }

        Sync::sync();   // every thread is done with stage st
        if (tid == 0 && k + 2 < nt) issue(k + 2);
    }
    kg += (uint32_t)nt;
    if (!ok) return false;
    if constexpr (SMEM_TOT) {
#pragma unroll
        for (int c = 0; c < PLANES; ++c)
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int i = 0; i < TL; ++i) tot[c][r][i] = s_tot[tidx(c, r, i)];
    }
    if constexpr (!std::is_same<Sink, PlainStore>::value) {
        static_assert(PLANES == 1, "sinks take the amplitude hologram");
        sink(tot[0]);
        return true;
    }

#pragma unroll
    for (int c = 0; c < PLANES; ++c)
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const int n = n0 + r;
            if (n >= height || m0 >= width) continue;
            float *row = dst + (long long)c * im_offset + (long long)n * width + m0;
            if (vec && m0 + TL <= width) {
#pragma unroll
                for (int i = 0; i < TL; i += 4)
                    *reinterpret_cast<float4 *>(row + i) =
                        make_float4(tot[c][r][i], tot[c][r][i + 1], tot[c][r][i + 2], tot[c][r][i + 3]);
            } else {
#pragma unroll
                for (int i = 0; i < TL; ++i)
                    if (m0 + i < width) row[i] = tot[c][r][i];
            }
        }
    return true;
}

template <int BX, int BY>
__device__ __forceinline__ void init_point_barriers(uint64_t *s_bar)
{
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
}

}  // namespace dev
}  // namespace cgh
