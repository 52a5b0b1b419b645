// a3: the separable factors of the GEMM form.
//
// The phase of Eq. 5 (restricted form) is 2 pi c_j ((m - x_j)^2 + (n - y_j)^2)
// = alpha_mj + beta_nj, so
//   cos(alpha + beta) = cos(alpha) cos(beta) - sin(alpha) sin(beta)
// and I = P Q^T with, for point j,
//   P[n][2j] = cos beta_nj,        P[n][2j+1] = sin beta_nj
//   Q[m][2j] = s A_j cos alpha_mj, Q[m][2j+1] = -s A_j sin alpha_mj
// (s = an optional amplitude scale, undone in the GEMM epilogue).
//
// Each angle is reduced in integers: with the point's 64-bit fixed-point
// constant C_j (prep.cu), the turn is the top 32 bits of C_j d^2 mod 2^64, d
// the integer distance along one axis (|d| < 2^15, so d^2 < 2^30).  Split
// FP16 (hi = fp16(v), lo = fp16(v - hi), 2^-22 of v): that exact turn for every
// entry, converted to t in [-1/2, 1/2) (error <= 2^-26 turn), and the hardware
// sine and cosine (MUFU, |2 pi t| <= pi, absolute error below 4e-7) give the
// pair -- ~1e-7 of the NRMS, which the accumulation dominates.  FP16 and BF16:
// the turn is exact at a band's first row and walks down the band by the
// second-order recurrence of Eqs. 6-8 (drift < 496 units of 2^-32 turn over 32
// rows), converted through its top 23 bits as a float mantissa -- 1.1e-6 rad at
// most, far below their rounding, and the kernel becomes HBM-write-bound.  No
// FP64 is needed on the GPU.
//
// For the imaginary part of the complex wave, sin(alpha + beta) =
// sin(alpha) cos(beta) + cos(alpha) sin(beta), so Im O = P Q'^T with the same P
// and Q'[m][2j] = s A_j sin alpha, Q'[m][2j+1] = s A_j cos alpha ("imag" launch,
// Q' rows only).
//
// One thread owns 4 consecutive points (8 columns, one 16-byte store per row
// and plane) and walks a band of rows, so the point constants are read once
// per band; rows [0, height) are P's, rows [height, height + width) are Q's.
#include "factors_dev.cuh"
#include "kernels.h"

namespace cgh {

namespace {

using namespace dev;

template <int MODE, bool IMAG>
__global__ void __launch_bounds__(kFactorThreads)
    factors_kernel(const int4 *__restrict__ geo, const uint2 *__restrict__ aux, int n_points, int slots,
                   int height, int width, uint16_t *__restrict__ P, uint16_t *__restrict__ Q, long long ld,
                   long long plane_p, long long plane_q, const float *__restrict__ amp_max, int row_begin,
                   const PhaseRef ref)
{
    const int j0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (j0 >= slots) return;
    float scale = 1.0f;
    if (amp_max != nullptr) {
        const float m = *amp_max;
        if (m > 0.0f) scale = 1.0f / m;
    }
    const int rows = height + width;
    const int r_begin = row_begin + blockIdx.y * kRowsPerBlock;
    const int r_end = min(rows, row_begin + (int)(blockIdx.y + 1) * kRowsPerBlock);
    factor_thread<MODE, IMAG>(j0, r_begin, r_end, geo, aux, n_points, height, width, P, Q, ld, plane_p, plane_q,
                              scale, ref);
}

// Grouped factors (groups.cu): for group g (plane constant C, column x_g,
// members in [first, first + count) of the gathered point arrays)
//   P'[n][2g] + i P'[n][2g+1] = s sum_members A_j exp(i 2 pi C (n - y_j)^2)
//   Q'[m][2g] + i Q'[m][2g+1] = exp(-i 2 pi C (m - x_g)^2)   (cos alpha, -sin alpha)
// so that sum_k P'[n][k] Q'[m][k] = s Re sum_g W_g(n) U_g(m) = s I(m, n);
// s = 1 / wscale keeps |P'| <= 1.
//
// A block covers kGroupRows rows (of P', or of Q' for the blocks past the P'
// rows) and kGroupTile group slots.  Each warp takes whole groups; lane l owns
// the rows r0 + l + 32 q, q = 0 .. 3, so the lanes of a warp run the same
// member loop (no divergence whatever the group sizes) and read each member's
// staged constants with one broadcast load for four terms.  The block's results
// meet in shared memory (slot-major, padded against bank conflicts) and leave as
// full 128-byte row segments.
//
// Per member and lane, row q = 0: the turn C (n - y)^2 mod 1 in 32-bit fixed
// point (rounded to 23 bits by the +256), its top 23 bits as the mantissa of f
// in [1, 2), and u = (f - 1.5) K1 in [-pi, pi): the angle minus a half turn, so
// the sine and cosine of u are minus those of the angle -- the members carry -A.
// K1 is 2 pi rounded to a float whose 1.5 multiple is exact, so the argument
// grid is symmetric about zero and the hardware sine's odd error cancels in the
// sum (as in the direct kernel).  Rows q = 1 .. 3 are 32 rows apart, where the
// phase differs by 32 E (up to the common C l^2, applied at the end): their
// terms are the row-0 phasor rotated by exp(i 2 pi 32 E), which the staging lane
// computes once per member with the accurate sincospif.  A term then costs a
// quarter of one hardware sincos and a complex multiply; each rotation adds
// about 1e-7 of relative error (three at most), against the sincos's 4e-7.
constexpr int kGroupTile = 32;
constexpr int kGroupThreads = 256;
constexpr int kGroupLaneRows = 4;                      // rows per lane
constexpr int kGroupRows = 32 * kGroupLaneRows;       // rows per block
constexpr int kTileStride = kGroupRows + 1;            // words per slot in the shared tile, +1 against conflicts

__device__ __forceinline__ void half_turn_sincos(uint32_t chi, uint32_t clo, uint32_t d, uint32_t add, float &s,
                                                 float &c)
{
    const uint32_t d2 = d * d;                                    // < 2^30
    const uint32_t g = chi * d2 + add + __umulhi(clo, d2);       // turn in 2^-32 units (add: +1/2 ulp of 23 bits, reference)
    const float f = __uint_as_float((g >> 9) | 0x3f800000u);
    __sincosf(fmaf(f, kTurnK1, -kTurnK0), &s, &c);
}

template <int MODE>
__global__ void __launch_bounds__(kGroupThreads)
    group_factors_kernel(const int4 *__restrict__ groups, int g_begin, int n_groups, int slots,
                         const unsigned long long *__restrict__ planes, const int2 *__restrict__ members,
                         int height, int width, uint16_t *__restrict__ P, uint16_t *__restrict__ Q, long long ld,
                         long long plane_p, long long plane_q, const float *__restrict__ wscale, const PhaseRef ref)
{
    __shared__ uint32_t tile_hi[kGroupTile * kTileStride];
    __shared__ uint32_t tile_lo[MODE == kFactorSplit16 ? kGroupTile * kTileStride : 1];
    __shared__ uint4 stage[kGroupThreads / 32][32];    // per warp: {G, E, -A, 0} of 32 members
    __shared__ float2 stage_r[kGroupThreads / 32][32];  // and their 32-row rotations exp(i 2 pi 32 E)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p_blocks = (height + kGroupRows - 1) / kGroupRows;
    const bool is_p = (int)blockIdx.y < p_blocks;
    const int r0 = (is_p ? (int)blockIdx.y : (int)blockIdx.y - p_blocks) * kGroupRows;
    const int s_base = blockIdx.x * kGroupTile;
    const float inv = 1.0f / *wscale;
    // reference phase of this lane's rows (P': ky n) or columns (Q': kx m + phi0)
    uint32_t radd[kGroupLaneRows];
#pragma unroll
    for (int q = 0; q < kGroupLaneRows; ++q) {
        const int line = r0 + lane + 32 * q;
        radd[q] = is_p ? ref_turn(ref, 0, line) - ref.phi0 : ref_turn(ref, line, 0);
    }
    for (int k = warp; k < kGroupTile; k += kGroupThreads / 32) {
        const int slot = s_base + k;
        float re[kGroupLaneRows], im[kGroupLaneRows];
#pragma unroll
        for (int q = 0; q < kGroupLaneRows; ++q) re[q] = im[q] = 0.0f;
        if (slot < n_groups) {
            const int4 d = groups[g_begin + slot];   // {first, count, plane, x}
            const unsigned long long C = planes[d.z];
            const uint32_t chi = (uint32_t)(C >> 32), clo = (uint32_t)C;
            if (is_p) {
                // (r0 + l - y)^2 = D^2 + 2 D l + l^2, D = r0 - y, l = lane + 32 q < 128: per member G = C D^2 and
                // E = 2 C D (top 32 bits, one lane each), per row the phase G + E l; each row's C l^2 (and the
                // reference) is one rotation of the sum at the end.  E l in 32 bits is off by at most l < 128
                // units of 2^-32.
                const unsigned long long C2 = C << 1;
                for (int base = 0; base < d.y; base += 32) {
                    const int j = base + lane;
                    if (j < d.y) {
                        const int2 v = members[d.x + j];
                        const int D = r0 - v.x;
                        const uint32_t d2 = (uint32_t)(D * D);   // < 2^30
                        const uint32_t G = chi * d2 + __umulhi(clo, d2);
                        const uint32_t E = (uint32_t)((C2 * (unsigned long long)(long long)D) >> 32);
                        stage[warp][lane] = make_uint4(G + 256u, E, (uint32_t)v.y, 0u);   // +2^8: round to 23 bits
                        // 32 rows on, the phase grows by 32 E: its rotation, accurate (once per member, shared by
                        // every lane); pi x with x = (32 E as a signed turn) * 2 is the angle in [-pi, pi)
                        float rs, rc;
                        sincospif((float)(int)(E << 5) * 4.656612873077393e-10f, &rs, &rc);
                        stage_r[warp][lane] = make_float2(rc, rs);
                    }
                    __syncwarp();
                    const int n = min(32, d.y - base);
                    for (int i = 0; i < n; ++i) {
                        const uint4 s = stage[warp][i];                              // same address in every lane
                        const float2 r = stage_r[warp][i];
                        const uint32_t t = s.x + s.y * (uint32_t)lane;
                        const float f = __uint_as_float(__funnelshift_r(t, 0x7fu, 9));   // 0x3f800000 | t >> 9
                        float sn, cs;
                        __sincosf(fmaf(f, kTurnK1, -kTurnK0), &sn, &cs);             // angle - pi
                        const float a = __uint_as_float(s.z);                         // members carry -A
                        float pc = a * cs, ps = a * sn;                               // A exp(i angle), row q = 0
#pragma unroll
                        for (int q = 0; q < kGroupLaneRows; ++q) {
                            re[q] += pc;
                            im[q] += ps;
                            if (q + 1 < kGroupLaneRows) {                             // on to row q + 1
                                const float nc = fmaf(pc, r.x, -ps * r.y);
                                ps = fmaf(pc, r.y, ps * r.x);
                                pc = nc;
                            }
                        }
                    }
                    __syncwarp();
                }
                // times exp(i 2 pi (C l^2 + reference)): half_turn_sincos gives minus its cosine and sine
#pragma unroll
                for (int q = 0; q < kGroupLaneRows; ++q) {
                    float sn, cs;
                    half_turn_sincos(chi, clo, (uint32_t)(lane + 32 * q), 256u + radd[q], sn, cs);
                    const float wr = -cs, wi = -sn;
                    const float r2 = re[q] * wr - im[q] * wi, i2 = re[q] * wi + im[q] * wr;
                    re[q] = r2 * inv;
                    im[q] = i2 * inv;
                }
            } else {
#pragma unroll
                for (int q = 0; q < kGroupLaneRows; ++q) {
                    float sn, cs;
                    half_turn_sincos(chi, clo, (uint32_t)(r0 + lane + 32 * q - d.w), 256u + radd[q], sn, cs);
                    re[q] = -cs;   // cos alpha
                    im[q] = sn;    // -sin alpha
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kGroupLaneRows; ++q) {
            tile_hi[k * kTileStride + lane + 32 * q] = pack(re[q], im[q], MODE, false);
            if (MODE == kFactorSplit16) tile_lo[k * kTileStride + lane + 32 * q] = pack(re[q], im[q], MODE, true);
        }
    }
    __syncthreads();
    // write-out: 8 lanes x 16 bytes (4 slots) per row, four rows per warp
    const int rows = is_p ? height : width;
    uint16_t *base = is_p ? P : Q;
    const long long lo_off = is_p ? plane_p : plane_q;
    for (int item = threadIdx.x; item < kGroupRows * (kGroupTile / 4); item += kGroupThreads) {
        const int row = item / (kGroupTile / 4), c = item % (kGroupTile / 4);
        const int s = s_base + 4 * c;
        if (r0 + row >= rows || s >= slots) continue;
        uint16_t *dst = base + (long long)(r0 + row) * ld + 2 * s;
        const int t = 4 * c * kTileStride + row;
        *reinterpret_cast<uint4 *>(dst) = make_uint4(tile_hi[t], tile_hi[t + kTileStride], tile_hi[t + 2 * kTileStride],
                                                     tile_hi[t + 3 * kTileStride]);
        if (MODE == kFactorSplit16)
            *reinterpret_cast<uint4 *>(dst + lo_off) = make_uint4(
                tile_lo[t], tile_lo[t + kTileStride], tile_lo[t + 2 * kTileStride], tile_lo[t + 3 * kTileStride]);
    }
}

}  // namespace

cudaError_t launch_group_factors(int mode, const int4 *groups, int g_begin, int n_groups,
                                 const unsigned long long *planes, const int2 *members, int height, int width,
                                 void *P, void *Q, int64_t ld, const float *wscale, cudaStream_t s,
                                 const PhaseRef &ref)
{
    const int slots = (int)(ld / 2);
    dim3 grid((slots + kGroupTile - 1) / kGroupTile, (height + kGroupRows - 1) / kGroupRows + (width + kGroupRows - 1) / kGroupRows);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    const long long plane_p = (long long)height * ld, plane_q = (long long)width * ld;
    auto *p = static_cast<uint16_t *>(P);
    auto *q = static_cast<uint16_t *>(Q);
    switch (mode) {
    case kFactorF16:
        group_factors_kernel<kFactorF16><<<grid, kGroupThreads, 0, s>>>(groups, g_begin, n_groups, slots, planes,
                                                                        members, height, width, p, q, ld, plane_p,
                                                                        plane_q, wscale, ref);
        break;
    case kFactorBF16:
        group_factors_kernel<kFactorBF16><<<grid, kGroupThreads, 0, s>>>(groups, g_begin, n_groups, slots, planes,
                                                                         members, height, width, p, q, ld, plane_p,
                                                                         plane_q, wscale, ref);
        break;
    default:
        group_factors_kernel<kFactorSplit16><<<grid, kGroupThreads, 0, s>>>(groups, g_begin, n_groups, slots,
                                                                            planes, members, height, width, p, q, ld,
                                                                            plane_p, plane_q, wscale, ref);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_factors(int mode, const int4 *geo, const uint2 *aux, int n_points, int height, int width,
                           void *P, void *Q, int64_t ld, const float *amp_max, cudaStream_t s, bool imag_q_only,
                           const PhaseRef &ref)
{
    const int slots = (int)(ld / 2);
    const int threads_x = (slots + 3) / 4;
    const int row_begin = imag_q_only ? height : 0;
    const int rows = height + width - row_begin;
    dim3 grid((threads_x + kFactorThreads - 1) / kFactorThreads, (rows + kRowsPerBlock - 1) / kRowsPerBlock);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    const long long plane_p = (long long)height * ld, plane_q = (long long)width * ld;
    auto *p = static_cast<uint16_t *>(P);
    auto *q = static_cast<uint16_t *>(Q);
    const bool im = imag_q_only;
#define CGH_FACTORS(M, I)                                                                                       \
    factors_kernel<M, I><<<grid, kFactorThreads, 0, s>>>(geo, aux, n_points, slots, height, width, p, q, ld, plane_p, \
                                                         plane_q, amp_max, row_begin, ref)
    switch (mode) {
    case kFactorF16:
        if (im) CGH_FACTORS(kFactorF16, true);
        else CGH_FACTORS(kFactorF16, false);
        break;
    case kFactorBF16:
        if (im) CGH_FACTORS(kFactorBF16, true);
        else CGH_FACTORS(kFactorBF16, false);
        break;
    default:
        if (im) CGH_FACTORS(kFactorSplit16, true);
        else CGH_FACTORS(kFactorSplit16, false);
        break;
    }
#undef CGH_FACTORS
    return cudaGetLastError();
}

}  // namespace cgh
