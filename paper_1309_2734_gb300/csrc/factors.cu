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
// Each angle is reduced exactly in integers: with the point's 64-bit
// fixed-point constant C_j (prep.cu), the turn is the top 32 bits of
// C_j d^2 mod 2^64, d the integer distance along one axis (|d| < 2^15, so
// d^2 < 2^30).  The signed 32-bit turn converts to t in [-1/2, 1/2) (error
// <= 2^-26 turn), and the hardware sine and cosine (MUFU, |2 pi t| <= pi,
// absolute error below 4e-7) give the pair, which is rounded to FP16 or BF16,
// or split into hi = fp16(v) and lo = fp16(v - hi).  That error is far below
// FP16/BF16 rounding and, in the split form, contributes ~1e-7 to the NRMS
// (the accumulation dominates).  The kernel is issue-bound; the MUFU leaves
// the issue slots to the integer phase work.  No FP64 is needed on the GPU.
//
// For the imaginary part of the complex wave, sin(alpha + beta) =
// sin(alpha) cos(beta) + cos(alpha) sin(beta), so Im O = P Q'^T with the same P
// and Q'[m][2j] = s A_j sin alpha, Q'[m][2j+1] = s A_j cos alpha ("imag" launch,
// Q' rows only).
//
// One thread owns 4 consecutive points (8 columns, one 16-byte store per row
// and plane) and walks a band of rows, so the point constants are read once
// per band; rows [0, height) are P's, rows [height, height + width) are Q's.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace cgh {

namespace {

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

template <int MODE>
__global__ void __launch_bounds__(kFactorThreads)
    factors_kernel(const int4 *__restrict__ geo, const uint2 *__restrict__ aux, int n_points, int slots,
                   int height, int width, uint16_t *__restrict__ P, uint16_t *__restrict__ Q, long long ld,
                   long long plane_p, long long plane_q, const float *__restrict__ amp_max, int row_begin,
                   bool imag)
{
    const int j0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (j0 >= slots) return;
    float scale = 1.0f;
    if (amp_max != nullptr) {
        const float m = *amp_max;
        if (m > 0.0f) scale = 1.0f / m;
    }
    int px[4], py[4];
    uint32_t chi[4], clo[4];
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
            a[q] = __uint_as_float(aux[j].y) * scale;
        } else {
            px[q] = py[q] = 0;
            chi[q] = clo[q] = 0u;
            a[q] = 0.0f;
        }
    }
    const int rows = height + width;
    const int r_end = min(rows, row_begin + (int)(blockIdx.y + 1) * kRowsPerBlock);
    for (int r = row_begin + blockIdx.y * kRowsPerBlock; r < r_end; ++r) {
        const bool is_p = r < height;
        const int line = is_p ? r : r - height;
        float v[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float c = 0.0f, s = 0.0f;
            if (live[q]) {
                const uint32_t d = (uint32_t)(line - (is_p ? py[q] : px[q]));
                const uint32_t d2 = d * d;                                   // < 2^30
                const uint32_t g = chi[q] * d2 + __umulhi(clo[q], d2);       // turn, 2^-32 units
                const float t = (float)(int)g * 2.3283064365386963e-10f;     // [-1/2, 1/2)
                sincos_turn(t, s, c);
                if (!is_p) {
                    const float cc = c;
                    c = imag ? a[q] * s : a[q] * c;
                    s = imag ? a[q] * cc : -a[q] * s;
                }
            }
            v[2 * q] = c;
            v[2 * q + 1] = s;
        }
        uint16_t *dst = (is_p ? P + (long long)line * ld : Q + (long long)line * ld) + 2 * j0;
        const uint4 hi = make_uint4(pack(v[0], v[1], MODE, false), pack(v[2], v[3], MODE, false),
                                    pack(v[4], v[5], MODE, false), pack(v[6], v[7], MODE, false));
        *reinterpret_cast<uint4 *>(dst) = hi;
        if (MODE == kFactorSplit16) {
            const uint4 lo = make_uint4(pack(v[0], v[1], MODE, true), pack(v[2], v[3], MODE, true),
                                        pack(v[4], v[5], MODE, true), pack(v[6], v[7], MODE, true));
            *reinterpret_cast<uint4 *>(dst + (is_p ? plane_p : plane_q)) = lo;
        }
    }
}

}  // namespace

cudaError_t launch_factors(int mode, const int4 *geo, const uint2 *aux, int n_points, int height, int width,
                           void *P, void *Q, int64_t ld, const float *amp_max, cudaStream_t s, bool imag_q_only)
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
    switch (mode) {
    case kFactorF16:
        factors_kernel<kFactorF16><<<grid, kFactorThreads, 0, s>>>(geo, aux, n_points, slots, height, width, p, q, ld,
                                                                   plane_p, plane_q, amp_max, row_begin, imag_q_only);
        break;
    case kFactorBF16:
        factors_kernel<kFactorBF16><<<grid, kFactorThreads, 0, s>>>(geo, aux, n_points, slots, height, width, p, q,
                                                                    ld, plane_p, plane_q, amp_max, row_begin,
                                                                    imag_q_only);
        break;
    default:
        factors_kernel<kFactorSplit16><<<grid, kFactorThreads, 0, s>>>(geo, aux, n_points, slots, height, width, p,
                                                                       q, ld, plane_p, plane_q, amp_max, row_begin,
                                                                       imag_q_only);
        break;
    }
    return cudaGetLastError();
}

}  // namespace cgh
