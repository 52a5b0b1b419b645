// a1: point preparation (device code shared by prep.cu and persist.cu).  One
// thread per (padded) point computes the point's
// fixed-point phase constants and checks its data.
//
// The phase of Eq. 5 in turns is c_j r^2 with c_j = p^2 / (2 lambda z_j)
// (Section 2.2 names the same constant P_j = 1/(2 lambda z_j) in metres).
// Because r^2 is an integer, only frac(c_j) matters modulo one turn; it is
// stored as the 64-bit fixed-point C_j = round(frac(c_j) 2^64).  Every phase
// the kernels form is then C_j * (integer) mod 2^64, exact up to C_j's own
// rounding (<= 2^-65 turn per px^2, i.e. < 2^-33 turn for r^2 < 2^32).
// FP64 is used only here, O(N) work.  With the piston of Eq. 2 the point
// carries frac(z_j / lambda) (the phase 2 pi z_j / lambda in turns) in place of
// the second difference, which the kernels then form from C_j itself.
#pragma once

#include "device_util.cuh"
#include "kernels.h"

namespace cgh {
namespace dev {

// Prepares point j < n_pad (padding beyond n: zero amplitude, zero phase).
__device__ __forceinline__ void prep_point(int j, const float *__restrict__ xyz, const float *__restrict__ amp, int n,
                                           double pitch, double lambda, int4 *__restrict__ geo,
                                           uint2 *__restrict__ aux, int *status, float *amp_max, int aux_x,
                                           float4 *__restrict__ ext, int width, int height, int tile_cols,
                                           int tile_rows)
{
    if (ext != nullptr) ext[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (j >= n) {  // padding: zero amplitude, zero phase
        geo[j] = make_int4(0, 0, 0, 0);
        aux[j] = make_uint2(0u, 0u);
        return;
    }
    const float fx = xyz[3 * j + 0], fy = xyz[3 * j + 1], fz = xyz[3 * j + 2];
    const float a = amp[j];
    const bool ok = isfinite(fx) && isfinite(fy) && isfinite(fz) && isfinite(a) && fz > 0.0f &&
                    fx == rintf(fx) && fy == rintf(fy) && fabsf(fx) <= (float)kMaxCoord &&
                    fabsf(fy) <= (float)kMaxCoord;
    if (!ok) {
        atomicOr(status, kStatusInput);
        geo[j] = make_int4(0, 0, 0, 0);
        aux[j] = make_uint2(0u, 0u);
        return;
    }
    const double c = (pitch * pitch) / (2.0 * lambda * (double)fz);   // turns per px^2
    const double fr = c - floor(c);                                  // [0, 1), exact
    const double scaled = ldexp(fr, 64);                              // exact power-of-two scaling
    unsigned long long C = (scaled >= 18446744073709551616.0) ? 0ull : __double2ull_rn(scaled);
    geo[j] = make_int4((int)fx, (int)fy, (int)(unsigned)(C >> 32), (int)(unsigned)(C & 0xffffffffull));
    unsigned w = aux_x == kAuxSecondDiff ? (unsigned)((C << 1) >> 32) : 0u;   // 2 c_j, top 32 bits
    if (aux_x == kAuxPiston) {   // frac(z / lambda) in 2^-32 turn (within ~2^-32 turn while z / lambda < 2^21)
        const double zt = (double)fz / lambda;
        const double pf = ldexp(zt - floor(zt), 32);
        w = pf >= 4294967295.5 ? 0u : (unsigned)__double2ull_rn(pf);
    }
    aux[j] = make_uint2(w, __float_as_uint(a));
    if (ext != nullptr) {
        // {(p / z)^2, z / (2 lambda)} as float pairs {hi, hi, lo, lo}, the spherical kernel's two flags in the
        // signs of the high parts.  Tile centres lie up
        // to half a thread tile (hx, hy) beyond the farthest pixel, so cx, cy bound |centre - point| per axis;
        // the quadratic in w = u - U0 is used when its truncation error Z max|h'''| wmax^3 / 6 = zh wmax^3 / 8
        // and its range max|d1 w + d2 w^2| <= zh (umax / 2) wmax + (zh / 4) wmax^2 are within bounds.
        const double pz = pitch / (double)fz, qz = pz * pz, zh = (double)fz / (2.0 * lambda);
        const double hx = 0.5 * (tile_cols - 1), hy = 0.5 * (tile_rows - 1);
        const double cx = fmax(fabs((double)fx), fabs((double)(width - 1) - (double)fx)) + hx;
        const double cy = fmax(fabs((double)fy), fabs((double)(height - 1) - (double)fy)) + hy;
        const double umax = (cx * cx + cy * cy) * qz;
        const double wmax = (2.0 * hx * cx + hx * hx + 2.0 * hy * cy + hy * hy) * qz;
        const bool quad = zh * wmax * wmax * wmax / 8.0 <= kSphFitTurns &&
                          zh * (0.5 * umax) * wmax + 0.25 * zh * wmax * wmax <= kSphRangeTurns;
        const float q = (float)qz, h = (float)zh;   // and the pair's low parts, for the double-float d0
        ext[j] = make_float4(quad ? q : -q, umax < kSeriesU ? h : -h, (float)(qz - (double)q), (float)(zh - (double)h));
    }
    if (amp_max != nullptr) atomicMax(reinterpret_cast<unsigned *>(amp_max), __float_as_uint(fabsf(a)));
}

}  // namespace dev
}  // namespace cgh
