// f3: step 1 of the wavefront-recording method (Section 2.3): the complex
// amplitude of the point cloud recorded on a virtual plane at distance z_wrp
// from the hologram (same grid), each point summed only over its window.
//
// Window.  The light of point j (distance d_j = z_j - z_wrp > 0 behind the
// plane) that can reach the hologram within the grid's largest diffraction
// angle, sin(theta) = lambda / (2 p), crosses the plane within radius
// d_j tan(theta): in pixels w = d s / sqrt(1 - s^2) / p, s = lambda / (2 p), and
// the window holds the pixels with (m - x_j)^2 + (n - y_j)^2 <= floor(w^2).
// That integer is computed in double with every operation rounded on its own
// (no contraction), so it is the same number on any IEEE machine.
//
// Phase (Eq. 2, at distance d_j): c_j r^2 turns, c_j = p^2 / (2 lambda d_j), in
// 64-bit fixed point as in the point preparation, plus the piston d_j / lambda
// with CGH_PHASE_FRESNEL_PISTON; sine and cosine from the hardware on the
// symmetric argument grid of the direct kernel.
//
// Gather, deterministic: one CTA per 32 x 32 pixel tile walks the points in
// index order, 256 at a time; the threads test the 256 window bounding boxes
// against the tile in parallel, compact the hits (warp ballots, order kept)
// and then every thread adds the hits to its four pixels.  No atomics, so the
// sums are bit-reproducible.  The points a tile walks are those of its band of
// 32 rows: for every band one CTA lists, in index order, the points whose
// window reaches the band (count, scan, fill; the same ballot compaction), so
// a tile skips the points of the other bands and the sums are unchanged.
#include "device_util.cuh"
#include "kernels.h"

namespace cgh {

namespace {

constexpr int kTile = 32;              // pixels per tile side
constexpr int kRecThreads = 256;       // 32 columns x 8 row groups of 4 rows
constexpr float kWK1 = 6.28318595886230469f;   // 2 pi rounded so that 1.5 K1 is a float
constexpr float kWK0 = 9.42477893829345703f;

__global__ void wrp_prep_kernel(const float *__restrict__ xyz, const float *__restrict__ amp, int n, int n_pad,
                                double pitch, double lambda, double z_wrp, bool piston, int4 *__restrict__ geo,
                                uint4 *__restrict__ win, int *status)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pad) return;
    if (j >= n) {
        geo[j] = make_int4(0, 0, 0, 0);
        win[j] = make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    const float fx = xyz[3 * j + 0], fy = xyz[3 * j + 1], fz = xyz[3 * j + 2];
    const float a = amp[j];
    const double d = __dadd_rn((double)fz, -z_wrp);
    const bool ok = isfinite(fx) && isfinite(fy) && isfinite(fz) && isfinite(a) && d > 0.0 && fx == rintf(fx) &&
                    fy == rintf(fy) && fabsf(fx) <= (float)kMaxCoord && fabsf(fy) <= (float)kMaxCoord;
    if (!ok) {
        atomicOr(status, kStatusInput);
        geo[j] = make_int4(0, 0, 0, 0);
        win[j] = make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    const double c = (pitch * pitch) / (2.0 * lambda * d);
    const double fr = c - floor(c);
    const double scaled = ldexp(fr, 64);
    const unsigned long long C = (scaled >= 18446744073709551616.0) ? 0ull : __double2ull_rn(scaled);
    geo[j] = make_int4((int)fx, (int)fy, (int)(unsigned)(C >> 32), (int)(unsigned)(C & 0xffffffffull));
    unsigned pist = 0u;
    if (piston) {
        const double zt = d / lambda;
        const double pf = ldexp(zt - floor(zt), 32);
        pist = pf >= 4294967295.5 ? 0u : (unsigned)__double2ull_rn(pf);
    }
    // squared window radius, each double operation rounded on its own
    const double s = __ddiv_rn(lambda, __dmul_rn(2.0, pitch));
    const double den = __dsqrt_rn(__dadd_rn(1.0, -__dmul_rn(s, s)));
    const double w = __ddiv_rn(__ddiv_rn(__dmul_rn(d, s), den), pitch);
    const double w2 = floor(__dmul_rn(w, w));
    const unsigned W2 = w2 >= 2147483647.0 ? 2147483647u : (unsigned)w2;
    unsigned R = (unsigned)sqrt((double)W2);   // integer radius: R^2 <= W2 < (R + 1)^2
    while ((unsigned long long)(R + 1) * (R + 1) <= W2) ++R;
    while ((unsigned long long)R * R > W2) --R;
    win[j] = make_uint4(pist, __float_as_uint(a), W2, R);
}

// Ballot compaction of one chunk: the position of this thread's hit among the
// chunk's hits (warp order, then lane order: index order kept) and their total.
__device__ __forceinline__ int compact_hits(bool hit, int *s_wcnt, int &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) s_wcnt[warp] = __popc(mask);
    __syncthreads();
    int before = 0;
    total = 0;
#pragma unroll
    for (int k = 0; k < kRecThreads / 32; ++k) {
        before += k < warp ? s_wcnt[k] : 0;
        total += s_wcnt[k];
    }
    return before + __popc(mask & ((1u << lane) - 1u));
}

__device__ __forceinline__ bool reaches_rows(const int4 q, const uint4 w, int y0)
{
    const int R = (int)w.w;
    return q.y + R >= y0 && q.y - R <= y0 + kTile - 1;
}

constexpr int kSegChunks = 16;   // chunks of kRecThreads points per segment of the band lists

// One CTA per (band of kTile rows, segment of kSegChunks x kRecThreads points):
// count (list == nullptr) or list, in index order, the segment's points whose
// window reaches the band.  A band's list is its segments' lists in order.
__global__ void __launch_bounds__(kRecThreads)
    wrp_band_kernel(const int4 *__restrict__ geo, const uint4 *__restrict__ win, int n_pad, int *count,
                    const int *__restrict__ offset, int *__restrict__ list)
{
    __shared__ int s_wcnt[kRecThreads / 32];
    const int y0 = blockIdx.x * kTile;
    const int cell = blockIdx.x * gridDim.y + blockIdx.y;   // band-major, then segment
    const int begin = blockIdx.y * kSegChunks * kRecThreads;
    const int end = min(n_pad, begin + kSegChunks * kRecThreads);
    int written = 0;
    for (int base = begin; base < end; base += kRecThreads) {
        const int j = base + threadIdx.x;
        const bool hit = reaches_rows(geo[j], win[j], y0);
        __syncthreads();   // s_wcnt of the previous chunk is read
        int total;
        const int pos = compact_hits(hit, s_wcnt, total);
        if (list != nullptr && hit) list[offset[cell] + written + pos] = j;
        written += total;
    }
    if (list == nullptr && threadIdx.x == 0) count[cell] = written;
}

// Exclusive scan of the (band, segment) counts in that order (one thread).
__global__ void wrp_band_scan(const int *count, int cells, int *offset)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int run = 0;
    for (int b = 0; b < cells; ++b) {
        offset[b] = run;
        run += count[b];
    }
    offset[cells] = run;
}

__global__ void __launch_bounds__(kRecThreads)
    wrp_record_kernel(const int4 *__restrict__ geo, const uint4 *__restrict__ win, int n_pad, int H, int W,
                      int tiles_x, int segs, const int *__restrict__ offset, const int *__restrict__ list,
                      float2 *__restrict__ pad, long long pad_ld, float *__restrict__ planes)
{
    __shared__ int4 s_geo[kRecThreads];
    __shared__ uint4 s_win[kRecThreads];
    __shared__ unsigned char s_hit[kRecThreads];
    __shared__ int s_wcnt[kRecThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int band = blockIdx.x / tiles_x;
    const int x0 = (blockIdx.x % tiles_x) * kTile, y0 = band * kTile;
    const int m = x0 + lane;
    const int nb = y0 + warp * 4;
    // the points to walk: the band's list, or all points
    const int first = list != nullptr ? offset[band * segs] : 0;
    const int count = list != nullptr ? offset[(band + 1) * segs] - first : n_pad;
    float re[4] = {0.0f, 0.0f, 0.0f, 0.0f}, im[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int base = 0; base < count; base += kRecThreads) {
        __syncthreads();   // the previous chunk is consumed
        const int k = base + tid;
        int4 q = make_int4(0, 0, 0, 0);
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        bool hit = false;
        if (k < count) {
            const int j = list != nullptr ? list[first + k] : k;
            q = geo[j];
            w = win[j];
            const int R = (int)w.w;
            hit = q.x + R >= x0 && q.x - R <= x0 + kTile - 1 && reaches_rows(q, w, y0);
        }
        s_geo[tid] = q;
        s_win[tid] = w;
        int total;
        const int pos = compact_hits(hit, s_wcnt, total);
        if (hit) s_hit[pos] = (unsigned char)tid;
        __syncthreads();
        for (int h = 0; h < total; ++h) {
            const int p = s_hit[h];
            const int4 g = s_geo[p];
            const uint4 v = s_win[p];
            if (g.y + (int)v.w < nb || g.y - (int)v.w > nb + 3) continue;   // the window misses this warp's rows
            const float a = -__uint_as_float(v.y);   // the half-turn shift below negates sine and cosine
            const int dx = m - g.x;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int dy = nb + i - g.y;
                const uint32_t r2 = (uint32_t)(dx * dx) + (uint32_t)(dy * dy);
                if (r2 > v.z) continue;
                const uint32_t t = (uint32_t)g.z * r2 + __umulhi((uint32_t)g.w, r2) + v.x + 256u;
                const float f = __uint_as_float((t >> 9) | 0x3f800000u);
                float sn, cs;
                __sincosf(fmaf(f, kWK1, -kWK0), &sn, &cs);   // angle - pi
                re[i] = fmaf(a, cs, re[i]);
                im[i] = fmaf(a, sn, im[i]);
            }
        }
    }
    if (m >= W) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int n = nb + i;
        if (n >= H) continue;
        if (pad != nullptr) {
            pad[(long long)n * pad_ld + m] = make_float2(re[i], im[i]);
        } else {
            planes[(long long)n * W + m] = re[i];
            planes[(long long)H * W + (long long)n * W + m] = im[i];
        }
    }
}

}  // namespace

cudaError_t launch_wrp_prep(const float *d_xyz, const float *d_amp, int n, int n_pad, double pitch, double lambda,
                            double z_wrp, bool piston, int4 *geo, uint4 *win, int *status, cudaStream_t s)
{
    if (n_pad <= 0) return cudaSuccess;
    wrp_prep_kernel<<<(n_pad + 255) / 256, 256, 0, s>>>(d_xyz, d_amp, n, n_pad, pitch, lambda, z_wrp, piston, geo, win,
                                                      status);
    return cudaGetLastError();
}

int wrp_band_cells(int H, int n_pad)
{
    const int segs = (n_pad + kSegChunks * kRecThreads - 1) / (kSegChunks * kRecThreads);
    return ((H + kTile - 1) / kTile) * (segs > 0 ? segs : 1);
}

static int wrp_segs(int n_pad)
{
    const int segs = (n_pad + kSegChunks * kRecThreads - 1) / (kSegChunks * kRecThreads);
    return segs > 0 ? segs : 1;
}

cudaError_t launch_wrp_bands(const int4 *geo, const uint4 *win, int n_pad, int H, int *count, int *offset, int *list,
                             cudaStream_t s)
{
    const dim3 grid((H + kTile - 1) / kTile, wrp_segs(n_pad));
    wrp_band_kernel<<<grid, kRecThreads, 0, s>>>(geo, win, n_pad, count, nullptr, nullptr);
    wrp_band_scan<<<1, 32, 0, s>>>(count, (int)(grid.x * grid.y), offset);
    wrp_band_kernel<<<grid, kRecThreads, 0, s>>>(geo, win, n_pad, count, offset, list);
    return cudaGetLastError();
}

cudaError_t launch_wrp_record(const int4 *geo, const uint4 *win, int n_pad, int H, int W, const int *offset,
                              const int *list, float2 *pad, int64_t pad_ld, float *planes, cudaStream_t s)
{
    const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
    wrp_record_kernel<<<tiles_x * tiles_y, kRecThreads, 0, s>>>(geo, win, n_pad, H, W, tiles_x, wrp_segs(n_pad),
                                                               offset, list, pad, (long long)pad_ld, planes);
    return cudaGetLastError();
}

}  // namespace cgh
