// a2: the direct kernels (device code of the term and of a unit of work in
// direct_dev.cuh): one hologram in the chunked layout (pixel tile x point
// chunk, partial planes), in the balanced layout (equal shares of the (pixel
// tile, point) pairs, a tile's parts summed by the last CTA to finish it), the
// complex object wave, and the per-form batch kernels.
#include <type_traits>

#include "direct_dev.cuh"
#include "host_util.h"
#include "kernels.h"

namespace cgh {

namespace {

using namespace dev;

// One hologram: blockIdx.x = pixel tile, blockIdx.y = point chunk (its own output plane).
template <int TL, int TR, int BX, int BY, bool SFU, bool EXTRA>
__global__ void __launch_bounds__(BX *BY, 2)
    direct_kernel(const int4 *__restrict__ geo, const uint2 *__restrict__ aux, int n_ptiles, int width,
                  int height, int tiles_x, int split, float *__restrict__ out, long long slice_stride,
                  bool vec, int *status, unsigned long long timeout_ns, int drop_tile, const PhaseRef ref)
{
    __shared__ alignas(128) int4 s_geo[2][kPointTile];
    __shared__ alignas(128) uint2 s_aux[2][kPointTile];
    __shared__ alignas(8) uint64_t s_bar[2];
    init_point_barriers<BX, BY>(s_bar);
    const int tile = blockIdx.x;
    const int t_begin = (int)((long long)blockIdx.y * n_ptiles / split);
    const int t_end = (int)((long long)(blockIdx.y + 1) * n_ptiles / split);
    uint32_t kg = 0;
    direct_unit<TL, TR, BX, BY, SFU, 1, EXTRA>(geo, aux, t_begin, t_end, (tile % tiles_x) * (BX * TL),
                                     (tile / tiles_x) * (BY * TR), width, height,
                                     out + (long long)blockIdx.y * slice_stride, vec, s_geo, s_aux, s_bar, kg,
                                     status, timeout_ns, blockIdx.y == 0 ? drop_tile : -1, 0, ref);
}

// One hologram over a flat work space: unit u = t N + j is (pixel tile t, point j), t < n_tiles, j < N, and
// CTA c of C takes units [c U / C, (c + 1) U / C) (U = n_tiles N), so every CTA has the same number of terms to
// within one point, whatever the tile count, and no padded point is evaluated.  A CTA walks its units tile by
// tile (segments); a segment that covers all N points of its tile stores the tile, any other stores its
// partial totals in the CTA's slot (0: its first segment, 1: its last) and counts itself on the tile's counter.
// The CTA that arrives last sums the tile's segments in the order of their CTAs (so the result does not depend
// on who arrives last) and writes the tile: no partial planes and no separate reduction pass.  counters (one
// per tile) are zero at launch; slots hold 2 C tiles of totals, thread-major float4s.
// What a CTA of the balanced layout knows about its current segment, kept in shared memory so that none of it
// occupies registers while the point loop runs.
struct StreamSeg {
    long long t;      // pixel tile
    int p0, p1;       // points [p0, p1) of it
    int last;         // this CTA finished the tile's last part
};

// The end of a segment: a whole tile is stored; a part goes to the CTA's slot and is counted on the tile, and the
// CTA that counts last sums the tile's parts in CTA order (so the result does not depend on who is last).
template <int TL, int TR, int BX, int BY>
struct StreamSink {
    StreamSeg *seg;
    float4 *slots;
    int *counters;
    float *out;
    long long units, C, N;
    int tiles_x, width, height;
    bool vec;
    int *status;

    __device__ long long owner(long long u) const { return ((u + 1) * C - 1) / units; }
    // slot of CTA cs's part of tile t: 0 when it is the CTA's first segment, else 1 (its last)
    __device__ int slot_of(long long cs, long long t) const { return (cs * units / C) / N == t ? 0 : 1; }

    __device__ void operator()(float (&tot)[TR][TL]) const
    {
        constexpr int NT = BX * BY;
        constexpr int Q4 = TL * TR / 4;   // float4s of totals per thread
        const int tid = threadIdx.x;
        const long long c = blockIdx.x;
        const long long t = seg->t;
        // the tile and the CTA's slot exist (CTA-uniform, so every thread skips alike)
        if (!CGH_DCHECK(t >= 0 && t < units / N && c < C, status)) return;
        if (!(seg->p0 == 0 && seg->p1 == N)) {
            float4 *mine = slots + (2 * c + slot_of(c, t)) * (long long)(Q4 * NT) + tid;
#pragma unroll
            for (int q = 0; q < Q4; ++q) {
                const int r = q * 4 / TL, i = q * 4 % TL;
                mine[q * NT] = make_float4(tot[r][i], tot[r][i + 1], tot[r][i + 2], tot[r][i + 3]);
            }
            __threadfence();
            __syncthreads();
            const long long lo = owner(t * N), hi = owner(t * N + N - 1);
            if (tid == 0) seg->last = atomicAdd(&counters[t], 1) == (int)(hi - lo);
            __syncthreads();
            if (!seg->last) return;
            __threadfence();
            // the tile's parts in CTA order, G float4s of every thread's block at a time: the G loads of one part
            // are independent, so a part costs one memory round trip per group rather than one per float4
            constexpr int G = 4;
            static_assert(Q4 % G == 0, "whole groups of float4s");
#pragma unroll
            for (int q0 = 0; q0 < Q4; q0 += G) {
                float4 a[G];
                for (long long cs = lo; cs <= hi; ++cs) {
                    float4 v[G];
                    if (cs == c) {
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            const int r = (q0 + g) * 4 / TL, i = (q0 + g) * 4 % TL;
                            v[g] = make_float4(tot[r][i], tot[r][i + 1], tot[r][i + 2], tot[r][i + 3]);
                        }
                    } else {
                        const float4 *part = slots + (2 * cs + slot_of(cs, t)) * (long long)(Q4 * NT) + tid;
#pragma unroll
                        for (int g = 0; g < G; ++g) v[g] = __ldcg(part + (q0 + g) * NT);
                    }
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        if (cs == lo) {
                            a[g] = v[g];
                        } else {
                            a[g].x += v[g].x;
                            a[g].y += v[g].y;
                            a[g].z += v[g].z;
                            a[g].w += v[g].w;
                        }
                    }
                }
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int r = (q0 + g) * 4 / TL, i = (q0 + g) * 4 % TL;
                    tot[r][i] = a[g].x;
                    tot[r][i + 1] = a[g].y;
                    tot[r][i + 2] = a[g].z;
                    tot[r][i + 3] = a[g].w;
                }
            }
        }
        const int m0 = (int)(t % tiles_x) * (BX * TL) + (tid % BX) * TL;
        const int n0 = (int)(t / tiles_x) * (BY * TR) + (tid / BX) * TR;
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const int n = n0 + r;
            if (n >= height || m0 >= width) continue;
            float *row = out + (long long)n * width + m0;
            if (vec && m0 + TL <= width) {
#pragma unroll
                for (int i = 0; i < TL; i += 4)
                    *reinterpret_cast<float4 *>(row + i) =
                        make_float4(tot[r][i], tot[r][i + 1], tot[r][i + 2], tot[r][i + 3]);
            } else {
#pragma unroll
                for (int i = 0; i < TL; ++i)
                    if (m0 + i < width) row[i] = tot[r][i];
            }
        }
    }
};

// One hologram over a flat work space: unit u = t N + j is (pixel tile t, point j), t < n_tiles, j < N, and
// CTA c of C takes units [c U / C, (c + 1) U / C) (U = n_tiles N), so every CTA has the same number of terms to
// within one point, whatever the tile count, and no padded point is evaluated.  A CTA walks its units tile by
// tile (segments); a segment that covers all N points of its tile stores the tile, any other stores its
// partial totals in the CTA's slot (0: its first segment, 1: its last) and counts itself on the tile's counter;
// the CTA that arrives last sums the tile's parts (StreamSink): no partial planes and no separate reduction
// pass.  counters (one per tile) are zero at launch; slots hold 2 C tiles of totals, thread-major float4s.
// SMEM_TOT: the running totals in shared memory (TR TL floats per thread, dynamic), which leaves the registers to a
// wider thread block's partial sums.
template <int TL, int TR, int BX, int BY, bool SFU, bool EXTRA, bool SMEM_TOT, bool TABLES>
__global__ void __launch_bounds__(BX *BY, 512 / (BX * BY))
    direct_stream_kernel(const int4 *__restrict__ geo, const uint2 *__restrict__ aux, int n_points, int width,
                         int height, int tiles_x, long long units, float *__restrict__ out,
                         float4 *__restrict__ slots, int *__restrict__ counters, bool vec, int *status,
                         unsigned long long timeout_ns, int drop_tile, const PhaseRef ref)
{
    constexpr int T = kPointTile;
    static_assert(TL % 4 == 0, "rows of float4s");
    __shared__ alignas(128) int4 s_geo[2][kPointTile];
    __shared__ alignas(128) uint2 s_aux[2][kPointTile];
    __shared__ alignas(8) uint64_t s_bar[2];
    __shared__ StreamSeg s_seg;
    extern __shared__ __align__(16) float s_dyn[];   // the running totals (SMEM_TOT), then the tables (TABLES)
    float *s_tot = s_dyn;
    float2 *s_tab = reinterpret_cast<float2 *>(s_dyn + (SMEM_TOT ? TL * TR * BX * BY : 0));
    init_point_barriers<BX, BY>(s_bar);
    const StreamSink<TL, TR, BX, BY> sink{&s_seg, slots, counters, out, units, (long long)gridDim.x,
                                          (long long)n_points, tiles_x, width, height, vec, status};
    uint32_t kg = 0;
    const long long w0 = (long long)blockIdx.x * units / gridDim.x;
    for (long long w = w0;;) {
        const long long w1 = ((long long)blockIdx.x + 1) * units / gridDim.x;
        if (w >= w1) break;
        const long long t = w / n_points;
        const int p0 = (int)(w - t * n_points);
        const int p1 = (int)min((long long)n_points, (long long)p0 + (w1 - w));
        if (threadIdx.x == 0) {
            s_seg.t = t;
            s_seg.p0 = p0;
            s_seg.p1 = p1;
        }
        __syncthreads();
        const int k0 = p0 / T, k1 = (p1 + T - 1) / T;
        const int drop = (blockIdx.x == 0 && w == w0) ? drop_tile : -1;
        if (!direct_unit<TL, TR, BX, BY, SFU, 1, EXTRA, SMEM_TOT, StreamSink<TL, TR, BX, BY>, CtaSync, T, TABLES>(
                geo, aux, k0, k1, (int)(t % tiles_x) * (BX * TL), (int)(t / tiles_x) * (BY * TR), width, height,
                out, vec, s_geo, s_aux, s_bar, kg, status, timeout_ns, drop, 0, ref, s_tot, p0 - k0 * T,
                p1 - (k1 - 1) * T, sink, s_tab))
            break;
        w = s_seg.t * n_points + s_seg.p1;
        __syncthreads();   // s_seg and the point stages are reused by the next segment
    }
}

// The complex object wave of one hologram: blockIdx.x = pixel tile, blockIdx.y =
// point chunk; chunk s writes real and imaginary planes at out + s * slice_stride
// and out + s * slice_stride + im_offset.  TABLES: the sines and cosines of a point's columns and rows taken once
// per CTA into shared-memory tables (dev::SepTable), after the totals.
template <int TL, int TR, int BX, int BY, bool EXTRA, bool TABLES>
__global__ void __launch_bounds__(BX *BY, 2)
    direct_wave_kernel(const int4 *__restrict__ geo, const uint2 *__restrict__ aux, int n_ptiles, int width,
                       int height, int tiles_x, int split, float *__restrict__ out, long long slice_stride,
                       long long im_offset, bool vec, int *status, unsigned long long timeout_ns,
                       const PhaseRef ref)
{
    __shared__ alignas(128) int4 s_geo[2][kPointTile];
    __shared__ alignas(128) uint2 s_aux[2][kPointTile];
    __shared__ alignas(8) uint64_t s_bar[2];
    extern __shared__ __align__(16) float s_tot[];   // the running totals: 2 TR TL floats per thread; the tables
    float2 *s_tab = reinterpret_cast<float2 *>(s_tot + 2 * TR * TL * BX * BY);
    init_point_barriers<BX, BY>(s_bar);
    const int tile = blockIdx.x;
    const int t_begin = (int)((long long)blockIdx.y * n_ptiles / split);
    const int t_end = (int)((long long)(blockIdx.y + 1) * n_ptiles / split);
    uint32_t kg = 0;
    direct_unit<TL, TR, BX, BY, true, 2, EXTRA, true, PlainStore, CtaSync, kPointTile, TABLES>(
        geo, aux, t_begin, t_end, (tile % tiles_x) * (BX * TL), (tile / tiles_x) * (BY * TR), width, height,
        out + (long long)blockIdx.y * slice_stride, vec, s_geo, s_aux, s_bar, kg, status, timeout_ns, -1, im_offset,
        ref, s_tot, 0, kPointTile, PlainStore(), s_tab);
}

// A batch: every CTA walks its list of {job, pixel tile} units over all points of the job.
template <int TL, int TR, int BX, int BY, bool SFU>
__global__ void __launch_bounds__(BX *BY, 2)
    direct_batch_kernel(const DirectJob *__restrict__ jobs, const int *__restrict__ cta_off,
                        const int2 *__restrict__ units, int *status, unsigned long long timeout_ns)
{
    __shared__ alignas(128) int4 s_geo[2][kPointTile];
    __shared__ alignas(128) uint2 s_aux[2][kPointTile];
    __shared__ alignas(8) uint64_t s_bar[2];
    init_point_barriers<BX, BY>(s_bar);
    uint32_t kg = 0;
    for (int i = cta_off[blockIdx.x]; i < cta_off[blockIdx.x + 1]; ++i) {
        const int2 w = units[i];
        const DirectJob &J = jobs[w.x];
        if (!direct_unit<TL, TR, BX, BY, SFU>(J.geo, J.aux, 0, J.n_ptiles, (w.y % J.tiles_x) * (BX * TL),
                                              (w.y / J.tiles_x) * (BY * TR), J.width, J.height, J.out,
                                              J.vec != 0, s_geo, s_aux, s_bar, kg, status, timeout_ns))
            break;
    }
}

constexpr int kTL = 8, kTR = 4, kBX = 32, kBY = 8;   // the wide shape: 256 x 32 pixels per CTA
constexpr int kTallBX = 16, kTallBY = 16;             // the tall shape: 128 x 64 pixels per CTA

template <int BX, int BY, bool SFU, bool EXTRA>
void direct_as(dim3 grid, cudaStream_t s, const int4 *geo, const uint2 *aux, int n_ptiles, int width, int height,
               int tiles_x, int split, float *out, long long ss, bool vec, int *status, uint64_t timeout_ns,
               int drop_tile, const PhaseRef &ref)
{
    direct_kernel<kTL, kTR, BX, BY, SFU, EXTRA><<<grid, BX * BY, 0, s>>>(
        geo, aux, n_ptiles, width, height, tiles_x, split, out, ss, vec, status, timeout_ns, drop_tile, ref);
}

template <int BX, int BY>
void direct_shaped(bool sfu, bool extra, dim3 grid, cudaStream_t s, const int4 *geo, const uint2 *aux, int n_ptiles,
                   int width, int height, int tiles_x, int split, float *out, long long ss, bool vec, int *status,
                   uint64_t timeout_ns, int drop_tile, const PhaseRef &ref)
{
    if (sfu && !extra)
        direct_as<BX, BY, true, false>(grid, s, geo, aux, n_ptiles, width, height, tiles_x, split, out, ss, vec,
                                       status, timeout_ns, drop_tile, ref);
    else if (sfu)
        direct_as<BX, BY, true, true>(grid, s, geo, aux, n_ptiles, width, height, tiles_x, split, out, ss, vec,
                                      status, timeout_ns, drop_tile, ref);
    else if (!extra)
        direct_as<BX, BY, false, false>(grid, s, geo, aux, n_ptiles, width, height, tiles_x, split, out, ss, vec,
                                        status, timeout_ns, drop_tile, ref);
    else
        direct_as<BX, BY, false, true>(grid, s, geo, aux, n_ptiles, width, height, tiles_x, split, out, ss, vec,
                                       status, timeout_ns, drop_tile, ref);
}

}  // namespace

DirectShape direct_shape(bool tall)
{
    return tall ? DirectShape{kTallBX * kTL, kTallBY * kTR, kTallBX * kTallBY, kTallBX}
                : DirectShape{kBX * kTL, kBY * kTR, kBX * kBY, kBX};
}

cudaError_t launch_direct(bool sfu, const DirectShape &sh, const int4 *geo, const uint2 *aux, int n_pad, int width,
                          int height, int split, float *out, int64_t slice_stride, int *status, uint64_t timeout_ns,
                          cudaStream_t s, int drop_tile, const PhaseRef &ref)
{
    const int tiles_x = (width + sh.tile_w - 1) / sh.tile_w;
    const int tiles_y = (height + sh.tile_h - 1) / sh.tile_h;
    const int n_ptiles = n_pad / kPointTile;
    if (split < 1) split = 1;
    dim3 grid(tiles_x * tiles_y, split);
    // 16-byte stores only when every row start of every slice is 16-byte aligned
    const bool vec = (width % 4 == 0) && (slice_stride % 4 == 0) && ((uintptr_t)out % 16 == 0);
    const long long ss = (long long)slice_stride;
    const bool extra = ref.any();
    if (sh.bx == kTallBX)
        direct_shaped<kTallBX, kTallBY>(sfu, extra, grid, s, geo, aux, n_ptiles, width, height, tiles_x, split, out,
                                        ss, vec, status, timeout_ns, drop_tile, ref);
    else
        direct_shaped<kBX, kBY>(sfu, extra, grid, s, geo, aux, n_ptiles, width, height, tiles_x, split, out, ss,
                                vec, status, timeout_ns, drop_tile, ref);
    return cudaGetLastError();
}

namespace {

// The balanced layout's thread blocks: TL x TR pixels per thread, BX x BY threads, totals in registers or shared
// memory.
template <int TL, int TR, int BX, int BY, bool SMEM_TOT, bool TABLES = false>
struct StreamCfg {
    static constexpr size_t kTotBytes = SMEM_TOT ? (size_t)TL * TR * BX * BY * sizeof(float) : 0;
    static constexpr size_t kDyn =
        kTotBytes + (TABLES ? (size_t)2 * kSepGroup * SepTable<BX * TL, BY * TR>::kPerPoint * sizeof(float2) : 0);

    template <bool SFU, bool EXTRA>
    static cudaError_t launch(int ctas, cudaStream_t s, const int4 *geo, const uint2 *aux, int n_points, int width,
                              int height, int tiles_x, long long units, float *out, float4 *slots, int *counters,
                              bool vec, int *status, uint64_t timeout_ns, int drop_tile, const PhaseRef &ref)
    {
        if constexpr (kDyn > 0) {   // with the static tiles the totals or tables exceed the default 48 KB
            static PerDeviceOnce configured;
            const cudaError_t e = configured.run([] {
                return cudaFuncSetAttribute(direct_stream_kernel<TL, TR, BX, BY, SFU, EXTRA, SMEM_TOT, TABLES>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDyn);
            });
            if (e != cudaSuccess) return e;
        }
        direct_stream_kernel<TL, TR, BX, BY, SFU, EXTRA, SMEM_TOT, TABLES><<<ctas, BX * BY, kDyn, s>>>(
            geo, aux, n_points, width, height, tiles_x, units, out, slots, counters, vec, status, timeout_ns,
            drop_tile, ref);
        return cudaGetLastError();
    }

    static cudaError_t dispatch(bool sfu, bool extra, int ctas, cudaStream_t s, const int4 *geo, const uint2 *aux,
                                int n_points, int width, int height, int tiles_x, long long units, float *out,
                                float4 *slots, int *counters, bool vec, int *status, uint64_t timeout_ns,
                                int drop_tile, const PhaseRef &ref)
    {
#define CGH_STREAM_ARGS ctas, s, geo, aux, n_points, width, height, tiles_x, units, out, slots, counters, vec, status, \
                        timeout_ns, drop_tile, ref
        if (sfu && !extra) return launch<true, false>(CGH_STREAM_ARGS);
        if (sfu) return launch<true, true>(CGH_STREAM_ARGS);
        if (!extra) return launch<false, false>(CGH_STREAM_ARGS);
        return launch<false, true>(CGH_STREAM_ARGS);
#undef CGH_STREAM_ARGS
    }

    static int resident(bool sfu)
    {
        if constexpr (kDyn > 0) {   // the limit the launch will set (occupancy counts it)
            static PerDeviceOnce configured;
            configured.run([] {
                cudaError_t e =
                    cudaFuncSetAttribute(direct_stream_kernel<TL, TR, BX, BY, true, false, SMEM_TOT, TABLES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDyn);
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(direct_stream_kernel<TL, TR, BX, BY, false, false, SMEM_TOT, TABLES>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDyn);
                return e;
            });
        }
        int n = 0;
        const cudaError_t e =
            sfu ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, direct_stream_kernel<TL, TR, BX, BY, true, false, SMEM_TOT, TABLES>, BX * BY, kDyn)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, direct_stream_kernel<TL, TR, BX, BY, false, false, SMEM_TOT, TABLES>, BX * BY, kDyn);
        if (e != cudaSuccess || n < 1) {
            cudaGetLastError();
            return 1;
        }
        return n;
    }
};

// (A 16 x 16 block of 12 x 4 pixels per thread with the totals in shared memory -- fewer per-point instructions
// per term -- was measured slower: 4.84 against 4.65 ms at 1920x1080, 10^4 points.)
using StreamTall = StreamCfg<kTL, kTR, kTallBX, kTallBY, false>;
using StreamWide = StreamCfg<kTL, kTR, kBX, kBY, false>;
// Blocks of 8 x 8 pixels per thread, 128 threads, totals in shared memory: 16 x 8 threads (the tall shape's
// 128 x 64 tile) or 32 x 4 (the wide shape's 256 x 32).  With the separable SFU evaluation a point costs a thread
// 16 hardware sines and cosines for 64 terms.
constexpr int kSqTL = 8, kSqTR = 8, kSqBX = 16, kSqBY = 8, kSqWideBX = 32, kSqWideBY = 4;
using StreamSquare = StreamCfg<kSqTL, kSqTR, kSqBX, kSqBY, true>;
using StreamSquareWide = StreamCfg<kSqTL, kSqTR, kSqWideBX, kSqWideBY, true>;
// The 8 x 4-pixel blocks with the tables of the tile (dev::SepTable): the sines and cosines of a point's columns
// and rows taken once per CTA.  The tall block keeps its totals in shared memory, the registers going to the
// unrolled point loop (1920x1080, 10^4 points: 2.27 against 2.30 ms); the wide one measured the other way (2.94
// in registers, 3.71 in shared memory).
using StreamTallTab = StreamCfg<kTL, kTR, kTallBX, kTallBY, true, true>;
using StreamWideTab = StreamCfg<kTL, kTR, kBX, kBY, false, true>;

}  // namespace

DirectShape direct_stream_shape(int variant)
{
    if (variant == 2) return DirectShape{kSqBX * kSqTL, kSqBY * kSqTR, kSqBX * kSqBY, kSqBX};
    if (variant == 3) return DirectShape{kSqWideBX * kSqTL, kSqWideBY * kSqTR, kSqWideBX * kSqWideBY, kSqWideBX};
    if (variant == 4 || variant == 5) {
        DirectShape sh = direct_shape(variant == 4);
        sh.tables = 1;
        return sh;
    }
    return direct_shape(variant == 1);
}

int direct_stream_per_sm(bool sfu, const DirectShape &sh)
{
    if (sh.tables) return sh.bx == kTallBX ? StreamTallTab::resident(sfu) : StreamWideTab::resident(sfu);
    if (sh.threads == kSqBX * kSqBY)
        return sh.bx == kSqBX ? StreamSquare::resident(sfu) : StreamSquareWide::resident(sfu);
    return sh.bx == kTallBX ? StreamTall::resident(sfu) : StreamWide::resident(sfu);
}

cudaError_t launch_direct_stream(bool sfu, const DirectShape &sh, int ctas, const int4 *geo, const uint2 *aux,
                                 int n_points, int width, int height, float *out, float *slots, int *counters,
                                 int *status, uint64_t timeout_ns, cudaStream_t s, int drop_tile, const PhaseRef &ref)
{
    const int tiles_x = (width + sh.tile_w - 1) / sh.tile_w;
    const int tiles_y = (height + sh.tile_h - 1) / sh.tile_h;
    const long long units = (long long)tiles_x * tiles_y * n_points;
    if (n_points < 1 || ctas < 1 || (long long)ctas > units || ((uintptr_t)slots % 16) != 0)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(counters, 0, (size_t)tiles_x * tiles_y * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const bool vec = (width % 4 == 0) && ((uintptr_t)out % 16 == 0);
    float4 *sl = reinterpret_cast<float4 *>(slots);
    const bool extra = ref.any();
#define CGH_STREAM_ARGS sfu, extra, ctas, s, geo, aux, n_points, width, height, tiles_x, units, out, sl, counters, vec, \
                        status, timeout_ns, drop_tile, ref
    if (sh.tables)
        return sh.bx == kTallBX ? StreamTallTab::dispatch(CGH_STREAM_ARGS) : StreamWideTab::dispatch(CGH_STREAM_ARGS);
    if (sh.threads == kSqBX * kSqBY)
        return sh.bx == kSqBX ? StreamSquare::dispatch(CGH_STREAM_ARGS) : StreamSquareWide::dispatch(CGH_STREAM_ARGS);
    if (sh.bx == kTallBX) return StreamTall::dispatch(CGH_STREAM_ARGS);
    return StreamWide::dispatch(CGH_STREAM_ARGS);
#undef CGH_STREAM_ARGS
}

}  // namespace cgh

namespace cgh {

cudaError_t launch_direct_batch(bool sfu, bool tall, const DirectJob *d_jobs, const int *d_cta_off,
                                const int2 *d_units, int ctas, int *status, uint64_t timeout_ns, cudaStream_t s)
{
    if (ctas <= 0) return cudaSuccess;
    if (sfu && tall)
        direct_batch_kernel<kTL, kTR, kTallBX, kTallBY, true><<<ctas, kTallBX * kTallBY, 0, s>>>(
            d_jobs, d_cta_off, d_units, status, timeout_ns);
    else if (sfu)
        direct_batch_kernel<kTL, kTR, kBX, kBY, true><<<ctas, kBX * kBY, 0, s>>>(d_jobs, d_cta_off, d_units, status,
                                                                                 timeout_ns);
    else if (tall)
        direct_batch_kernel<kTL, kTR, kTallBX, kTallBY, false><<<ctas, kTallBX * kTallBY, 0, s>>>(
            d_jobs, d_cta_off, d_units, status, timeout_ns);
    else
        direct_batch_kernel<kTL, kTR, kBX, kBY, false><<<ctas, kBX * kBY, 0, s>>>(d_jobs, d_cta_off, d_units,
                                                                                  status, timeout_ns);
    return cudaGetLastError();
}

int direct_ctas_per_sm(bool sfu, bool tall)
{
    int n = 0;
    cudaError_t e;
    if (sfu && tall)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, direct_batch_kernel<kTL, kTR, kTallBX, kTallBY, true>,
                                                          kTallBX * kTallBY, 0);
    else if (sfu)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, direct_batch_kernel<kTL, kTR, kBX, kBY, true>,
                                                          kBX * kBY, 0);
    else if (tall)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, direct_batch_kernel<kTL, kTR, kTallBX, kTallBY, false>,
                                                          kTallBX * kTallBY, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, direct_batch_kernel<kTL, kTR, kBX, kBY, false>,
                                                          kBX * kBY, 0);
    if (e != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 1;
    }
    return n;
}

}  // namespace cgh

namespace cgh {

namespace {
constexpr int kWaveTL = 8, kWaveTR = 4;   // two planes of partial sums in registers, the totals in shared memory

// The tall block takes the tables (two CTAs an SM with 8-point groups); the wide one's tables would leave one CTA
// an SM, so it keeps each thread's own sines and cosines.
template <int BX, int BY>
void wave_as(bool extra, dim3 grid, cudaStream_t s, const int4 *geo, const uint2 *aux, int n_ptiles, int width,
             int height, int tiles_x, int split, float *out, long long ss, long long im, bool vec, int *status,
             uint64_t timeout_ns, const PhaseRef &ref)
{
    constexpr bool kTables = BX == kTallBX;
    constexpr size_t dyn_bytes =
        (size_t)2 * kWaveTR * kWaveTL * BX * BY * sizeof(float) +
        (kTables ? (size_t)2 * sep_group<2>() * SepTable<BX * kWaveTL, BY * kWaveTR>::kPerPoint * sizeof(float2)
                 : 0);
    static PerDeviceOnce configured;   // the running totals exceed the default 48 KB of dynamic shared memory
    const cudaError_t e = configured.run([&] {
        cudaError_t r = cudaFuncSetAttribute(direct_wave_kernel<kWaveTL, kWaveTR, BX, BY, true, kTables>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_bytes);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(direct_wave_kernel<kWaveTL, kWaveTR, BX, BY, false, kTables>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_bytes);
        return r;
    });
    if (e != cudaSuccess) return;
    if (extra)
        direct_wave_kernel<kWaveTL, kWaveTR, BX, BY, true, kTables><<<grid, BX * BY, dyn_bytes, s>>>(
            geo, aux, n_ptiles, width, height, tiles_x, split, out, ss, im, vec, status, timeout_ns, ref);
    else
        direct_wave_kernel<kWaveTL, kWaveTR, BX, BY, false, kTables><<<grid, BX * BY, dyn_bytes, s>>>(
            geo, aux, n_ptiles, width, height, tiles_x, split, out, ss, im, vec, status, timeout_ns, ref);
}
}  // namespace

DirectShape direct_wave_shape(bool tall)
{
    return tall ? DirectShape{kTallBX * kWaveTL, kTallBY * kWaveTR, kTallBX * kTallBY, kTallBX}
                : DirectShape{kBX * kWaveTL, kBY * kWaveTR, kBX * kBY, kBX};
}

cudaError_t launch_direct_wave(const DirectShape &sh, const int4 *geo, const uint2 *aux, int n_pad, int width,
                               int height, int split, float *out, int64_t slice_stride, int64_t im_offset,
                               int *status, uint64_t timeout_ns, cudaStream_t s, const PhaseRef &ref)
{
    const int tiles_x = (width + sh.tile_w - 1) / sh.tile_w;
    const int tiles_y = (height + sh.tile_h - 1) / sh.tile_h;
    const int n_ptiles = n_pad / kPointTile;
    if (split < 1) split = 1;
    dim3 grid(tiles_x * tiles_y, split);
    const bool vec = (width % 4 == 0) && (slice_stride % 4 == 0) && (im_offset % 4 == 0) &&
                     ((uintptr_t)out % 16 == 0);
    if (sh.bx == kTallBX)
        wave_as<kTallBX, kTallBY>(ref.any(), grid, s, geo, aux, n_ptiles, width, height, tiles_x, split, out,
                                  (long long)slice_stride, (long long)im_offset, vec, status, timeout_ns, ref);
    else
        wave_as<kBX, kBY>(ref.any(), grid, s, geo, aux, n_ptiles, width, height, tiles_x, split, out,
                          (long long)slice_stride, (long long)im_offset, vec, status, timeout_ns, ref);
    return cudaGetLastError();
}

}  // namespace cgh
