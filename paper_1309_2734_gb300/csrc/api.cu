// The C ABI (include/cgh.h): argument checks, the context and its workspace,
// and the order of kernel launches for each entry point.  No arithmetic of
// the method runs here; every step of the hologram runs in the kernels.
#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "context.h"
#include "tuner.h"

using namespace cgh;

namespace cgh {

// Direct form: prep, then the direct kernel.  By default one launch in which the CTAs take equal shares of the
// (pixel tile, point) pairs and the last CTA to finish a tile sums its parts (no partial planes).  With
// CGH_OPT_POINT_SPLIT > 0: point chunks into partial planes and the fixed-order chunk reduction after.
constexpr int kStreamMinPoints = 64;      // fewest points of one CTA's share in the balanced layout
constexpr int kStreamSharePoints = 1024;  // points per share from which CTAs beyond the resident ones are added
constexpr int kStreamWaves = 2;           // at most this many CTAs per resident slot

int run_direct(cgh_ctx *ctx, bool sfu, int width, int height, double pitch, double lambda, const float *d_xyz,
               const float *d_amp, int64_t n, float *d_out)
{
    const int64_t n_pad = padded_points(n);
    const int64_t n_ptiles = n_pad / kPointTile;
    const size_t geo_bytes = align_up((size_t)n_pad * sizeof(int4), 256);
    const size_t aux_bytes = align_up((size_t)n_pad * sizeof(uint2), 256);
    const int64_t plane = (int64_t)width * height;
    const uint64_t tmo = (uint64_t)ctx->timeout_ms * 1000000ull;
    const bool stream_k = ctx->point_split == 0;
    DirectShape sh;
    int split = 1, ctas = 0;
    size_t ws_rest = 0;
    if (stream_k) {
        // the shape with the fewer padded pixels; up to kStreamWaves CTAs per resident slot (measured at
        // 1920x1080, 10^4 points, 8 x 8 pixels a thread, four 128-thread CTAs per SM: 608 CTAs 3.02 ms, 1216 2.995,
        // 1824 3.017, 2432 3.22; DRAM writes 0.1 / 3.9 / 18.4 MB per launch, the parts L2 no longer holds), each
        // share of at least kStreamSharePoints points beyond the first wave and kStreamMinPoints within it
        auto padded = [&](const DirectShape &s) {
            return (int64_t)((width + s.tile_w - 1) / s.tile_w) * s.tile_w *
                   (((int64_t)height + s.tile_h - 1) / s.tile_h) * s.tile_h;
        };
        // blocks of 8 x 4 pixels with the tables of the tile, 16 x 16 threads (a 128 x 64 tile) unless 32 x 8 (256 x
        // 32) pads a fifth fewer pixels (at equal padding the tall block measured 16 % faster: a point's 192 table
        // entries over 256 threads instead of 288); CGH_OPT_DIRECT_SHAPE pins any block
        if (ctx->direct_shape > 0) {
            sh = direct_stream_shape(ctx->direct_shape - 1);
        } else {
            sh = direct_stream_shape(4);
            if (padded(direct_stream_shape(5)) * 6 < padded(sh) * 5) sh = direct_stream_shape(5);
        }
        const int64_t tiles = (int64_t)((width + sh.tile_w - 1) / sh.tile_w) * ((height + sh.tile_h - 1) / sh.tile_h);
        const int64_t units = tiles * n;
        const int64_t slots = (int64_t)ctx->num_sms * direct_stream_per_sm(sfu, sh);
        int64_t want = units >= slots * kStreamSharePoints
                           ? std::min<int64_t>(kStreamWaves * slots, units / kStreamSharePoints)
                           : std::min<int64_t>(slots, units / kStreamMinPoints);
        if (ctx->direct_ctas > 0) want = std::min<int64_t>(ctx->direct_ctas, units);
        ctas = (int)std::max<int64_t>(1, want);
        ws_rest = align_up((size_t)2 * ctas * sh.tile_w * sh.tile_h * sizeof(float), 256) +
                  align_up((size_t)tiles * sizeof(int), 256);
    } else {
        const DirectLayout lay = choose_direct_layout(false, width, height, n_ptiles, ctx->num_sms, ctx->point_split);
        sh = lay.shape;
        split = lay.split;
        ws_rest = split > 1 ? (size_t)split * plane * sizeof(float) : 0;
    }
    int rc = ensure(ctx, &ctx->ws, &ctx->ws_bytes, geo_bytes + aux_bytes + ws_rest);
    if (rc) return rc;
    char *base = static_cast<char *>(ctx->ws);
    int4 *geo = reinterpret_cast<int4 *>(base);
    uint2 *aux = reinterpret_cast<uint2 *>(base + geo_bytes);
    float *rest = reinterpret_cast<float *>(base + geo_bytes + aux_bytes);
    cudaError_t e;
    {
        ProfileScope ps(ctx, "prep_points", 1);
        e = launch_prep_points(d_xyz, d_amp, (int)n, (int)n_pad, pitch, lambda, geo, aux, ctx->d_status,
                               nullptr, ctx->stream, aux_mode(ctx));
    }
    if (e != cudaSuccess) return cuda_status(e);
    if (stream_k) {
        int *counters = reinterpret_cast<int *>(
            reinterpret_cast<char *>(rest) + align_up((size_t)2 * ctas * sh.tile_w * sh.tile_h * sizeof(float), 256));
        ProfileScope ps(ctx, sfu ? "direct_sfu" : "direct_accurate", 1);   // and the counters' memset
        return cuda_status(launch_direct_stream(sfu, sh, ctas, geo, aux, (int)n, width, height, d_out, rest,
                                                counters, ctx->d_status, tmo, ctx->stream, ctx->drop_tile,
                                                phase_ref(ctx)));
    }
    {
        ProfileScope ps(ctx, sfu ? "direct_sfu" : "direct_accurate", 1);
        e = launch_direct(sfu, sh, geo, aux, (int)n_pad, width, height, split, split > 1 ? rest : d_out, plane,
                          ctx->d_status, tmo, ctx->stream, ctx->drop_tile, phase_ref(ctx));
    }
    if (e != cudaSuccess || split == 1) return cuda_status(e);
    ProfileScope ps(ctx, "reduce_slices", 1);
    return cuda_status(launch_reduce_slices(rest, split, plane, plane, d_out, ctx->stream));
}

// k-blocks per TMEM accumulation chain of the split-FP16 form (3 passes each)
constexpr int kSplit16ChunkKb = 8;
// smallest point chunk worth a pipeline stage of its own
constexpr int64_t kPipelineMinPoints = 8192;
// CGH_OPT_GEMM_GROUP = 0 tries the grouped form from this many points
constexpr int64_t kGroupMinPoints = 65536;

int factor_mode(int form)
{
    return form == CGH_GEMM_BF16 ? kFactorBF16 : (form == CGH_GEMM_SPLIT16 ? kFactorSplit16 : kFactorF16);
}

// Factor generation for K units [u0, u0 + nu) (points, or groups of points)
// into P and Q with leading dimension ld, on stream s.
using FactorLaunch = std::function<cudaError_t(int64_t u0, int64_t nu, void *P, void *Q, int64_t ld, cudaStream_t s)>;

// The GEMM over K units: per chunk of units the factors P and Q and the
// tcgen05 GEMM over K splits, later chunks adding to the planes of the first;
// then the fixed-order split reduction when there is more than one split.
// Chunks bound the factor workspace (CGH_OPT_FACTOR_BUDGET_MB: 10^6 points of
// a 4096x4096 split-FP16 hologram would otherwise need 65 GB) and can pipeline
// the two halves of the form: with CGH_OPT_GEMM_PIPELINE > 1 the factors of
// chunk c + 1 are generated on a second stream (double-buffered) while the
// tensor cores run the GEMM of chunk c.  (Measured on GB300 at 1920x1080 with
// 5x10^4 points: 0.428 ms without, 0.428-0.46 ms with 2-4 stages, so it is
// off by default.)  The epilogue multiplies by *scale, the factor of Q (or
// P) that keeps the FP16 operands within range.
// Points (K units) per factor chunk when one chunk's P and Q may take budget bytes.
static int64_t gemm_chunk_units(int mode, int width, int height, int64_t budget)
{
    const int planes = mode == kFactorSplit16 ? 2 : 1;
    const int64_t bytes_per_unit = (int64_t)planes * (width + height) * 2 * 2;
    const int64_t chunk = budget / bytes_per_unit / 32 * 32;
    return chunk < 32 ? 32 : chunk;
}

int gemm_units(cgh_ctx *ctx, int mode, int width, int height, int64_t n, const char *factor_name,
               const FactorLaunch &factors, const float *scale, float *d_out)
{
    const int planes = mode == kFactorSplit16 ? 2 : 1;
    const int depth = ctx->gemm_pipeline;
    const int64_t budget = (ctx->factor_budget_mb << 20) / (depth > 1 ? 2 : 1);   // per factor buffer
    int64_t chunk = gemm_chunk_units(mode, width, height, budget);
    if (depth > 1 && n >= (int64_t)depth * kPipelineMinPoints) {
        const int64_t even = ((n + depth - 1) / depth + 31) / 32 * 32;
        if (even < chunk) chunk = even;
    }
    if (chunk >= n) chunk = n;
    const int64_t n_chunks = (n + chunk - 1) / chunk;
    const int64_t ld_max = (2 * chunk + 63) / 64 * 64;
    const int64_t nkb_max = ld_max / 64;
    GemmPlan plan;
    plan.mode = mode;
    plan.ctas = gemm_max_ctas(ctx->num_sms);
    const GemmLayout lay = choose_gemm_layout(width, height, nkb_max, plan.ctas, mode == kFactorSplit16,
                                              ctx->gemm_bn, ctx->gemm_splitk, ctx->gemm_trans, ctx->gemm_pair);
    plan.pair = lay.pair;
    plan.bn = lay.bn;
    plan.splits = lay.splits;
    plan.trans = lay.trans;
    if (!gemm_bn_supported(plan.bn)) return CGH_ENOTSUP;
    plan.chunk_kb = ctx->gemm_chunk > 0 ? ctx->gemm_chunk : (mode == kFactorSplit16 ? kSplit16ChunkKb : 0);
    plan.accumulate = false;
    // every chunk must write every partial plane: no more splits than the last chunk has k-blocks
    const int64_t last = n - (n_chunks - 1) * chunk;
    const int64_t nkb_last = (2 * last + 63) / 64;
    if (plan.splits > nkb_last) plan.splits = (int)nkb_last;
    const int64_t plane = (int64_t)width * height;
    const int nbuf = n_chunks > 1 ? 2 : 1;
    const size_t p_bytes = align_up((size_t)planes * height * ld_max * 2, 256);
    const size_t q_bytes = align_up((size_t)planes * width * ld_max * 2, 256);
    const size_t part_bytes = plan.splits > 1 ? (size_t)plan.splits * plane * sizeof(float) : 0;
    int rc = ensure(ctx, &ctx->ws, &ctx->ws_bytes, nbuf * (p_bytes + q_bytes) + part_bytes);
    if (rc) return rc;
    char *fac = static_cast<char *>(ctx->ws);
    float *parts = reinterpret_cast<float *>(fac + nbuf * (p_bytes + q_bytes));
    cudaError_t e;
    const uint64_t tmo = (uint64_t)ctx->timeout_ms * 1000000ull;
    // factors on the side stream when pipelining, else on the main stream
    cudaStream_t fs = ctx->stream;
    if (nbuf == 2) {
        rc = ensure_side_stream(ctx);
        if (rc) return rc;
        fs = ctx->side_stream;
        e = cudaEventRecord(ctx->ev_ready, ctx->stream);       // prep (and earlier work) done
        if (e == cudaSuccess) e = cudaStreamWaitEvent(fs, ctx->ev_ready, 0);
        if (e != cudaSuccess) return cuda_status(e);
    }
    for (int64_t c = 0; c < n_chunks; ++c) {
        const int64_t c0 = c * chunk;
        const int64_t nc = n - c0 < chunk ? n - c0 : chunk;
        const int64_t ld = (2 * nc + 63) / 64 * 64;
        const int b = (int)(c & 1) % nbuf;
        void *P = fac + b * (p_bytes + q_bytes);
        void *Q = fac + b * (p_bytes + q_bytes) + p_bytes;
        if (nbuf == 2 && c >= 2) {
            e = cudaStreamWaitEvent(fs, ctx->ev_gemm[b], 0);   // the GEMM of chunk c - 2 has read buffer b
            if (e != cudaSuccess) return cuda_status(e);
        }
        {
            ProfileScope ps(ctx, factor_name, 1, fs);
            e = factors(c0, nc, P, Q, ld, fs);
        }
        if (e != cudaSuccess) return cuda_status(e);
        if (nbuf == 2) {
            e = cudaEventRecord(ctx->ev_fact[b], fs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_fact[b], 0);
            if (e != cudaSuccess) return cuda_status(e);
        }
        GemmPlan pc = plan;
        pc.accumulate = c > 0;
        {
            ProfileScope ps(ctx, "gemm_tcgen05", 1);
            e = launch_gemm(pc, P, Q, height, width, ld, plan.splits > 1 ? parts : d_out, plane, scale,
                            ctx->d_status, tmo, ctx->stream);
        }
        if (e != cudaSuccess) return cuda_status(e);
        if (nbuf == 2) {
            e = cudaEventRecord(ctx->ev_gemm[b], ctx->stream);
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    if (plan.splits == 1) return CGH_OK;
    ProfileScope ps(ctx, "reduce_slices", 1);
    return cuda_status(launch_reduce_slices(parts, plan.splits, plane, plane, d_out, ctx->stream));
}

}  // namespace cgh

extern "C" int cgh_gemm_layout(int width, int height, int64_t n_points, int form, int num_sms, int *layout)
{
    using namespace cgh;
    if (width < 1 || height < 1 || width > kMaxSide || height > kMaxSide || n_points < 1 || num_sms < 1 || !layout)
        return CGH_EINVAL;
    if (form < CGH_GEMM_F16 || form > CGH_GEMM_SPLIT16) return CGH_EINVAL;
    const int mode = factor_mode(form);
    int64_t chunk = gemm_chunk_units(mode, width, height, kDefaultFactorBudgetMb << 20);
    if (chunk > n_points) chunk = n_points;
    const GemmLayout lay = choose_gemm_layout(width, height, (2 * chunk + 63) / 64, gemm_max_ctas(num_sms),
                                              mode == kFactorSplit16, 0, 0, 0, 0);
    const int64_t last = n_points - (n_points - 1) / chunk * chunk;
    const int64_t nkb_last = (2 * last + 63) / 64;
    layout[0] = lay.trans ? 1 : 0;
    layout[1] = lay.bn;
    layout[2] = lay.splits > nkb_last ? (int)nkb_last : lay.splits;
    layout[3] = lay.pair ? 1 : 0;
    return CGH_OK;
}

namespace cgh {

// Copies n ints of device memory to the context's pinned buffer and waits for
// them (bounded like cgh_sync); the grouped form's two reads of counts.
int read_counts(cgh_ctx *ctx, const int *d_src, int n, int *out)
{
    if (!ctx->h_meta) {
        if (cudaMallocHost(&ctx->h_meta, 16 * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            ctx->h_meta = nullptr;
            return CGH_ENOMEM;
        }
    }
    cudaError_t e = cudaMemcpyAsync(ctx->h_meta, d_src, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaStreamQuery(ctx->stream);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_status(q);
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
        if (ms.count() > 2 * ctx->timeout_ms + 1000) return CGH_ETIMEOUT;
        std::this_thread::yield();
    }
    std::memcpy(out, ctx->h_meta, n * sizeof(int));
    return CGH_OK;
}

// GEMM form: prep into the point workspace, then (CGH_OPT_GEMM_GROUP) either
// the grouped form -- points of one depth plane and one column summed into a
// single K unit before the GEMM -- or one K unit per point.
int run_gemm(cgh_ctx *ctx, int form, int width, int height, double pitch, double lambda, const float *d_xyz,
             const float *d_amp, int64_t n, float *d_out)
{
    const int mode = factor_mode(form);
    const int64_t n_pad = padded_points(n);
    // with the piston, points of equal C may still differ in depth: no grouping
    bool try_group = !piston_on(ctx) && (ctx->gemm_group == 2 || (ctx->gemm_group == 0 && n >= kGroupMinPoints));
    const PhaseRef ref = phase_ref(ctx);
    if (try_group) {   // the grouped form reads counts back: not while a graph is being captured
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) {
            cudaGetLastError();
            try_group = false;
        } else if (cs != cudaStreamCaptureStatusNone) {
            try_group = false;
        }
    }
    if (ctx->gemm_persistent && !try_group && !piston_on(ctx) && !ref.any()) {
        // the persistent kernel: factor generation of later K chunks overlaps the GEMM of earlier ones; all
        // factors at once, so within the factor budget; not while the stream is captured (a new plan copies
        // its tables to the device and synchronises)
        const int planes = mode == kFactorSplit16 ? 2 : 1;
        const int64_t fbytes = (int64_t)planes * (width + height) * ((2 * n + 63) / 64 * 64) * 2;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const bool capturing = cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess ||
                               cs != cudaStreamCaptureStatusNone;
        cudaGetLastError();
        if (!capturing && fbytes <= (ctx->factor_budget_mb << 20)) {
            const cgh_instance inst{width, height, pitch, lambda, d_xyz, d_amp, n, d_out};
            return run_single_persistent(ctx, form, inst);
        }
    }
    const size_t geo_bytes = align_up((size_t)n_pad * sizeof(int4), 256);
    const size_t aux_bytes = align_up((size_t)n_pad * sizeof(uint2), 256);
    const size_t meta_bytes = 256;   // amax, wscale, meta[4]
    const size_t gscratch_bytes = try_group ? align_up(group_workspace_bytes((int)n, kMaxPlanes), 256) : 0;
    const size_t groups_bytes = try_group ? align_up((size_t)n * sizeof(int4), 256) : 0;
    const size_t gathered_bytes = try_group ? align_up((size_t)n * sizeof(int2), 256) : 0;
    int rc = ensure(ctx, &ctx->pws, &ctx->pws_bytes,
                    geo_bytes + aux_bytes + meta_bytes + gscratch_bytes + groups_bytes + gathered_bytes);
    if (rc) return rc;
    char *base = static_cast<char *>(ctx->pws);
    int4 *geo = reinterpret_cast<int4 *>(base);
    uint2 *aux = reinterpret_cast<uint2 *>(base + geo_bytes);
    float *amax = reinterpret_cast<float *>(base + geo_bytes + aux_bytes);
    float *wscale = amax + 1;
    int *meta = reinterpret_cast<int *>(amax + 4);
    char *gscratch = base + geo_bytes + aux_bytes + meta_bytes;
    int4 *groups = reinterpret_cast<int4 *>(gscratch + gscratch_bytes);
    int2 *members = reinterpret_cast<int2 *>(gscratch + gscratch_bytes + groups_bytes);
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(float), ctx->stream);
    if (e != cudaSuccess) return cuda_status(e);
    {
        ProfileScope ps(ctx, "prep_points", 1);
        e = launch_prep_points(d_xyz, d_amp, (int)n, (int)n_pad, pitch, lambda, geo, aux, ctx->d_status, amax,
                               ctx->stream, aux_mode(ctx));
    }
    if (e != cudaSuccess) return cuda_status(e);
    if (try_group) {
        int m[4] = {0, 0, 0, 0};
        {
            ProfileScope ps(ctx, "group_planes", 2);
            e = launch_planes(geo, (int)n, gscratch, meta, ctx->stream);
        }
        if (e != cudaSuccess) return cuda_status(e);
        rc = read_counts(ctx, meta, 1, m);
        if (rc) return rc;
        const int n_planes = m[0];
        if (n_planes >= 1 && n_planes <= kMaxPlanes) {
            {
                ProfileScope ps(ctx, "group_count", 4);
                e = launch_group_count(geo, (int)n, n_planes, gscratch, meta, groups, ctx->stream);
            }
            if (e != cudaSuccess) return cuda_status(e);
            rc = read_counts(ctx, meta, 4, m);
            if (rc) return rc;
            const int n_groups = m[2], largest = m[3];
            const bool pays = ctx->gemm_group == 2 || 2 * (int64_t)n_groups <= n;
            if (n_groups >= 1 && largest <= kMaxGroupPoints && pays) {
                {
                    ProfileScope ps(ctx, "group_build", 4);
                    e = launch_group_build(geo, aux, (int)n, n_planes, n_groups, gscratch, meta, groups, amax,
                                           wscale, members, ctx->stream);
                }
                if (e != cudaSuccess) return cuda_status(e);
                const FactorLaunch gf = [&](int64_t u0, int64_t nu, void *P, void *Q, int64_t ld, cudaStream_t s) {
                    return launch_group_factors(mode, groups, (int)u0, (int)nu, group_plane_table(gscratch), members,
                                                height, width, P, Q, ld, wscale, s, ref);
                };
                return gemm_units(ctx, mode, width, height, n_groups, "group_factors", gf, wscale, d_out);
            }
        }
    }
    const FactorLaunch pf = [&](int64_t u0, int64_t nu, void *P, void *Q, int64_t ld, cudaStream_t s) {
        return launch_factors(mode, geo + u0, aux + u0, (int)nu, height, width, P, Q, ld, amax, s, false, ref);
    };
    return gemm_units(ctx, mode, width, height, n, "factors", pf, amax, d_out);
}

// The complex object wave: real plane at d_out, imaginary plane at d_out + W H.
// Direct form: one pass accumulating both parts.  GEMM forms: per chunk of
// points, Re = P Q^T and Im = P Q'^T (the same P), later chunks adding.
int run_wave(cgh_ctx *ctx, int form, const float *d_xyz, const float *d_amp, int64_t n, float *d_out)
{
    const int width = ctx->width, height = ctx->height;
    const int64_t plane = (int64_t)width * height;
    const int64_t n_pad = padded_points(n);
    const size_t geo_bytes = align_up((size_t)n_pad * sizeof(int4), 256);
    const size_t aux_bytes = align_up((size_t)n_pad * sizeof(uint2), 256);
    const uint64_t tmo = (uint64_t)ctx->timeout_ms * 1000000ull;
    cudaError_t e;
    if (form == CGH_DIRECT_SFU) {
        const int64_t n_ptiles = n_pad / kPointTile;
        const DirectLayout lay = choose_direct_layout(true, width, height, n_ptiles, ctx->num_sms, ctx->point_split);
        const DirectShape sh = lay.shape;
        const int split = lay.split;
        const size_t part_bytes = split > 1 ? (size_t)split * 2 * plane * sizeof(float) : 0;
        int rc = ensure(ctx, &ctx->ws, &ctx->ws_bytes, geo_bytes + aux_bytes + part_bytes);
        if (rc) return rc;
        char *base = static_cast<char *>(ctx->ws);
        int4 *geo = reinterpret_cast<int4 *>(base);
        uint2 *aux = reinterpret_cast<uint2 *>(base + geo_bytes);
        float *parts = reinterpret_cast<float *>(base + geo_bytes + aux_bytes);
        {
            ProfileScope ps(ctx, "prep_points", 1);
            e = launch_prep_points(d_xyz, d_amp, (int)n, (int)n_pad, ctx->pitch, ctx->lambda, geo, aux, ctx->d_status,
                                   nullptr, ctx->stream, aux_mode(ctx));
        }
        if (e != cudaSuccess) return cuda_status(e);
        {
            ProfileScope ps(ctx, "direct_wave", 1);
            e = launch_direct_wave(sh, geo, aux, (int)n_pad, width, height, split, split > 1 ? parts : d_out,
                                   2 * plane, plane, ctx->d_status, tmo, ctx->stream, phase_ref(ctx));
        }
        if (e != cudaSuccess || split == 1) return cuda_status(e);
        ProfileScope ps(ctx, "reduce_slices", 2);
        e = launch_reduce_slices(parts, split, plane, 2 * plane, d_out, ctx->stream);
        if (e == cudaSuccess) e = launch_reduce_slices(parts + plane, split, plane, 2 * plane, d_out + plane, ctx->stream);
        return cuda_status(e);
    }
    if (form < CGH_GEMM_F16 || form > CGH_GEMM_SPLIT16) return CGH_ENOTSUP;
    const int mode = factor_mode(form);
    const int planes = mode == kFactorSplit16 ? 2 : 1;
    const int64_t bytes_per_point = (int64_t)planes * (width + height) * 2 * 2;
    int64_t chunk = (ctx->factor_budget_mb << 20) / bytes_per_point / 32 * 32;
    if (chunk < 32) chunk = 32;
    if (chunk >= n) chunk = n;
    const int64_t ld_max = (2 * chunk + 63) / 64 * 64;
    GemmPlan plan;
    plan.mode = mode;
    plan.ctas = gemm_max_ctas(ctx->num_sms);
    // one CTA per tile: the complex wave's two output planes have no two-SM form
    const GemmLayout lay = choose_gemm_layout(width, height, ld_max / 64, plan.ctas, mode == kFactorSplit16,
                                              ctx->gemm_bn, ctx->gemm_splitk, ctx->gemm_trans, 2);
    plan.bn = lay.bn;
    plan.splits = lay.splits;
    plan.trans = lay.trans;
    if (!gemm_bn_supported(plan.bn)) return CGH_ENOTSUP;
    plan.chunk_kb = ctx->gemm_chunk > 0 ? ctx->gemm_chunk : (mode == kFactorSplit16 ? kSplit16ChunkKb : 0);
    plan.accumulate = false;
    const int64_t last = n - (n - 1) / chunk * chunk;
    if (plan.splits > (2 * last + 63) / 64) plan.splits = (int)((2 * last + 63) / 64);
    const size_t amax_bytes = 256;
    const size_t p_bytes = align_up((size_t)planes * height * ld_max * 2, 256);
    const size_t q_bytes = align_up((size_t)planes * width * ld_max * 2, 256);
    const size_t part_bytes = plan.splits > 1 ? (size_t)plan.splits * 2 * plane * sizeof(float) : 0;
    int rc = ensure(ctx, &ctx->ws, &ctx->ws_bytes, geo_bytes + aux_bytes + amax_bytes + p_bytes + q_bytes + part_bytes);
    if (rc) return rc;
    char *base = static_cast<char *>(ctx->ws);
    int4 *geo = reinterpret_cast<int4 *>(base);
    uint2 *aux = reinterpret_cast<uint2 *>(base + geo_bytes);
    float *amax = reinterpret_cast<float *>(base + geo_bytes + aux_bytes);
    void *P = base + geo_bytes + aux_bytes + amax_bytes;
    void *Q = base + geo_bytes + aux_bytes + amax_bytes + p_bytes;
    float *parts = reinterpret_cast<float *>(base + geo_bytes + aux_bytes + amax_bytes + p_bytes + q_bytes);
    e = cudaMemsetAsync(amax, 0, sizeof(float), ctx->stream);
    if (e != cudaSuccess) return cuda_status(e);
    {
        ProfileScope ps(ctx, "prep_points", 1);
        e = launch_prep_points(d_xyz, d_amp, (int)n, (int)n_pad, ctx->pitch, ctx->lambda, geo, aux, ctx->d_status,
                               amax, ctx->stream, aux_mode(ctx));
    }
    if (e != cudaSuccess) return cuda_status(e);
    const PhaseRef ref = phase_ref(ctx);
    float *re_out = plan.splits > 1 ? parts : d_out;
    float *im_out = plan.splits > 1 ? parts + (int64_t)plan.splits * plane : d_out + plane;
    for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        const int64_t nc = n - c0 < chunk ? n - c0 : chunk;
        const int64_t ld = (2 * nc + 63) / 64 * 64;
        GemmPlan pc = plan;
        pc.accumulate = c0 > 0;
        for (int part = 0; part < 2; ++part) {
            {
                ProfileScope ps(ctx, "factors", 1);
                e = launch_factors(mode, geo + c0, aux + c0, (int)nc, height, width, P, Q, ld, amax, ctx->stream,
                                   part == 1, ref);
            }
            if (e != cudaSuccess) return cuda_status(e);
            {
                ProfileScope ps(ctx, "gemm_tcgen05", 1);
                e = launch_gemm(pc, P, Q, height, width, ld, part == 0 ? re_out : im_out, plane, amax, ctx->d_status,
                                tmo, ctx->stream);
            }
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    if (plan.splits == 1) return CGH_OK;
    ProfileScope ps(ctx, "reduce_slices", 2);
    e = launch_reduce_slices(re_out, plan.splits, plane, plane, d_out, ctx->stream);
    if (e == cudaSuccess) e = launch_reduce_slices(im_out, plan.splits, plane, plane, d_out + plane, ctx->stream);
    return cuda_status(e);
}

// The exact spherical wave (Eq. 1): prep with the piston and the spherical
// constants, the spherical kernel over point chunks, then the chunk reduction.
// planes = 1: the amplitude hologram at d_out; 2: the complex wave (real part
// at d_out, imaginary part at d_out + W H).
int run_spherical(cgh_ctx *ctx, int width, int height, double pitch, double lambda, const float *d_xyz,
                  const float *d_amp, int64_t n, int planes, float *d_out)
{
    const int64_t n_pad = padded_points(n);
    const int64_t n_ptiles = n_pad / kPointTile;
    const DirectShape shapes[3] = {spherical_shape(planes, 0), spherical_shape(planes, 1), spherical_shape(planes, 2)};
    const DirectLayout lay = choose_layout(shapes, 3, width, height, n_ptiles, ctx->num_sms, ctx->point_split);
    const DirectShape sh = lay.shape;
    const int split = lay.split;
    const int64_t plane = (int64_t)width * height;
    const size_t geo_bytes = align_up((size_t)n_pad * sizeof(int4), 256);
    const size_t aux_bytes = align_up((size_t)n_pad * sizeof(uint2), 256);
    const size_t ext_bytes = align_up((size_t)n_pad * sizeof(float4), 256);
    const size_t part_bytes = split > 1 ? (size_t)split * planes * plane * sizeof(float) : 0;
    int rc = ensure(ctx, &ctx->ws, &ctx->ws_bytes, geo_bytes + aux_bytes + ext_bytes + part_bytes);
    if (rc) return rc;
    char *base = static_cast<char *>(ctx->ws);
    int4 *geo = reinterpret_cast<int4 *>(base);
    uint2 *aux = reinterpret_cast<uint2 *>(base + geo_bytes);
    float4 *ext = reinterpret_cast<float4 *>(base + geo_bytes + aux_bytes);
    float *parts = reinterpret_cast<float *>(base + geo_bytes + aux_bytes + ext_bytes);
    cudaError_t e;
    {
        ProfileScope ps(ctx, "prep_points", 1);
        e = launch_prep_points(d_xyz, d_amp, (int)n, (int)n_pad, pitch, lambda, geo, aux, ctx->d_status, nullptr,
                               ctx->stream, kAuxPiston, ext, width, height, sph_tile_cols(planes),
                               sph_tile_rows(planes));
    }
    if (e != cudaSuccess) return cuda_status(e);
    {
        ProfileScope ps(ctx, planes == 2 ? "spherical_wave" : "spherical", 1);
        e = launch_spherical(sh, geo, aux, ext, (int)n_pad, width, height, split, planes, split > 1 ? parts : d_out,
                             (int64_t)planes * plane, plane, phase_ref(ctx), ctx->stream);
    }
    if (e != cudaSuccess || split == 1) return cuda_status(e);
    ProfileScope ps(ctx, "reduce_slices", planes);
    for (int c = 0; c < planes && e == cudaSuccess; ++c)
        e = launch_reduce_slices(parts + c * plane, split, plane, (int64_t)planes * plane, d_out + c * plane,
                                 ctx->stream);
    return cuda_status(e);
}

// Fresnel diffraction state of the context, made on first use: the own FFT's
// grid (Ly x Lx, powers of two), its twiddle tables, the padded work plane and
// the chirp's spectrum; for grids beyond its lengths, a cuFFT plan of 2H x 2W.
int ensure_fft(cgh_ctx *ctx)
{
    if (ctx->fft_ready) return CGH_OK;
    const FftGrid g = fft_grid(ctx->height, ctx->width);
    const size_t words = g.ok ? (size_t)g.Ly * g.Lx : (size_t)4 * ctx->width * ctx->height;
    auto fail = [&](int rc) {
        cudaGetLastError();
        for (float2 **p : {&ctx->fft_pad, &ctx->fft_spec, &ctx->fft_twx, &ctx->fft_twy})
            if (*p) {
                cudaFree(*p);
                *p = nullptr;
            }
        return rc;
    };
    if (cudaMalloc(&ctx->fft_pad, words * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&ctx->fft_spec, words * sizeof(float2)) != cudaSuccess)
        return fail(CGH_ENOMEM);
    if (g.ok) {
        // e^{-2 pi i k / L} in double, rounded once
        for (int pass = 0; pass < 2; ++pass) {
            const int L = pass == 0 ? g.Lx : g.Ly;
            float2 **dst = pass == 0 ? &ctx->fft_twx : &ctx->fft_twy;
            std::vector<float2> t((size_t)L);
            for (int k = 0; k < L; ++k) {
                const double a = -2.0 * 3.14159265358979323846 * (double)k / (double)L;
                t[(size_t)k] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
            if (cudaMalloc(dst, (size_t)L * sizeof(float2)) != cudaSuccess) return fail(CGH_ENOMEM);
            if (cudaMemcpy(*dst, t.data(), (size_t)L * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(CGH_ECUDA);
        }
    } else if (!fft_plan_2d(2 * ctx->height, 2 * ctx->width, &ctx->fft_plan, ctx->stream)) {
        ctx->fft_plan = nullptr;
        return fail(CGH_ECUDA);
    }
    ctx->fft_g = g;
    ctx->fft_spec_z = 0.0;
    ctx->fft_ready = true;
    return CGH_OK;
}

// Fresnel diffraction by z into d_out ([2][H][W]) of the input planes in, or
// (in == nullptr) of the plane already in the work plane (rows < H, columns
// < W).  The chirp's spectrum carries the prefactor exp(i 2 pi z / lambda) /
// (i lambda z) p^2 and the inverse transform's 1 / (grid size); it is kept for
// the next call with the same z.
int fresnel_run(cgh_ctx *ctx, double z, const float *in, float *d_out)
{
    const int H = ctx->height, W = ctx->width;
    const FftGrid &g = ctx->fft_g;
    const double cells = g.ok ? (double)g.Ly * g.Lx : 4.0 * H * W;
    cudaError_t e = cudaSuccess;
    if (ctx->fft_spec_z != z) {
        const double zt = z / ctx->lambda;
        const double a0 = 6.283185307179586476925286766559 * (zt - std::rint(zt));
        const double s = ctx->pitch * ctx->pitch / (ctx->lambda * z) / cells;
        const unsigned long long C = turns_fixed64(ctx->pitch * ctx->pitch / (2.0 * ctx->lambda * z));
        if (g.ok) {
            ProfileScope ps(ctx, "fresnel_spectrum", 5);
            e = launch_fft_chirp_spectrum(g, ctx->fft_spec, C, s * std::sin(a0), -s * std::cos(a0), ctx->fft_twx,
                                          ctx->fft_twy, ctx->stream);
        } else {
            {
                ProfileScope ps(ctx, "fresnel_chirp", 1);
                e = launch_chirp(ctx->fft_spec, H, W, C, s * std::sin(a0), -s * std::cos(a0), ctx->stream);
            }
            if (e == cudaSuccess && !fft_exec(ctx->fft_plan, ctx->fft_spec, false, ctx->stream)) return CGH_ECUDA;
        }
        if (e != cudaSuccess) return cuda_status(e);
        ctx->fft_spec_z = z;
    }
    if (g.ok) {
        ProfileScope ps(ctx, "fresnel_fft", 5);
        return cuda_status(launch_fft_convolve(g, in, H, W, ctx->fft_pad, ctx->fft_spec, ctx->fft_twx, ctx->fft_twy,
                                               d_out, ctx->stream));
    }
    if (in != nullptr) {
        ProfileScope ps(ctx, "fresnel_expand", 1);
        e = launch_expand(in, H, W, ctx->fft_pad, ctx->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    {
        ProfileScope ps(ctx, "cufft_c2c", 1);
        if (!fft_exec(ctx->fft_plan, ctx->fft_pad, false, ctx->stream)) return CGH_ECUDA;
    }
    {
        ProfileScope ps(ctx, "fresnel_mul", 1);
        e = launch_cmul(ctx->fft_pad, ctx->fft_spec, 4ll * H * W, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_status(e);
    {
        ProfileScope ps(ctx, "cufft_c2c", 1);
        if (!fft_exec(ctx->fft_plan, ctx->fft_pad, true, ctx->stream)) return CGH_ECUDA;
    }
    ProfileScope ps(ctx, "fresnel_crop", 1);
    return cuda_status(launch_crop(ctx->fft_pad, H, W, d_out, ctx->stream));
}

// Largest band-list workspace of the WRP record (points x bands x 4 bytes).
constexpr size_t kMaxBandListBytes = (size_t)1 << 30;

// WRP step 1 into the padded work plane (pad, zeroed first) or into planes.
int wrp_record(cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n, double z_wrp, float2 *pad,
               float *planes)
{
    const int64_t n_pad = padded_points(n);
    const size_t geo_bytes = align_up((size_t)n_pad * sizeof(int4), 256);
    const size_t win_bytes = align_up((size_t)n_pad * sizeof(uint4), 256);
    // band lists hold at most every point in every band; beyond kMaxBandListBytes the tiles walk all points
    const int bands = (ctx->height + 31) / 32;
    const int cells = wrp_band_cells(ctx->height, (int)n_pad);
    const size_t list_bytes = (size_t)n_pad * bands * sizeof(int);
    const bool binned = list_bytes <= kMaxBandListBytes;
    const size_t band_bytes = binned ? align_up((size_t)(2 * cells + 1) * sizeof(int), 256) + list_bytes : 0;
    int rc = ensure(ctx, &ctx->ws, &ctx->ws_bytes, geo_bytes + win_bytes + band_bytes);
    if (rc) return rc;
    int4 *geo = reinterpret_cast<int4 *>(ctx->ws);
    uint4 *win = reinterpret_cast<uint4 *>(static_cast<char *>(ctx->ws) + geo_bytes);
    int *count = reinterpret_cast<int *>(static_cast<char *>(ctx->ws) + geo_bytes + win_bytes);
    int *offset = count + cells;
    int *list = binned ? reinterpret_cast<int *>(reinterpret_cast<char *>(count) +
                                                 align_up((size_t)(2 * cells + 1) * sizeof(int), 256))
                       : nullptr;
    cudaError_t e;
    {
        ProfileScope ps(ctx, "wrp_prep", 1);
        e = launch_wrp_prep(d_xyz, d_amp, (int)n, (int)n_pad, ctx->pitch, ctx->lambda, z_wrp, piston_on(ctx), geo, win,
                            ctx->d_status, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_status(e);
    // the own FFT reads only the rows < H, columns < W of the work plane; the cuFFT path reads all of it
    const bool own = ctx->fft_g.ok;
    if (pad != nullptr && !own) {
        e = cudaMemsetAsync(pad, 0, (size_t)4 * ctx->width * ctx->height * sizeof(float2), ctx->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    const int64_t pad_ld = own ? ctx->fft_g.Lx : 2 * ctx->width;
    if (binned) {
        ProfileScope ps(ctx, "wrp_bands", 3);
        e = launch_wrp_bands(geo, win, (int)n_pad, ctx->height, count, offset, list, ctx->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    ProfileScope ps(ctx, "wrp_record", 1);
    return cuda_status(launch_wrp_record(geo, win, (int)n_pad, ctx->height, ctx->width, offset, list, pad, pad_ld,
                                         planes, ctx->stream));
}

int resolve_form(cgh_ctx *ctx, int width, int height, int64_t n)
{
    if (ctx->phase_model == CGH_PHASE_SPHERICAL)   // one form computes Eq. 1
        return (ctx->form == CGH_FORM_AUTO || ctx->form == CGH_DIRECT_SFU) ? CGH_DIRECT_SFU : -1;
    if (ctx->form != CGH_FORM_AUTO) return ctx->form;
    return tune_choose_form(ctx, width, height, n, (double)ctx->tol_e9 * 1e-9);
}

int compute_hologram(cgh_ctx *ctx, int width, int height, double pitch, double lambda, const float *d_xyz,
                     const float *d_amp, int64_t n, float *d_out)
{
    if (n == 0) return cuda_status(cudaMemsetAsync(d_out, 0, (size_t)width * height * sizeof(float), ctx->stream));
    const int form = resolve_form(ctx, width, height, n);
    if (ctx->phase_model == CGH_PHASE_SPHERICAL)
        return form == CGH_DIRECT_SFU ? run_spherical(ctx, width, height, pitch, lambda, d_xyz, d_amp, n, 1, d_out)
                                      : CGH_ENOTSUP;
    switch (form) {
    case CGH_DIRECT_SFU:
        return run_direct(ctx, true, width, height, pitch, lambda, d_xyz, d_amp, n, d_out);
    case CGH_DIRECT_ACCURATE:
        return run_direct(ctx, false, width, height, pitch, lambda, d_xyz, d_amp, n, d_out);
    case CGH_GEMM_F16:
    case CGH_GEMM_BF16:
    case CGH_GEMM_SPLIT16:
        return run_gemm(ctx, form, width, height, pitch, lambda, d_xyz, d_amp, n, d_out);
    default:
        return CGH_ENOTSUP;
    }
}

}  // namespace cgh

extern "C" {

int cgh_abi_version(void)
{
    return CGH_ABI_VERSION;
}

const char *cgh_status_string(int status)
{
    switch (status) {
    case CGH_OK: return "ok";
    case CGH_EINVAL: return "invalid argument";
    case CGH_ENOMEM: return "device memory allocation failed";
    case CGH_ECUDA: return "CUDA error or no usable CUDA device";
    case CGH_ETIMEOUT: return "bounded wait ran out";
    case CGH_EINPUT: return "invalid point data (z <= 0, NaN, or non-integer / out-of-range x, y)";
    case CGH_ENOTSUP: return "form or option not supported for this problem";
    case CGH_EBOUNDS: return "a bounds check of the debug build failed";
    default: return "unknown status";
    }
}

int cgh_create(int width, int height, double pitch_m, double lambda_m, cgh_ctx **out)
{
    if (!out) return CGH_EINVAL;
    *out = nullptr;
    if (!valid_size(width, height) || !finite_positive(pitch_m) || !finite_positive(lambda_m)) return CGH_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CGH_ECUDA;
    }
    int major = 0, minor = 0, sms = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return CGH_ECUDA;
    }
    if (major != 10 || minor != 3) return CGH_ECUDA;   // the kernels are built for sm_103a only
    cgh_ctx *ctx = new (std::nothrow) cgh_ctx();
    if (!ctx) return CGH_ENOMEM;
    ctx->width = width;
    ctx->height = height;
    ctx->pitch = pitch_m;
    ctx->lambda = lambda_m;
    ctx->device = dev;
    ctx->num_sms = sms;
    if (cudaMalloc(&ctx->d_status, 4 * sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, 4 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_status) cudaFree(ctx->d_status);
        delete ctx;
        return CGH_ENOMEM;
    }
    *out = ctx;
    return CGH_OK;
}

int cgh_destroy(cgh_ctx *ctx)
{
    if (!ctx) return CGH_OK;
    DeviceGuard g(ctx->device);
    int rc = cgh_sync(ctx);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->pws) cudaFree(ctx->pws);
    for (float2 *p : {ctx->fft_pad, ctx->fft_spec, ctx->fft_twx, ctx->fft_twy})
        if (p) cudaFree(p);
    fft_plan_destroy(ctx->fft_plan);
    if (ctx->h_meta) cudaFreeHost(ctx->h_meta);
    if (ctx->io) cudaFree(ctx->io);
    if (ctx->d_status) cudaFree(ctx->d_status);
    for (auto &p : ctx->pending) {
        cudaEventDestroy(p.start);
        cudaEventDestroy(p.stop);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
    for (cudaEvent_t ev : {ctx->ev_ready, ctx->ev_fact[0], ctx->ev_fact[1], ctx->ev_gemm[0], ctx->ev_gemm[1]})
        if (ev) cudaEventDestroy(ev);
    destroy_batch_plan(ctx->batch);
    destroy_batch_plan(ctx->single);
    destroy_tune_state(ctx->tune);
    delete ctx;
    return rc == CGH_ETIMEOUT ? rc : CGH_OK;
}

int cgh_set_stream(cgh_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return CGH_EINVAL;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return CGH_OK;
}

int cgh_set_form(cgh_ctx *ctx, int form)
{
    if (!ctx || form < CGH_FORM_AUTO || form > CGH_GEMM_SPLIT16) return CGH_EINVAL;
    ctx->form = form;
    return CGH_OK;
}

int cgh_measure_mufu(cgh_ctx *ctx, double *results_per_s)
{
    if (!ctx || !results_per_s) return CGH_EINVAL;
    DeviceGuard g(ctx->device);
    const double r = measure_mufu_rate(ctx->num_sms, ctx->stream);
    if (!(r > 0.0)) return CGH_ECUDA;
    *results_per_s = r;
    return CGH_OK;
}

int cgh_set_reference(cgh_ctx *ctx, double sin_x, double sin_y, double phase0_rad)
{
    if (!ctx || !std::isfinite(sin_x) || !std::isfinite(sin_y) || !std::isfinite(phase0_rad)) return CGH_EINVAL;
    if (std::fabs(sin_x) > 1.0 || std::fabs(sin_y) > 1.0 || std::fabs(phase0_rad) > 1e6) return CGH_EINVAL;
    ctx->ref_sx = sin_x;
    ctx->ref_sy = sin_y;
    ctx->ref_phase0 = phase0_rad;
    return CGH_OK;
}

int cgh_set_option(cgh_ctx *ctx, int key, int64_t value)
{
    if (!ctx) return CGH_EINVAL;
    switch (key) {
    case CGH_OPT_TIMEOUT_MS:
        if (value < 1 || value > 3600000) return CGH_EINVAL;
        ctx->timeout_ms = value;
        return CGH_OK;
    case CGH_OPT_POINT_SPLIT:
        if (value < 0 || value > 4096) return CGH_EINVAL;
        ctx->point_split = (int)value;
        return CGH_OK;
    case CGH_OPT_GEMM_SPLITK:
        if (value < 0 || value > 64) return CGH_EINVAL;
        ctx->gemm_splitk = (int)value;
        return CGH_OK;
    case CGH_OPT_GEMM_BN:
        if (value != 0 && !gemm_bn_supported((int)value)) return CGH_EINVAL;
        ctx->gemm_bn = (int)value;
        return CGH_OK;
    case CGH_OPT_TOLERANCE_E9:
        if (value < 1) return CGH_EINVAL;
        ctx->tol_e9 = value;
        return CGH_OK;
    case CGH_OPT_GEMM_CHUNK:
        if (value < 0 || value > (1 << 24)) return CGH_EINVAL;
        ctx->gemm_chunk = (int)value;
        return CGH_OK;
    case CGH_OPT_TEST_DROP_TILE:
        if (value < -1 || value > 0x7fffffff) return CGH_EINVAL;
        ctx->drop_tile = (int)value;
        return CGH_OK;
    case CGH_OPT_FACTOR_BUDGET_MB:
        if (value < 1 || value > (1 << 22)) return CGH_EINVAL;
        ctx->factor_budget_mb = value;
        return CGH_OK;
    case CGH_OPT_GEMM_TRANSPOSE:
        if (value < 0 || value > 2) return CGH_EINVAL;
        ctx->gemm_trans = (int)value;
        return CGH_OK;
    case CGH_OPT_GEMM_PIPELINE:
        if (value < 1 || value > 64) return CGH_EINVAL;
        ctx->gemm_pipeline = (int)value;
        return CGH_OK;
    case CGH_OPT_GEMM_GROUP:
        if (value < 0 || value > 2) return CGH_EINVAL;
        ctx->gemm_group = (int)value;
        return CGH_OK;
    case CGH_OPT_PHASE_MODEL:
        if (value != CGH_PHASE_FRESNEL && value != CGH_PHASE_FRESNEL_PISTON && value != CGH_PHASE_SPHERICAL)
            return CGH_EINVAL;
        ctx->phase_model = (int)value;
        return CGH_OK;
    case CGH_OPT_DIRECT_CTAS:
        if (value < 0 || value > (1 << 24)) return CGH_EINVAL;
        ctx->direct_ctas = (int)value;
        return CGH_OK;
    case CGH_OPT_BATCH_MODE:
        if (value != 0 && value != 1) return CGH_EINVAL;
        ctx->batch_mode = (int)value;
        return CGH_OK;
    case CGH_OPT_BATCH_OVERLAP:
        if (value != 0 && value != 1) return CGH_EINVAL;
        ctx->batch_overlap = (int)value;
        return CGH_OK;
    case CGH_OPT_TEST_ALLOC_FAIL:
        if (value < 0 || value > 1000) return CGH_EINVAL;
        ctx->test_alloc_fail = (int)value;
        return CGH_OK;
    case CGH_OPT_DIRECT_SHAPE:
        if (value < 0 || value > 6) return CGH_EINVAL;
        ctx->direct_shape = (int)value;
        return CGH_OK;
    case CGH_OPT_GEMM_PERSISTENT:
        if (value != 0 && value != 1) return CGH_EINVAL;
        ctx->gemm_persistent = (int)value;
        return CGH_OK;
    case CGH_OPT_GEMM_PAIR:
        if (value < 0 || value > 2) return CGH_EINVAL;
        ctx->gemm_pair = (int)value;
        return CGH_OK;
    case CGH_OPT_BATCH_CHUNK_MB:
        if (value < 0 || value > (1 << 20)) return CGH_EINVAL;
        ctx->batch_chunk_mb = (int)value;
        return CGH_OK;
    case CGH_OPT_BATCH_PREMADE_PCT:
        if (value < 0 || value > 100) return CGH_EINVAL;
        ctx->batch_premade_pct = (int)value;
        return CGH_OK;
    case CGH_OPT_PROFILE:
        if (value != 0 && value != 1) return CGH_EINVAL;
        ctx->profile = value == 1;
        return CGH_OK;
    default:
        return CGH_EINVAL;
    }
}

int cgh_point_cloud(cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n_points, float *d_out)
{
    if (!ctx || !d_out || n_points < 0 || n_points > 0x7fffffffll) return CGH_EINVAL;
    if (n_points > 0 && (!d_xyz || !d_amp)) return CGH_EINVAL;
    DeviceGuard g(ctx->device);
    return compute_hologram(ctx, ctx->width, ctx->height, ctx->pitch, ctx->lambda, d_xyz, d_amp, n_points, d_out);
}

int cgh_point_cloud_host(cgh_ctx *ctx, const float *h_xyz, const float *h_amp, int64_t n_points, float *h_out)
{
    if (!ctx || !h_out || n_points < 0 || n_points > 0x7fffffffll) return CGH_EINVAL;
    if (n_points > 0 && (!h_xyz || !h_amp)) return CGH_EINVAL;
    DeviceGuard g(ctx->device);
    const size_t xyz_b = align_up((size_t)n_points * 3 * sizeof(float), 256);
    const size_t amp_b = align_up((size_t)n_points * sizeof(float), 256);
    const size_t out_b = (size_t)ctx->width * ctx->height * sizeof(float);
    int rc = ensure(ctx, &ctx->io, &ctx->io_bytes, xyz_b + amp_b + out_b);
    if (rc) return rc;
    char *base = static_cast<char *>(ctx->io);
    float *d_xyz = reinterpret_cast<float *>(base);
    float *d_amp = reinterpret_cast<float *>(base + xyz_b);
    float *d_out = reinterpret_cast<float *>(base + xyz_b + amp_b);
    if (n_points > 0) {
        if (cudaMemcpyAsync(d_xyz, h_xyz, (size_t)n_points * 3 * sizeof(float), cudaMemcpyHostToDevice,
                            ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(d_amp, h_amp, (size_t)n_points * sizeof(float), cudaMemcpyHostToDevice, ctx->stream) !=
                cudaSuccess)
            return cuda_status(cudaGetLastError());
    }
    rc = compute_hologram(ctx, ctx->width, ctx->height, ctx->pitch, ctx->lambda, d_xyz, d_amp, n_points, d_out);
    if (rc) return rc;
    if (cudaMemcpyAsync(h_out, d_out, out_b, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        return cuda_status(cudaGetLastError());
    return cgh_sync(ctx);
}

int cgh_factors(cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n_points, int dtype_form, void *d_p,
                void *d_q, int64_t ld)
{
    if (!ctx || !d_p || !d_q || n_points < 0 || n_points > 0x3fffffffll) return CGH_EINVAL;
    if (n_points > 0 && (!d_xyz || !d_amp)) return CGH_EINVAL;
    if (dtype_form != CGH_GEMM_F16 && dtype_form != CGH_GEMM_BF16 && dtype_form != CGH_GEMM_SPLIT16)
        return CGH_EINVAL;
    if (ld < 2 * n_points || ld % 64 != 0 || ld <= 0) return CGH_EINVAL;
    if ((uintptr_t)d_p % 16 != 0 || (uintptr_t)d_q % 16 != 0) return CGH_EINVAL;
    DeviceGuard g(ctx->device);
    const int64_t n_pad = padded_points(n_points);
    const size_t geo_bytes = align_up((size_t)n_pad * sizeof(int4), 256);
    const size_t aux_bytes = align_up((size_t)n_pad * sizeof(uint2), 256);
    int rc = ensure(ctx, &ctx->ws, &ctx->ws_bytes, geo_bytes + aux_bytes + 256);
    if (rc) return rc;
    char *base = static_cast<char *>(ctx->ws);
    int4 *geo = reinterpret_cast<int4 *>(base);
    uint2 *aux = reinterpret_cast<uint2 *>(base + geo_bytes);
    cudaError_t e;
    {
        ProfileScope ps(ctx, "prep_points", 1);
        e = launch_prep_points(d_xyz, d_amp, (int)n_points, (int)n_pad, ctx->pitch, ctx->lambda, geo, aux,
                               ctx->d_status, nullptr, ctx->stream, aux_mode(ctx));
    }
    if (e != cudaSuccess) return cuda_status(e);
    ProfileScope ps(ctx, "factors", 1);
    return cuda_status(launch_factors(factor_mode(dtype_form), geo, aux, (int)n_points, ctx->height, ctx->width,
                                      d_p, d_q, ld, nullptr, ctx->stream, false, phase_ref(ctx)));
}

int cgh_batch(cgh_ctx *ctx, const cgh_instance *inst, int n_inst)
{
    if (!ctx || n_inst < 0 || (n_inst > 0 && !inst)) return CGH_EINVAL;
    for (int i = 0; i < n_inst; ++i) {
        const cgh_instance &b = inst[i];
        if (!valid_size(b.width, b.height) || !finite_positive(b.pitch_m) || !finite_positive(b.lambda_m) ||
            !b.d_out || b.n_points < 0 || b.n_points > 0x3fffffffll || (b.n_points > 0 && (!b.d_xyz || !b.d_amp)))
            return CGH_EINVAL;
    }
    if (ctx->phase_model != CGH_PHASE_FRESNEL || phase_ref(ctx).any()) return CGH_ENOTSUP;
    if (n_inst == 0) return CGH_OK;
    DeviceGuard g(ctx->device);
    return run_batch(ctx, inst, n_inst);
}

int cgh_batch_forms(cgh_ctx *ctx, int *forms, int max_entries, int *n_entries)
{
    if (!ctx || !n_entries || max_entries < 0 || (max_entries > 0 && !forms)) return CGH_EINVAL;
    *n_entries = batch_forms(ctx, forms, max_entries);
    return CGH_OK;
}

int cgh_autotune(cgh_ctx *ctx, int force)
{
    if (!ctx) return CGH_EINVAL;
    DeviceGuard g(ctx->device);
    return tune_calibrate(ctx, force != 0);
}

int cgh_wave(cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n_points, float *d_out)
{
    if (!ctx || !d_out || n_points < 0 || n_points > 0x7fffffffll) return CGH_EINVAL;
    if (n_points > 0 && (!d_xyz || !d_amp)) return CGH_EINVAL;
    DeviceGuard g(ctx->device);
    const int64_t plane = (int64_t)ctx->width * ctx->height;
    if (n_points == 0) return cuda_status(cudaMemsetAsync(d_out, 0, (size_t)2 * plane * sizeof(float), ctx->stream));
    int form = resolve_form(ctx, ctx->width, ctx->height, n_points);
    if (ctx->phase_model == CGH_PHASE_SPHERICAL)
        return form == CGH_DIRECT_SFU ? run_spherical(ctx, ctx->width, ctx->height, ctx->pitch, ctx->lambda, d_xyz,
                                                      d_amp, n_points, 2, d_out)
                                      : CGH_ENOTSUP;
    if (form == CGH_DIRECT_ACCURATE) {
        if (ctx->form == CGH_DIRECT_ACCURATE) return CGH_ENOTSUP;
        form = CGH_DIRECT_SFU;   // the automatic choice falls back to the other FP32 form
    }
    return run_wave(ctx, form, d_xyz, d_amp, n_points, d_out);
}

int cgh_fresnel(cgh_ctx *ctx, const float *d_in, double z_m, float *d_out)
{
    if (!ctx || !d_in || !d_out || !std::isfinite(z_m) || z_m == 0.0) return CGH_EINVAL;
    DeviceGuard g(ctx->device);
    int rc = ensure_fft(ctx);
    if (rc) return rc;
    return fresnel_run(ctx, z_m, d_in, d_out);
}

static int wrp_args(const cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n, double z_wrp,
                    const float *d_out)
{
    if (!ctx || !d_out || n < 0 || n > 0x7fffff00ll || !std::isfinite(z_wrp) || !(z_wrp > 0.0)) return CGH_EINVAL;
    if (n > 0 && (!d_xyz || !d_amp)) return CGH_EINVAL;
    if (ctx->phase_model == CGH_PHASE_SPHERICAL || phase_ref(ctx).reference()) return CGH_ENOTSUP;
    return CGH_OK;
}

int cgh_wrp_record(cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n_points, double z_wrp_m,
                   float *d_plane)
{
    int rc = wrp_args(ctx, d_xyz, d_amp, n_points, z_wrp_m, d_plane);
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    return wrp_record(ctx, d_xyz, d_amp, n_points, z_wrp_m, nullptr, d_plane);
}

int cgh_wrp(cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n_points, double z_wrp_m, float *d_out)
{
    int rc = wrp_args(ctx, d_xyz, d_amp, n_points, z_wrp_m, d_out);
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    rc = ensure_fft(ctx);
    if (rc) return rc;
    rc = wrp_record(ctx, d_xyz, d_amp, n_points, z_wrp_m, ctx->fft_pad, nullptr);
    if (rc) return rc;
    return fresnel_run(ctx, z_wrp_m, nullptr, d_out);
}

int cgh_quantize8(cgh_ctx *ctx, const float *d_field, int64_t n, int mode, uint8_t *d_out)
{
    if (!ctx || n < 0 || (n > 0 && (!d_field || !d_out))) return CGH_EINVAL;
    if (mode != CGH_Q_AMPLITUDE_MINMAX && mode != CGH_Q_PHASE) return CGH_EINVAL;
    DeviceGuard g(ctx->device);
    if (mode == CGH_Q_PHASE) {
        ProfileScope ps(ctx, "kinoform8", 1);
        return cuda_status(launch_kinoform8(d_field, d_field + n, n, d_out, ctx->stream));
    }
    ProfileScope ps(ctx, "quantize8", 3);
    return cuda_status(
        launch_quantize8(d_field, n, d_out, reinterpret_cast<uint32_t *>(ctx->d_status + 1), ctx->stream));
}

int cgh_profile_read(cgh_ctx *ctx, cgh_kernel_time *out, int max_entries, int *n_entries, int reset)
{
    if (!ctx || max_entries < 0 || (max_entries > 0 && !out)) return CGH_EINVAL;
    DeviceGuard g(ctx->device);
    if (!ctx->pending.empty()) {
        const auto t0 = std::chrono::steady_clock::now();
        cudaEvent_t last = ctx->pending.back().stop;
        for (;;) {
            cudaError_t q = cudaEventQuery(last);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) return cuda_status(q);
            const auto ms =
                std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
            if (ms.count() > ctx->timeout_ms) return CGH_ETIMEOUT;
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        for (auto &p : ctx->pending) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, p.start, p.stop) != cudaSuccess) {
                cudaGetLastError();
                ms = 0.0f;
            }
            bool found = false;
            for (auto &t : ctx->totals)
                if (t.name == p.name) {
                    t.launches += p.launches;
                    t.ms += ms;
                    found = true;
                    break;
                }
            if (!found) ctx->totals.push_back({p.name, (int64_t)p.launches, (double)ms});
            ctx->event_pool.push_back(p.start);
            ctx->event_pool.push_back(p.stop);
        }
        ctx->pending.clear();
    }
    const int n = (int)ctx->totals.size();
    for (int i = 0; i < n && i < max_entries; ++i) {
        std::memset(out[i].name, 0, sizeof(out[i].name));
        std::strncpy(out[i].name, ctx->totals[i].name.c_str(), sizeof(out[i].name) - 1);
        out[i].launches = ctx->totals[i].launches;
        out[i].total_ms = ctx->totals[i].ms;
    }
    if (n_entries) *n_entries = n;
    if (reset) ctx->totals.clear();
    return CGH_OK;
}

int cgh_sync(cgh_ctx *ctx)
{
    if (!ctx) return CGH_EINVAL;
    DeviceGuard g(ctx->device);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaStreamQuery(ctx->stream);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_status(q);
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
        // the device-side waits give up after timeout_ms; leave them room to report
        if (ms.count() > 2 * ctx->timeout_ms + 1000) return CGH_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    int bits = 0;
    if (cudaMemcpy(&bits, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_status(cudaGetLastError());
    if (bits != 0 && cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) return cuda_status(cudaGetLastError());
    if (bits & kStatusTimeout) return CGH_ETIMEOUT;
    if (bits & kStatusInput) return CGH_EINPUT;
    if (bits & kStatusBounds) return CGH_EBOUNDS;
    return CGH_OK;
}

}  // extern "C"
