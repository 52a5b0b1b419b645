// a7: many holograms per cgh_batch call, captured in a CUDA graph.
//
// The first cgh_batch call with a given set of instances builds a plan: a form
// per instance (the context's form, or the autotuner's choice under the
// tolerance) and, for GEMM instances, a tile width; one device arena for
// every instance's prepared points, factors and the unit tables; and a CUDA
// graph of the batch.  Later calls with the same instances (shapes,
// parameters and buffers) only replay the graph on the context's stream.
//
// Default (CGH_OPT_BATCH_MODE = 0): ONE persistent launch (persist.cu) that
// dequeues every unit of the batch -- point preparation, factor generation,
// direct units on the SIMT warps, GEMM units on the tensor cores -- from two
// global queues, with bounded waits on per-job counters; GEMM jobs are queued
// longest units first.  Mode 1 (kept for comparison): per instance the point
// preparation and factor generation, then one persistent GEMM launch over
// per-CTA unit lists and one persistent direct launch per direct form.
#include <algorithm>
#include <cstring>
#include <vector>

#include "context.h"
#include "tuner.h"

namespace cgh {

struct BatchPlan {
    std::vector<uint64_t> key;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    cudaStream_t capture = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int> forms;
};

void destroy_batch_plan(BatchPlan *p)
{
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->arena) cudaFree(p->arena);
    if (p->capture) cudaStreamDestroy(p->capture);
    delete p;
}

namespace {

uint64_t bits_of(double v)
{
    uint64_t b;
    std::memcpy(&b, &v, sizeof b);
    return b;
}

std::vector<uint64_t> plan_key(const cgh_ctx *ctx, const cgh_instance *inst, int n)
{
    std::vector<uint64_t> k;
    k.reserve(4 + (size_t)n * 8);
    k.push_back((uint64_t)n);
    k.push_back((uint64_t)ctx->form);
    k.push_back((uint64_t)ctx->tol_e9);
    k.push_back(((uint64_t)ctx->gemm_bn << 32) | (uint64_t)(uint32_t)ctx->gemm_chunk);
    k.push_back((uint64_t)ctx->batch_mode | ((uint64_t)ctx->batch_overlap << 8) |
                ((uint64_t)ctx->batch_chunk_mb << 16) | ((uint64_t)(ctx->batch_premade_pct + 1) << 40));
    k.push_back((uint64_t)(uint32_t)ctx->drop_tile);
    for (int i = 0; i < n; ++i) {
        const cgh_instance &b = inst[i];
        k.push_back(((uint64_t)(uint32_t)b.width << 32) | (uint32_t)b.height);
        k.push_back(bits_of(b.pitch_m));
        k.push_back(bits_of(b.lambda_m));
        k.push_back((uint64_t)(uintptr_t)b.d_xyz);
        k.push_back((uint64_t)(uintptr_t)b.d_amp);
        k.push_back((uint64_t)b.n_points);
        k.push_back((uint64_t)(uintptr_t)b.d_out);
    }
    return k;
}

// Greedy assignment: units in the given order, each to the least-loaded CTA.
void assign(const std::vector<int2> &units, const std::vector<double> &cost, int ctas, std::vector<int> &off,
            std::vector<int2> &ordered)
{
    std::vector<std::vector<int2>> per(ctas);
    std::vector<double> load(ctas, 0.0);
    for (size_t i = 0; i < units.size(); ++i) {
        int best = 0;
        for (int c = 1; c < ctas; ++c)
            if (load[c] < load[best]) best = c;
        per[best].push_back(units[i]);
        load[best] += cost[i];
    }
    off.assign(ctas + 1, 0);
    ordered.clear();
    for (int c = 0; c < ctas; ++c) {
        off[c] = (int)ordered.size();
        ordered.insert(ordered.end(), per[c].begin(), per[c].end());
    }
    off[ctas] = (int)ordered.size();
}

struct Layout {
    size_t bytes = 0;
    size_t take(size_t n, size_t align = 256)
    {
        bytes = (bytes + align - 1) / align * align;
        const size_t at = bytes;
        bytes += n;
        return at;
    }
};

constexpr int kSplit16ChunkKbBatch = 8;

// Form (and, for the GEMM forms, tile width) of every instance: the context's form, or the autotuner's choice.
// forced > 0: that form for every instance.
void choose_forms(cgh_ctx *ctx, const cgh_instance *inst, int n, BatchPlan *plan, std::vector<int> &bn,
                  int forced = 0)
{
    const double tol = (double)ctx->tol_e9 * 1e-9;
    plan->forms.assign(n, CGH_DIRECT_SFU);
    bn.assign(n, 256);
    for (int i = 0; i < n; ++i) {
        if (inst[i].n_points == 0) continue;
        const int f = forced > 0 ? forced
                      : ctx->form != CGH_FORM_AUTO
                          ? ctx->form
                          : tune_choose_form(ctx, inst[i].width, inst[i].height, inst[i].n_points, tol);
        plan->forms[i] = f;
        if (f >= CGH_GEMM_F16)
            bn[i] = ctx->gemm_bn > 0 ? ctx->gemm_bn
                                     : (ctx->form == CGH_FORM_AUTO ? tune_choose_bn(ctx, inst[i].width, inst[i].height, f)
                                                                   : choose_gemm_bn(inst[i].width));
    }
}

// (Re)allocates the plan's arena for at least `bytes` (a pending CGH_OPT_TEST_ALLOC_FAIL is taken as a failure).
int ensure_arena(cgh_ctx *ctx, BatchPlan *plan, size_t bytes)
{
    if (bytes <= plan->arena_bytes) return CGH_OK;
    if (ctx->test_alloc_fail > 0) {
        --ctx->test_alloc_fail;
        return CGH_ENOMEM;
    }
    if (plan->arena) {
        cudaFree(plan->arena);
        plan->arena = nullptr;
        plan->arena_bytes = 0;
    }
    if (cudaMalloc(&plan->arena, bytes) != cudaSuccess) {
        cudaGetLastError();
        return CGH_ENOMEM;
    }
    plan->arena_bytes = bytes;
    return CGH_OK;
}

// Ends the capture on the plan's stream and instantiates the graph.
int finish_capture(BatchPlan *plan, cudaError_t e)
{
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(plan->capture, &graph);
    if (e != cudaSuccess || ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return CGH_ECUDA;
    }
    ec = cudaGraphInstantiate(&plan->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) {
        plan->exec = nullptr;
        return cuda_status(ec);
    }
    return CGH_OK;
}

int begin_capture(BatchPlan *plan)
{
    if (!plan->capture && cudaStreamCreateWithFlags(&plan->capture, cudaStreamNonBlocking) != cudaSuccess)
        return cuda_status(cudaGetLastError());
    if (plan->exec) {
        cudaGraphExecDestroy(plan->exec);
        plan->exec = nullptr;
    }
    if (cudaStreamBeginCapture(plan->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return cuda_status(cudaGetLastError());
    return CGH_OK;
}

// The persistent batch's GEMM tile: width 192 or 224 (so that the 224-wide kernel with its five-stage operand ring
// serves every job) and orientation (A = P: 128-row tiles of hologram rows; transposed: of hologram columns), by
// padded area times the relative cost of the width (128-wide tiles measured about 35 % slower per flop at
// 1920x1080, 192-wide 3 %).  A forced CGH_OPT_GEMM_BN / CGH_OPT_GEMM_TRANSPOSE wins.
void choose_persist_tile(const cgh_ctx *ctx, int width, int height, int &bn, bool &trans)
{
    static const int cands[] = {224, 192, 128};
    static const double eff[] = {1.0, 1.03, 1.35};
    double best = 1e300;
    bn = 224;
    trans = false;
    for (int tr = 0; tr < 2; ++tr) {
        if ((ctx->gemm_trans == 1 && tr) || (ctx->gemm_trans == 2 && !tr)) continue;
        const int64_t a_rows = tr ? width : height, b_rows = tr ? height : width;
        for (int c = 0; c < 3; ++c) {
            const int w = ctx->gemm_bn > 0 ? ctx->gemm_bn : cands[c];
            if (ctx->gemm_bn > 0 && c > 0) break;
            const double cost = (double)((a_rows + 127) / 128 * 128) * (double)((b_rows + w - 1) / w * w) *
                                (ctx->gemm_bn > 0 ? 1.0 : eff[c]);
            if (cost < best * (1.0 - 1e-9)) {
                best = cost;
                bn = w;
                trans = tr != 0;
            }
        }
    }
}

// K chunks of the persistent batch's GEMM units.  A unit is one tile over one K chunk, and its producer streams
// the k-blocks behind the factor generation (it waits for the factors of each k-block).  Where the batch has tiles
// enough for the CTAs, a chunk's operands (both factors, all planes) take about kBatchChunkMb: the CTAs on one
// hologram then sweep a K range that L2 holds, and one hologram's chunks follow each other closely (measured on
// the 64-frame video batch: 32 / 64 / 128 / 256 / 512 MB and the whole K gave 119 / 111 / 103 / 104 / 107 / 107 ms
// at NRMS 1e-5 and 52 / 37.4 / 36.1 / 36.1 / 36.9 / 39.8 ms at 2e-3).  Otherwise K is cut into chunks by the
// rounds model of the one-hologram GEMM (rounds of units over this job's share of the CTAs, times k-blocks per
// unit, each extra chunk 1 % slower).  The chunks of a tile add to the output in K order.
constexpr int kBatchChunkMb = 128;
constexpr int kBatchPremadePct = 0;   // share of the batch's factor bytes made before the persistent launch

static int persist_kchunks(int64_t tiles, int64_t total_tiles, int64_t nkb, int step, int ctas)
{
    if (total_tiles >= 2 * (int64_t)ctas) return 1;
    const double share = (double)ctas * (double)tiles / (double)total_tiles;   // this job's CTAs
    int best = 1;
    double best_t = 1e300;
    for (int s = 1; s <= 16 && (int64_t)s * step <= nkb; ++s) {
        const int64_t kcs = ((nkb + s - 1) / s + step - 1) / step * step;
        const int64_t chunks = (nkb + kcs - 1) / kcs;
        const double rounds = std::ceil((double)(tiles * chunks) / std::max(1.0, share));
        const double t = rounds * (double)kcs * (1.0 + 0.01 * (double)(chunks - 1));
        if (t < best_t * (1.0 - 1e-9)) {
            best_t = t;
            best = s;
        }
    }
    return best;
}

constexpr int kDirectChunkPoints = 2048;   // points per direct unit of the persistent batch (at most 64 chunks)
constexpr int kDirectMaxChunks = 64;

// The persistent plan: one job per instance with points, the SIMT and GEMM unit queues, and a graph of
// (memset of the counters, memsets of the empty instances' outputs, ONE persistent launch).
int build_plan_persist(cgh_ctx *ctx, const cgh_instance *inst, int n, BatchPlan *plan, int forced_form = 0)
{
    std::vector<int> bn;
    choose_forms(ctx, inst, n, plan, bn, forced_form);
    const int rows_f = persist_factor_rows(), pts_f = persist_factor_points();
    const int dtw = persist_direct_tile_w(), dth = persist_direct_tile_h();
    constexpr int kQ4NT = 8 * 256;   // float4s of one direct tile's totals
    std::vector<int> job_of(n, -1), inst_of;
    for (int i = 0; i < n; ++i)
        if (inst[i].n_points > 0) {
            job_of[i] = (int)inst_of.size();
            inst_of.push_back(i);
        }
    const int nj = (int)inst_of.size();
    std::vector<PersistJob> jobs(nj);
    std::vector<char> jtrans(nj, 0);
    std::vector<int64_t> jtiles(nj, 0);
    int64_t total_tiles = 0;
    for (int j = 0; j < nj; ++j) {
        const int i = inst_of[j];
        if (plan->forms[i] < CGH_GEMM_F16) continue;
        bool tr = false;
        choose_persist_tile(ctx, inst[i].width, inst[i].height, bn[i], tr);
        jtrans[j] = tr ? 1 : 0;
        const int a_rows = tr ? inst[i].width : inst[i].height, b_rows = tr ? inst[i].height : inst[i].width;
        jtiles[j] = (int64_t)((a_rows + 127) / 128) * ((b_rows + bn[i] - 1) / bn[i]);
        total_tiles += jtiles[j];
    }
    const int gctas_max = gemm_max_ctas(ctx->num_sms);
    // arena: the zeroed counters first (one memset), then per-job buffers, then the tables
    Layout L;
    const size_t z_heads = L.take(64 * sizeof(int));
    const size_t z_prep = L.take((size_t)nj * sizeof(int));
    const size_t z_fact = L.take((size_t)nj * sizeof(int));
    const size_t z_amax = L.take((size_t)nj * sizeof(float));
    std::vector<size_t> z_count(nj, 0), z_chunk(nj, 0), o_geo(nj), o_aux(nj), o_p(nj, 0), o_q(nj, 0),
        o_parts(nj, 0);
    std::vector<int64_t> work(nj, 0);
    int bn_max = 0;
    for (int j = 0; j < nj; ++j) {
        const cgh_instance &b = inst[inst_of[j]];
        PersistJob &J = jobs[j];
        std::memset(&J, 0, sizeof J);
        J.form = plan->forms[inst_of[j]];
        J.n = (int)b.n_points;
        J.n_pad = (int)padded_points(b.n_points);
        J.width = b.width;
        J.height = b.height;
        if (J.form >= CGH_GEMM_F16) {
            const int i = inst_of[j];
            const int64_t nkb = (2 * b.n_points + 63) / 64;
            const int kc = J.form == CGH_GEMM_SPLIT16 ? (ctx->gemm_chunk > 0 ? ctx->gemm_chunk : kSplit16ChunkKbBatch)
                                                      : 1;
            // a multiple of the factor units' 32 k-blocks (so a chunk's factors are whole factor groups) and of
            // the TMEM chain kc
            const int gkb = 2 * persist_factor_points() / 64;
            const int step = kc % gkb == 0 ? kc : (gkb % kc == 0 ? gkb : gkb * kc);
            const int s = persist_kchunks(jtiles[j], total_tiles, nkb, step, gctas_max);
            int64_t kcs = ((nkb + s - 1) / s + step - 1) / step * step;
            // chunks of an operand size: pinned, or by default where the batch has tiles enough for the CTAs
            const int chunk_mb = ctx->batch_chunk_mb > 0 ? ctx->batch_chunk_mb
                                                         : (total_tiles >= 2 * (int64_t)gctas_max ? kBatchChunkMb : 0);
            if (chunk_mb > 0) {   // no longer than the split
                const int planes = J.form == CGH_GEMM_SPLIT16 ? 2 : 1;
                const int a_rows = jtrans[j] ? b.width : b.height, b_rows = jtrans[j] ? b.height : b.width;
                const double row_bytes = (double)planes *
                                         (double)((a_rows + 127) / 128 * 128 + (b_rows + bn[i] - 1) / bn[i] * bn[i]) *
                                         128.0;
                const int64_t by = (int64_t)((double)chunk_mb * 1048576.0 / row_bytes) / step * step;
                kcs = std::min(kcs, std::max<int64_t>(step, by));
            }
            J.kchunks = (int)((nkb + kcs - 1) / kcs);
            J.kchunk_kb = (int)kcs;
            if (J.kchunks > 1) z_count[j] = L.take((size_t)jtiles[j] * 4 * sizeof(int));
            const int64_t slots = (2 * b.n_points + 63) / 64 * 32;   // point slots: ld / 2
            z_chunk[j] = L.take((size_t)((slots + pts_f - 1) / pts_f) * sizeof(int));
        } else {
            J.tiles_x = (b.width + dtw - 1) / dtw;
            const int tiles = J.tiles_x * ((b.height + dth - 1) / dth);
            J.chunks = (int)std::min<int64_t>(kDirectMaxChunks,
                                              std::max<int64_t>(1, (b.n_points + kDirectChunkPoints - 1) / kDirectChunkPoints));
            if (J.chunks > 1) z_count[j] = L.take((size_t)tiles * sizeof(int));
        }
    }
    const size_t z_end = L.take(0);
    for (int j = 0; j < nj; ++j) {
        const cgh_instance &b = inst[inst_of[j]];
        PersistJob &J = jobs[j];
        o_geo[j] = L.take((size_t)J.n_pad * sizeof(int4));
        o_aux[j] = L.take((size_t)J.n_pad * sizeof(uint2));
        if (J.form >= CGH_GEMM_F16) {
            const int planes = J.form == CGH_GEMM_SPLIT16 ? 2 : 1;
            J.ld = (2 * b.n_points + 63) / 64 * 64;
            o_p[j] = L.take((size_t)planes * b.height * J.ld * 2);
            o_q[j] = L.take((size_t)planes * b.width * J.ld * 2);
            bn_max = std::max(bn_max, bn[inst_of[j]]);
        } else if (J.chunks > 1) {
            const int tiles = J.tiles_x * ((b.height + dth - 1) / dth);
            o_parts[j] = L.take((size_t)tiles * J.chunks * kQ4NT * sizeof(float4));
        }
    }
    const size_t t_jobs = L.take((size_t)nj * sizeof(PersistJob), 128);
    // units
    std::vector<int4> simt;
    std::vector<int4> gunits;
    std::vector<int> gemm_order, direct_order;
    for (int j = 0; j < nj; ++j) {
        const cgh_instance &b = inst[inst_of[j]];
        const int f = jobs[j].form;
        if (f >= CGH_GEMM_F16) {
            // per-unit cost: k-blocks x passes x tile width (LPT order: the longest units first)
            work[j] = (int64_t)jobs[j].kchunk_kb * (f == CGH_GEMM_SPLIT16 ? 3 : 1) * bn[inst_of[j]];
            gemm_order.push_back(j);
        } else {
            work[j] = (int64_t)((b.n_points + jobs[j].chunks - 1) / jobs[j].chunks);
            direct_order.push_back(j);
        }
    }
    auto by_work = [&](int a, int c) { return work[a] > work[c] || (work[a] == work[c] && a < c); };
    std::sort(gemm_order.begin(), gemm_order.end(), by_work);
    std::sort(direct_order.begin(), direct_order.end(), by_work);
    // The first GEMM jobs in queue order, up to a share of all factor bytes, get their points and factors from
    // the plain kernels before the persistent launch (full occupancy, about three times the rate of the SIMT
    // groups), so the tensor cores start at once and the SIMT groups begin ahead of them on the rest.
    {
        double total = 0.0, done = 0.0;
        for (int j : gemm_order) total += (double)(inst[inst_of[j]].width + inst[inst_of[j]].height) * jobs[j].ld;
        const double share = (ctx->batch_premade_pct >= 0 ? ctx->batch_premade_pct : kBatchPremadePct) / 100.0;
        for (int j : gemm_order) {
            if (done >= share * total) break;
            jobs[j].premade = 1;
            done += (double)(inst[inst_of[j]].width + inst[inst_of[j]].height) * jobs[j].ld;
        }
    }
    for (int j = 0; j < nj; ++j) {
        jobs[j].prep_units = jobs[j].premade ? 0 : jobs[j].n_pad / kPointTile;
        for (int blk = 0; blk < jobs[j].prep_units; ++blk) simt.push_back(make_int4(kPersistPrep, j, blk, 0));
    }
    for (int j : gemm_order) {
        const cgh_instance &b = inst[inst_of[j]];
        const int a_rows = jtrans[j] ? b.width : b.height, b_rows = jtrans[j] ? b.height : b.width;
        const int tiles = ((a_rows + 127) / 128) * ((b_rows + bn[inst_of[j]] - 1) / bn[inst_of[j]]);
        for (int c = 0; c < jobs[j].kchunks; ++c)
            for (int t = 0; t < tiles; ++t) gunits.push_back(make_int4(j, t, c, 0));
    }
    for (int j : gemm_order) {
        const cgh_instance &b = inst[inst_of[j]];
        PersistJob &J = jobs[j];
        J.point_slots = (int)(J.ld / 2);
        const int bands = (b.height + b.width + rows_f - 1) / rows_f;
        const int groups = (J.point_slots + pts_f - 1) / pts_f;
        J.fact_units = J.premade ? 0 : bands * groups;
        J.fact_bands = bands;
        J.fact_groups = groups;
        if (J.premade) continue;
        // in K order within every K chunk, the chunks side by side, so the GEMM units of all chunks find the
        // factors of their first k-blocks first
        const int per_chunk = J.kchunk_kb / (2 * pts_f / 64);   // factor groups of one K chunk
        for (int pos = 0; pos < per_chunk; ++pos)
            for (int c = 0; c < J.kchunks; ++c) {
                const int g = c * per_chunk + pos;
                if (g >= groups) continue;
                for (int band = 0; band < bands; ++band) simt.push_back(make_int4(kPersistFactor, j, band, g));
            }
    }
    for (int j : direct_order) {
        const cgh_instance &b = inst[inst_of[j]];
        const int tiles = jobs[j].tiles_x * ((b.height + dth - 1) / dth);
        for (int t = 0; t < tiles; ++t)
            for (int c = 0; c < jobs[j].chunks; ++c) simt.push_back(make_int4(kPersistDirect, j, t, c));
    }
    if (ctx->drop_tile >= 0 && nj > 0) {
        // test hook: job 0 waits for one unit more than exists, so a bounded wait runs out (kStatusTimeout)
        if (jobs[0].form >= CGH_GEMM_F16) {
            ++jobs[0].fact_units;
            jobs[0].chunk_extra = 1;
        } else {
            ++jobs[0].prep_units;
        }
    }
    const size_t t_simt = L.take(simt.size() * sizeof(int4));
    const size_t t_gemm = L.take(gunits.size() * sizeof(int4));
    int rc = ensure_arena(ctx, plan, L.bytes);
    if (rc) return rc;
    char *A = static_cast<char *>(plan->arena);
    for (int j = 0; j < nj; ++j) {
        const cgh_instance &b = inst[inst_of[j]];
        PersistJob &J = jobs[j];
        J.xyz = b.d_xyz;
        J.amp = b.d_amp;
        J.geo = reinterpret_cast<int4 *>(A + o_geo[j]);
        J.aux = reinterpret_cast<uint2 *>(A + o_aux[j]);
        J.amax = reinterpret_cast<float *>(A + z_amax) + j;
        J.out = b.d_out;
        J.pitch = b.pitch_m;
        J.lambda = b.lambda_m;
        J.vec = (b.width % 4 == 0) && ((uintptr_t)b.d_out % 16 == 0);
        if (J.form >= CGH_GEMM_F16) {
            J.P = reinterpret_cast<uint16_t *>(A + o_p[j]);
            J.Q = reinterpret_cast<uint16_t *>(A + o_q[j]);
            J.plane_p = (long long)b.height * J.ld;
            J.plane_q = (long long)b.width * J.ld;
            const int kc = J.form == CGH_GEMM_SPLIT16 ? (ctx->gemm_chunk > 0 ? ctx->gemm_chunk : kSplit16ChunkKbBatch)
                                                      : ctx->gemm_chunk;
            if (!fill_gemm_job(&J.g, factor_mode(J.form), bn[inst_of[j]], J.P, J.Q, b.height, b.width, J.ld, kc,
                               b.d_out, J.amax, jtrans[j] != 0))
                return CGH_ECUDA;
            if (J.kchunks > 1) J.tile_seq = reinterpret_cast<int *>(A + z_count[j]);
            J.group_done = reinterpret_cast<int *>(A + z_chunk[j]);
        } else if (J.chunks > 1) {
            J.parts = reinterpret_cast<float4 *>(A + o_parts[j]);
            J.tile_count = reinterpret_cast<int *>(A + z_count[j]);
        }
    }
    auto up = [&](size_t at, const void *src, size_t bytes) {
        return bytes == 0 || cudaMemcpy(A + at, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!up(t_jobs, jobs.data(), jobs.size() * sizeof(PersistJob)) || !up(t_simt, simt.data(), simt.size() * sizeof(int4)) ||
        !up(t_gemm, gunits.data(), gunits.size() * sizeof(int4)))
        return cuda_status(cudaGetLastError());
    PersistParams pp;
    pp.jobs = reinterpret_cast<const PersistJob *>(A + t_jobs);
    pp.simt_units = reinterpret_cast<const int4 *>(A + t_simt);
    pp.simt_total = (int)simt.size();
    pp.gemm_units = reinterpret_cast<const int4 *>(A + t_gemm);
    pp.gemm_total = (int)gunits.size();
    pp.n_jobs = nj;
    pp.heads = reinterpret_cast<int *>(A + z_heads);
    pp.prep_done = reinterpret_cast<int *>(A + z_prep);
    pp.fact_done = reinterpret_cast<int *>(A + z_fact);
    pp.fact_all = 0;
    if (ctx->batch_overlap == 0)
        for (int j : gemm_order) pp.fact_all += jobs[j].fact_units;

    rc = begin_capture(plan);
    if (rc) return rc;
    cudaStream_t s = plan->capture;
    cudaError_t e = cudaMemsetAsync(A, 0, z_end, s);
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        if (inst[i].n_points == 0) e = cudaMemsetAsync(inst[i].d_out, 0, (size_t)inst[i].width * inst[i].height * sizeof(float), s);
    for (int j : gemm_order) {
        if (e != cudaSuccess || !jobs[j].premade) continue;
        const cgh_instance &b = inst[inst_of[j]];
        const PersistJob &J = jobs[j];
        e = launch_prep_points(b.d_xyz, b.d_amp, J.n, J.n_pad, b.pitch_m, b.lambda_m, J.geo, J.aux, ctx->d_status,
                               J.amax, s);
        if (e == cudaSuccess)
            e = launch_factors(factor_mode(J.form), J.geo, J.aux, J.n, b.height, b.width, J.P, J.Q, J.ld, J.amax, s);
    }
    if (e == cudaSuccess && nj > 0)
        e = launch_persist(pp, ctx->num_sms, bn_max, ctx->d_status, (uint64_t)ctx->timeout_ms * 1000000ull, s);
    rc = finish_capture(plan, e);
    if (rc) return rc;
    plan->key = plan_key(ctx, inst, n);
    return CGH_OK;
}

int build_plan_kinds(cgh_ctx *ctx, const cgh_instance *inst, int n, BatchPlan *plan)
{
    std::vector<int> bn;
    choose_forms(ctx, inst, n, plan, bn);
    // arena layout
    Layout L;
    struct Off {
        size_t geo, aux, amax, p, q;
        int64_t n_pad, ld;
    };
    std::vector<Off> off(n);
    int n_gemm = 0, n_dsfu = 0, n_dacc = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t np = inst[i].n_points;
        if (np == 0) continue;
        Off &o = off[i];
        o.n_pad = padded_points(np);
        o.geo = L.take((size_t)o.n_pad * sizeof(int4));
        o.aux = L.take((size_t)o.n_pad * sizeof(uint2));
        o.amax = L.take(sizeof(float));
        const int f = plan->forms[i];
        if (f >= CGH_GEMM_F16) {
            const int planes = f == CGH_GEMM_SPLIT16 ? 2 : 1;
            o.ld = (2 * np + 63) / 64 * 64;
            o.p = L.take((size_t)planes * inst[i].height * o.ld * 2);
            o.q = L.take((size_t)planes * inst[i].width * o.ld * 2);
            ++n_gemm;
        } else if (f == CGH_DIRECT_SFU) {
            ++n_dsfu;
        } else {
            ++n_dacc;
        }
    }
    // job tables and unit lists
    std::vector<GemmJob> gjobs;
    std::vector<DirectJob> djobs[2];
    std::vector<int2> gunits, dunits[2];
    std::vector<double> gcost, dcost[2];
    // the direct batch kernels' CTA shape: the one with fewer padded pixels over the direct instances (weighted by
    // their points, as the work is)
    double pad_work[2] = {0.0, 0.0};
    for (int i = 0; i < n; ++i) {
        if (inst[i].n_points == 0 || plan->forms[i] >= CGH_GEMM_F16) continue;
        for (int tall = 0; tall < 2; ++tall) {
            const DirectShape sh = direct_shape(tall != 0);
            pad_work[tall] += (double)((inst[i].width + sh.tile_w - 1) / sh.tile_w * sh.tile_w) *
                              (double)((inst[i].height + sh.tile_h - 1) / sh.tile_h * sh.tile_h) *
                              (double)off[i].n_pad;
        }
    }
    const bool dtall = pad_work[1] < pad_work[0];
    const DirectShape dsh = direct_shape(dtall);
    for (int i = 0; i < n; ++i) {
        if (inst[i].n_points == 0) continue;
        const int f = plan->forms[i];
        if (f >= CGH_GEMM_F16) {
            const int j = (int)gjobs.size();
            gjobs.emplace_back();
            // device pointers are filled after the arena exists; remember the instance
            const int tiles = ((inst[i].height + 127) / 128) * ((inst[i].width + bn[i] - 1) / bn[i]);
            const double c = (double)((2 * inst[i].n_points + 63) / 64) * (f == CGH_GEMM_SPLIT16 ? 3.0 : 1.0) * bn[i];
            for (int t = 0; t < tiles; ++t) {
                gunits.push_back(make_int2(j, t));
                gcost.push_back(c);
            }
        } else {
            const int which = f == CGH_DIRECT_SFU ? 0 : 1;
            const int j = (int)djobs[which].size();
            djobs[which].emplace_back();
            const int tiles_x = (inst[i].width + dsh.tile_w - 1) / dsh.tile_w;
            const int tiles = tiles_x * ((inst[i].height + dsh.tile_h - 1) / dsh.tile_h);
            for (int t = 0; t < tiles; ++t) {
                dunits[which].push_back(make_int2(j, t));
                dcost[which].push_back((double)off[i].n_pad);
            }
        }
    }
    const int gctas = gunits.empty() ? 0 : std::min<int>(gemm_max_ctas(ctx->num_sms), (int)gunits.size());
    int dctas[2];
    std::vector<int> goff, doff[2];
    std::vector<int2> gord, dord[2];
    if (gctas) assign(gunits, gcost, gctas, goff, gord);
    for (int w = 0; w < 2; ++w) {
        dctas[w] = dunits[w].empty() ? 0
                                     : std::min<int>(ctx->num_sms * direct_ctas_per_sm(w == 0, dtall),
                                                     (int)dunits[w].size());
        if (dctas[w]) assign(dunits[w], dcost[w], dctas[w], doff[w], dord[w]);
    }
    const size_t t_gjobs = L.take(gjobs.size() * sizeof(GemmJob), 128);
    const size_t t_goff = L.take(goff.size() * sizeof(int));
    const size_t t_gunits = L.take(gord.size() * sizeof(int2));
    size_t t_djobs[2], t_doff[2], t_dunits[2];
    for (int w = 0; w < 2; ++w) {
        t_djobs[w] = L.take(djobs[w].size() * sizeof(DirectJob));
        t_doff[w] = L.take(doff[w].size() * sizeof(int));
        t_dunits[w] = L.take(dord[w].size() * sizeof(int2));
    }
    const int arc = ensure_arena(ctx, plan, L.bytes);
    if (arc) return arc;
    char *A = static_cast<char *>(plan->arena);
    // fill the job tables with device pointers
    {
        int gj = 0, dj[2] = {0, 0};
        for (int i = 0; i < n; ++i) {
            if (inst[i].n_points == 0) continue;
            const int f = plan->forms[i];
            const Off &o = off[i];
            if (f >= CGH_GEMM_F16) {
                if (!fill_gemm_job(&gjobs[gj], factor_mode(f), bn[i], A + o.p, A + o.q, inst[i].height,
                                   inst[i].width, o.ld,
                                   f == CGH_GEMM_SPLIT16 ? (ctx->gemm_chunk > 0 ? ctx->gemm_chunk : kSplit16ChunkKbBatch)
                                                         : ctx->gemm_chunk,
                                   inst[i].d_out, reinterpret_cast<float *>(A + o.amax)))
                    return CGH_ECUDA;
                ++gj;
            } else {
                const int w = f == CGH_DIRECT_SFU ? 0 : 1;
                DirectJob &J = djobs[w][dj[w]++];
                J.geo = reinterpret_cast<const int4 *>(A + o.geo);
                J.aux = reinterpret_cast<const uint2 *>(A + o.aux);
                J.out = inst[i].d_out;
                J.n_ptiles = (int)(o.n_pad / kPointTile);
                J.width = inst[i].width;
                J.height = inst[i].height;
                J.tiles_x = (inst[i].width + dsh.tile_w - 1) / dsh.tile_w;
                J.vec = (inst[i].width % 4 == 0) && ((uintptr_t)inst[i].d_out % 16 == 0);
                J.pad = 0;
            }
        }
    }
    auto up = [&](size_t at, const void *src, size_t bytes) {
        return bytes == 0 || cudaMemcpy(A + at, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!up(t_gjobs, gjobs.data(), gjobs.size() * sizeof(GemmJob)) || !up(t_goff, goff.data(), goff.size() * sizeof(int)) ||
        !up(t_gunits, gord.data(), gord.size() * sizeof(int2)))
        return cuda_status(cudaGetLastError());
    for (int w = 0; w < 2; ++w)
        if (!up(t_djobs[w], djobs[w].data(), djobs[w].size() * sizeof(DirectJob)) ||
            !up(t_doff[w], doff[w].data(), doff[w].size() * sizeof(int)) ||
            !up(t_dunits[w], dord[w].data(), dord[w].size() * sizeof(int2)))
            return cuda_status(cudaGetLastError());

    // capture the whole batch
    const int crc = begin_capture(plan);
    if (crc) return crc;
    const uint64_t tmo = (uint64_t)ctx->timeout_ms * 1000000ull;
    cudaStream_t s = plan->capture;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const cgh_instance &b = inst[i];
        if (b.n_points == 0) {
            e = cudaMemsetAsync(b.d_out, 0, (size_t)b.width * b.height * sizeof(float), s);
            continue;
        }
        const int f = plan->forms[i];
        const Off &o = off[i];
        float *amax = reinterpret_cast<float *>(A + o.amax);
        const bool gemm = f >= CGH_GEMM_F16;
        if (gemm) e = cudaMemsetAsync(amax, 0, sizeof(float), s);
        if (e == cudaSuccess)
            e = launch_prep_points(b.d_xyz, b.d_amp, (int)b.n_points, (int)o.n_pad, b.pitch_m, b.lambda_m,
                                   reinterpret_cast<int4 *>(A + o.geo), reinterpret_cast<uint2 *>(A + o.aux),
                                   ctx->d_status, gemm ? amax : nullptr, s);
        if (e == cudaSuccess && gemm)
            e = launch_factors(factor_mode(f), reinterpret_cast<const int4 *>(A + o.geo),
                               reinterpret_cast<const uint2 *>(A + o.aux), (int)b.n_points, b.height, b.width,
                               A + o.p, A + o.q, o.ld, amax, s);
    }
    if (e == cudaSuccess && gctas) {
        int bn_max = 0;
        for (int i = 0; i < n; ++i)
            if (inst[i].n_points > 0 && plan->forms[i] >= CGH_GEMM_F16 && bn[i] > bn_max) bn_max = bn[i];
        e = launch_gemm_batch(reinterpret_cast<const GemmJob *>(A + t_gjobs), reinterpret_cast<const int *>(A + t_goff),
                              reinterpret_cast<const int2 *>(A + t_gunits), gctas, bn_max, ctx->d_status, tmo, s);
    }
    for (int w = 0; w < 2 && e == cudaSuccess; ++w)
        if (dctas[w])
            e = launch_direct_batch(w == 0, dtall, reinterpret_cast<const DirectJob *>(A + t_djobs[w]),
                                    reinterpret_cast<const int *>(A + t_doff[w]),
                                    reinterpret_cast<const int2 *>(A + t_dunits[w]), dctas[w], ctx->d_status, tmo, s);
    const int frc = finish_capture(plan, e);
    if (frc) return frc;
    plan->key = plan_key(ctx, inst, n);
    return CGH_OK;
}

}  // namespace

int run_single_persistent(cgh_ctx *ctx, int form, const cgh_instance &inst)
{
    if (!ctx->single) ctx->single = new BatchPlan();
    BatchPlan *plan = ctx->single;
    std::vector<uint64_t> key = plan_key(ctx, &inst, 1);
    key.push_back((uint64_t)form);
    if (!(plan->exec && plan->key == key)) {
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_status(cudaGetLastError());
        plan->key.clear();
        const int rc = build_plan_persist(ctx, &inst, 1, plan, form);
        if (rc) return rc;
        plan->key = key;
    }
    ProfileScope ps(ctx, "gemm_persist", 1);
    return cuda_status(cudaGraphLaunch(plan->exec, ctx->stream));
}

int batch_forms(const cgh_ctx *ctx, int *forms, int max_entries)
{
    if (!ctx->batch) return 0;
    const int n = (int)ctx->batch->forms.size();
    for (int i = 0; i < n && i < max_entries; ++i) forms[i] = ctx->batch->forms[i];
    return n;
}

int run_batch(cgh_ctx *ctx, const cgh_instance *inst, int n)
{
    if (!ctx->batch) ctx->batch = new BatchPlan();
    BatchPlan *plan = ctx->batch;
    const std::vector<uint64_t> key = plan_key(ctx, inst, n);
    if (!(plan->exec && plan->key == key)) {
        // the previous graph may still be running on the context's stream
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_status(cudaGetLastError());
        plan->key.clear();
        const int rc = ctx->batch_mode == 1 ? build_plan_kinds(ctx, inst, n, plan) : build_plan_persist(ctx, inst, n, plan);
        if (rc) return rc;
    }
    ProfileScope ps(ctx, ctx->batch_mode == 1 ? "batch_graph" : "batch_persist", 1);
    return cuda_status(cudaGraphLaunch(plan->exec, ctx->stream));
}

}  // namespace cgh
