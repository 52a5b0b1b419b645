// a7: the whole batch of holograms in ONE persistent launch.
//
// One CTA per SM, 14 warps, two groups that work side by side:
//   warps 0..5   the tcgen05 GEMM roles (gemm_dev.cuh): TMA producer, MMA
//                issuer, four epilogue warps; they take GEMM units {job, tile}
//                from a global queue (atomic counter), the producer publishing
//                each unit to the MMA issuer and the epilogue through a ring of
//                unit ids in shared memory;
//   warps 6..13  the SIMT group (256 threads, named barrier 1): point
//                preparation, factor generation and direct units, from a
//                second global queue.
// So the tensor cores run the GEMM of one hologram while the same SMs' FP32,
// integer and MUFU pipes prepare the points and the factors of the next ones,
// and direct holograms run on the SIMT group.
//
// Dependencies are counters in global memory, waited on with a bounded spin:
// a factor or direct unit of job j waits for all preparation units of j, a
// GEMM unit of j for all factor units of j.  The SIMT queue lists every
// preparation unit before any factor unit and every factor unit before any
// direct unit, and no SIMT unit waits on a GEMM unit, so every unit waited on
// was dequeued earlier by a CTA that is running it: the launch always makes
// progress, whatever the number of co-resident CTAs.  A wait that runs out
// (kStatusTimeout) stops its group; every other wait is bounded too, so the
// launch ends.
//
// Writes made with ordinary stores and read by the TMA engine (prepared points
// read by bulk copies, factors read by tensor-map loads) are published with
// fence.proxy.async.global and a release (__threadfence + atomicAdd) and taken
// with an acquire load and fence.proxy.async.global.
//
// Direct units {job, pixel tile, point chunk}: a job's points are cut into
// chunks so that the units balance; a tile's chunks leave their totals in
// slots and the last one to finish sums them in chunk order (fixed order, so
// the result does not depend on timing) and writes the tile.
#include "../../include/cgh.h"
#include "direct_dev.cuh"
#include "factors_dev.cuh"
#include "gemm_dev.cuh"
#include "host_util.h"
#include "kernels.h"
#include "prep_dev.cuh"

namespace cgh {

namespace {

using namespace dev;

constexpr int kGemmWarps = 6;
constexpr int kSimtBase = kGemmWarps * 32;                  // first thread of the SIMT group
constexpr int kSimtThreads = 256;
constexpr int kPersistThreads = kSimtBase + kSimtThreads;   // 448
constexpr int kSimtTile = 64;                               // points per shared-memory tile of a direct unit
constexpr int kRing = 4;                                    // GEMM unit ids in flight between the roles
constexpr int kFactorRows = 32;                             // rows of a factor unit
constexpr int kFactorPoints = kSimtThreads * 4;             // point slots of a factor unit
constexpr int kGroupKb = 2 * kFactorPoints / 64;            // k-blocks (of 64 K elements) of one factor unit: 32
// the direct units' CTA shape: 16 x 16 threads of 8 x 4 pixels (128 x 64-pixel tiles)
constexpr int kDTL = 8, kDTR = 4, kDBX = 16, kDBY = 16;
// shared memory for the GEMM ring: the 227 KB a CTA may use, less the alignment slack, the barriers and the
// static shared memory of the SIMT group and the unit ring (below 4 KB)
constexpr int kPersistRoom = 232448 - 1024 - 256 - 4096;

using SimtSync = GroupSync<1, kSimtThreads, kSimtBase>;

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// GEMM units {job, tile, K chunk} from the global queue.  The producer hands a unit to the MMA issuer and the
// epilogue through the ring of unit ids at once, and before it loads a k-block it waits (bounded) until the factor
// units of that k-block are written, so the GEMM of a hologram streams behind its factor generation and no role
// reads factors that are not there.
struct QueueUnits {
    const PersistJob *jobs;
    const int4 *units;   // {job, tile, K chunk, 0}
    int total;
    int *head;
    const int *fact_done;
    int *ring_u;
    uint64_t *ring_full, *ring_empty;   // 1 arrival; 5 arrivals (the MMA issuer and the four epilogue warps)
    int *status;
    unsigned long long timeout_ns;
    const int *fact_all_done;   // factor units done over all jobs
    int fact_all;               // > 0: wait for that many instead of the job's own
    int n_jobs;

    struct Cursor {
        uint32_t i;
    };
    __device__ Cursor start() const { return Cursor{0u}; }

    __device__ UnitInfo get(int u) const
    {
        const int4 w = units[u];
        const PersistJob &P = jobs[w.x];
        const GemmJob &J = P.g;
        UnitInfo x;
        x.mp = &J.p;
        x.mq = &J.q;
        x.mpl = &J.pl;
        x.mql = &J.ql;
        x.out = J.out;
        x.amp_max = J.amp_max;
        x.tm = w.y % J.tiles_m;
        x.row0 = x.tm * kBM;
        x.tn = w.y / J.tiles_m;
        x.kb0 = w.z * P.kchunk_kb;
        x.kb1 = min(J.nkb, x.kb0 + P.kchunk_kb);
        x.bn = J.bn;
        x.passes = J.passes;
        x.kc = J.kc;
        x.height = J.height;
        x.width = J.width;
        x.idesc = J.idesc;
        x.vec = J.vec != 0;
        x.accumulate = w.z > 0;
        x.trans = J.trans != 0;
        x.job = w.x;
        x.seq = P.kchunks > 1 ? P.tile_seq + 4 * w.y : nullptr;
        x.seq_k = w.z;
        return x;
    }

    __device__ bool next(int role, Cursor &c, UnitInfo &x) const
    {
        const int slot = (int)(c.i % kRing);
        const uint32_t ph = (c.i / kRing) & 1u;
        ++c.i;
        int u;
        if (role == 0) {
            if (!mbar_wait(&ring_empty[slot], ph ^ 1u, timeout_ns)) {
                atomicOr(status, kStatusTimeout);
                return false;
            }
            u = atomicAdd(head, 1);
            if (u >= total) u = -1;
            bool fail = false;
            if (u >= 0) {
                const int4 w = units[u];
                // the unit names a job, a tile and a K range that exist
                if (!CGH_DCHECK(w.x >= 0 && w.x < n_jobs && w.y >= 0 &&
                                    w.y < jobs[w.x].g.tiles_m * jobs[w.x].g.tiles_n && w.z >= 0 &&
                                    w.z * jobs[w.x].kchunk_kb < jobs[w.x].g.nkb,
                                status)) {
                    fail = true;
                    u = -1;
                }
            }
            if (u >= 0 && fact_all > 0) {   // every job's factors before any GEMM unit
                if (wait_count(fact_all_done, fact_all, timeout_ns)) {
                    fence_proxy_async_global();   // the factors' ordinary stores, for the TMA loads that follow
                } else {
                    atomicOr(status, kStatusTimeout);
                    fail = true;
                    u = -1;
                }
            }
            ring_u[slot] = u;
            mbar_arrive(&ring_full[slot]);
            if (fail) return false;
        } else {
            // the producer may wait up to the limit for the unit's factors first
            if (!mbar_wait(&ring_full[slot], ph, 2 * timeout_ns)) {
                atomicOr(status, kStatusTimeout);
                return false;
            }
            u = ring_u[slot];
            if (role == 1) {
                mbar_arrive(&ring_empty[slot]);
            } else {
                __syncwarp();
                if ((threadIdx.x & 31) == 0) mbar_arrive(&ring_empty[slot]);
            }
        }
        if (u < 0) return false;
        x = get(u);
        return true;
    }

    // The factor units of k-blocks [x.kb0, kb_end): every band of each group of kGroupKb k-blocks; upto is the
    // first group not yet seen complete (-1: none checked for this unit).
    __device__ bool ready(const UnitInfo &x, int kb_end, int &upto, unsigned long long timeout_ns) const
    {
        if (fact_all > 0) return true;   // next() waited for all of them
        const PersistJob &J = jobs[x.job];
        if (J.premade) return true;      // written before this launch
        if (upto < 0) upto = x.kb0 / kGroupKb;
        const int g_end = min(J.fact_groups, (kb_end + kGroupKb - 1) / kGroupKb);
        if (upto >= g_end) return true;
        for (; upto < g_end; ++upto)
            if (!wait_count(&J.group_done[upto], J.fact_bands + J.chunk_extra, timeout_ns)) return false;
        fence_proxy_async_global();   // the factors' ordinary stores, for the TMA loads that follow
        return true;
    }

    // after a failure the producer ends the sequence for the other roles
    __device__ void abort(Cursor &c, unsigned long long timeout_ns) const
    {
        const int slot = (int)(c.i % kRing);
        const uint32_t ph = (c.i / kRing) & 1u;
        ++c.i;
        if (!mbar_wait(&ring_empty[slot], ph ^ 1u, timeout_ns)) return;
        ring_u[slot] = -1;
        mbar_arrive(&ring_full[slot]);
    }
};

// All threads of the SIMT group: the unit's writes (ordinary stores) become visible to every CTA and to the
// async proxy, then one arrival on the counter.
__device__ __forceinline__ void publish(int *count)
{
    fence_proxy_async_global();
    __threadfence();
    SimtSync::sync();
    if (SimtSync::tid() == 0) atomicAdd(count, 1);
}

// Thread 0 of the group waits; the group learns the outcome.
__device__ __forceinline__ bool group_wait(const int *count, int need, unsigned long long timeout_ns)
{
    bool ok = true;
    if (SimtSync::tid() == 0) {
        ok = wait_count(count, need, timeout_ns);
        fence_proxy_async_global();
    }
    const bool failed = SimtSync::sync_or(!ok);
    __threadfence();
    return !failed;
}

// The end of a direct unit: one chunk stores its tile; otherwise the part goes to its slot and the last chunk of
// the tile to finish sums the parts in chunk order.
struct PersistDirectSink {
    const PersistJob *J;
    int tile, chunk;
    int *s_last;

    __device__ void operator()(float (&tot)[kDTR][kDTL]) const
    {
        constexpr int NT = kDBX * kDBY;
        constexpr int Q4 = kDTL * kDTR / 4;
        const int t = SimtSync::tid();
        if (J->chunks > 1) {
            float4 *base = J->parts + (long long)tile * J->chunks * (Q4 * NT) + t;
#pragma unroll
            for (int q = 0; q < Q4; ++q) {
                const int r = q * 4 / kDTL, i = q * 4 % kDTL;
                base[((long long)chunk * Q4 + q) * NT] = make_float4(tot[r][i], tot[r][i + 1], tot[r][i + 2], tot[r][i + 3]);
            }
            __threadfence();
            SimtSync::sync();
            if (t == 0) *s_last = atomicAdd(&J->tile_count[tile], 1) == J->chunks - 1;
            SimtSync::sync();
            if (!*s_last) return;
            __threadfence();
#pragma unroll
            for (int q = 0; q < Q4; ++q) {
                const int r = q * 4 / kDTL, i = q * 4 % kDTL;
                float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                for (int b = 0; b < J->chunks; ++b) {
                    const float4 v = b == chunk ? make_float4(tot[r][i], tot[r][i + 1], tot[r][i + 2], tot[r][i + 3])
                                                : __ldcg(base + ((long long)b * Q4 + q) * NT);
                    if (b == 0) {
                        a = v;
                    } else {
                        a.x += v.x;
                        a.y += v.y;
                        a.z += v.z;
                        a.w += v.w;
                    }
                }
                tot[r][i] = a.x;
                tot[r][i + 1] = a.y;
                tot[r][i + 2] = a.z;
                tot[r][i + 3] = a.w;
            }
        }
        const int m0 = (tile % J->tiles_x) * (kDBX * kDTL) + (t % kDBX) * kDTL;
        const int n0 = (tile / J->tiles_x) * (kDBY * kDTR) + (t / kDBX) * kDTR;
#pragma unroll
        for (int r = 0; r < kDTR; ++r) {
            const int n = n0 + r;
            if (n >= J->height || m0 >= J->width) continue;
            float *row = J->out + (long long)n * J->width + m0;
            if (J->vec && m0 + kDTL <= J->width) {
#pragma unroll
                for (int i = 0; i < kDTL; i += 4)
                    *reinterpret_cast<float4 *>(row + i) = make_float4(tot[r][i], tot[r][i + 1], tot[r][i + 2], tot[r][i + 3]);
            } else {
#pragma unroll
                for (int i = 0; i < kDTL; ++i)
                    if (m0 + i < J->width) row[i] = tot[r][i];
            }
        }
    }
};

template <bool SFU>
__device__ __forceinline__ bool run_direct_unit(const PersistJob &J, int tile, int chunk, int4 (*s_geo)[kSimtTile],
                                                uint2 (*s_aux)[kSimtTile], uint64_t *s_bar, uint32_t &kg,
                                                int *s_last, int *status, unsigned long long timeout_ns)
{
    const int p0 = (int)((long long)chunk * J.n / J.chunks), p1 = (int)((long long)(chunk + 1) * J.n / J.chunks);
    if (p1 <= p0) return true;   // cannot happen with chunks <= n
    const int k0 = p0 / kSimtTile, k1 = (p1 + kSimtTile - 1) / kSimtTile;
    const PersistDirectSink sink{&J, tile, chunk, s_last};
    return direct_unit<kDTL, kDTR, kDBX, kDBY, SFU, 1, false, false, PersistDirectSink, SimtSync, kSimtTile>(
        J.geo, J.aux, k0, k1, (tile % J.tiles_x) * (kDBX * kDTL), (tile / J.tiles_x) * (kDBY * kDTR), J.width,
        J.height, J.out, J.vec != 0, s_geo, s_aux, s_bar, kg, status, timeout_ns, -1, 0, PhaseRef(), nullptr,
        p0 - k0 * kSimtTile, p1 - (k1 - 1) * kSimtTile, sink);
}

template <int MODE>
__device__ __forceinline__ void run_factor_unit(const PersistJob &J, int band, int group)
{
    float scale = 1.0f;
    const float m = __ldcg(J.amax);   // written by other SMs in this launch: from L2, never a stale L1 line
    if (m > 0.0f) scale = 1.0f / m;
    const int j0 = group * kFactorPoints + SimtSync::tid() * 4;
    const int r0 = band * kFactorRows;
    const int r1 = min(J.height + J.width, r0 + kFactorRows);
    if (j0 < J.point_slots)
        factor_thread<MODE, false>(j0, r0, r1, J.geo, J.aux, J.n, J.height, J.width, J.P, J.Q, J.ld, J.plane_p,
                                   J.plane_q, scale, PhaseRef());
}

__device__ void simt_group(const PersistParams &p, int4 (*s_geo)[kSimtTile], uint2 (*s_aux)[kSimtTile],
                           uint64_t *s_bar, int4 *s_unit, int *s_last, int *status, unsigned long long timeout_ns)
{
    const int t = SimtSync::tid();
    uint32_t kg = 0;   // point tiles consumed by this group's direct units (stage and barrier parity)
    for (;;) {
        if (t == 0) {
            const int u = atomicAdd(&p.heads[0], 1);
            *s_unit = u < p.simt_total ? p.simt_units[u] : make_int4(-1, 0, 0, 0);
        }
        SimtSync::sync();
        const int4 w = *s_unit;
        SimtSync::sync();
        if (w.x < 0) return;
        // the unit names a job and a block, band or tile of it that exist (uniform over the group)
        if (!CGH_DCHECK(w.y >= 0 && w.y < p.n_jobs, status)) return;
        const PersistJob &J = p.jobs[w.y];
        if (!CGH_DCHECK(w.x == kPersistPrep ? w.z >= 0 && w.z < J.n_pad / kPointTile
                        : w.x == kPersistFactor
                            ? w.z >= 0 && w.z * kFactorRows < J.height + J.width && w.w >= 0 &&
                                  w.w * kFactorPoints < J.point_slots
                            : w.z >= 0 && w.z < J.tiles_x * ((J.height + kDBY * kDTR - 1) / (kDBY * kDTR)) &&
                                  w.w >= 0 && w.w < J.chunks,
                        status))
            return;
        bool ok = true;
        if (w.x == kPersistPrep) {
            const int j = w.z * kPointTile + t;
            if (j < J.n_pad)
                prep_point(j, J.xyz, J.amp, J.n, J.pitch, J.lambda, J.geo, J.aux, status,
                           J.form >= CGH_GEMM_F16 ? J.amax : nullptr, kAuxSecondDiff, nullptr, 0, 0, 4, 4);
            publish(&p.prep_done[w.y]);
        } else if (w.x == kPersistFactor) {
            ok = group_wait(&p.prep_done[w.y], J.prep_units, timeout_ns);
            if (ok) {
                if (J.form == CGH_GEMM_F16) run_factor_unit<kFactorF16>(J, w.z, w.w);
                else if (J.form == CGH_GEMM_BF16) run_factor_unit<kFactorBF16>(J, w.z, w.w);
                else run_factor_unit<kFactorSplit16>(J, w.z, w.w);
                publish(&J.group_done[w.w]);
                if (t == 0) {
                    atomicAdd(&p.fact_done[w.y], 1);
                    atomicAdd(&p.heads[2], 1);
                }
            }
        } else {
            ok = group_wait(&p.prep_done[w.y], J.prep_units, timeout_ns);
            if (ok)
                ok = J.form == CGH_DIRECT_SFU
                         ? run_direct_unit<true>(J, w.z, w.w, s_geo, s_aux, s_bar, kg, s_last, status, timeout_ns)
                         : run_direct_unit<false>(J, w.z, w.w, s_geo, s_aux, s_bar, kg, s_last, status, timeout_ns);
        }
        if (!ok) {
            if (t == 0) atomicOr(status, kStatusTimeout);
            return;
        }
    }
}

// 14 warps, so one sub-partition holds four of them: at most 128 registers a thread (4 x 32 x 128 = the
// sub-partition's 16,384)
template <int BN_MAX>
__global__ void __launch_bounds__(kPersistThreads, 1)
    persist_kernel(const __grid_constant__ PersistParams p, int *status, unsigned long long timeout_ns)
{
    using C = GemmCfg<BN_MAX, kPersistRoom>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const GemmBars bars = gemm_bars<C>(smem);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars.drain + 1);
    __shared__ int ring_u[kRing];
    __shared__ alignas(8) uint64_t ring_full[kRing], ring_empty[kRing];
    __shared__ alignas(128) int4 s_geo[2][kSimtTile];
    __shared__ alignas(128) uint2 s_aux[2][kSimtTile];
    __shared__ alignas(8) uint64_t s_bar[2];
    __shared__ int4 s_unit;
    __shared__ int s_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool gemm = p.gemm_total > 0;
    if (threadIdx.x == 0) {
        gemm_init_barriers<C>(bars);
        for (int i = 0; i < kRing; ++i) {
            mbar_init(&ring_full[i], 1);
            mbar_init(&ring_empty[i], 1 + 4);
        }
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_barrier_init();
    }
    if (gemm && warp == 1) {
        tmem_alloc(tmem_slot, C::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp < kGemmWarps) {
        if (gemm) {
            const uint32_t tmem_base = *tmem_slot;
            const QueueUnits src{p.jobs,  p.gemm_units, p.gemm_total, &p.heads[1], p.fact_done, ring_u,
                                 ring_full, ring_empty,   status,       timeout_ns,  &p.heads[2], p.fact_all,
                                 p.n_jobs};
            if (warp == 0) {
                if (lane == 0) gemm_producer<C>(src, smem, bars, status, timeout_ns);
            } else if (warp == 1) {
                if (lane == 0) gemm_mma<C>(src, smem, bars, tmem_base, status, timeout_ns);
            } else {
                gemm_epilogue<C, QueueUnits, 32>(src, bars, tmem_base, warp, lane, status, timeout_ns);
            }
        }
    } else {
        simt_group(p, s_geo, s_aux, s_bar, &s_unit, &s_last, status, timeout_ns);
    }
    __syncthreads();
    if (gemm && warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(*tmem_slot, C::kTmemCols);
    }
}

template <int BN_MAX>
cudaError_t launch_persist_as(const PersistParams &p, int ctas, int *status, uint64_t timeout_ns, cudaStream_t s)
{
    using C = GemmCfg<BN_MAX, kPersistRoom>;
    static PerDeviceOnce configured;
    const cudaError_t e = configured.run([] {
        return cudaFuncSetAttribute(persist_kernel<BN_MAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    C::kSmemBytes);
    });
    if (e != cudaSuccess) return e;
    persist_kernel<BN_MAX><<<ctas, kPersistThreads, C::kSmemBytes, s>>>(p, status, timeout_ns);
    return cudaGetLastError();
}

}  // namespace

int persist_factor_rows() { return kFactorRows; }
int persist_factor_points() { return kFactorPoints; }
int persist_direct_tile_w() { return kDBX * kDTL; }
int persist_direct_tile_h() { return kDBY * kDTR; }

cudaError_t launch_persist(const PersistParams &p, int ctas, int bn_max, int *status, uint64_t timeout_ns,
                           cudaStream_t s)
{
    if (ctas <= 0) return cudaSuccess;
    if (bn_max <= 224) return launch_persist_as<224>(p, ctas, status, timeout_ns, s);
    return launch_persist_as<256>(p, ctas, status, timeout_ns, s);
}

}  // namespace cgh
