// Device-side code of the tcgen05 GEMM form, shared by its kernels (gemm.cu)
// and by the persistent batch kernel (persist.cu): the shared-memory ring and
// the three roles of a warp-specialised CTA.
//
//   producer   (one thread)   TMA loads of a 128 x 64 A tile and a bn x 64 B
//                             tile per stage into the ring (full/empty mbarriers);
//   MMA issuer (one thread)   tcgen05.mma (M = 128, N = bn, K = 16) into one of
//                             two TMEM accumulators, stage commits back to the
//                             ring, chunk commits to the accumulator's barrier;
//   epilogue   (four warps)   tcgen05.ld of the accumulator (warp w owns lanes
//                             32 (w % 4) .. + 31), chunk folding, stores.
//
// Units (a template parameter) hands every role the same sequence of units of
// work: Cursor, start(), next(role, cursor, info) with role 0 = producer, 1 =
// MMA issuer, 2 = epilogue (called by all 128 epilogue threads), ready(info,
// kb_end, state, timeout) -- the producer's bounded wait, before it loads a
// k-block, for the unit's operands of k-blocks below kb_end (state starts at
// -1 for every unit) -- and abort(cursor, timeout), which the producer calls
// after a failure so that the consumers stop.
#pragma once

#include <cuda.h>

#include "device_util.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace cgh {
namespace dev {

constexpr int kBM = 128;
constexpr int kBK = 64;   // 64 16-bit elements = one 128-byte swizzle row
constexpr int kGemmThreads = 192;
// Shared memory left for the operand ring: the 227 KB a CTA may use, less the 1024-byte alignment slack and the
// barriers.
constexpr int kStageRoom = 232448 - 1024 - 256;

template <int BN, int ROOM = kStageRoom>
struct GemmCfg {
    static constexpr int kStageA = kBM * kBK * 2;
    static constexpr int kStageB = BN * kBK * 2;
    static constexpr int kStageBytes = kStageA + kStageB;
    static constexpr int kStages = ROOM / kStageBytes > 8 ? 8 : ROOM / kStageBytes;
    static constexpr int kAccStride = BN <= 128 ? 128 : 256;   // TMEM columns between the two accumulators
    static constexpr int kTmemCols = 2 * kAccStride;
    static constexpr int kBarrierBytes = 256;
    static constexpr int kSmemBytes = 1024 + kStages * kStageBytes + kBarrierBytes;
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
    static_assert(kStageBytes % 1024 == 0, "stages must keep 1024-byte alignment");
    static_assert(kStages >= 2, "at least a double-buffered ring");
};

// Everything one unit of work needs.
struct UnitInfo {
    const CUtensorMap *mp, *mq, *mpl, *mql;
    float *out;                  // output (or partial) plane of this unit
    const float *amp_max;
    int tm, tn, kb0, kb1, bn, passes, kc, height, width;
    uint32_t idesc;
    bool vec;
    bool accumulate;             // add to the output already there (later point chunks)
    bool trans;                  // A = Q, B = P: accumulator rows are hologram columns
    int job = 0;                 // a batch's job (the readiness wait of a queue of units)
    int row0 = 0;                // the hologram row (transposed: column) of this CTA's accumulator lane 0
    // A K chunk of a batch's tile: epilogue warp q stores (adds) its quarter of the tile once seq[q] >= seq_k,
    // then sets seq[q] = seq_k + 1, so the chunks of a tile reach the output in K order; nullptr: no ordering.
    int *seq = nullptr;
    int seq_k = 0;
};

// The barriers of the ring and of the two accumulators.
struct GemmBars {
    uint64_t *full, *empty;   // [kStages] each
    uint64_t *tfull;          // [2]
    uint64_t *tempty;         // [2], 128 arrivals (the epilogue threads)
    uint64_t *drain;          // [1]
};

template <class C>
__device__ __forceinline__ GemmBars gemm_bars(uint8_t *smem)
{
    GemmBars b;
    b.full = reinterpret_cast<uint64_t *>(smem + C::kStages * C::kStageBytes);
    b.empty = b.full + C::kStages;
    b.tfull = b.empty + C::kStages;
    b.tempty = b.tfull + 2;
    b.drain = b.tempty + 2;
    return b;
}

// One thread; fenced for the async proxy.
template <class C>
__device__ __forceinline__ void gemm_init_barriers(const GemmBars &b)
{
    for (int s = 0; s < C::kStages; ++s) {
        mbar_init(&b.full[s], 1);
        mbar_init(&b.empty[s], 1);
    }
    mbar_init(&b.tfull[0], 1);
    mbar_init(&b.tfull[1], 1);
    mbar_init(&b.tempty[0], 128);
    mbar_init(&b.tempty[1], 128);
    mbar_init(b.drain, 1);
    fence_barrier_init();
}

template <class C, class Units>
__device__ __forceinline__ void gemm_producer(const Units &src, uint8_t *smem, const GemmBars &bars, int *status,
                                              unsigned long long timeout_ns)
{
    uint64_t *full = bars.full, *empty = bars.empty;
    uint32_t it = 0;
    bool ok = true;
    typename Units::Cursor cur = src.start();
    UnitInfo x;
    while (ok && src.next(0, cur, x)) {
        const uint32_t stage_bytes = (uint32_t)(C::kStageA + x.bn * kBK * 2);
        int upto = -1;   // the unit source's record of the operands known to be there
        for (int c0 = x.kb0; c0 < x.kb1 && ok; c0 += x.kc) {
            const int c1 = min(x.kb1, c0 + x.kc);
            for (int pass = 0; pass < x.passes && ok; ++pass) {
                const CUtensorMap *ma = (pass == 2) ? x.mpl : x.mp;
                const CUtensorMap *mb = (pass == 1) ? x.mql : x.mq;
                for (int kb = c0; kb < c1; ++kb, ++it) {
                    const int s = (int)(it % C::kStages);
                    const uint32_t ph = (it / C::kStages) & 1u;
                    // the operands of k-block kb (a batch: its factors) are there
                    if (pass == 0 && !src.ready(x, kb + 1, upto, timeout_ns)) {
                        atomicOr(status, kStatusTimeout);
                        ok = false;
                        break;
                    }
                    if (!mbar_wait(&empty[s], ph ^ 1u, timeout_ns)) {
                        atomicOr(status, kStatusTimeout);
                        ok = false;
                        break;
                    }
                    uint8_t *sa = smem + s * C::kStageBytes;
                    mbar_arrive_expect_tx(&full[s], stage_bytes);
                    tma_load_2d(sa, ma, &full[s], kb * kBK, x.tm * kBM);
                    tma_load_2d(sa + C::kStageA, mb, &full[s], kb * kBK, x.tn * x.bn);
                }
            }
        }
    }
    if (!ok) {
        src.abort(cur, timeout_ns);   // the consumers stop at once rather than at their own limits
        // drain: wait (bounded) for the loads of the last kStages issues
        for (uint32_t j = (it > (uint32_t)C::kStages ? it - C::kStages : 0); j < it; ++j)
            mbar_wait(&full[j % C::kStages], (j / C::kStages) & 1u, timeout_ns);
    }
}

template <class C, class Units>
__device__ __forceinline__ void gemm_mma(const Units &src, uint8_t *smem, const GemmBars &bars, uint32_t tmem_base,
                                         int *status, unsigned long long timeout_ns)
{
    uint64_t *full = bars.full, *empty = bars.empty, *tfull = bars.tfull, *tempty = bars.tempty,
             *drain = bars.drain;
    uint32_t it = 0;
    uint32_t uses[2] = {0u, 0u};   // chunks each accumulator has received
    int nb = 0;                    // accumulator of the next unit's first chunk
    bool ok = true;
    typename Units::Cursor cur = src.start();
    UnitInfo x;
    while (ok && src.next(1, cur, x)) {
        const int nch = x.kb1 > x.kb0 ? (x.kb1 - x.kb0 + x.kc - 1) / x.kc : 1;
        const int tb = nb;   // the unit's total
        for (int c = 0; c < nch && ok; ++c) {
            const int c0 = x.kb0 + c * x.kc, c1 = min(x.kb1, c0 + x.kc);
            const int b = c == 0 ? tb : 1 - tb;
            const uint32_t uph = uses[b] & 1u;
            ++uses[b];
            if (!mbar_wait(&tempty[b], uph ^ 1u, timeout_ns)) {
                atomicOr(status, kStatusTimeout);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + (uint32_t)(b * C::kAccStride);
            uint32_t acc = 0;
            for (int pass = 0; pass < x.passes && ok; ++pass) {
                for (int kb = c0; kb < c1; ++kb, ++it) {
                    const int s = (int)(it % C::kStages);
                    const uint32_t ph = (it / C::kStages) & 1u;
                    if (!mbar_wait(&full[s], ph, timeout_ns)) {
                        atomicOr(status, kStatusTimeout);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_addr = smem_addr(smem + s * C::kStageBytes);
                    const uint64_t adesc = sw128_kmajor_desc(a_addr);
                    const uint64_t bdesc = sw128_kmajor_desc(a_addr + C::kStageA);
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        // +32 bytes per K step of 16 elements inside the swizzled row
                        umma_f16(d_tmem, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk), x.idesc,
                                 acc);
                        acc = 1;
                    }
                    umma_commit(&empty[s]);
                }
            }
            if (!ok) break;
            // an empty K range issues no MMA; the epilogue then writes zeros itself
            umma_commit(&tfull[b]);
        }
        nb = 1 - tb;   // the other accumulator is released first
    }
    // every MMA issued so far completes before TMEM is freed
    umma_commit(drain);
    mbar_wait(drain, 0, timeout_ns);
}

// The producer of a CTA of a two-SM pair: this CTA's 128 rows of A (at row0) and its half of the bn rows of B
// into its own stages; the loads of both CTAs are counted on the even CTA's full barrier, on which only the even
// CTA's producer arrives (with both CTAs' bytes).  Stages are freed by the even CTA's MMA commits, which arrive on
// both CTAs' empty barriers.
template <class C, class Units>
__device__ __forceinline__ void gemm_producer_pair(const Units &src, uint8_t *smem, const GemmBars &bars,
                                                   uint32_t rank, int *status, unsigned long long timeout_ns)
{
    uint64_t *full = bars.full, *empty = bars.empty;
    uint32_t it = 0;
    bool ok = true;
    typename Units::Cursor cur = src.start();
    UnitInfo x;
    while (ok && src.next(0, cur, x)) {
        const int half = x.bn / 2;
        const uint32_t pair_bytes = 2u * (uint32_t)(C::kStageA + half * kBK * 2);
        for (int c0 = x.kb0; c0 < x.kb1 && ok; c0 += x.kc) {
            const int c1 = min(x.kb1, c0 + x.kc);
            for (int pass = 0; pass < x.passes && ok; ++pass) {
                const CUtensorMap *ma = (pass == 2) ? x.mpl : x.mp;
                const CUtensorMap *mb = (pass == 1) ? x.mql : x.mq;
                for (int kb = c0; kb < c1; ++kb, ++it) {
                    const int s = (int)(it % C::kStages);
                    const uint32_t ph = (it / C::kStages) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u, timeout_ns)) {
                        atomicOr(status, kStatusTimeout);
                        ok = false;
                        break;
                    }
                    uint8_t *sa = smem + s * C::kStageBytes;
                    if (rank == 0) mbar_arrive_expect_tx(&full[s], pair_bytes);
                    const uint32_t bar = cluster_map(&full[s], 0);
                    tma_load_2d_pair(sa, ma, bar, kb * kBK, x.row0);
                    tma_load_2d_pair(sa + C::kStageA, mb, bar, kb * kBK, x.tn * x.bn + (int)rank * half);
                }
            }
        }
    }
    if (!ok && rank == 0) {
        // drain: wait (bounded) for the loads of the last kStages issues
        for (uint32_t j = (it > (uint32_t)C::kStages ? it - C::kStages : 0); j < it; ++j)
            mbar_wait(&full[j % C::kStages], (j / C::kStages) & 1u, timeout_ns);
    }
}

// The MMA issuer of a two-SM pair (one thread of the even CTA): M = 256 (128 rows of each CTA), N = bn (half of
// its rows in each CTA), commits to both CTAs' barriers; the epilogues of both CTAs release an accumulator on the
// even CTA's tempty barrier (256 arrivals).
template <class C, class Units>
__device__ __forceinline__ void gemm_mma_pair(const Units &src, uint8_t *smem, const GemmBars &bars,
                                              uint32_t tmem_base, int *status, unsigned long long timeout_ns)
{
    uint64_t *full = bars.full, *empty = bars.empty, *tfull = bars.tfull, *tempty = bars.tempty,
             *drain = bars.drain;
    uint32_t it = 0;
    uint32_t uses[2] = {0u, 0u};
    int nb = 0;
    bool ok = true;
    typename Units::Cursor cur = src.start();
    UnitInfo x;
    while (ok && src.next(1, cur, x)) {
        const int nch = x.kb1 > x.kb0 ? (x.kb1 - x.kb0 + x.kc - 1) / x.kc : 1;
        const int tb = nb;
        for (int c = 0; c < nch && ok; ++c) {
            const int c0 = x.kb0 + c * x.kc, c1 = min(x.kb1, c0 + x.kc);
            const int b = c == 0 ? tb : 1 - tb;
            const uint32_t uph = uses[b] & 1u;
            ++uses[b];
            if (!mbar_wait(&tempty[b], uph ^ 1u, timeout_ns)) {
                atomicOr(status, kStatusTimeout);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + (uint32_t)(b * C::kAccStride);
            uint32_t acc = 0;
            for (int pass = 0; pass < x.passes && ok; ++pass) {
                for (int kb = c0; kb < c1; ++kb, ++it) {
                    const int s = (int)(it % C::kStages);
                    const uint32_t ph = (it / C::kStages) & 1u;
                    if (!mbar_wait(&full[s], ph, timeout_ns)) {
                        atomicOr(status, kStatusTimeout);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_addr = smem_addr(smem + s * C::kStageBytes);
                    const uint64_t adesc = sw128_kmajor_desc(a_addr);
                    const uint64_t bdesc = sw128_kmajor_desc(a_addr + C::kStageA);
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        umma_f16_pair(d_tmem, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk), x.idesc, acc);
                        acc = 1;
                    }
                    umma_commit_pair(&empty[s]);
                }
            }
            if (!ok) break;
            umma_commit_pair(&tfull[b]);
        }
        nb = 1 - tb;
    }
    umma_commit_pair(drain);   // both CTAs learn when every MMA into their tensor memory is done
    mbar_wait(drain, 0, timeout_ns);
}

// ROUND: columns of the accumulator per store round (64 or 32; 32 holds half the registers).  PAIR: a CTA of a
// two-SM pair; the accumulators are released on the even CTA's barriers (the MMA issuer's), remotely from the
// odd CTA.
template <class C, class Units, int ROUND = 64, bool PAIR = false>
__device__ __forceinline__ void gemm_epilogue(const Units &src, const GemmBars &bars, uint32_t tmem_base, int warp,
                                              int lane, int *status, unsigned long long timeout_ns)
{
    uint64_t *tfull = bars.tfull, *tempty = bars.tempty;
    auto release = [&](int b) {
        if constexpr (PAIR) mbar_arrive_cluster(cluster_map(&tempty[b], 0));
        else mbar_arrive(&tempty[b]);
    };
    const int q = warp & 3;   // TMEM lane quarter this warp may access
    const int row_in_tile = q * 32 + lane;
    const uint32_t lane_base = tmem_base + ((uint32_t)(q * 32) << 16);
    uint32_t uses[2] = {0u, 0u};
    int nb = 0;
    bool ok = true;
    typename Units::Cursor cur = src.start();
    UnitInfo x;
    while (ok && src.next(2, cur, x)) {
        const bool empty_range = x.kb1 <= x.kb0;
        const int nch = x.kb1 > x.kb0 ? (x.kb1 - x.kb0 + x.kc - 1) / x.kc : 1;
        const int row = x.row0 + row_in_tile;
        float *dst = x.out + (long long)row * x.width;
        const int tb = nb;
        nb = 1 - tb;
        const uint32_t taddr = lane_base + (uint32_t)(tb * C::kAccStride);          // the unit's total
        const uint32_t xaddr = lane_base + (uint32_t)((1 - tb) * C::kAccStride);    // its later chunks
        if (!mbar_wait(&tfull[tb], uses[tb] & 1u, timeout_ns)) {
            atomicOr(status, kStatusTimeout);
            ok = false;
            break;
        }
        ++uses[tb];
        tc_fence_after();
        // the factors' scale, read once the unit's MMAs are done (so after every load of its operands), and from
        // L2: in a persistent batch other SMs wrote it during this launch and this SM's L1 may hold an old line
        float unscale = 1.0f;
        if (x.amp_max != nullptr) {
            const float m = __ldcg(x.amp_max);
            if (m > 0.0f) unscale = m;
        }
        for (int c = 1; c < nch; ++c) {
            // total += chunk c, in FP32 and chunk order
            if (!mbar_wait(&tfull[1 - tb], uses[1 - tb] & 1u, timeout_ns)) {
                atomicOr(status, kStatusTimeout);
                ok = false;
                break;
            }
            ++uses[1 - tb];
            tc_fence_after();
            // FOLD columns per tensor-memory round trip (32 where the registers allow; bn is a multiple of 16)
            constexpr int FOLD = ROUND >= 64 ? 32 : 16;
#pragma unroll 1
            for (int cc = 0; cc < x.bn; cc += FOLD) {
                const bool two = FOLD == 32 && cc + 16 < x.bn;
                uint32_t a[2][16], t[2][16];
                tmem_ld16(xaddr + (uint32_t)cc, a[0]);
                tmem_ld16(taddr + (uint32_t)cc, t[0]);
                if (two) {
                    tmem_ld16(xaddr + (uint32_t)(cc + 16), a[1]);
                    tmem_ld16(taddr + (uint32_t)(cc + 16), t[1]);
                }
                tmem_ld_wait();
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h == 1 && !two) break;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        t[h][i] = __float_as_uint(__uint_as_float(t[h][i]) + __uint_as_float(a[h][i]));
                    tmem_st16(taddr + (uint32_t)(cc + 16 * h), t[h]);
                }
            }
            tmem_st_wait();
            tc_fence_before();
            release(1 - tb);
        }
        if (!ok) break;
        if (x.seq != nullptr) {
            // the tile's previous K chunk has left this warp's quarter first
            bool got = true;
            if (lane == 0) got = wait_count(&x.seq[q], x.seq_k, timeout_ns);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) {
                if (lane == 0) atomicOr(status, kStatusTimeout);
                ok = false;
                break;
            }
        }
        // the tile to global memory: stored, or added to what earlier point chunks left there (read from L2:
        // in a batch another SM may have written it during this launch)
        const bool first = !x.accumulate;
        // a later K chunk of an ordered tile: the earlier chunks' values are final and visible (sequence flag), so
        // the additions go to L2 as reductions (the same FP32 sums in the same order, without reading the tile
        // back into the SM first)
        const bool reduce = !first && x.seq != nullptr;
        if (x.trans) {
            // accumulator row = hologram column m (the warp's 32 lanes hold 32
            // consecutive m), accumulator column = hologram row n: every store
            // instruction writes 128 contiguous bytes of out[n][m0 .. m0 + 31]
            const int m = row;
            const bool in_m = m < x.width;
            constexpr int TR = ROUND / 2;   // accumulator columns per round: 32 (or 16)
            constexpr int TG = TR / 16;
#pragma unroll 1
            for (int cc = 0; cc < x.bn; cc += TR) {
                const int ncol = min(TR, x.bn - cc);   // a multiple of 16
                const int n0 = x.tn * x.bn + cc;
                float old[TR];
                if (!first && !reduce && in_m) {
#pragma unroll
                    for (int i = 0; i < TR; ++i)
                        old[i] = (i < ncol && n0 + i < x.height) ? __ldcg(x.out + (long long)(n0 + i) * x.width + m)
                                                                 : 0.0f;
                }
                uint32_t r[TG][16];
#pragma unroll
                for (int g = 0; g < TG; ++g)
                    if (g == 0 || ncol > 16 * g) tmem_ld16(taddr + (uint32_t)(cc + 16 * g), r[g]);
                tmem_ld_wait();
                if (!in_m) continue;
#pragma unroll
                for (int i = 0; i < TR; ++i) {
                    if (i >= ncol || n0 + i >= x.height) continue;
                    float v = empty_range ? 0.0f : __uint_as_float(r[i >> 4][i & 15]) * unscale;
                    if (reduce) {
                        atomicAdd(x.out + (long long)(n0 + i) * x.width + m, v);
                        continue;
                    }
                    if (!first) v += old[i];
                    x.out[(long long)(n0 + i) * x.width + m] = v;
                }
            }
        } else {
#pragma unroll 1
            for (int cc = 0; cc < x.bn; cc += ROUND) {
                // ROUND columns per round (groups of 16): the previous partial sums (if any) are loaded first,
                // all at once, so the global-memory latency is paid once per round and overlaps the
                // tensor-memory reads
                constexpr int G = ROUND / 16;
                const int ncol = min(ROUND, x.bn - cc);   // a multiple of 16
                const int col0 = x.tn * x.bn + cc;
                const bool in_row = row < x.height;
                bool gvec[G];
#pragma unroll
                for (int gq = 0; gq < G; ++gq)
                    gvec[gq] = x.vec && in_row && gq * 16 < ncol && col0 + gq * 16 + 16 <= x.width;
                float4 old[4 * G];
#pragma unroll
                for (int gq = 0; gq < G; ++gq)
                    if (!first && !reduce && gvec[gq]) {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            old[4 * gq + i] = __ldcg(reinterpret_cast<const float4 *>(dst + col0 + 16 * gq) + i);
                    }
                uint32_t r[G][16];
#pragma unroll
                for (int gq = 0; gq < G; ++gq)
                    if (gq == 0 || ncol > 16 * gq) tmem_ld16(taddr + (uint32_t)(cc + 16 * gq), r[gq]);
                tmem_ld_wait();
                if (!in_row) continue;
#pragma unroll
                for (int gq = 0; gq < G; ++gq) {
                    if (gq * 16 >= ncol) continue;
                    float v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = empty_range ? 0.0f : __uint_as_float(r[gq][i]) * unscale;
                    float *d16 = dst + col0 + 16 * gq;
                    if (reduce) {
                        if (gvec[gq]) {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                atomicAdd(reinterpret_cast<float4 *>(d16) + i,
                                          make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (col0 + 16 * gq + i < x.width) atomicAdd(d16 + i, v[i]);
                        }
                        continue;
                    }
                    if (gvec[gq]) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float4 w = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                            if (!first) {
                                w.x += old[4 * gq + i].x;
                                w.y += old[4 * gq + i].y;
                                w.z += old[4 * gq + i].z;
                                w.w += old[4 * gq + i].w;
                            }
                            reinterpret_cast<float4 *>(d16)[i] = w;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (col0 + 16 * gq + i < x.width) d16[i] = first ? v[i] : __ldcg(d16 + i) + v[i];
                    }
                }
            }
        }
        if (x.seq != nullptr) {   // this warp's quarter of the tile is out: the next K chunk may add to it
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release(&x.seq[q], x.seq_k + 1);
        }
        tc_fence_before();
        release(tb);
    }
}

}  // namespace dev
}  // namespace cgh
