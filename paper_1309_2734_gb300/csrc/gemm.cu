// a4: the tensor-core form of the hologram, out[n][m] = sum_k P[n][k] Q[m][k]
// (I = P Q^T with the separable factors of factors.cu; K = 2N, both operands
// K-major 16-bit, FP32 accumulation in tensor memory).
//
// One persistent CTA per SM (192 threads):
//   warp 0      TMA producer: 2-D tiled loads (128-byte swizzle, no multicast)
//               of a 128 x 64 P tile and a BN x 64 Q tile per stage into a
//               ring of shared-memory stages guarded by full/empty mbarriers;
//   warp 1      TMEM allocation, and one thread issuing tcgen05.mma
//               (M = 128, N = BN, K = 16 per instruction) into one of two
//               TMEM accumulators, committing each stage back to its empty
//               barrier and each finished tile to the accumulator's full barrier;
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (each warp owns one
//               32-lane quarter = 32 rows), scaling, and stores to global
//               memory, then release of the accumulator.
// Two accumulators let the epilogue of one tile overlap the MMAs of the next.
//
// Work units are (K split, tile) pairs, numbered so that the units in flight
// at the same time share a K range: the P and Q slices they stream are then
// read from HBM about once and re-served from L2.
//
// Split FP16 (three products P_hi Q_hi^T + P_hi Q_lo^T + P_lo Q_hi^T) runs the
// three passes of a unit into the same accumulator.
//
// Accumulation chunks.  Long accumulation chains in TMEM lose accuracy much
// faster than round-to-nearest FP32 would (measured on GB300: NRMS ~1.5e-5
// after 9000 K elements of split FP16, growing about linearly with the
// chain), so a unit's K range is cut into chunks of kc k-blocks: each chunk
// is accumulated in TMEM from zero, and the epilogue adds it to the tile in
// global memory (L2-resident) in FP32, in a fixed order.
//
// Every wait is bounded; on a timeout the CTA latches kStatusTimeout, drains
// what it issued (again bounded), frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "device_util.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace cgh {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;   // 64 16-bit elements = one 128-byte swizzle row
constexpr int kGemmThreads = 192;

template <int BN>
struct GemmCfg {
    static constexpr int kStageA = kBM * kBK * 2;
    static constexpr int kStageB = BN * kBK * 2;
    static constexpr int kStageBytes = kStageA + kStageB;
    static constexpr int kStages = (200 * 1024) / kStageBytes > 8 ? 8 : (200 * 1024) / kStageBytes;
    static constexpr int kAccStride = BN <= 128 ? 128 : 256;   // TMEM columns between the two accumulators
    static constexpr int kTmemCols = 2 * kAccStride;
    static constexpr int kBarrierBytes = 256;
    static constexpr int kSmemBytes = 1024 + kStages * kStageBytes + kBarrierBytes;
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
    static_assert(kStageBytes % 1024 == 0, "stages must keep 1024-byte alignment");
};

template <int BN, bool SPLIT3>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tm_p, const __grid_constant__ CUtensorMap tm_q,
                const __grid_constant__ CUtensorMap tm_pl, const __grid_constant__ CUtensorMap tm_ql, int height,
                int width, int nkb, int splits, int tiles_m, int tiles_n, int kc, uint32_t idesc,
                float *__restrict__ out, long long slice_stride, bool vec, const float *__restrict__ amp_max,
                int *status, unsigned long long timeout_ns)
{
    using C = GemmCfg<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::kStages * C::kStageBytes);
    uint64_t *empty = full + C::kStages;
    uint64_t *tfull = empty + C::kStages;   // [2]
    uint64_t *tempty = tfull + 2;           // [2]
    uint64_t *drain = tempty + 2;           // [1]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = tiles_m * tiles_n;
    const int n_units = n_tiles * splits;
    constexpr int kPasses = SPLIT3 ? 3 : 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&tfull[0], 1);
        mbar_init(&tfull[1], 1);
        mbar_init(&tempty[0], 128);
        mbar_init(&tempty[1], 128);
        mbar_init(drain, 1);
        fence_barrier_init();
        tma_prefetch_map(&tm_p);
        tma_prefetch_map(&tm_q);
        if (SPLIT3) {
            tma_prefetch_map(&tm_pl);
            tma_prefetch_map(&tm_ql);
        }
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, C::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            uint32_t it = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
                const int split = u / n_tiles, t = u % n_tiles;
                const int tm = t % tiles_m, tn = t / tiles_m;
                const int kb0 = (int)((long long)split * nkb / splits);
                const int kb1 = (int)((long long)(split + 1) * nkb / splits);
                for (int c0 = kb0; c0 < kb1 && ok; c0 += kc) {
                    const int c1 = min(kb1, c0 + kc);
                    for (int pass = 0; pass < kPasses && ok; ++pass) {
                        const CUtensorMap *ma = (pass == 2) ? &tm_pl : &tm_p;
                        const CUtensorMap *mb = (pass == 1) ? &tm_ql : &tm_q;
                        for (int kb = c0; kb < c1; ++kb, ++it) {
                            const int s = (int)(it % C::kStages);
                            const uint32_t ph = (it / C::kStages) & 1u;
                            if (!mbar_wait(&empty[s], ph ^ 1u, timeout_ns)) {
                                atomicOr(status, kStatusTimeout);
                                ok = false;
                                break;
                            }
                            uint8_t *sa = smem + s * C::kStageBytes;
                            mbar_arrive_expect_tx(&full[s], C::kStageBytes);
                            tma_load_2d(sa, ma, &full[s], kb * kBK, tm * kBM);
                            tma_load_2d(sa + C::kStageA, mb, &full[s], kb * kBK, tn * BN);
                        }
                    }
                }
            }
            if (!ok) {
                // drain: wait (bounded) for the loads of the last kStages issues
                for (uint32_t j = (it > (uint32_t)C::kStages ? it - C::kStages : 0); j < it; ++j)
                    mbar_wait(&full[j % C::kStages], (j / C::kStages) & 1u, timeout_ns);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            uint32_t it = 0, ch = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
                const int split = u / n_tiles;
                const int kb0 = (int)((long long)split * nkb / splits);
                const int kb1 = (int)((long long)(split + 1) * nkb / splits);
                const int nch = kb1 > kb0 ? (kb1 - kb0 + kc - 1) / kc : 1;
              for (int c = 0; c < nch && ok; ++c, ++ch) {
                const int c0 = kb0 + c * kc, c1 = min(kb1, c0 + kc);
                const int b = (int)(ch & 1u);
                const uint32_t uph = (ch >> 1) & 1u;
                if (!mbar_wait(&tempty[b], uph ^ 1u, timeout_ns)) {
                    atomicOr(status, kStatusTimeout);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(b * C::kAccStride);
                uint32_t acc = 0;
                for (int pass = 0; pass < kPasses && ok; ++pass) {
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
                            umma_f16(d_tmem, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk), idesc, acc);
                            acc = 1;
                        }
                        umma_commit(&empty[s]);
                    }
                }
                if (!ok) break;
                // an empty K range issues no MMA; the epilogue then writes zeros itself
                umma_commit(&tfull[b]);
              }
            }
            // every MMA issued so far completes before TMEM is freed
            umma_commit(drain);
            mbar_wait(drain, 0, timeout_ns);
        }
    } else {
        // ---------------- epilogue ----------------
        const int q = warp & 3;   // TMEM lane quarter this warp may access
        const int row_in_tile = q * 32 + lane;
        float unscale = 1.0f;
        if (amp_max != nullptr) {
            const float m = *amp_max;
            if (m > 0.0f) unscale = m;
        }
        uint32_t ch = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
            const int split = u / n_tiles, t = u % n_tiles;
            const int tm = t % tiles_m, tn = t / tiles_m;
            const int kb0 = (int)((long long)split * nkb / splits);
            const int kb1 = (int)((long long)(split + 1) * nkb / splits);
            const bool empty_range = kb1 <= kb0;
            const int nch = kb1 > kb0 ? (kb1 - kb0 + kc - 1) / kc : 1;
          for (int c = 0; c < nch; ++c, ++ch) {
            // the first chunk stores, later chunks add (FP32, fixed order): each TMEM
            // accumulation chain stays kc k-blocks long
            const bool first = c == 0;
            const int b = (int)(ch & 1u);
            const uint32_t uph = (ch >> 1) & 1u;
            const bool arrived = mbar_wait(&tfull[b], uph, timeout_ns);
            if (!arrived) {
                atomicOr(status, kStatusTimeout);
                ok = false;
                break;
            }
            tc_fence_after();
            const int row = tm * kBM + row_in_tile;
            float *dst = out + (long long)split * slice_stride + (long long)row * width;
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * C::kAccStride);
#pragma unroll 1
            for (int c = 0; c < BN; c += 16) {
                uint32_t r[16];
                tmem_ld16(taddr + (uint32_t)c, r);
                tmem_ld_wait();
                if (row < height) {
                    const int col0 = tn * BN + c;
                    float v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = empty_range ? 0.0f : __uint_as_float(r[i]) * unscale;
                    if (vec && col0 + 16 <= width) {
#pragma unroll
                        for (int i = 0; i < 16; i += 4) {
                            float4 *p4 = reinterpret_cast<float4 *>(dst + col0 + i);
                            float4 w = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                            if (!first) {
                                const float4 o = *p4;
                                w.x += o.x;
                                w.y += o.y;
                                w.z += o.z;
                                w.w += o.w;
                            }
                            *p4 = w;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (col0 + i < width) dst[col0 + i] = first ? v[i] : dst[col0 + i] + v[i];
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[b]);
          }
        }
    }
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, C::kTmemCols);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// K-major 16-bit matrix [rows][ld] with 64 x box_rows boxes, 128-byte swizzle.
bool make_map(CUtensorMap *m, const void *base, bool bf16, int64_t ld, int64_t rows, int box_rows)
{
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                     const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int BN, bool SPLIT3>
cudaError_t launch_bn(const GemmPlan &plan, const CUtensorMap &p, const CUtensorMap &q, const CUtensorMap &pl,
                      const CUtensorMap &ql, int height, int width, int nkb, uint32_t idesc, float *out,
                      int64_t slice_stride, bool vec, const float *amp_max, int *status, uint64_t timeout_ns,
                      cudaStream_t s)
{
    using C = GemmCfg<BN>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(gemm_kernel<BN, SPLIT3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             C::kSmemBytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int tiles_m = (height + kBM - 1) / kBM;
    const int tiles_n = (width + BN - 1) / BN;
    const int units = tiles_m * tiles_n * plan.splits;
    const int ctas = plan.ctas < units ? plan.ctas : units;
    const int kc = plan.chunk_kb > 0 ? plan.chunk_kb : nkb;
    gemm_kernel<BN, SPLIT3><<<ctas, kGemmThreads, C::kSmemBytes, s>>>(
        p, q, pl, ql, height, width, nkb, plan.splits, tiles_m, tiles_n, kc, idesc, out, (long long)slice_stride,
        vec, amp_max, status, timeout_ns);
    return cudaGetLastError();
}

}  // namespace

int gemm_max_ctas(int num_sms)
{
    return num_sms;
}

cudaError_t launch_gemm(const GemmPlan &plan, const void *P, const void *Q, int height, int width, int64_t ld,
                        float *out, int64_t slice_stride, const float *amp_max, int *status, uint64_t timeout_ns,
                        cudaStream_t s)
{
    if (ld % kBK != 0 || plan.splits < 1 || plan.ctas < 1) return cudaErrorInvalidValue;
    const bool bf16 = plan.mode == kFactorBF16;
    const bool split3 = plan.mode == kFactorSplit16;
    const int bn = plan.bn;
    CUtensorMap tp, tq, tpl, tql;
    const uint16_t *p16 = static_cast<const uint16_t *>(P);
    const uint16_t *q16 = static_cast<const uint16_t *>(Q);
    if (!make_map(&tp, P, bf16, ld, height, kBM) || !make_map(&tq, Q, bf16, ld, width, bn)) return cudaErrorInvalidValue;
    if (split3) {
        if (!make_map(&tpl, p16 + (int64_t)height * ld, false, ld, height, kBM) ||
            !make_map(&tql, q16 + (int64_t)width * ld, false, ld, width, bn))
            return cudaErrorInvalidValue;
    } else {
        tpl = tp;
        tql = tq;
    }
    const int nkb = (int)(ld / kBK);
    const uint32_t idesc = umma_idesc_f16(bf16, kBM, bn);
    const bool vec = (width % 4 == 0) && (slice_stride % 4 == 0) && ((uintptr_t)out % 16 == 0);
#define CGH_GEMM_CASE(BNV)                                                                                         \
    case BNV:                                                                                                      \
        return split3 ? launch_bn<BNV, true>(plan, tp, tq, tpl, tql, height, width, nkb, idesc, out, slice_stride, \
                                             vec, amp_max, status, timeout_ns, s)                                  \
                      : launch_bn<BNV, false>(plan, tp, tq, tpl, tql, height, width, nkb, idesc, out,              \
                                              slice_stride, vec, amp_max, status, timeout_ns, s);
    switch (bn) {
        CGH_GEMM_CASE(128)
        CGH_GEMM_CASE(192)
        CGH_GEMM_CASE(240)
        CGH_GEMM_CASE(256)
    default:
        return cudaErrorInvalidValue;
    }
#undef CGH_GEMM_CASE
}

}  // namespace cgh
