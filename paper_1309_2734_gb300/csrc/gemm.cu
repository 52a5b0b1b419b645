// a4: the tensor-core form of the hologram, out[n][m] = sum_k P[n][k] Q[m][k]
// (I = P Q^T with the separable factors of factors.cu; K = 2N, both operands
// K-major 16-bit, FP32 accumulation in tensor memory).
//
// One persistent CTA per SM (192 threads):
//   warp 0      TMA producer: 2-D tiled loads (128-byte swizzle, no multicast)
//               of a 128 x 64 P tile and a bn x 64 Q tile per stage into a
//               ring of shared-memory stages guarded by full/empty mbarriers;
//   warp 1      TMEM allocation, and one thread issuing tcgen05.mma
//               (M = 128, N = bn, K = 16 per instruction) into one of two
//               TMEM accumulators, committing each stage back to its empty
//               barrier and each finished chunk to the accumulator's full barrier;
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (each warp owns one
//               32-lane quarter = 32 rows), scaling, and stores to global
//               memory, then release of the accumulator.
// Two accumulators let the epilogue of one chunk overlap the MMAs of the next.
//
// Work units.  For one hologram, units are (K split, tile) pairs, numbered so
// that the units in flight at the same time share a K range: the P and Q
// slices they stream are then read from HBM about once and re-served from L2.
// For a batch of holograms, every CTA walks its own list of (job, tile) units,
// and each job (one hologram) carries its own tensor maps, shape, tile width,
// pass count and output in global memory, so holograms of different sizes and
// precisions share one launch.
//
// Split FP16 (three products P_hi Q_hi^T + P_hi Q_lo^T + P_lo Q_hi^T) runs the
// three passes of a chunk into the same accumulator.
//
// Accumulation chunks.  Long accumulation chains in TMEM lose accuracy much
// faster than round-to-nearest FP32 would (measured on GB300: NRMS ~1.5e-5
// after 9000 K elements of split FP16, growing about linearly with the
// chain), so a unit's K range is cut into chunks of kc k-blocks, each
// accumulated in TMEM from zero.  A unit of several chunks keeps its running
// total in tensor memory: the first chunk goes to one accumulator (the
// total), every later chunk to the other, and the epilogue adds it to the
// total (tcgen05.ld both, FP32 add, tcgen05.st) in a fixed order; the tile
// reaches global memory once.  The next unit's total takes the accumulator
// the last chunk used, so its first chunk overlaps the previous write-out.
//
// Every wait is bounded; on a timeout the CTA latches kStatusTimeout, drains
// what it issued (again bounded), frees its TMEM and returns.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "gemm_dev.cuh"
#include "host_util.h"
#include "kernels.h"

namespace cgh {

namespace {

using namespace dev;

// One hologram: everything in the (grid-constant) kernel parameters.
struct alignas(64) SingleUnits {
    CUtensorMap p, q, pl, ql;
    float *out;
    const float *amp_max;
    long long slice_stride;
    int height, width, nkb, splits, tiles_m, tiles_n, kc, passes, bn;
    uint32_t idesc;
    int vec;
    int accumulate;
    int trans;

    // every role walks units blockIdx.x, blockIdx.x + gridDim.x, ...
    struct Cursor {
        int u;
    };
    __device__ Cursor start() const { return Cursor{(int)blockIdx.x}; }
    __device__ bool next(int, Cursor &c, UnitInfo &x) const
    {
        if (c.u >= tiles_m * tiles_n * splits) return false;
        x = get(c.u);
        c.u += gridDim.x;
        return true;
    }
    __device__ bool ready(const UnitInfo &, int, int &, unsigned long long) const { return true; }
    __device__ void abort(Cursor &, unsigned long long) const {}
    __device__ UnitInfo get(int u) const
    {
        const int n_tiles = tiles_m * tiles_n;
        const int split = u / n_tiles, t = u % n_tiles;
        UnitInfo x;
        x.mp = &p;
        x.mq = &q;
        x.mpl = &pl;
        x.mql = &ql;
        x.out = out + (long long)split * slice_stride;
        x.amp_max = amp_max;
        x.tm = t % tiles_m;
        x.row0 = x.tm * kBM;
        x.tn = t / tiles_m;
        x.kb0 = (int)((long long)split * nkb / splits);
        x.kb1 = (int)((long long)(split + 1) * nkb / splits);
        x.bn = bn;
        x.passes = passes;
        x.kc = kc;
        x.height = height;
        x.width = width;
        x.idesc = idesc;
        x.vec = vec != 0;
        x.accumulate = accumulate != 0;
        x.trans = trans != 0;
        return x;
    }
};

// A batch: per-CTA unit lists over a job table in global memory.
struct BatchUnits {
    const GemmJob *jobs;
    const int *cta_off;     // [ctas + 1]
    const int2 *units;      // {job, tile}

    // every role walks the CTA's own list
    struct Cursor {
        int i;
    };
    __device__ Cursor start() const { return Cursor{cta_off[blockIdx.x]}; }
    __device__ bool next(int, Cursor &c, UnitInfo &x) const
    {
        if (c.i >= cta_off[blockIdx.x + 1]) return false;
        x = get(c.i);
        ++c.i;
        return true;
    }
    __device__ bool ready(const UnitInfo &, int, int &, unsigned long long) const { return true; }
    __device__ void abort(Cursor &, unsigned long long) const {}
    __device__ UnitInfo get(int i) const
    {
        const int2 w = units[i];
        const GemmJob &J = jobs[w.x];
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
        x.kb0 = 0;
        x.kb1 = J.nkb;
        x.bn = J.bn;
        x.passes = J.passes;
        x.kc = J.kc;
        x.height = J.height;
        x.width = J.width;
        x.idesc = J.idesc;
        x.vec = J.vec != 0;
        x.accumulate = false;
        x.trans = J.trans != 0;
        return x;
    }
};

template <int BN_MAX, class Units>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_kernel(const __grid_constant__ Units src, int *status, unsigned long long timeout_ns)
{
    using C = GemmCfg<BN_MAX>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const GemmBars bars = gemm_bars<C>(smem);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars.drain + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) gemm_init_barriers<C>(bars);
    if (warp == 1) {
        tmem_alloc(tmem_slot, C::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    if (warp == 0) {
        if (lane == 0) gemm_producer<C>(src, smem, bars, status, timeout_ns);
    } else if (warp == 1) {
        if (lane == 0) gemm_mma<C>(src, smem, bars, tmem_base, status, timeout_ns);
    } else {
        gemm_epilogue<C>(src, bars, tmem_base, warp, lane, status, timeout_ns);
    }
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, C::kTmemCols);
    }
}

// ---- the two-SM form: clusters of two CTAs, M = 256 ----------------------------------------------------------

// Stages of a CTA of the pair: its 128 x 64 tile of A and its half (BN/2 rows) of the BN x 64 tile of B, so a
// stage is 30 KB at BN = 224 and seven fit where five of the single-CTA form's 44 KB stages did.
template <int BN>
struct GemmPairCfg {
    static constexpr int kStageA = kBM * kBK * 2;
    static constexpr int kStageB = (BN / 2) * kBK * 2;
    static constexpr int kStageBytes = kStageA + kStageB;
    static constexpr int kStages = kStageRoom / kStageBytes > 8 ? 8 : kStageRoom / kStageBytes;
    static constexpr int kAccStride = BN <= 128 ? 128 : 256;
    static constexpr int kTmemCols = 2 * kAccStride;
    static constexpr int kBarrierBytes = 256;
    static constexpr int kSmemBytes = 1024 + kStages * kStageBytes + kBarrierBytes;
    static_assert(BN % 32 == 0 && BN >= 64 && BN <= 256, "UMMA N for M = 256, halves of whole swizzle atoms");
    static_assert(kStageBytes % 1024 == 0, "stages must keep 1024-byte alignment");
};

// One hologram in 256-row tiles: cluster c (CTAs 2c and 2c + 1) walks units c, c + clusters, ...; CTA rank r
// holds rows [256 tm + 128 r, + 128) of the tile.
struct alignas(64) PairUnits {
    CUtensorMap p, q, pl, ql;   // B maps with boxes of bn / 2 rows
    float *out;
    const float *amp_max;
    long long slice_stride;
    int height, width, nkb, splits, tiles_m, tiles_n, kc, passes, bn;
    uint32_t idesc;
    int vec;
    int accumulate;
    int trans;

    struct Cursor {
        int u;
    };
    __device__ Cursor start() const { return Cursor{(int)(blockIdx.x >> 1)}; }
    __device__ bool next(int, Cursor &c, UnitInfo &x) const
    {
        if (c.u >= tiles_m * tiles_n * splits) return false;
        x = get(c.u);
        c.u += (int)(gridDim.x >> 1);
        return true;
    }
    __device__ bool ready(const UnitInfo &, int, int &, unsigned long long) const { return true; }
    __device__ void abort(Cursor &, unsigned long long) const {}
    __device__ UnitInfo get(int u) const
    {
        const int n_tiles = tiles_m * tiles_n;
        const int split = u / n_tiles, t = u % n_tiles;
        UnitInfo x;
        x.mp = &p;
        x.mq = &q;
        x.mpl = &pl;
        x.mql = &ql;
        x.out = out + (long long)split * slice_stride;
        x.amp_max = amp_max;
        x.tm = t % tiles_m;
        x.tn = t / tiles_m;
        x.row0 = x.tm * 2 * kBM + (int)cluster_rank() * kBM;
        x.kb0 = (int)((long long)split * nkb / splits);
        x.kb1 = (int)((long long)(split + 1) * nkb / splits);
        x.bn = bn;
        x.passes = passes;
        x.kc = kc;
        x.height = height;
        x.width = width;
        x.idesc = idesc;
        x.vec = vec != 0;
        x.accumulate = accumulate != 0;
        x.trans = trans != 0;
        return x;
    }
};

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_pair_kernel(const __grid_constant__ PairUnits src, int *status, unsigned long long timeout_ns)
{
    using C = GemmPairCfg<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const GemmBars bars = gemm_bars<C>(smem);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars.drain + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) {
            mbar_init(&bars.full[s], 1);
            mbar_init(&bars.empty[s], 1);
        }
        mbar_init(&bars.tfull[0], 1);
        mbar_init(&bars.tfull[1], 1);
        mbar_init(&bars.tempty[0], 256);   // both CTAs' epilogue threads (only the even CTA's are used)
        mbar_init(&bars.tempty[1], 256);
        mbar_init(bars.drain, 1);
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc_pair(tmem_slot, C::kTmemCols);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    cluster_sync();   // both CTAs' barriers initialised and tensor memory allocated
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    if (warp == 0) {
        if (lane == 0) gemm_producer_pair<C>(src, smem, bars, rank, status, timeout_ns);
    } else if (warp == 1) {
        if (lane == 0) {
            if (rank == 0) gemm_mma_pair<C>(src, smem, bars, tmem_base, status, timeout_ns);
            else mbar_wait(bars.drain, 0, timeout_ns);   // the even CTA's last commit: its MMAs are done
        }
    } else {
        gemm_epilogue<C, PairUnits, 64, true>(src, bars, tmem_base, warp, lane, status, timeout_ns);
    }
    tc_fence_before();
    cluster_sync();   // no CTA leaves while the other may still arrive on its barriers
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc_pair(tmem_base, C::kTmemCols);
    }
}

template <int BN>
cudaError_t launch_pair(const PairUnits &u, int clusters, int *status, uint64_t timeout_ns, cudaStream_t s)
{
    using C = GemmPairCfg<BN>;
    static PerDeviceOnce configured;
    cudaError_t e = configured.run([] {
        return cudaFuncSetAttribute(gemm_pair_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    });
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters, 1, 1);
    cfg.blockDim = dim3(kGemmThreads, 1, 1);
    cfg.dynamicSmemBytes = C::kSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, gemm_pair_kernel<BN>, u, status, (unsigned long long)timeout_ns);
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

template <int BN_MAX, class Units>
cudaError_t configure()
{
    static PerDeviceOnce done;
    return done.run([] {
        return cudaFuncSetAttribute(gemm_kernel<BN_MAX, Units>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    GemmCfg<BN_MAX>::kSmemBytes);
    });
}

template <int BN>
cudaError_t launch_single(const SingleUnits &u, int ctas, int *status, uint64_t timeout_ns, cudaStream_t s)
{
    cudaError_t e = configure<BN, SingleUnits>();
    if (e != cudaSuccess) return e;
    gemm_kernel<BN, SingleUnits><<<ctas, kGemmThreads, GemmCfg<BN>::kSmemBytes, s>>>(u, status, timeout_ns);
    return cudaGetLastError();
}

}  // namespace

// K-major 16-bit matrix [rows][ld] with 64 x box_rows boxes, 128-byte swizzle.
bool make_operand_map(CUtensorMap *m, const void *base, bool bf16, int64_t ld, int64_t rows, int box_rows)
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

int gemm_max_ctas(int num_sms)
{
    return num_sms;
}

bool gemm_bn_supported(int bn)
{
    return bn == 128 || bn == 192 || bn == 224 || bn == 240 || bn == 256;
}

cudaError_t launch_gemm(const GemmPlan &plan, const void *P, const void *Q, int height, int width, int64_t ld,
                        float *out, int64_t slice_stride, const float *amp_max, int *status, uint64_t timeout_ns,
                        cudaStream_t s)
{
    if (ld % kBK != 0 || plan.splits < 1 || plan.ctas < 1 || !gemm_bn_supported(plan.bn))
        return cudaErrorInvalidValue;
    const bool bf16 = plan.mode == kFactorBF16;
    const bool split3 = plan.mode == kFactorSplit16;
    const int bn = plan.bn;
    SingleUnits u;
    // A operand: 128-row tiles of P (or of Q when transposed); B operand: bn-row tiles of the other
    const bool tr = plan.trans;
    const void *A = tr ? Q : P, *B = tr ? P : Q;
    const int a_rows = tr ? width : height, b_rows = tr ? height : width;
    const uint16_t *a16 = static_cast<const uint16_t *>(A);
    const uint16_t *b16 = static_cast<const uint16_t *>(B);
    if (!make_operand_map(&u.p, A, bf16, ld, a_rows, kBM) || !make_operand_map(&u.q, B, bf16, ld, b_rows, bn))
        return cudaErrorInvalidValue;
    if (split3) {
        if (!make_operand_map(&u.pl, a16 + (int64_t)a_rows * ld, false, ld, a_rows, kBM) ||
            !make_operand_map(&u.ql, b16 + (int64_t)b_rows * ld, false, ld, b_rows, bn))
            return cudaErrorInvalidValue;
    } else {
        u.pl = u.p;
        u.ql = u.q;
    }
    u.trans = tr ? 1 : 0;
    u.nkb = (int)(ld / kBK);
    u.out = out;
    u.amp_max = amp_max;
    u.slice_stride = (long long)slice_stride;
    u.height = height;
    u.width = width;
    u.splits = plan.splits;
    u.tiles_m = (a_rows + kBM - 1) / kBM;
    u.tiles_n = (b_rows + bn - 1) / bn;
    u.kc = plan.chunk_kb > 0 ? plan.chunk_kb : u.nkb;
    u.passes = split3 ? 3 : 1;
    u.bn = bn;
    u.idesc = umma_idesc_f16(bf16, kBM, bn);
    u.vec = (width % 4 == 0) && (slice_stride % 4 == 0) && ((uintptr_t)out % 16 == 0);
    u.accumulate = plan.accumulate ? 1 : 0;
    if (plan.pair) {
        // the two-SM form: 256-row tiles, B maps with boxes of bn / 2 rows (whole 32-row groups: not at 240)
        if (bn == 240) return cudaErrorInvalidValue;
        PairUnits v;
        v.p = u.p;
        v.pl = u.pl;
        if (!make_operand_map(&v.q, B, bf16, ld, b_rows, bn / 2)) return cudaErrorInvalidValue;
        if (split3) {
            if (!make_operand_map(&v.ql, b16 + (int64_t)b_rows * ld, false, ld, b_rows, bn / 2))
                return cudaErrorInvalidValue;
        } else {
            v.ql = v.q;
        }
        v.out = u.out;
        v.amp_max = u.amp_max;
        v.slice_stride = u.slice_stride;
        v.height = u.height;
        v.width = u.width;
        v.nkb = u.nkb;
        v.splits = u.splits;
        v.tiles_m = (a_rows + 2 * kBM - 1) / (2 * kBM);
        v.tiles_n = u.tiles_n;
        v.kc = u.kc;
        v.passes = u.passes;
        v.bn = bn;
        v.idesc = umma_idesc_f16(bf16, 2 * kBM, bn);
        v.vec = u.vec;
        v.accumulate = u.accumulate;
        v.trans = u.trans;
        const int pair_units = v.tiles_m * v.tiles_n * v.splits;
        const int clusters = std::min(plan.ctas / 2, pair_units);
        switch (bn) {
        case 128: return launch_pair<128>(v, clusters, status, timeout_ns, s);
        case 192: return launch_pair<192>(v, clusters, status, timeout_ns, s);
        case 224: return launch_pair<224>(v, clusters, status, timeout_ns, s);
        default: return launch_pair<256>(v, clusters, status, timeout_ns, s);
        }
    }
    const int units = u.tiles_m * u.tiles_n * u.splits;
    const int ctas = plan.ctas < units ? plan.ctas : units;
    switch (bn) {
    case 128: return launch_single<128>(u, ctas, status, timeout_ns, s);
    case 192: return launch_single<192>(u, ctas, status, timeout_ns, s);
    case 224: return launch_single<224>(u, ctas, status, timeout_ns, s);
    case 240: return launch_single<240>(u, ctas, status, timeout_ns, s);
    default: return launch_single<256>(u, ctas, status, timeout_ns, s);
    }
}

bool fill_gemm_job(GemmJob *job, int mode, int bn, const void *P, const void *Q, int height, int width, int64_t ld,
                   int chunk_kb, float *out, const float *amp_max, bool trans)
{
    if (ld % kBK != 0 || !gemm_bn_supported(bn)) return false;
    const bool bf16 = mode == kFactorBF16;
    const bool split3 = mode == kFactorSplit16;
    // A operand: 128-row tiles of P (or of Q when transposed); B operand: bn-row tiles of the other
    const void *A = trans ? Q : P, *B = trans ? P : Q;
    const int a_rows = trans ? width : height, b_rows = trans ? height : width;
    const uint16_t *a16 = static_cast<const uint16_t *>(A);
    const uint16_t *b16 = static_cast<const uint16_t *>(B);
    if (!make_operand_map(&job->p, A, bf16, ld, a_rows, kBM) || !make_operand_map(&job->q, B, bf16, ld, b_rows, bn))
        return false;
    if (split3) {
        if (!make_operand_map(&job->pl, a16 + (int64_t)a_rows * ld, false, ld, a_rows, kBM) ||
            !make_operand_map(&job->ql, b16 + (int64_t)b_rows * ld, false, ld, b_rows, bn))
            return false;
    } else {
        job->pl = job->p;
        job->ql = job->q;
    }
    job->out = out;
    job->amp_max = amp_max;
    job->height = height;
    job->width = width;
    job->nkb = (int)(ld / kBK);
    job->tiles_m = (a_rows + kBM - 1) / kBM;
    job->tiles_n = (b_rows + bn - 1) / bn;
    job->kc = chunk_kb > 0 ? chunk_kb : job->nkb;
    job->passes = split3 ? 3 : 1;
    job->bn = bn;
    job->idesc = umma_idesc_f16(bf16, kBM, bn);
    job->vec = (width % 4 == 0) && ((uintptr_t)out % 16 == 0);
    job->trans = trans ? 1 : 0;
    return true;
}

template <int BN_MAX>
cudaError_t launch_batch_as(const GemmJob *d_jobs, const int *d_cta_off, const int2 *d_units, int ctas, int *status,
                            uint64_t timeout_ns, cudaStream_t s)
{
    cudaError_t e = configure<BN_MAX, BatchUnits>();
    if (e != cudaSuccess) return e;
    BatchUnits u{d_jobs, d_cta_off, d_units};
    gemm_kernel<BN_MAX, BatchUnits><<<ctas, kGemmThreads, GemmCfg<BN_MAX>::kSmemBytes, s>>>(u, status, timeout_ns);
    return cudaGetLastError();
}

cudaError_t launch_gemm_batch(const GemmJob *d_jobs, const int *d_cta_off, const int2 *d_units, int ctas,
                              int bn_max, int *status, uint64_t timeout_ns, cudaStream_t s)
{
    if (ctas <= 0) return cudaSuccess;
    if (bn_max <= 224) return launch_batch_as<224>(d_jobs, d_cta_off, d_units, ctas, status, timeout_ns, s);
    return launch_batch_as<256>(d_jobs, d_cta_off, d_units, ctas, status, timeout_ns, s);
}

}  // namespace cgh
