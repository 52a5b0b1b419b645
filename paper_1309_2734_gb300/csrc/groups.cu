// Point groups for the grouped GEMM form (depth-layered clouds).
//
// Points that share a depth plane (the same fixed-point constant C) and a
// column x share the column factor exp(i alpha(m)) of the separable form, so
//   I(m, n) = Re sum_g U_g(m) W_g(n),
//   U_g(m) = exp(i 2 pi c_g (m - x_g)^2),
//   W_g(n) = sum_{j in g} A_j exp(i 2 pi c_j (n - y_j)^2),
// and the GEMM runs over K = 2 G (G = number of groups) instead of 2 N.  For
// 10^6 points on 16 planes of a 4096-wide hologram G <= 16 x 4096: 15x less
// tensor work, the same sum (only rounding differs).
//
// Grouping, all on the device except two small reads of counts:
//   1. distinct C values (at most kMaxPlanes) in a small open-addressing hash
//      set, then sorted, so plane ids are deterministic;
//   2. key = plane id * kXSpan + (x + kMaxCoord), a counting sort: histogram,
//      exclusive scans of the counts and of the non-empty flags, scatter;
//   3. each group's members sorted by point index (fixed summation order) and
//      gathered, in group order, as compact {y, -A} records.
// The host reads the plane count after step 1 and the group count and largest
// group after step 2, and keeps the ungrouped form when grouping does not pay.
#include "device_util.cuh"
#include "kernels.h"

namespace cgh {

namespace {

constexpr int kPlaneSlots = 2 * kMaxPlanes;    // hash set capacity (load factor <= 1/2)
constexpr unsigned long long kEmptySlot = ~0ull;
constexpr int kScanBlock = 1024;
static_assert(kXSpan == 2 * kMaxCoord + 1, "one key per column a point may occupy");

__device__ __forceinline__ unsigned long long c_of(const int4 g)
{
    return ((unsigned long long)(uint32_t)g.z << 32) | (uint32_t)g.w;
}

// Distinct C values: each block first collects its points' values in a shared-memory set of the same capacity
// and inserts only those into the global set, so a layered cloud costs one global probe sequence per (block,
// plane), and a cloud with more than kMaxPlanes depths stops at its first block (no block walks a full set).
__global__ void planes_insert(const int4 *__restrict__ geo, int n, unsigned long long *slots, int *overflow)
{
    __shared__ unsigned long long local[kPlaneSlots];
    __shared__ int n_local, full;
    if (threadIdx.x == 0) {
        n_local = 0;
        full = *(volatile int *)overflow;   // already more planes than the set holds
    }
    for (int i = threadIdx.x; i < kPlaneSlots; i += blockDim.x) local[i] = kEmptySlot;
    __syncthreads();
    if (full) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        const unsigned long long c = c_of(geo[j]);
        unsigned int h = (unsigned int)((c * 0x9e3779b97f4a7c15ull) >> 40) % kPlaneSlots;
        for (int probe = 0; probe < kPlaneSlots && !*(volatile int *)&full; ++probe) {
            const unsigned long long prev = atomicCAS(&local[h], kEmptySlot, c);
            if (prev == c) break;
            if (prev == kEmptySlot) {
                if (atomicAdd(&n_local, 1) >= kMaxPlanes) atomicExch(&full, 1);
                break;
            }
            h = (h + 1) % kPlaneSlots;
        }
    }
    __syncthreads();
    if (full || n_local > kMaxPlanes) {
        if (threadIdx.x == 0) atomicExch(overflow, 1);
        return;
    }
    for (int i = threadIdx.x; i < kPlaneSlots; i += blockDim.x) {
        const unsigned long long c = local[i];
        if (c == kEmptySlot) continue;
        unsigned int h = (unsigned int)((c * 0x9e3779b97f4a7c15ull) >> 40) % kPlaneSlots;
        int probe = 0;
        for (; probe < kPlaneSlots; ++probe) {
            // plain read first: a present value costs reads, not contended atomics
            const unsigned long long seen = *(volatile unsigned long long *)&slots[h];
            if (seen == c) break;
            if (seen == kEmptySlot) {
                const unsigned long long prev = atomicCAS(&slots[h], kEmptySlot, c);
                if (prev == kEmptySlot || prev == c) break;
            }
            h = (h + 1) % kPlaneSlots;
        }
        if (probe == kPlaneSlots) atomicExch(overflow, 1);
    }
}

// One block: the distinct values, sorted; meta[0] = count (or -1 beyond kMaxPlanes).
__global__ void planes_finalize(const unsigned long long *slots, unsigned long long *planes, int *meta,
                                const int *overflow)
{
    __shared__ unsigned long long v[kPlaneSlots];
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < kPlaneSlots; i += blockDim.x) {
        const unsigned long long s = slots[i];
        if (s != kEmptySlot) v[atomicAdd(&cnt, 1)] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int c = cnt;
        for (int i = 1; i < c; ++i) {   // insertion sort of <= kPlaneSlots values
            const unsigned long long x = v[i];
            int k = i - 1;
            while (k >= 0 && v[k] > x) {
                v[k + 1] = v[k];
                --k;
            }
            v[k + 1] = x;
        }
        for (int i = 0; i < c; ++i) planes[i] = v[i];
        meta[0] = (*overflow || c > kMaxPlanes) ? -1 : c;
    }
}

__device__ __forceinline__ int plane_id(const unsigned long long *planes, int np, unsigned long long c)
{
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (planes[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void group_histogram(const int4 *__restrict__ geo, int n, const unsigned long long *planes, int np,
                                int *key_of, int *counts)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int4 g = geo[j];
    const int key = plane_id(planes, np, c_of(g)) * kXSpan + (g.x + kMaxCoord);
    key_of[j] = key;
    atomicAdd(&counts[key], 1);
}

// Exclusive scans of counts (-> offsets) and of non-empty flags (-> group index), per block of kScanBlock.
__global__ void scan_blocks(const int *__restrict__ counts, int nkeys, int2 *__restrict__ scan, int2 *block_sums)
{
    __shared__ int2 s[kScanBlock];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    const int c = i < nkeys ? counts[i] : 0;
    s[threadIdx.x] = make_int2(c, c > 0 ? 1 : 0);
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {   // Hillis-Steele inclusive scan
        int2 add = make_int2(0, 0);
        if ((int)threadIdx.x >= off) add = s[threadIdx.x - off];
        __syncthreads();
        s[threadIdx.x].x += add.x;
        s[threadIdx.x].y += add.y;
        __syncthreads();
    }
    const int2 incl = s[threadIdx.x];
    if (i < nkeys) scan[i] = make_int2(incl.x - c, incl.y - (c > 0 ? 1 : 0));
    if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = incl;
}

// One block: exclusive scan of the block sums in place; meta[1] = points, meta[2] = groups.
__global__ void scan_sums(int2 *block_sums, int nblocks, int *meta)
{
    if (threadIdx.x != 0) return;
    int2 run = make_int2(0, 0);
    for (int b = 0; b < nblocks; ++b) {
        const int2 v = block_sums[b];
        block_sums[b] = run;
        run.x += v.x;
        run.y += v.y;
    }
    meta[1] = run.x;
    meta[2] = run.y;
}

// Adds the block offsets; writes each non-empty key's group descriptor.
__global__ void scan_finish(const int *__restrict__ counts, int nkeys, int2 *scan, const int2 *block_sums,
                            int4 *groups, int *max_count)
{
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i >= nkeys) return;
    const int2 b = block_sums[blockIdx.x];
    int2 v = scan[i];
    v.x += b.x;
    v.y += b.y;
    scan[i] = v;
    const int c = counts[i];
    if (c > 0) {
        groups[v.y] = make_int4(v.x, c, i / kXSpan, i % kXSpan - kMaxCoord);   // {first, count, plane, x}
        atomicMax(max_count, c);
    }
}

__global__ void group_scatter(const int *__restrict__ key_of, int n, const int2 *__restrict__ scan, int *cursor,
                              int *perm)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int key = key_of[j];
    perm[scan[key].x + atomicAdd(&cursor[key], 1)] = j;
}

// Each group's members in ascending point order (a fixed summation order).
// Groups hold at most kMaxGroupPoints points when this runs (the host checks
// the largest count first), so the insertion sort is bounded.
__global__ void group_order(const int4 *__restrict__ groups, const int *meta, int *perm)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= meta[2]) return;   // groups beyond the count were never written
    const int4 d = groups[g];
    int *p = perm + d.x;
    for (int i = 1; i < d.y; ++i) {
        const int x = p[i];
        int k = i - 1;
        while (k >= 0 && p[k] > x) {
            p[k + 1] = p[k];
            --k;
        }
        p[k + 1] = x;
    }
}

// Members in group order as {y, -A}: the row factor needs only these (the
// plane constant comes from the sorted plane table, the column from the group).
__global__ void group_gather(const int *__restrict__ perm, int n, const int4 *__restrict__ geo,
                             const uint2 *__restrict__ aux, int2 *__restrict__ members)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = perm[i];
    members[i] = make_int2(geo[j].y, (int)(__float_as_uint(-__uint_as_float(aux[j].y))));
}

__global__ void group_scale(const float *amp_max, const int *max_count, float *wscale)
{
    const float a = *amp_max > 0.0f ? *amp_max : 1.0f;
    *wscale = a * (float)max(*max_count, 1);
}

int blocks(long long n, int t)
{
    return (int)((n + t - 1) / t);
}

}  // namespace

namespace {

constexpr size_t kHeaderBytes = 2 * kPlaneSlots * sizeof(unsigned long long) + 256;

struct GroupScratch {
    unsigned long long *slots, *planes;
    int *overflow, *counts, *cursor, *key_of, *perm;
    int2 *scan, *bsums;
    long long nkeys;
    int nblocks;
};

GroupScratch carve(void *scratch, int n, int n_planes)
{
    GroupScratch w;
    w.slots = static_cast<unsigned long long *>(scratch);
    w.planes = w.slots + kPlaneSlots;
    w.overflow = reinterpret_cast<int *>(w.planes + kPlaneSlots);
    char *base = static_cast<char *>(scratch) + kHeaderBytes;
    w.nkeys = (long long)n_planes * kXSpan;
    w.nblocks = (int)((w.nkeys + kScanBlock - 1) / kScanBlock);
    w.counts = reinterpret_cast<int *>(base);
    w.cursor = w.counts + w.nkeys;
    w.scan = reinterpret_cast<int2 *>(w.cursor + w.nkeys);
    w.bsums = w.scan + w.nkeys;
    w.key_of = reinterpret_cast<int *>(w.bsums + w.nblocks);
    w.perm = w.key_of + n;
    return w;
}

}  // namespace

size_t group_workspace_bytes(int n, int n_planes)
{
    const size_t nkeys = (size_t)n_planes * kXSpan;
    const size_t nblocks = (nkeys + kScanBlock - 1) / kScanBlock;
    return kHeaderBytes + nkeys * (2 * sizeof(int) + sizeof(int2)) + nblocks * sizeof(int2) +
           (size_t)n * 2 * sizeof(int) + 256;
}

const unsigned long long *group_plane_table(const void *scratch)
{
    return static_cast<const unsigned long long *>(scratch) + kPlaneSlots;
}

cudaError_t launch_planes(const int4 *geo, int n, void *scratch, int *meta, cudaStream_t s)
{
    const GroupScratch w = carve(scratch, n, 0);
    cudaError_t e = cudaMemsetAsync(w.slots, 0xff, kPlaneSlots * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.overflow, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (n > 0) planes_insert<<<blocks(n, 256), 256, 0, s>>>(geo, n, w.slots, w.overflow);
    planes_finalize<<<1, 128, 0, s>>>(w.slots, w.planes, meta, w.overflow);
    return cudaGetLastError();
}

cudaError_t launch_group_count(const int4 *geo, int n, int n_planes, void *scratch, int *meta, int4 *groups,
                               cudaStream_t s)
{
    const GroupScratch w = carve(scratch, n, n_planes);
    cudaError_t e = cudaMemsetAsync(w.counts, 0, (size_t)w.nkeys * 2 * sizeof(int), s);   // counts and cursors
    if (e == cudaSuccess) e = cudaMemsetAsync(meta + 3, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (n > 0) group_histogram<<<blocks(n, 256), 256, 0, s>>>(geo, n, w.planes, n_planes, w.key_of, w.counts);
    scan_blocks<<<w.nblocks, kScanBlock, 0, s>>>(w.counts, (int)w.nkeys, w.scan, w.bsums);
    scan_sums<<<1, 32, 0, s>>>(w.bsums, w.nblocks, meta);
    scan_finish<<<w.nblocks, kScanBlock, 0, s>>>(w.counts, (int)w.nkeys, w.scan, w.bsums, groups, meta + 3);
    return cudaGetLastError();
}

cudaError_t launch_group_build(const int4 *geo, const uint2 *aux, int n, int n_planes, int n_groups, void *scratch,
                               const int *meta, const int4 *groups, const float *amp_max, float *wscale,
                               int2 *members, cudaStream_t s)
{
    const GroupScratch w = carve(scratch, n, n_planes);
    if (n > 0) {
        group_scatter<<<blocks(n, 256), 256, 0, s>>>(w.key_of, n, w.scan, w.cursor, w.perm);
        if (n_groups > 0) group_order<<<blocks(n_groups, 128), 128, 0, s>>>(groups, meta, w.perm);
        group_gather<<<blocks(n, 256), 256, 0, s>>>(w.perm, n, geo, aux, members);
    }
    group_scale<<<1, 1, 0, s>>>(amp_max, meta + 3, wscale);
    return cudaGetLastError();
}

}  // namespace cgh
