// cgh_point_cloud_noalloc: the direct SFU hologram for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs where the
// allocator is forbidden or already exhausted (a host that hands out only
// pre-registered buffers, a real-time loop that may not allocate, a plug-in
// inside another program's memory budget).  cgh_create() allocates a
// context, and cgh_point_cloud() grows a workspace on demand, so neither suits
// them.  This entry point needs no context and allocates nothing: the
// prepared points live in one fixed scratch array in the library's own
// device memory, defined below, which every GPU that loads the library holds
// until the process exits.
//
// The scratch is shared by every call on a device and keeps the last call's
// contents.  The preparation kernel rewrites every entry a call reads, and the
// status word is cleared at the start of each call.  Calls that overlap on
// the GPU (from several host threads, or on several streams) race on the
// scratch and give wrong results: serialise them.
#include <cmath>
#include <mutex>

#include "../../include/cgh.h"
#include "device_util.cuh"
#include "kernels.h"

namespace {

using namespace cgh;

constexpr int64_t kMaxPoints = CGH_NOALLOC_MAX_POINTS;   // 131072 points
constexpr size_t kGeoBytes = (size_t)kMaxPoints * sizeof(int4);
constexpr size_t kAuxBytes = (size_t)kMaxPoints * sizeof(uint2);
constexpr size_t kScratchBytes = kGeoBytes + kAuxBytes + 256;   // + status word
constexpr int kMaxDevices = 64;

// 3 MiB + 256 B: prepared points (geo, aux) and the status word.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device and kept for the life of the
// process: after cudaDeviceReset() the module is loaded again and the kept address is stale, so the header tells
// callers not to use this entry point after a reset.
int scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return CGH_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return CGH_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return CGH_OK;
}

}  // namespace

// The direct kernel's CTA shape with the fewer padded pixels (one point chunk: no split to balance).
static cgh::DirectShape noalloc_shape(int width, int height)
{
    const cgh::DirectShape wide = cgh::direct_shape(false), tall = cgh::direct_shape(true);
    auto padded = [&](const cgh::DirectShape &sh) {
        return (int64_t)((width + sh.tile_w - 1) / sh.tile_w) * sh.tile_w *
               ((int64_t)((height + sh.tile_h - 1) / sh.tile_h) * sh.tile_h);
    };
    return padded(tall) < padded(wide) ? tall : wide;
}

extern "C" int cgh_point_cloud_noalloc(int width, int height, double pitch_m, double lambda_m, const float *d_xyz,
                                       const float *d_amp, int64_t n_points, float *d_out, void *cuda_stream)
{
    if (width < 1 || height < 1 || width > kMaxSide || height > kMaxSide) return CGH_EINVAL;
    if (!std::isfinite(pitch_m) || !std::isfinite(lambda_m) || !(pitch_m > 0.0) || !(lambda_m > 0.0))
        return CGH_EINVAL;
    if (!d_out || n_points < 0 || (n_points > 0 && (!d_xyz || !d_amp))) return CGH_EINVAL;
    if (n_points > kMaxPoints) return CGH_EINVAL;   // beyond the fixed scratch: use cgh_point_cloud
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CGH_ECUDA;
    }
    unsigned char *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    int4 *geo = reinterpret_cast<int4 *>(base);
    uint2 *aux = reinterpret_cast<uint2 *>(base + kGeoBytes);
    int *status = reinterpret_cast<int *>(base + kGeoBytes + kAuxBytes);
    const int64_t plane = (int64_t)width * height;
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return CGH_ECUDA;
    }
    if (n_points == 0) {
        if (cudaMemsetAsync(d_out, 0, (size_t)plane * sizeof(float), s) != cudaSuccess) {
            cudaGetLastError();
            return CGH_ECUDA;
        }
    } else {
        const int64_t n_pad = (n_points + kPointTile - 1) / kPointTile * kPointTile;   // <= kMaxPoints
        cudaError_t e = launch_prep_points(d_xyz, d_amp, (int)n_points, (int)n_pad, pitch_m, lambda_m, geo, aux,
                                           status, nullptr, s);
        if (e == cudaSuccess)
            e = launch_direct(true, noalloc_shape(width, height), geo, aux, (int)n_pad, width, height, 1, d_out,
                              plane, status, 5000000000ull, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return CGH_ECUDA;
        }
    }
    // wait for this call's work and read its status word (no allocation involved)
    int bits = 0;
    if (cudaMemcpyAsync(&bits, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return CGH_ECUDA;
    }
    if (bits & kStatusTimeout) return CGH_ETIMEOUT;
    if (bits & kStatusInput) return CGH_EINPUT;
    return CGH_OK;
}
