// Host-side launchers of the library's kernels (internal; not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cgh {

// Points per shared-memory tile of the direct kernel; prepared point arrays
// are padded to a multiple of it.
constexpr int kPointTile = 256;

// a1: per-point constants and validation (prep.cu).
cudaError_t launch_prep_points(const float *d_xyz, const float *d_amp, int n, int n_pad, double pitch,
                               double lambda, int4 *geo, uint2 *aux, int *status, cudaStream_t s);

// a2: direct kernel (direct.cu).
struct DirectShape {
    int tile_w, tile_h;   // pixels covered by one CTA
    int threads;          // threads per CTA
};
DirectShape direct_shape(bool sfu);
cudaError_t launch_direct(bool sfu, const int4 *geo, const uint2 *aux, int n_pad, int width, int height,
                          int split, float *out, int64_t slice_stride, int *status, uint64_t timeout_ns,
                          cudaStream_t s);

// a5: fixed-order sum of `slices` planes of n floats (reduce.cu).
cudaError_t launch_reduce_slices(const float *parts, int slices, int64_t n, int64_t slice_stride, float *out,
                                 cudaStream_t s);

// a6: 8-bit min/max quantiser (quantize.cu). scratch holds 2 uint32.
cudaError_t launch_quantize8(const float *field, int64_t n, uint8_t *out, uint32_t *scratch, cudaStream_t s);

}  // namespace cgh
