// a1: point preparation.  One thread per (padded) point computes the point's
// fixed-point phase constants and checks its data.
//
// The phase of Eq. 5 in turns is c_j r^2 with c_j = p^2 / (2 lambda z_j)
// (Section 2.2 names the same constant P_j = 1/(2 lambda z_j) in metres).
// Because r^2 is an integer, only frac(c_j) matters modulo one turn; it is
// stored as the 64-bit fixed-point C_j = round(frac(c_j) 2^64).  Every phase
// the kernels form is then C_j * (integer) mod 2^64, exact up to C_j's own
// rounding (<= 2^-65 turn per px^2, i.e. < 2^-33 turn for r^2 < 2^32).
// FP64 is used only here, O(N) work.  With the piston of Eq. 2 the point
// carries frac(z_j / lambda) (the phase 2 pi z_j / lambda in turns) in place of
// the second difference, which the kernels then form from C_j itself.
#include "prep_dev.cuh"

namespace cgh {

__global__ void prep_points_kernel(const float *__restrict__ xyz, const float *__restrict__ amp, int n,
                                   int n_pad, double pitch, double lambda, int4 *__restrict__ geo,
                                   uint2 *__restrict__ aux, int *status, float *amp_max, int aux_x,
                                   float4 *__restrict__ ext, int width, int height, int tile_cols, int tile_rows)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pad) return;
    dev::prep_point(j, xyz, amp, n, pitch, lambda, geo, aux, status, amp_max, aux_x, ext, width, height, tile_cols,
                    tile_rows);
}

cudaError_t launch_prep_points(const float *d_xyz, const float *d_amp, int n, int n_pad, double pitch,
                               double lambda, int4 *geo, uint2 *aux, int *status, float *amp_max,
                               cudaStream_t s, int aux_x, float4 *ext, int width, int height, int tile_cols, int tile_rows)
{
    if (n_pad <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (n_pad + threads - 1) / threads;
    prep_points_kernel<<<blocks, threads, 0, s>>>(d_xyz, d_amp, n, n_pad, pitch, lambda, geo, aux, status,
                                                         amp_max, aux_x, ext, width, height, tile_cols, tile_rows);
    return cudaGetLastError();
}

}  // namespace cgh
