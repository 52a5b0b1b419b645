// Host-side launchers of the library's kernels (internal; not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace cgh {

// Points per shared-memory tile of the direct kernel; prepared point arrays
// are padded to a multiple of it.
constexpr int kPointTile = 256;

// a1: per-point constants and validation (prep.cu).  amp_max (optional, zeroed
// by the caller) receives max_j |A_j|.  geo[j] = {x, y, C_hi, C_lo},
// aux[j] = {w, A} with w per aux_x: kAuxSecondDiff: the second difference
// 2 C_j (top 32 bits) of the recurrence; kAuxPiston: the piston
// frac(z_j / lambda) in 2^-32 turn (the phase of Eq. 2 with its first term);
// kAuxZero: 0 (a piston slot for kernels that add one, none wanted).  ext
// (optional, the spherical form) receives {(p / z_j)^2, z_j / (2 lambda)} as
// float pairs {hi, hi, lo, lo}.
enum { kAuxSecondDiff = 0, kAuxPiston = 1, kAuxZero = 2 };
// The spherical kernel's thread tile (pixels: sph_tile_rows(planes) rows of
// sph_tile_cols(planes) columns) and the bounds behind the two
// flags prep writes into ext's signs (both checked at every pixel of the
// width x height hologram): ext.x >= 0 when the distance remainder may be taken
// as a quadratic about each thread tile's centre (truncation error at most
// kSphFitTurns, range within kSphRangeTurns); ext.y >= 0 when u = r^2 / z^2
// stays below kSeriesU.
__host__ __device__ constexpr int sph_tile_rows(int planes) { return planes == 1 ? 8 : 4; }
__host__ __device__ constexpr int sph_tile_cols(int planes) { return planes == 1 ? 8 : 4; }
constexpr double kSphFitTurns = 2.98023223876953125e-8;   // 2^-25 turn
constexpr double kSphRangeTurns = 0.45;
constexpr double kSeriesU = 0.05;
cudaError_t launch_prep_points(const float *d_xyz, const float *d_amp, int n, int n_pad, double pitch,
                               double lambda, int4 *geo, uint2 *aux, int *status, float *amp_max,
                               cudaStream_t s, int aux_x = kAuxSecondDiff, float4 *ext = nullptr, int width = 0,
                               int height = 0, int tile_cols = 4, int tile_rows = 4);

// The plane-wave reference phase of Eq. 5, phi_r(m, n) = kx m + ky n + phi0,
// common to every point of a launch: kx, ky in 2^-64 turn per pixel, phi0 in
// 2^-32 turn; piston: the points were prepared with their piston in aux.x.
// All zero: the restricted phase of Eq. 5.
struct PhaseRef {
    unsigned long long kx = 0, ky = 0;
    uint32_t phi0 = 0;
    uint32_t piston = 0;
    bool reference() const { return kx != 0 || ky != 0 || phi0 != 0; }
    bool any() const { return reference() || piston != 0; }
};

#ifdef __CUDACC__
// phi_r at pixel (m, n) >= 0, top 32 bits of the 64-bit fixed point, plus phi0.
__device__ __forceinline__ uint32_t ref_turn(const PhaseRef &r, int m, int n)
{
    return (uint32_t)((r.kx * (unsigned long long)m + r.ky * (unsigned long long)n) >> 32) + r.phi0;
}
// Its change per column (per row): kx (ky) rounded to 2^-32 turn.
__device__ __forceinline__ uint32_t ref_step(unsigned long long k)
{
    return (uint32_t)((k >> 32) + ((k >> 31) & 1ull));
}
#endif

// a2: direct kernel (direct.cu).
struct DirectShape {
    int tile_w, tile_h;   // pixels covered by one CTA
    int threads;          // threads per CTA
    int bx;               // threads per CTA row: 32 (the wide shape) or 16 (the tall and short shapes)
    int per_sm = 2;       // CTAs resident per SM
    int tables = 0;       // 1: the balanced layout's kernel with per-CTA tables of the column and row sines
};
// The CTA shapes of the direct kernels (256 threads, 8 columns of pixels per
// thread): wide = 32 x 8 threads, tall = 16 x 16 threads.
DirectShape direct_shape(bool tall = false);
// drop_tile >= 0 is a test hook: the first point chunk never loads that tile,
// so its bounded wait runs out and the launch ends with kStatusTimeout.
cudaError_t launch_direct(bool sfu, const DirectShape &sh, const int4 *geo, const uint2 *aux, int n_pad, int width,
                          int height, int split, float *out, int64_t slice_stride, int *status, uint64_t timeout_ns,
                          cudaStream_t s, int drop_tile = -1, const PhaseRef &ref = PhaseRef());

// The direct form over a flat (pixel tile, point) work space split evenly over ctas CTAs, with the partial
// tiles at range boundaries summed in CTA order by the last CTA to finish each tile (direct.cu): out receives
// the hologram, no padded point is evaluated.  slots: 2 ctas x tile_w x tile_h floats (16-byte aligned);
// counters: one int per pixel tile (zeroed by the launch).  drop_tile >= 0: CTA 0 never loads that point tile
// of its range (test hook).
// variant 0: 32 x 8 threads of 8 x 4 pixels (256 x 32 tiles); 1: 16 x 16 threads of 8 x 4 (128 x 64).
DirectShape direct_stream_shape(int variant);
int direct_stream_per_sm(bool sfu, const DirectShape &sh);
cudaError_t launch_direct_stream(bool sfu, const DirectShape &sh, int ctas, const int4 *geo, const uint2 *aux,
                                 int n_points, int width, int height, float *out, float *slots, int *counters,
                                 int *status, uint64_t timeout_ns, cudaStream_t s, int drop_tile = -1,
                                 const PhaseRef &ref = PhaseRef());

// Complex object wave (Eq. 2, restricted form), SFU form: real part at out,
// imaginary part at out + im_offset; point chunk s at out + s * slice_stride.
DirectShape direct_wave_shape(bool tall = false);
cudaError_t launch_direct_wave(const DirectShape &sh, const int4 *geo, const uint2 *aux, int n_pad, int width,
                               int height, int split, float *out, int64_t slice_stride, int64_t im_offset,
                               int *status, uint64_t timeout_ns, cudaStream_t s, const PhaseRef &ref = PhaseRef());

// f2: the exact spherical wave of Eq. 1 (spherical.cu), direct SFU form.
// Points prepared with the piston and ext.  planes = 1: the amplitude
// hologram (Eq. 5, middle line) at out; planes = 2: the complex wave, real part
// at out and imaginary part at out + im_offset.  Point chunk s at out + s * slice_stride.
// variant 0: 32 x 8 threads (wide), 1: 16 x 16 (tall), 2: 16 x 8 (short, four CTAs per SM).
DirectShape spherical_shape(int planes, int variant = 0);
cudaError_t launch_spherical(const DirectShape &sh, const int4 *geo, const uint2 *aux, const float4 *ext, int n_pad,
                             int width, int height, int split, int planes, float *out, int64_t slice_stride,
                             int64_t im_offset, const PhaseRef &ref, cudaStream_t s);

// a7: one job (hologram) of a batched direct launch; units are {job, pixel tile}.
struct DirectJob {
    const int4 *geo;
    const uint2 *aux;
    float *out;
    int n_ptiles, width, height, tiles_x, vec, pad;
};
// tall: the 16 x 16-thread CTA shape (tiles of direct_shape(true)), else the wide one.
cudaError_t launch_direct_batch(bool sfu, bool tall, const DirectJob *d_jobs, const int *d_cta_off,
                                const int2 *d_units, int ctas, int *status, uint64_t timeout_ns, cudaStream_t s);
// CTAs of the batched direct kernel resident per SM (occupancy calculator).
int direct_ctas_per_sm(bool sfu, bool tall);

// a3: separable factors P [height][ld], Q [width][ld] (factors.cu).  For
// kFactorSplit16 the lo planes follow the hi planes (offset rows * ld).
// amp_max (optional) scales Q by 1 / max|A|.
enum { kFactorF16 = 0, kFactorBF16 = 1, kFactorSplit16 = 2 };
// imag_q_only: write only Q' (the factor of the imaginary part) into Q.
// The reference phase goes to both factors (ky n into P, kx m + phi0 into Q),
// the piston (aux.x) into Q.
cudaError_t launch_factors(int mode, const int4 *geo, const uint2 *aux, int n_points, int height, int width,
                           void *P, void *Q, int64_t ld, const float *amp_max, cudaStream_t s,
                           bool imag_q_only = false, const PhaseRef &ref = PhaseRef());

// Grouped GEMM form (groups.cu, factors.cu).  Groups: points with the same
// plane constant C and the same column x.  meta (device, 4 ints): [0] planes
// (-1 beyond kMaxPlanes), [1] points, [2] groups, [3] largest group.  groups[g]
// = {first, count, plane, x} into members[] = {y, -A} (sized n, group order);
// the plane ids index the sorted table of plane constants in the scratch.
constexpr int kMaxPlanes = 64;
constexpr int kXSpan = 2 * 16384 + 1;
constexpr int kMaxGroupPoints = 1024;   // larger groups: the ungrouped form
size_t group_workspace_bytes(int n, int n_planes);
const unsigned long long *group_plane_table(const void *scratch);
cudaError_t launch_planes(const int4 *geo, int n, void *scratch, int *meta, cudaStream_t s);
cudaError_t launch_group_count(const int4 *geo, int n, int n_planes, void *scratch, int *meta, int4 *groups,
                               cudaStream_t s);
cudaError_t launch_group_build(const int4 *geo, const uint2 *aux, int n, int n_planes, int n_groups, void *scratch,
                               const int *meta, const int4 *groups, const float *amp_max, float *wscale,
                               int2 *members, cudaStream_t s);
cudaError_t launch_group_factors(int mode, const int4 *groups, int g_begin, int n_groups,
                                 const unsigned long long *planes, const int2 *members, int height, int width,
                                 void *P, void *Q, int64_t ld, const float *wscale, cudaStream_t s,
                                 const PhaseRef &ref = PhaseRef());

// f3: Fresnel diffraction (fresnel.cu) and the wavefront-recording method (wrp.cu).
// Padded planes are [2H][2W] interleaved complex; input/output planes [2][H][W].
bool fft_plan_2d(int rows, int cols, void **plan, cudaStream_t s);
void fft_plan_destroy(void *plan);
bool fft_exec(void *plan, float2 *data, bool inverse, cudaStream_t s);
// h = pre * exp(i 2 pi C (k^2 + l^2) / 2^64) at the signed offsets of the 2H x 2W grid
cudaError_t launch_chirp(float2 *h, int H, int W, unsigned long long C, double pre_re, double pre_im, cudaStream_t s);
cudaError_t launch_expand(const float *in, int H, int W, float2 *pad, cudaStream_t s);
cudaError_t launch_cmul(float2 *a, const float2 *b, int64_t n, cudaStream_t s);
cudaError_t launch_crop(const float2 *pad, int H, int W, float *out, cudaStream_t s);
// The library's own FFT path (fft.cu): padded grid Ly x Lx (powers of two >= 2H - 1, 2W - 1, at most
// kFftMaxLen), Ly = L1 L2 for the column four-step; pad and spec are [Ly][Lx] complex, twx / twy the
// tables e^{-2 pi i k / Lx}, e^{-2 pi i k / Ly}.  Larger grids use cuFFT.
constexpr int kFftMaxLen = 16384;
struct FftGrid {
    int Ly = 0, Lx = 0, L1 = 0, L2 = 0;
    bool ok = false;
};
FftGrid fft_grid(int H, int W);
// The chirp pre * exp(i 2 pi C (k^2 + l^2) / 2^64) on the grid, transformed: its spectrum in the
// scrambled column order the convolution uses.
cudaError_t launch_fft_chirp_spectrum(const FftGrid &g, float2 *spec, unsigned long long C, double pre_re,
                                      double pre_im, const float2 *twx, const float2 *twy, cudaStream_t s);
// out ([2][H][W]) = crop(IFFT(FFT(input) * spec)); input = the planes in, or (in == nullptr) the rows
// y < H, columns x < W of pad.
cudaError_t launch_fft_convolve(const FftGrid &g, const float *in, int H, int W, float2 *pad, const float2 *spec,
                                const float2 *twx, const float2 *twy, float *out, cudaStream_t s);

// win[j] = {piston (or 0), A, floor(w_j^2), floor(w_j)}; geo as in the point preparation, at d_j = z_j - z_wrp
cudaError_t launch_wrp_prep(const float *d_xyz, const float *d_amp, int n, int n_pad, double pitch, double lambda,
                            double z_wrp, bool piston, int4 *geo, uint4 *win, int *status, cudaStream_t s);
// Band lists (32 rows each, built per segment of 4096 points): count[cells], offset[cells + 1],
// list[sum of counts] (at most n_pad * bands), cells = bands x segments.
int wrp_band_cells(int H, int n_pad);
cudaError_t launch_wrp_bands(const int4 *geo, const uint4 *win, int n_pad, int H, int *count, int *offset, int *list,
                             cudaStream_t s);
// into pad (row stride pad_ld) when pad is not null, else into planes [2][H][W]; list == nullptr: every tile
// walks all points (the same sums)
cudaError_t launch_wrp_record(const int4 *geo, const uint4 *win, int n_pad, int H, int W, const int *offset,
                              const int *list, float2 *pad, int64_t pad_ld, float *planes, cudaStream_t s);

// Hardware-sine throughput (results per second) of the whole GPU, measured; -1 on failure (probe.cu).
double measure_mufu_rate(int num_sms, cudaStream_t s);

// a4: tcgen05 GEMM, out[n][m] (+)= sum_k P[n][k] Q[m][k] over K splits (gemm.cu).
struct GemmPlan {
    int mode;          // kFactorF16 / kFactorBF16 / kFactorSplit16
    int bn;            // tile width in columns of the hologram (Q rows)
    int splits;        // K splits; > 1 writes partial planes
    int ctas;          // persistent CTAs
    int chunk_kb;      // k-blocks (of 64) per TMEM accumulation chain; 0 = whole split
    bool accumulate;   // add to the output (or partial planes) instead of overwriting
    bool trans;        // A = Q (128-row tiles of hologram columns), B = P; writes out transposed back
    bool pair = false; // the two-SM form (clusters of two CTAs, 256-row tiles, half of B in each CTA); bn != 240
};
int gemm_max_ctas(int num_sms);
bool gemm_bn_supported(int bn);
cudaError_t launch_gemm(const GemmPlan &plan, const void *P, const void *Q, int height, int width, int64_t ld,
                        float *out, int64_t slice_stride, const float *amp_max, int *status, uint64_t timeout_ns,
                        cudaStream_t s);

// a7: one job (hologram) of a batched GEMM launch; lives in global memory,
// written once per plan.  Units are {job, tile} pairs in per-CTA lists.
struct alignas(64) GemmJob {
    CUtensorMap p, q, pl, ql;
    float *out;
    const float *amp_max;
    int height, width, nkb, tiles_m, tiles_n, kc, passes, bn;
    uint32_t idesc;
    int vec;
    int trans;
};
// trans: A = Q (128-row tiles of hologram columns), B = P; the epilogue writes the tile back transposed.
bool fill_gemm_job(GemmJob *job, int mode, int bn, const void *P, const void *Q, int height, int width, int64_t ld,
                   int chunk_kb, float *out, const float *amp_max, bool trans = false);
// bn_max: the widest tile of the jobs; at most 224 selects the kernel whose
// shared-memory ring has room for 5 stages of 224-wide tiles (4 at 256).
cudaError_t launch_gemm_batch(const GemmJob *d_jobs, const int *d_cta_off, const int2 *d_units, int ctas,
                              int bn_max, int *status, uint64_t timeout_ns, cudaStream_t s);

// a7: the persistent batch kernel (persist.cu).  One job per hologram; the SIMT queue holds units
// {kind, job, a, b}: kPersistPrep (a = block of kPointTile points), kPersistFactor (a = band of
// persist_factor_rows() stacked rows, b = group of persist_factor_points() point slots), kPersistDirect
// (a = pixel tile of persist_direct_tile_w() x persist_direct_tile_h(), b = point chunk); the GEMM queue holds
// {job, tile, K chunk} (the chunks of a tile add to the output in K order; before it loads a k-block the producer
// waits for the factor units of that k-block).  heads[3], prep_done[jobs], fact_done[jobs], every job's
// amax, tile_count, tile_seq and group_done are zero at launch.
enum { kPersistPrep = 0, kPersistFactor = 1, kPersistDirect = 2 };
struct alignas(64) PersistJob {
    GemmJob g;                  // GEMM forms: tensor maps, shape, output
    const float *xyz, *amp;     // the caller's points
    int4 *geo;                  // prepared points (padded to kPointTile)
    uint2 *aux;
    float *amax;                // max |A| (GEMM forms)
    uint16_t *P, *Q;            // factors, [planes][rows][ld]
    float *out;                 // [height][width]
    float4 *parts;              // direct units with chunks > 1: [tiles][chunks][totals of a tile]
    int *tile_count;            // direct units with chunks > 1: one counter per pixel tile
    double pitch, lambda;
    long long ld, plane_p, plane_q;
    int n, n_pad, point_slots, width, height, form;
    int prep_units, fact_units; // what a factor (direct) unit and a GEMM unit wait for
    int tiles_x, chunks, vec;
    int kchunk_kb, kchunks;     // GEMM: k-blocks of one K chunk of a unit (a multiple of the factor units'
                                // 32), and chunks per tile
    int *tile_seq;              // GEMM with kchunks > 1: [tiles][4], the next K chunk each epilogue quarter takes
    int *group_done;            // GEMM: [fact_groups], factor units (bands) done of each group of point slots
    int fact_bands, fact_groups;// GEMM: factor units = bands (of stacked rows) x groups (of point slots)
    int chunk_extra;            // test hook: every factor group waits for this many bands more than exist
    int premade;                // GEMM: points and factors written by launches before the persistent one
};
struct PersistParams {
    const PersistJob *jobs;
    const int4 *simt_units;
    int simt_total;
    const int4 *gemm_units;     // {job, tile, K chunk, 0}
    int gemm_total;
    int n_jobs;
    int *heads;                 // [0]: next SIMT unit, [1]: next GEMM unit, [2]: factor units done (all jobs)
    int *prep_done, *fact_done; // per job
    int fact_all;               // > 0: every GEMM unit waits for heads[2] >= fact_all (all jobs' factors first)
};
int persist_factor_rows();
int persist_factor_points();
int persist_direct_tile_w();
int persist_direct_tile_h();
// ctas persistent CTAs (one per SM); bn_max: the widest GEMM tile of the jobs (224: five ring stages of
// 224-wide tiles; up to 256: four).
cudaError_t launch_persist(const PersistParams &p, int ctas, int bn_max, int *status, uint64_t timeout_ns,
                           cudaStream_t s);

// a5: fixed-order sum of `slices` planes of n floats (reduce.cu).
cudaError_t launch_reduce_slices(const float *parts, int slices, int64_t n, int64_t slice_stride, float *out,
                                 cudaStream_t s);

// a6: 8-bit min/max quantiser (quantize.cu). scratch holds 2 uint32.
cudaError_t launch_quantize8(const float *field, int64_t n, uint8_t *out, uint32_t *scratch, cudaStream_t s);
// Kinoform (phase-only hologram, Eq. 3) quantiser: 255/(2 pi) per radian of
// atan2(im, re) taken in [0, 2 pi).
cudaError_t launch_kinoform8(const float *re, const float *im, int64_t n, uint8_t *out, cudaStream_t s);

}  // namespace cgh
