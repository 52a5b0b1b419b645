/*
 * cgh.h - C ABI of the GB300 point-cloud Fresnel hologram library (libcgh.so).
 *
 * The library computes, on one NVIDIA GB300 (sm_103a), the amplitude
 * computer-generated hologram of a point cloud
 *
 *     I(m, n) = sum_j A_j cos( pi p^2 / (lambda z_j) * ((m - x_j)^2 + (n - y_j)^2) )
 *
 * which is Eq. 5 of the paper (Section 2.1: the interference term of Eq. 4
 * with the Fresnel approximation of Eq. 2), without the per-point piston
 * 2 pi z_j / lambda, the reference phase phi_r and the constant 2 A_r.
 * m is the hologram column, n the row (both in [0, width) x [0, height));
 * x_j, y_j are the point's position in pixel units (integers, origin at pixel
 * (0, 0)); z_j is its distance in metres; p is the pixel pitch and lambda the
 * wavelength, in metres.  Holograms are row-major float32, out[n * width + m]
 * (Section 4.1: adr = j + WIDTH * i).
 *
 * Two forms compute the same sum:
 *   - direct: per pixel and per point, the phase is built incrementally in
 *     exact 32/64-bit fixed-point turns (the recurrence of Eqs. 6-8,
 *     Section 2.2) and fed to a single-precision cosine;
 *   - separable GEMM: exp(i phi) factors exactly into a column term and a row
 *     term, so I = P Q^T with P [height][2N] and Q [width][2N]; the product
 *     runs on the tcgen05 tensor cores in FP16, BF16 or split hi+lo FP16 with
 *     FP32 accumulation.
 *
 * Conventions for every entry point:
 *   - Return value: CGH_OK (0) or a cgh_status code; no exception or signal
 *     ever leaves the library.  Arguments that the host can check (null
 *     pointers, sizes, non-finite scalars) are rejected at once and nothing is
 *     launched.  Errors found by the GPU in the data (z <= 0, NaN, non-integer
 *     or out-of-range coordinates) are latched in the context's status word
 *     and returned by cgh_sync(); the output is then unspecified.
 *   - Pointers named d_* are device pointers (cudaMalloc / torch CUDA
 *     tensors) on the context's device; h_* are host pointers.  The caller
 *     owns every buffer it passes; the library never frees them.  The
 *     context owns its own workspace and frees it in cgh_destroy().
 *   - Work is enqueued on the context's stream (cgh_set_stream) and is
 *     asynchronous unless stated otherwise; cgh_sync() waits for it.
 *   - A context is not thread safe: use one per host thread.
 *   - There is no CPU fallback: a build without a usable CUDA device returns
 *     CGH_ECUDA from cgh_create().
 */
#ifndef CGH_H
#define CGH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CGH_ABI_VERSION 1

/* Status codes. */
enum {
    CGH_OK = 0,
    CGH_EINVAL = 1,    /* bad argument, checked on the host */
    CGH_ENOMEM = 2,    /* device allocation failed */
    CGH_ECUDA = 3,     /* CUDA runtime/driver error, or no usable device */
    CGH_ETIMEOUT = 4,  /* a bounded wait (device or host) ran out */
    CGH_EINPUT = 5,    /* bad point data, found on the device */
    CGH_ENOTSUP = 6,   /* form or option not available for this problem */
    CGH_EBOUNDS = 7    /* debug build (CGH_DEBUG) only: a device-side bounds check failed, the access was
                          skipped; the release build never returns it */
};

/* How the hologram is computed. */
enum {
    CGH_FORM_AUTO = 0,          /* autotuner's choice for the accuracy class */
    CGH_DIRECT_SFU = 1,         /* direct sum, hardware (MUFU) cosine */
    CGH_DIRECT_ACCURATE = 2,    /* direct sum, polynomial cosine on the FMA pipe */
    CGH_GEMM_F16 = 3,           /* I = P Q^T, FP16 factors, FP32 accumulate */
    CGH_GEMM_BF16 = 4,          /* I = P Q^T, BF16 factors, FP32 accumulate */
    CGH_GEMM_SPLIT16 = 5        /* I = Ph Qh^T + Ph Ql^T + Pl Qh^T, hi+lo FP16 */
};

/* 8-bit quantisation rules (cgh_quantize8). */
enum {
    CGH_Q_AMPLITUDE_MINMAX = 0, /* floor((v - min) * s), s = 255 / (max - min) rounded up */
    CGH_Q_PHASE = 1             /* kinoform: floor(255/(2 pi) * arg), arg of (re, im) in [0, 2 pi) */
};

/* Phase models (CGH_OPT_PHASE_MODEL), Section 2.1; r^2 = p^2 ((m - x_j)^2 + (n - y_j)^2). */
enum {
    CGH_PHASE_FRESNEL = 0,         /* Eq. 5 without the piston: pi r^2 / (lambda z_j) (the default) */
    CGH_PHASE_FRESNEL_PISTON = 1,  /* Eq. 2 / Eq. 5 (third line): 2 pi / lambda (z_j + r^2 / (2 z_j)) */
    CGH_PHASE_SPHERICAL = 2        /* Eq. 1 / Eq. 5 (second line): 2 pi / lambda sqrt(r^2 + z_j^2); CGH_DIRECT_SFU
                                      (or CGH_FORM_AUTO) only, the exact distance is not separable */
};

/* Options (cgh_set_option). */
enum {
    CGH_OPT_TIMEOUT_MS = 1,     /* bound on every device-side wait; host-side waits allow 2x + 1 s; default 5000 */
    CGH_OPT_POINT_SPLIT = 2,    /* direct forms: 0 = automatic (the amplitude hologram: every CTA takes an
                                   equal share of the (pixel tile, point) pairs and the last CTA to finish a tile
                                   sums its parts; the complex wave: point chunks as the critical-path model
                                   picks them); s > 0: s point chunks, each a plane of partial sums, reduced
                                   after */
    CGH_OPT_GEMM_SPLITK = 3,    /* GEMM forms: K splits reduced afterwards; 0 = automatic */
    CGH_OPT_GEMM_BN = 4,        /* GEMM forms: tile width, one of 128, 192, 224, 240, 256; 0 = automatic */
    CGH_OPT_TOLERANCE_E9 = 5,   /* CGH_FORM_AUTO: largest admissible NRMS, in units of 1e-9 */
    CGH_OPT_PROFILE = 6,        /* 1: bracket every kernel launch with CUDA events (cgh_profile_read) */
    CGH_OPT_GEMM_CHUNK = 7,     /* GEMM forms: k-blocks of 64 per tensor-memory accumulation chain; 0 = default */
    CGH_OPT_TEST_DROP_TILE = 8, /* test hook, direct forms: never load point tile k (>= 0) of the first chunk, so the
                                   kernel's bounded wait runs out and cgh_sync returns CGH_ETIMEOUT; -1 = off */
    CGH_OPT_FACTOR_BUDGET_MB = 9, /* GEMM forms: device memory for the factors of the points in flight; default 2048 */
    CGH_OPT_GEMM_PIPELINE = 10, /* GEMM forms: point chunks (>= 8192 points each) whose factor generation overlaps
                                   the previous chunk's GEMM on a second stream; default 1 = no overlap (on GB300
                                   the overlap measured no faster at 1920x1080 with 5x10^4 points) */
    CGH_OPT_GEMM_TRANSPOSE = 11, /* GEMM forms: 0 = automatic, 1 = 128-row tiles of P (hologram rows), 2 = 128-row
                                   tiles of Q (hologram columns; the result is written back transposed) */
    CGH_OPT_GEMM_GROUP = 12,    /* GEMM forms, cgh_point_cloud: points on one depth plane (equal z, so equal
                                   constant of Eq. 5) and one column x share the column factor of the separable
                                   form, so their row factors are summed first and the GEMM runs over K = 2 x the
                                   number of such groups.  0 = automatic: tried from 65536 points, used when it at
                                   least halves K; 1 = never; 2 = whenever it applies.  It applies with at most 64
                                   distinct depths and at most 1024 points per group, and never while the stream is
                                   being captured into a graph (it reads two counts back to the host, which waits for
                                   the stream).  Results agree with the ungrouped form to rounding.  Not with the
                                   piston (CGH_PHASE_FRESNEL_PISTON): points of equal C may differ in depth. */
    CGH_OPT_PHASE_MODEL = 13,   /* CGH_PHASE_* above; default CGH_PHASE_FRESNEL.  cgh_batch supports the default
                                   only (CGH_ENOTSUP otherwise). */
    CGH_OPT_DIRECT_CTAS = 14,   /* direct SFU amplitude form with CGH_OPT_POINT_SPLIT = 0: the CTAs that share
                                   the (pixel tile, point) pairs; 0 = automatic (up to three per resident CTA slot,
                                   each with at least 1024 points; the hardware schedules those beyond the resident
                                   ones as others finish) */
    CGH_OPT_BATCH_MODE = 15,    /* cgh_batch: 0 = one persistent launch for the whole batch (default; GEMM units on
                                   the tensor cores beside point preparation, factor generation and direct units
                                   on the same SMs); 1 = per-kind launches (preparation and factors per instance,
                                   then one GEMM launch and one direct launch per direct form) */
    CGH_OPT_BATCH_OVERLAP = 16, /* cgh_batch, persistent launch: 1 = a GEMM unit starts as soon as its own
                                   hologram's factors are written (default); 0 = once every hologram's factors
                                   are written */
    CGH_OPT_TEST_ALLOC_FAIL = 17, /* test hook: the next n growths of the context's workspace fail as a failed
                                   cudaMalloc would (the call returns CGH_ENOMEM, nothing is launched, and the
                                   context stays usable); 0 = off */
    CGH_OPT_DIRECT_SHAPE = 18,  /* direct SFU amplitude form with CGH_OPT_POINT_SPLIT = 0: the thread block;
                                   0 = automatic (5 or 6 by the padded pixels), 1 = 32 x 8 threads of 8 x 4
                                   pixels, 2 = 16 x 16 threads of 8 x 4, 3 = 16 x 8 threads of 8 x 8, 4 = 32 x 4
                                   threads of 8 x 8 (each thread its own sines and cosines); 5 = 16 x 16 threads of
                                   8 x 4, 6 = 32 x 8 threads of 8 x 4, with the sines and cosines of a point's
                                   columns and rows taken once per CTA into shared-memory tables */
    CGH_OPT_GEMM_PERSISTENT = 19, /* GEMM forms, cgh_point_cloud: 1 = the hologram as a one-instance batch in the
                                   persistent kernel (its factors generated K chunk by K chunk while the tensor
                                   cores run the GEMM of the chunks already there; a CUDA graph replayed while the
                                   buffers stay the same), when all its factors fit CGH_OPT_FACTOR_BUDGET_MB, it is
                                   not grouped, has no piston or reference and the stream is not being captured;
                                   0 = the separate factor and GEMM launches */
    CGH_OPT_GEMM_PAIR = 20,     /* GEMM forms, cgh_point_cloud: the two-SM tcgen05 form (clusters of two CTAs,
                                   256-row tiles, each CTA holding half of the B tile, so more operand stages fit)
                                   or one CTA per 128-row tile.  0 = chosen with the tile width and K splits by the
                                   measured time model (default), 1 = always the two-SM form (not at width 240),
                                   2 = never */
    CGH_OPT_BATCH_CHUNK_MB = 21, /* cgh_batch persistent launch (and CGH_OPT_GEMM_PERSISTENT): a GEMM unit covers
                                   one K chunk of its tile whose operands (both factors, all planes) take about
                                   this many MiB, the chunks of a tile added to the output in K order; 0 = 128 MiB
                                   where the batch has two tiles or more per SM, else chunks that balance the
                                   tiles over the SMs (default) */
    CGH_OPT_BATCH_PREMADE_PCT = 22 /* cgh_batch persistent launch: the first GEMM holograms in queue order, up to
                                   this percentage of the batch's factor bytes, get their points and factors
                                   from the plain kernels launched before the persistent one (in the same
                                   graph); the SIMT groups make the rest */
};

typedef struct cgh_ctx cgh_ctx;

/*
 * Creates a context for width x height holograms of pixel pitch pitch_m and
 * wavelength lambda_m (Section 4.1 fixes the CGH size, pitch P and wavelength
 * WL of each run).  1 <= width, height <= 16384; pitch_m and lambda_m finite
 * and > 0.  Binds the current CUDA device and the legacy default stream.
 * *out receives the context; on failure *out is NULL.
 */
int cgh_create(int width, int height, double pitch_m, double lambda_m, cgh_ctx **out);

/* Waits for the context's work (bounded), frees its workspace and the context. NULL is allowed. */
int cgh_destroy(cgh_ctx *ctx);

/* Binds a CUDA stream (a cudaStream_t passed as void*; NULL = legacy default stream). */
int cgh_set_stream(cgh_ctx *ctx, void *cuda_stream);

/*
 * Sets the reference wave R = A_r exp(i phi_r) of Eq. 4 to a plane wave,
 *   phi_r(x_h, y_h) = 2 pi / lambda (x_h sin_x + y_h sin_y) + phase0_rad,
 * x_h = m p, y_h = n p.  Eq. 5 adds phi_r to the phase of every term, so the
 * amplitude hologram becomes sum_j A_j cos(theta_j + phi_r) and the complex
 * wave (cgh_wave) sum_j A_j exp(i (theta_j + phi_r)).  (Eq. 4 written out
 * would give theta_j - phi_r; Eq. 5's sign is the one implemented: negate all
 * three arguments for the other.)  |sin_x|, |sin_y| <= 1, |phase0_rad| <= 1e6,
 * all finite; (0, 0, 0), the default, is no reference phase.  All forms except
 * cgh_batch (CGH_ENOTSUP with a reference set).
 */
int cgh_set_reference(cgh_ctx *ctx, double sin_x, double sin_y, double phase0_rad);

/*
 * Fresnel diffraction, Eq. 10 (Section 2.3): propagates the complex plane d_in
 * by z_m (metres, nonzero, either sign) onto d_out, both [2][H][W] float32
 * (real plane, then imaginary plane; the context's width W x height H, pitch
 * p), device memory; d_out may equal d_in.  The integral is the sum over cells
 * of area p^2 with the prefactor exp(i 2 pi z / lambda) / (i lambda z):
 *   O(m, n) = exp(i 2 pi z/lambda)/(i lambda z) p^2 sum u(m', n') exp(i pi p^2 ((m-m')^2 + (n-n')^2)/(lambda z)),
 * evaluated as the paper does by zero-padding (to the powers of two >= 2H - 1,
 * 2W - 1), FFT, product with the chirp's spectrum (cached per z), inverse FFT
 * and crop, in single precision, with the library's own FFT (cuFFT for grids
 * beyond 16384 a side).  Allocates two padded complex planes and the twiddle
 * tables on first use.
 */
int cgh_fresnel(cgh_ctx *ctx, const float *d_in, double z_m, float *d_out);

/*
 * The wavefront-recording method (Section 2.3), step 1: records the point
 * cloud's complex amplitude on a virtual plane at distance z_wrp_m (> 0) from
 * the hologram, on the hologram's grid, into d_plane ([2][H][W], device).
 * Each point (z_j > z_wrp_m, else CGH_EINPUT) contributes only inside its
 * window, the pixels within d tan(asin(lambda/2p)) / p of (x_j, y_j) with
 * d = z_j - z_wrp_m (the squared radius floored to an integer), with the
 * phase of Eq. 2 at distance d: without the piston (CGH_PHASE_FRESNEL) or with
 * it (CGH_PHASE_FRESNEL_PISTON).  CGH_ENOTSUP for CGH_PHASE_SPHERICAL or with
 * a reference wave set.
 */
int cgh_wrp_record(cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n_points, double z_wrp_m,
                   float *d_plane);

/*
 * The wavefront-recording method, both steps: cgh_wrp_record, then Fresnel
 * diffraction (cgh_fresnel) by z_wrp_m onto the hologram: the complex object
 * wave at d_out ([2][H][W], device); cgh_quantize8 with CGH_Q_PHASE turns it
 * into the kinoform of Eq. 3.
 */
int cgh_wrp(cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n_points, double z_wrp_m, float *d_out);

/*
 * Measures the throughput of the hardware sine (one MUFU operation per
 * result; eight independent chains per thread, every SM busy), the pipe that
 * bounds CGH_DIRECT_SFU, and stores it in *results_per_s.  For stating the
 * direct kernel's roofline against a measured peak; the paper has no
 * counterpart.  Synchronises the context's stream.  CGH_ECUDA on failure.
 */
int cgh_measure_mufu(cgh_ctx *ctx, double *results_per_s);

/* Selects the form (CGH_FORM_* above). */
int cgh_set_form(cgh_ctx *ctx, int form);

/* Sets an option (CGH_OPT_* above). */
int cgh_set_option(cgh_ctx *ctx, int key, int64_t value);

/*
 * The hologram of one point cloud (Eq. 5, restricted form; Section 2.1).
 *   d_xyz : float32 [n_points][3], x and y in pixel units, z in metres.
 *           x and y must be integers with |x|, |y| <= 16384; z finite and > 0.
 *   d_amp : float32 [n_points], amplitudes A_j (finite).
 *   d_out : float32 [height][width], row-major; fully overwritten.
 * n_points == 0 writes zeros.  n_points <= 2^31 - 1.
 */
int cgh_point_cloud(cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n_points,
                    float *d_out);

/*
 * Same as cgh_point_cloud, with host buffers: copies h_xyz and h_amp to the
 * device, computes, copies the hologram back to h_out and waits (bounded).
 * Page-locked host memory makes the copies faster but is not required.
 */
int cgh_point_cloud_host(cgh_ctx *ctx, const float *h_xyz, const float *h_amp, int64_t n_points,
                         float *h_out);

/*
 * The separable factors of one point cloud (the GEMM form's operands).
 * With alpha = 2 pi c_j (m - x_j)^2, beta = 2 pi c_j (n - y_j)^2,
 * c_j = p^2 / (2 lambda z_j), so that the phase of Eq. 5 is alpha + beta:
 *   P[n][2j] = cos beta,        P[n][2j+1] = sin beta          (d_p: [height][ld])
 *   Q[m][2j] = A_j cos alpha,   Q[m][2j+1] = -A_j sin alpha    (d_q: [width][ld])
 * dtype_form is CGH_GEMM_F16 or CGH_GEMM_BF16 (16-bit elements), or
 * CGH_GEMM_SPLIT16, for which d_p and d_q each hold two planes, hi then lo,
 * of [rows][ld] FP16 elements (lo = fp16(v - hi)).  ld >= 2 n_points counts
 * elements and must be a multiple of 64; columns [2 n_points, ld) are zeroed.
 */
int cgh_factors(cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n_points,
                int dtype_form, void *d_p, void *d_q, int64_t ld);

/*
 * The complex object wave of one point cloud (Eq. 2 with the same restriction
 * as above), O(m, n) = sum_j A_j exp(i 2 pi c_j r^2): its real part is the
 * amplitude hologram of cgh_point_cloud and its argument gives the phase-only
 * hologram (kinoform) of Eq. 3, the workload the paper times (Section 5).
 *   d_out : float32 [2][height][width]: the real plane, then the imaginary plane.
 * Forms: CGH_DIRECT_SFU (both parts in one direct pass: hardware sine pairs at
 * the first column of each thread's row and for its first column step, the
 * other terms by complex rotation along the row, since the phase is quadratic
 * in the column, Eqs. 6-8; NRMS about 1.3e-6) and the GEMM forms (Re O = P Q^T and Im O = P Q'^T, with
 * Q'[m][2j] = A_j sin alpha, Q'[m][2j+1] = A_j cos alpha).  CGH_FORM_AUTO
 * picks among those; CGH_DIRECT_ACCURATE returns CGH_ENOTSUP.
 */
int cgh_wave(cgh_ctx *ctx, const float *d_xyz, const float *d_amp, int64_t n_points, float *d_out);

/* One instance of a batch: a whole hologram problem. */
typedef struct {
    int width, height;
    double pitch_m, lambda_m;
    const float *d_xyz;     /* float32 [n_points][3] */
    const float *d_amp;     /* float32 [n_points] */
    int64_t n_points;
    float *d_out;           /* float32 [height][width] */
} cgh_instance;

/*
 * Many holograms (for example the frames of a holographic video) in one
 * persistent launch.  inst is a host array of n_inst instances (the context's
 * own width/height/pitch/lambda are not used).  The form of each instance is
 * the autotuner's choice under the context's tolerance (CGH_FORM_AUTO) or the
 * context's form.  The first call with a given set of shapes builds the work
 * list and captures the launch in a CUDA graph; later calls with the same
 * shapes and buffers replay it.
 */
int cgh_batch(cgh_ctx *ctx, const cgh_instance *inst, int n_inst);

/*
 * The forms (CGH_DIRECT_SFU ... CGH_GEMM_SPLIT16) the last plan of cgh_batch
 * chose, one per instance in the order given (instances without points report
 * CGH_DIRECT_SFU and compute nothing).  Writes min(count, max_entries) entries
 * to the host array forms and the count to *n_entries; 0 entries before the
 * first cgh_batch call.  Host only: no device work.  Not part of the paper's
 * method: it reports the autotuner's choices.
 */
int cgh_batch_forms(cgh_ctx *ctx, int *forms, int max_entries, int *n_entries);

/*
 * Calibrates the autotuner on this device: times every form on three small
 * synthetic clouds and fits, per form, t = c0 + c1 W H N + c2 (W + H) N, from
 * which CGH_FORM_AUTO picks the fastest form whose stated NRMS bound meets
 * CGH_OPT_TOLERANCE_E9; GEMM tile widths are timed per hologram shape on first
 * use.  Runs on the context's stream and waits; must not be called during
 * stream capture.  The first CGH_FORM_AUTO call calibrates by itself if this
 * was not called.  force != 0 re-measures even if a calibration exists.  With
 * the environment variable CGH_TUNE_CACHE=<file>, measurements are read from
 * and saved to that JSON file (keyed by device name and ABI version).
 */
int cgh_autotune(cgh_ctx *ctx, int force);

/*
 * 8-bit quantisation.  CGH_Q_PHASE: d_field holds a complex field as two
 * planes of n floats (real, then imaginary; the layout of cgh_wave); each
 * output is floor(fl(psi * fl(255/(2 pi)))) clamped to [0, 255], with
 * psi = atan2f(im, re) plus 2 pi when negative, as the listings of
 * Section 4.1 quantise their kinoforms.
 * CGH_Q_AMPLITUDE_MINMAX, a float32 field of n values:
 *   lo = min, hi = max over the field (NaN ignored); if !(hi > lo) all 0;
 *   s  = the smallest float >= 255 / ((double)hi - (double)lo) (at most FLT_MAX);
 *   q  = floor(fl(fl(v - lo) * s)), each operation rounded to nearest, no FMA;
 *        255 if q >= 255, 0 if q < 0 or NaN.
 * The paper quantises its phase-only CGHs with 255/(2 pi) (Section 4.1); this
 * is the amplitude counterpart.  d_field and d_out may not overlap.
 */
int cgh_quantize8(cgh_ctx *ctx, const float *d_field, int64_t n, int mode, uint8_t *d_out);

/* Device time of one kernel of the library, summed over its launches (CGH_OPT_PROFILE). */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} cgh_kernel_time;

/*
 * Reads the per-kernel device times recorded since the last reset while
 * CGH_OPT_PROFILE was on.  The events are recorded on the context's stream
 * around each launch; this call waits (bounded) for them.  Up to max_entries
 * entries go to out; *n_entries receives the number of distinct kernels.
 * reset != 0 clears the record afterwards.
 */
int cgh_profile_read(cgh_ctx *ctx, cgh_kernel_time *out, int max_entries, int *n_entries, int reset);

/*
 * For callers that cannot allocate device memory (no cudaMalloc allowed, as
 * in a real-time loop, a host that only hands out pre-registered buffers, or
 * a plug-in living inside another program's memory budget): the direct SFU
 * hologram of one point cloud with no context and no allocation.  The paper
 * has no counterpart; it is this library's own entry point.
 *
 * Arguments as cgh_create() and cgh_point_cloud(); cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  The point constants go to a
 * fixed scratch array of CGH_NOALLOC_MAX_POINTS entries (3 MiB) in the
 * library's own device memory, which every GPU that loads libcgh.so holds
 * until the process exits; n_points > CGH_NOALLOC_MAX_POINTS returns
 * CGH_EINVAL before anything is launched (use cgh_point_cloud instead).
 * The call allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.  Every call blocks: it synchronises cuda_stream to read
 * its status word back, and returns CGH_OK, CGH_EINPUT (bad point data) or
 * CGH_ETIMEOUT.  The first call on a device looks up the scratch address for
 * that device (cudaGetSymbolAddress) and keeps it for the life of the
 * process; make that first call before any stream capture, and do not call
 * this entry point again after cudaDeviceReset() in the same process (the
 * kept address would no longer name the scratch).  Every call shares the
 * scratch and it keeps the last call's contents; calls that overlap on the
 * GPU (several host threads or streams at once) race on it and must be
 * serialised by the caller.
 */
#define CGH_NOALLOC_MAX_POINTS 131072
int cgh_point_cloud_noalloc(int width, int height, double pitch_m, double lambda_m, const float *d_xyz,
                            const float *d_amp, int64_t n_points, float *d_out, void *cuda_stream);

/*
 * Checks an autotuner cache file (the JSON that cgh_autotune writes to
 * CGH_TUNE_CACHE) without touching a GPU: *accepted = 1 when the file at path
 * was written for device_name (the cache's "device" string) and this ABI and
 * holds a complete table of finite, non-negative time coefficients, else 0 --
 * such a file (truncated, edited, another device or ABI, unreadable) is
 * ignored by cgh_autotune, which then calibrates and rewrites it.  Not part of
 * the paper's method: a diagnostic of the autotuner's cache.
 */
int cgh_tune_cache_check(const char *path, const char *device_name, int *accepted);

/*
 * The launch shape cgh_point_cloud gives the GEMM of a hologram of
 * width x height pixels and n_points points in form (CGH_GEMM_F16,
 * CGH_GEMM_BF16 or CGH_GEMM_SPLIT16; not grouped) on a device of num_sms SMs
 * with every option at its default, written to layout[0..3]: 1 when the
 * 128-row A tiles are tiles of hologram columns (the product written back
 * transposed), else 0; the tile width (columns of the B tile); the K splits;
 * 1 for the two-SM form (CGH_OPT_GEMM_PAIR), else 0.  Host only: no GPU is
 * touched.  Returns CGH_EINVAL for sides outside [1, 16384], n_points < 1,
 * num_sms < 1, another form or a null layout.  Not part of the paper's
 * method: a diagnostic of the GEMM's launch-shape choice (Section 2.1,
 * Eq. 5, written as the product of the factors).
 */
int cgh_gemm_layout(int width, int height, int64_t n_points, int form, int num_sms, int *layout);

/* Waits for the context's work (bounded by CGH_OPT_TIMEOUT_MS); returns and clears the latched status. */
int cgh_sync(cgh_ctx *ctx);

/* Static text for a status code. */
const char *cgh_status_string(int status);

/* CGH_ABI_VERSION of the loaded library. */
int cgh_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CGH_H */
