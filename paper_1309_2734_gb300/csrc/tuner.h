// Launch-shape selection and the measured autotuner (host side).
#pragma once

#include <cstdint>

#include "kernels.h"

struct cgh_ctx;

namespace cgh {

// Point chunks for the direct kernels: the shortest critical path, rounds of
// (pixel tiles x chunks) over the resident CTAs times the longest chunk.
int choose_point_split(int64_t pixel_tiles, int64_t point_tiles, int num_sms);

// The direct kernels' CTA shape (wide or tall, the one with less padding and the
// better fill) and its point split; force_split > 0 pins the split.
struct DirectLayout {
    DirectShape shape;
    int split;
};
DirectLayout choose_direct_layout(bool wave, int width, int height, int64_t point_tiles, int num_sms,
                                  int force_split);
// The same choice among n_shapes CTA shapes (each with its threads and CTAs per SM); step_cost, if given, scales
// each shape's predicted path by the relative time of one of its point-tile steps.
DirectLayout choose_layout(const DirectShape *shapes, int n_shapes, int width, int height, int64_t point_tiles,
                           int num_sms, int force_split, const double *step_cost = nullptr);

// GEMM orientation, tile width, K splits and form (one CTA per 128-row tile, or the two-SM form: clusters of two
// CTAs on 256-row tiles) with the shortest predicted time: rounds of units over the ctas CTAs (ctas / 2 clusters)
// times a unit's k-blocks times the measured time of one k-block at that width and form, plus the split
// reduction.  force_* > 0 pin a choice (force_trans: 1 = never transposed, 2 = always; force_pair: 1 = always
// the two-SM form, 2 = never).
struct GemmLayout {
    bool trans;
    int bn;
    int splits;
    bool pair;
};
GemmLayout choose_gemm_layout(int width, int height, int64_t k_blocks, int ctas, bool split_form, int force_bn,
                              int force_splits, int force_trans, int force_pair);

// GEMM tile width (columns of the hologram per tile) with the least padding.
int choose_gemm_bn(int width);

// K splits of the GEMM so that (tiles x splits) units balance over ctas
// persistent CTAs; each split keeps at least 4 k-blocks of 64.
int choose_gemm_splits(int64_t tiles, int64_t k_blocks, int ctas);

// Stated NRMS bound of a form against the FP64 oracle.
double form_nrms_bound(int form);

// Form without measurements (static rule).
int choose_form(int width, int height, int64_t n_points, double tol, int num_sms);

// Measured: calibrate the per-form time model on this device (once; cached).
int tune_calibrate(cgh_ctx *ctx, bool force);
// Predicted seconds per hologram of a form.
double tune_predict(cgh_ctx *ctx, int form, int width, int height, int64_t n);
// Fastest admissible form by the calibrated model.
int tune_choose_form(cgh_ctx *ctx, int width, int height, int64_t n, double tol);
// Fastest GEMM tile width for a shape and form, timed on that shape.
int tune_choose_bn(cgh_ctx *ctx, int width, int height, int form);

}  // namespace cgh
