// Launch-shape and form selection (host side).
#pragma once

#include <cstdint>

namespace cgh {

// Point chunks for the direct kernel so that (pixel tiles x chunks) fills
// whole waves of resident CTAs; 1 when one wave is already nearly full.
int choose_point_split(int64_t pixel_tiles, int64_t point_tiles, int num_sms);

// GEMM tile width (columns of the hologram per tile) with the least padding.
int choose_gemm_bn(int width);

// K splits of the GEMM so that (tiles x splits) units balance over ctas
// persistent CTAs; each split keeps at least 4 k-blocks of 64.
int choose_gemm_splits(int64_t tiles, int64_t k_blocks, int ctas);

// Form for CGH_FORM_AUTO: the fastest form whose stated NRMS bound is within tol.
int choose_form(int width, int height, int64_t n_points, double tol, int num_sms);

}  // namespace cgh
