// Launch-shape and form selection (host side).
#include "tuner.h"

#include "../../include/cgh.h"

namespace cgh {

namespace {
constexpr int kDirectCtasPerSm = 2;
}

int choose_point_split(int64_t pixel_tiles, int64_t point_tiles, int num_sms)
{
    if (pixel_tiles <= 0 || point_tiles <= 1) return 1;
    const int64_t slots = (int64_t)num_sms * kDirectCtasPerSm;
    auto efficiency = [&](int64_t s) {
        const int64_t units = pixel_tiles * s;
        const int64_t waves = (units + slots - 1) / slots;
        return (double)units / (double)(waves * slots);
    };
    int best = 1;
    double best_eff = efficiency(1);
    for (int64_t s = 2; s <= 32 && s * 2 <= point_tiles; ++s) {
        const double e = efficiency(s);
        // each extra chunk costs one more plane of partial sums; demand a clear gain
        if (e > best_eff + 0.03) {
            best = (int)s;
            best_eff = e;
        }
        if (best_eff > 0.97) break;
    }
    return best;
}

int choose_gemm_bn(int width)
{
    static const int cands[] = {256, 240, 192, 128};
    int best = 256;
    double best_waste = 1e30;
    for (int bn : cands) {
        const int tiles = (width + bn - 1) / bn;
        const double waste = (double)(tiles * bn - width) / (double)width + 1e-3 * (256 - bn) / 256.0;
        if (waste < best_waste) {
            best_waste = waste;
            best = bn;
        }
    }
    return best;
}

int choose_gemm_splits(int64_t tiles, int64_t k_blocks, int ctas)
{
    if (tiles <= 0 || ctas <= 0) return 1;
    int best = 1;
    double best_time = 1e30;
    for (int64_t s = 1; s <= 32 && s * 4 <= (k_blocks > 4 ? k_blocks : 4); ++s) {
        const int64_t units = tiles * s;
        const int64_t rounds = (units + ctas - 1) / ctas;
        // time in units of one whole-K tile; each extra split costs a partial plane
        const double t = (double)rounds / (double)s + 0.01 * (double)(s - 1);
        if (t < best_time - 1e-9) {
            best_time = t;
            best = (int)s;
        }
    }
    return best;
}

int choose_form(int width, int height, int64_t n_points, double tol, int num_sms)
{
    (void)width;
    (void)height;
    (void)n_points;
    (void)num_sms;
    (void)tol;
    return CGH_DIRECT_SFU;
}

}  // namespace cgh
