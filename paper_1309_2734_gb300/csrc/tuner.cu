// Autotuner and launch-shape selection (host side).
//
// Static rules (no measurement):
//   choose_point_split  point chunks of the direct kernel, to fill whole waves;
//   choose_direct_layout  the direct kernels' CTA shape (less padding) with its split;
//   choose_gemm_bn      GEMM tile width with the least padding of the width;
//   choose_gemm_splits  K splits of the GEMM, to balance tiles over the CTAs.
//
// Measured rules (a context, outside any stream capture):
//   tune_calibrate      times every form on three synthetic clouds on this
//                       device and fits, per form, t = c0 + c1 W H N + c2 (W + H) N;
//   tune_choose_form    the fastest form whose stated NRMS bound is within the
//                       requested tolerance, by that model;
//   tune_choose_bn      the fastest GEMM tile width for a hologram shape and
//                       form, timed on that shape with 4096 points, cached.
// With CGH_TUNE_CACHE=<path> in the environment the measurements are read
// from and written to a small JSON file keyed by the device name.
#include "tuner.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "context.h"

namespace cgh {

namespace {
constexpr int kDirectCtasPerSm = 2;
constexpr int kForms = 6;
}  // namespace

// Critical path of a direct launch in point-tile steps of one CTA: rounds of pixel tiles x splits over the
// resident CTA slots, times the longest point chunk (chunks differ by at most one tile); each extra chunk adds a
// plane of partial sums, written and read back by the reduction: 0.2 % per chunk.
static double direct_path(int64_t pixel_tiles, int64_t point_tiles, int64_t s, int64_t slots)
{
    const int64_t rounds = (pixel_tiles * s + slots - 1) / slots;
    const int64_t longest = (point_tiles + s - 1) / s;
    return (double)rounds * (double)longest * (1.0 + 0.002 * (double)(s - 1));
}

static int split_for(int64_t pixel_tiles, int64_t point_tiles, int64_t slots)
{
    if (pixel_tiles <= 0 || point_tiles <= 1) return 1;
    int best = 1;
    double best_t = direct_path(pixel_tiles, point_tiles, 1, slots);
    for (int64_t s = 2; s <= 64 && s * 2 <= point_tiles; ++s) {
        const double t = direct_path(pixel_tiles, point_tiles, s, slots);
        if (t < best_t * (1.0 - 1e-9)) {
            best = (int)s;
            best_t = t;
        }
    }
    return best;
}

int choose_point_split(int64_t pixel_tiles, int64_t point_tiles, int num_sms)
{
    return split_for(pixel_tiles, point_tiles, (int64_t)num_sms * kDirectCtasPerSm);
}

DirectLayout choose_layout(const DirectShape *shapes, int n_shapes, int width, int height, int64_t point_tiles,
                           int num_sms, int force_split, const double *step_cost)
{
    DirectLayout best{};
    double best_t = 1e300, best_area = 0.0;
    for (int k = 0; k < n_shapes; ++k) {
        const DirectShape &sh = shapes[k];
        const int64_t slots = (int64_t)num_sms * sh.per_sm;
        const int64_t tiles = (int64_t)((width + sh.tile_w - 1) / sh.tile_w) * ((height + sh.tile_h - 1) / sh.tile_h);
        int s = force_split > 0 ? force_split : split_for(tiles, point_tiles, slots);
        if (s > point_tiles) s = (int)(point_tiles > 0 ? point_tiles : 1);
        // in point-tile steps of one CTA: the shapes keep the same warps per SM (threads x CTAs per SM) and the
        // same pixels per thread, so a step takes the same time whatever the shape
        const double t =
            direct_path(tiles, point_tiles > 0 ? point_tiles : 1, s, slots) * (step_cost ? step_cost[k] : 1.0);
        const double area = (double)tiles * sh.tile_w * sh.tile_h;
        // a shorter path wins; on equal paths, fewer padded pixels computed
        if (t < best_t * (1.0 - 1e-9) || (t <= best_t * (1.0 + 1e-9) && area < best_area)) {
            best_t = t;
            best_area = area;
            best = DirectLayout{sh, s};
        }
    }
    return best;
}

// The complex wave's tall block reads the tile's tables, its wide block takes each thread's own sines and
// cosines: a point-tile step of the wide block takes 1.78 times as long (5.71 against 3.20 ms at 1920x1080,
// 10^4 points), so the wide block wins only where it needs far fewer rounds.
constexpr double kWaveWideStepCost = 1.78;

DirectLayout choose_direct_layout(bool wave, int width, int height, int64_t point_tiles, int num_sms,
                                  int force_split)
{
    const DirectShape shapes[2] = {wave ? direct_wave_shape(false) : direct_shape(false),
                                   wave ? direct_wave_shape(true) : direct_shape(true)};
    const double wave_cost[2] = {kWaveWideStepCost, 1.0};
    return choose_layout(shapes, 2, width, height, point_tiles, num_sms, force_split, wave ? wave_cost : nullptr);
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

// Time of one k-block (64 K elements) of one GEMM unit, in microseconds, by tile width, for the one-CTA and the
// two-SM form (index 0 and 1) of the FP16/BF16 GEMM and of split FP16 (three products per k-block).  Measured on
// GB300 (least time per k-block of a unit over 1024x1024, 1920x1080 and 3840x2160 holograms, 4 10^3 to 1.5 10^5
// points, every width, split and orientation): up to a width of 224 it hardly depends on the width, so a unit is
// bound by its operand stream, not by its MMAs; the 4-stage ring of the 256-wide one-CTA tile is slower, the
// two-SM form's 256-wide tile (half of B per CTA) is not.  240 is interpolated (one-CTA form only).
struct KbCost {
    int bn;
    double f16[2], split[2];
};
static const KbCost kKbCost[] = {
    {128, {0.273, 0.269}, {0.908, 0.969}}, {192, {0.271, 0.269}, {0.924, 0.992}},
    {224, {0.272, 0.275}, {0.939, 1.025}}, {240, {0.295, 0.0}, {0.99, 0.0}},
    {256, {0.318, 0.274}, {1.048, 1.035}},
};
// Effective bandwidth of the split reduction, bytes per microsecond.
constexpr double kReduceBytesPerUs = 3.0e6;

GemmLayout choose_gemm_layout(int width, int height, int64_t k_blocks, int ctas, bool split_form, int force_bn,
                              int force_splits, int force_trans, int force_pair)
{
    GemmLayout best{false, 256, 1, false};
    double best_t = 1e300;
    for (int pair = 0; pair < 2; ++pair) {
        if ((force_pair == 1 && !pair) || (force_pair == 2 && pair)) continue;   // 1: always, 2: never
        if (pair && ctas < 2) continue;
        const int tile_m = pair ? 256 : 128;
        const int slots = pair ? ctas / 2 : ctas;   // the two-SM form's units run on clusters of two CTAs
        for (int tr = 0; tr < 2; ++tr) {
            if (force_trans == 1 && tr) continue;    // 1: never transposed
            if (force_trans == 2 && !tr) continue;   // 2: always transposed
            const int64_t a_rows = tr ? width : height, b_rows = tr ? height : width;
            const int64_t tiles_m = (a_rows + tile_m - 1) / tile_m;
            for (const KbCost &kc : kKbCost) {
                const int bn = kc.bn;
                if (force_bn > 0 && bn != force_bn) continue;
                const double c = split_form ? kc.split[pair] : kc.f16[pair];
                if (c <= 0.0) continue;   // no two-SM form of this width (halves of whole 32-row groups)
                const int64_t tiles = tiles_m * ((b_rows + bn - 1) / bn);
                for (int64_t s = 1; s <= 16; ++s) {
                    if (force_splits > 0 && s != force_splits) continue;
                    if (force_splits <= 0 && s > 1 && s * 4 > k_blocks) break;
                    const int64_t rounds = (tiles * s + slots - 1) / slots;
                    // critical path: rounds of units of ceil(k_blocks / s) k-blocks (each split a little
                    // slower: the units in flight spread over more K ranges), then the split reduction
                    double t = (double)rounds * (double)((k_blocks + s - 1) / s) * c * (1.0 + 0.01 * (double)(s - 1));
                    if (s > 1) t += (double)(s + 1) * (double)width * (double)height * 4.0 / kReduceBytesPerUs;
                    // the transposed write-out (32 lanes, 32 consecutive columns) breaks ties
                    if (tr) t *= 0.995;
                    if (t < best_t * (1.0 - 1e-9)) {
                        best_t = t;
                        best = GemmLayout{tr != 0, bn, (int)s, pair != 0};
                    }
                }
            }
        }
    }
    if (best_t == 1e300 && force_pair == 1)   // no two-SM form of the forced width
        return choose_gemm_layout(width, height, k_blocks, ctas, split_form, force_bn, force_splits, force_trans, 2);
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

// Stated NRMS bound of each form against the FP64 oracle (measured values are
// below these: direct SFU ~4e-7, direct accurate ~1e-7, split FP16 ~3e-6,
// FP16 ~3e-4, BF16 ~2e-3 on the display-size clouds).
double form_nrms_bound(int form)
{
    switch (form) {
    case CGH_DIRECT_SFU: return 1e-5;
    case CGH_DIRECT_ACCURATE: return 2e-6;
    case CGH_GEMM_F16: return 2e-3;
    case CGH_GEMM_BF16: return 1e-2;
    case CGH_GEMM_SPLIT16: return 1e-5;
    default: return 1.0;
    }
}

struct TuneState {
    bool calibrated = false;
    double coef[kForms][3] = {};   // seconds: c0, per W*H*N, per (W+H)*N
    std::map<std::string, int> bn;
    std::string device;
};

void destroy_tune_state(TuneState *t)
{
    delete t;
}

namespace {

std::string device_name(int dev)
{
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    return std::string(p.name) + ":" + std::to_string(p.multiProcessorCount);
}

const char *cache_path()
{
    const char *p = std::getenv("CGH_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

void save_cache(const TuneState &t)
{
    const char *path = cache_path();
    if (!path) return;
    FILE *f = std::fopen(path, "w");
    if (!f) return;
    std::fprintf(f, "{\n \"abi\": %d,\n \"device\": \"%s\",\n \"coef\": [", CGH_ABI_VERSION, t.device.c_str());
    for (int i = 0; i < kForms; ++i)
        std::fprintf(f, "%s[%.9e, %.9e, %.9e]", i ? ", " : "", t.coef[i][0], t.coef[i][1], t.coef[i][2]);
    std::fprintf(f, "],\n \"bn\": {");
    bool first = true;
    for (const auto &kv : t.bn) {
        std::fprintf(f, "%s\"%s\": %d", first ? "" : ", ", kv.first.c_str(), kv.second);
        first = false;
    }
    std::fprintf(f, "}\n}\n");
    std::fclose(f);
}

// Parses a cache written by save_cache: accepted only when it names this device and ABI and every one of the
// kForms x 3 coefficients is finite and not negative (they are seconds, and seconds per evaluation); anything
// else -- a truncated or edited file, another device, another ABI -- is refused as a whole and the tuner
// calibrates instead.  Tile widths that the GEMM does not support are skipped.
bool parse_cache(const std::string &text, const std::string &device, TuneState &out)
{
    const std::string dev_key = "\"device\": \"" + device + "\"";
    const std::string abi_key = "\"abi\": " + std::to_string(CGH_ABI_VERSION) + ",";
    if (text.find(dev_key) == std::string::npos || text.find(abi_key) == std::string::npos) return false;
    size_t c = text.find("\"coef\": [");
    if (c == std::string::npos) return false;
    double coef[kForms][3];
    const char *p = text.c_str() + c + 9;
    for (int i = 0; i < kForms; ++i) {
        double a, b, d;
        int n = 0;
        if (std::sscanf(p, " [%lf, %lf, %lf]%n", &a, &b, &d, &n) != 3 || n <= 0) return false;
        for (double v : {a, b, d})
            if (!std::isfinite(v) || v < 0.0) return false;
        coef[i][0] = a;
        coef[i][1] = b;
        coef[i][2] = d;
        p += n;
        while (*p == ',' || *p == ' ') ++p;
    }
    if (*p != ']') return false;
    std::map<std::string, int> bn;
    size_t bpos = text.find("\"bn\": {");
    if (bpos == std::string::npos) return false;
    const char *q = text.c_str() + bpos + 7;
    for (;;) {
        char key[128];
        int val, n = 0;
        if (std::sscanf(q, " \"%127[^\"]\": %d%n", key, &val, &n) != 2) break;
        if (gemm_bn_supported(val)) bn[key] = val;
        q += n;
        while (*q == ',' || *q == ' ') ++q;
    }
    while (*q == ' ' || *q == '\n') ++q;
    if (*q != '}') return false;   // a truncated tile-width table
    std::memcpy(out.coef, coef, sizeof coef);
    out.bn = bn;
    out.calibrated = true;
    return true;
}

bool read_file(const char *path, std::string &text)
{
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
    std::fclose(f);
    return true;
}

// Reads the cache of CGH_TUNE_CACHE for this device, if there is an acceptable one.
bool load_cache(TuneState &t)
{
    const char *path = cache_path();
    std::string text;
    if (!path || !read_file(path, text)) return false;
    return parse_cache(text, t.device, t);
}

// Deterministic synthetic cloud (integer positions inside the hologram,
// z in [0.3, 1] m, A in [0.5, 1]) for the measurements.
void synth_points(int width, int height, int64_t n, std::vector<float> &xyz, std::vector<float> &amp)
{
    xyz.resize((size_t)n * 3);
    amp.resize((size_t)n);
    uint64_t s = 0x9e3779b97f4a7c15ull;
    auto next = [&]() {
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        return s;
    };
    for (int64_t j = 0; j < n; ++j) {
        xyz[3 * j + 0] = (float)(next() % (uint64_t)width);
        xyz[3 * j + 1] = (float)(next() % (uint64_t)height);
        xyz[3 * j + 2] = 0.3f + 0.7f * (float)((next() >> 11) * (1.0 / 9007199254740992.0));
        amp[j] = 0.5f + 0.5f * (float)((next() >> 11) * (1.0 / 9007199254740992.0));
    }
}

struct Scratch {
    float *xyz = nullptr, *amp = nullptr, *out = nullptr;
    ~Scratch()
    {
        if (xyz) cudaFree(xyz);
        if (amp) cudaFree(amp);
        if (out) cudaFree(out);
    }
};

// Seconds per hologram of `form` (tile width bn, 0 = default) on a synthetic cloud.
double time_form(cgh_ctx *ctx, int form, int bn, int width, int height, int64_t n, int reps)
{
    std::vector<float> hx, ha;
    synth_points(width, height, n, hx, ha);
    Scratch s;
    if (cudaMalloc(&s.xyz, hx.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&s.amp, ha.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&s.out, (size_t)width * height * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return -1.0;
    }
    cudaMemcpy(s.xyz, hx.data(), hx.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(s.amp, ha.data(), ha.size() * sizeof(float), cudaMemcpyHostToDevice);
    const int saved_form = ctx->form, saved_bn = ctx->gemm_bn, saved_model = ctx->phase_model;
    const int saved_group = ctx->gemm_group;
    const bool saved_profile = ctx->profile;
    ctx->form = form;
    ctx->gemm_bn = bn;
    ctx->profile = false;
    ctx->phase_model = CGH_PHASE_FRESNEL;   // the forms' own cost; the piston and reference add none per term
    ctx->gemm_group = 1;                    // synthetic depths are continuous: no grouping
    double sec = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
        compute_hologram(ctx, width, height, ctx->pitch, ctx->lambda, s.xyz, s.amp, n, s.out) == CGH_OK) {
        cudaEventRecord(e0, ctx->stream);
        bool ok = true;
        for (int r = 0; r < reps && ok; ++r)
            ok = compute_hologram(ctx, width, height, ctx->pitch, ctx->lambda, s.xyz, s.amp, n, s.out) == CGH_OK;
        cudaEventRecord(e1, ctx->stream);
        if (ok && cudaEventSynchronize(e1) == cudaSuccess) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) sec = ms * 1e-3 / reps;
        }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ctx->form = saved_form;
    ctx->gemm_bn = saved_bn;
    ctx->phase_model = saved_model;
    ctx->gemm_group = saved_group;
    ctx->profile = saved_profile;
    return sec;
}

// Least squares for t = c0 + c1 x1 + c2 x2 over the samples; coefficients kept >= 0.
void fit3(const std::vector<double> &t, const std::vector<double> &x1, const std::vector<double> &x2, double c[3])
{
    const size_t m = t.size();
    double A[3][3] = {}, b[3] = {};
    for (size_t i = 0; i < m; ++i) {
        const double r[3] = {1.0, x1[i], x2[i]};
        for (int p = 0; p < 3; ++p) {
            b[p] += r[p] * t[i];
            for (int q = 0; q < 3; ++q) A[p][q] += r[p] * r[q];
        }
    }
    // Cramer's rule on the normal equations, then clamp
    auto det3 = [](double M[3][3]) {
        return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
               M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    };
    const double d = det3(A);
    for (int k = 0; k < 3; ++k) {
        double M[3][3];
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) M[p][q] = (q == k) ? b[p] : A[p][q];
        c[k] = d != 0.0 ? det3(M) / d : 0.0;
    }
    if (c[0] < 0.0 || c[1] < 0.0 || c[2] < 0.0) {
        // fall back to a proportional model through the largest sample
        size_t big = 0;
        for (size_t i = 1; i < m; ++i)
            if (x1[i] > x1[big]) big = i;
        c[0] = 0.0;
        c[1] = x1[big] > 0 ? t[big] / x1[big] : 0.0;
        c[2] = 0.0;
    }
}

std::string bn_key(int width, int height, int form)
{
    return std::to_string(width) + "x" + std::to_string(height) + ":" + std::to_string(form);
}

TuneState *state(cgh_ctx *ctx)
{
    if (!ctx->tune) {
        ctx->tune = new TuneState();
        ctx->tune->device = device_name(ctx->device);
        load_cache(*ctx->tune);
    }
    return ctx->tune;
}

}  // namespace

int tune_calibrate(cgh_ctx *ctx, bool force)
{
    TuneState *t = state(ctx);
    if (t->calibrated && !force) return CGH_OK;
    struct Shape {
        int w, h;
        int64_t n;
    };
    const Shape shapes[3] = {{256, 256, 2048}, {1024, 512, 8192}, {1024, 1024, 16384}};
    const int forms[5] = {CGH_DIRECT_SFU, CGH_DIRECT_ACCURATE, CGH_GEMM_F16, CGH_GEMM_BF16, CGH_GEMM_SPLIT16};
    for (int f : forms) {
        std::vector<double> ts, x1, x2;
        for (const Shape &s : shapes) {
            const double sec = time_form(ctx, f, 0, s.w, s.h, s.n, 3);
            if (sec <= 0.0) return CGH_ECUDA;
            ts.push_back(sec);
            x1.push_back((double)s.w * s.h * (double)s.n);
            x2.push_back((double)(s.w + s.h) * (double)s.n);
        }
        fit3(ts, x1, x2, t->coef[f]);
    }
    t->calibrated = true;
    save_cache(*t);
    return CGH_OK;
}

double tune_predict(cgh_ctx *ctx, int form, int width, int height, int64_t n)
{
    TuneState *t = state(ctx);
    const double *c = t->coef[form];
    return c[0] + c[1] * (double)width * height * (double)n + c[2] * (double)(width + height) * (double)n;
}

int tune_choose_form(cgh_ctx *ctx, int width, int height, int64_t n, double tol)
{
    if (tune_calibrate(ctx, false) != CGH_OK) return CGH_DIRECT_SFU;
    const int forms[5] = {CGH_DIRECT_SFU, CGH_DIRECT_ACCURATE, CGH_GEMM_F16, CGH_GEMM_BF16, CGH_GEMM_SPLIT16};
    int best = -1;
    double best_t = 1e300;
    for (int f : forms) {
        if (form_nrms_bound(f) > tol) continue;
        const double tp = tune_predict(ctx, f, width, height, n);
        if (tp < best_t) {
            best_t = tp;
            best = f;
        }
    }
    // nothing meets a tolerance tighter than every bound: the most accurate form
    return best >= 0 ? best : CGH_DIRECT_ACCURATE;
}

int tune_choose_bn(cgh_ctx *ctx, int width, int height, int form)
{
    TuneState *t = state(ctx);
    const std::string key = bn_key(width, height, form);
    auto it = t->bn.find(key);
    if (it != t->bn.end()) return it->second;
    static const int cands[] = {256, 240, 224, 192, 128};
    int best = choose_gemm_bn(width);
    double best_t = 1e300;
    for (int bn : cands) {
        const double sec = time_form(ctx, form, bn, width, height, 4096, 3);
        if (sec > 0.0 && sec < best_t) {
            best_t = sec;
            best = bn;
        }
    }
    t->bn[key] = best;
    save_cache(*t);
    return best;
}

int choose_form(int width, int height, int64_t n_points, double tol, int num_sms)
{
    (void)width;
    (void)height;
    (void)n_points;
    (void)num_sms;
    // without measurements: the direct SFU form when it is admissible, else the accurate one
    return form_nrms_bound(CGH_DIRECT_SFU) <= tol ? CGH_DIRECT_SFU
                                                   : (tol >= form_nrms_bound(CGH_GEMM_F16) ? CGH_GEMM_F16
                                                                                            : CGH_DIRECT_ACCURATE);
}

}  // namespace cgh

extern "C" int cgh_tune_cache_check(const char *path, const char *device_name, int *accepted)
{
    if (!path || !device_name || !accepted) return CGH_EINVAL;
    *accepted = 0;
    std::string text;
    if (!cgh::read_file(path, text)) return CGH_OK;
    cgh::TuneState t;
    *accepted = cgh::parse_cache(text, device_name, t) ? 1 : 0;
    return CGH_OK;
}
