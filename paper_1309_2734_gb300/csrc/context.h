// Internal: the context behind the C ABI's opaque cgh_ctx, its workspace
// helpers, and the pipeline entry points shared by api.cu, batch.cu and tuner.cu.
#pragma once

#include <chrono>
#include <cmath>
#include <cstdint>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/cgh.h"
#include "device_util.cuh"
#include "kernels.h"

namespace cgh {
constexpr int64_t kDefaultFactorBudgetMb = 2048;   // factor workspace of one chunk of points, MiB
struct BatchPlan;
struct TuneState;
void destroy_batch_plan(BatchPlan *plan);
void destroy_tune_state(TuneState *t);
}  // namespace cgh

struct cgh_ctx {
    int width = 0, height = 0;
    double pitch = 0.0, lambda = 0.0;
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    int form = CGH_FORM_AUTO;
    int64_t timeout_ms = 5000;
    int point_split = 0;
    int direct_ctas = 0;      // CGH_OPT_DIRECT_CTAS
    int direct_shape = 0;     // CGH_OPT_DIRECT_SHAPE
    int test_alloc_fail = 0;  // CGH_OPT_TEST_ALLOC_FAIL: workspace growths still to refuse
    int batch_mode = 0;       // CGH_OPT_BATCH_MODE
    int batch_overlap = 1;    // CGH_OPT_BATCH_OVERLAP
    int gemm_splitk = 0;
    int gemm_bn = 0;
    int gemm_chunk = 0;
    int drop_tile = -1;       // CGH_OPT_TEST_DROP_TILE
    int64_t factor_budget_mb = cgh::kDefaultFactorBudgetMb;   // CGH_OPT_FACTOR_BUDGET_MB
    int gemm_trans = 0;                // CGH_OPT_GEMM_TRANSPOSE
    int gemm_pipeline = 1;             // CGH_OPT_GEMM_PIPELINE (measured: no gain on GB300, off)
    cudaStream_t side_stream = nullptr;   // factor generation of the next point chunk
    cudaEvent_t ev_ready = nullptr, ev_fact[2] = {nullptr, nullptr}, ev_gemm[2] = {nullptr, nullptr};
    int64_t tol_e9 = 10000;   // 1e-5
    int *d_status = nullptr;  // [0] status bits, [1..2] quantiser scratch, [3] spare
    void *ws = nullptr;       // grow-only workspace
    size_t ws_bytes = 0;
    void *pws = nullptr;      // GEMM forms: prepared points and their groups (grow-only)
    size_t pws_bytes = 0;
    int *h_meta = nullptr;    // pinned: counts the grouped GEMM form reads back
    int gemm_group = 0;       // CGH_OPT_GEMM_GROUP
    int gemm_persistent = 0;  // CGH_OPT_GEMM_PERSISTENT
    int gemm_pair = 0;        // CGH_OPT_GEMM_PAIR
    int batch_chunk_mb = 0;   // CGH_OPT_BATCH_CHUNK_MB
    int batch_premade_pct = -1;   // CGH_OPT_BATCH_PREMADE_PCT (-1: the default)
    int phase_model = CGH_PHASE_FRESNEL;                 // CGH_OPT_PHASE_MODEL
    // Fresnel diffraction: cuFFT plan for the 2H x 2W grid, padded work plane,
    // and the chirp's spectrum for the distance fft_spec_z (0: none yet)
    void *fft_plan = nullptr;          // cuFFT, only for grids beyond the own FFT's lengths
    cgh::FftGrid fft_g;                // the own FFT's grid (fft_g.ok)
    float2 *fft_twx = nullptr, *fft_twy = nullptr;
    float2 *fft_pad = nullptr, *fft_spec = nullptr;
    bool fft_ready = false;
    double fft_spec_z = 0.0;
    double ref_sx = 0.0, ref_sy = 0.0, ref_phase0 = 0.0;   // cgh_set_reference
    void *io = nullptr;       // device staging of cgh_point_cloud_host
    size_t io_bytes = 0;
    // CGH_OPT_PROFILE: events around each launch, folded into per-kernel totals on read
    bool profile = false;
    struct Pending {
        const char *name;
        int launches;
        cudaEvent_t start, stop;
    };
    struct Total {
        std::string name;
        int64_t launches;
        double ms;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    std::vector<Total> totals;
    cgh::BatchPlan *batch = nullptr;   // cgh_batch: cached plan and CUDA graph
    cgh::BatchPlan *single = nullptr;  // CGH_OPT_GEMM_PERSISTENT: one hologram's persistent plan and graph
    cgh::TuneState *tune = nullptr;    // autotuner measurements
};

namespace cgh {

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
        dev_ = dev;
    }
    ~DeviceGuard()
    {
        if (prev_ != dev_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = 0, dev_ = 0;
};

inline bool finite_positive(double v)
{
    return std::isfinite(v) && v > 0.0;
}

inline bool valid_size(int w, int h)
{
    return w >= 1 && h >= 1 && w <= kMaxSide && h <= kMaxSide;
}

inline size_t align_up(size_t v, size_t a)
{
    return (v + a - 1) / a * a;
}

// Grows a workspace buffer to at least `need` bytes (contents are not kept).  A pending injected failure
// (CGH_OPT_TEST_ALLOC_FAIL) is taken instead of a growth: the buffer is left as it was and CGH_ENOMEM returned,
// as when cudaMalloc fails.
inline int ensure(cgh_ctx *ctx, void **buf, size_t *cap, size_t need)
{
    if (need <= *cap) return CGH_OK;
    if (ctx->test_alloc_fail > 0) {
        --ctx->test_alloc_fail;
        return CGH_ENOMEM;
    }
    if (*buf) {
        cudaFree(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    size_t want = align_up(need + need / 4, 1 << 20);
    if (cudaMalloc(buf, want) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return CGH_ENOMEM;
    }
    *cap = want;
    return CGH_OK;
}

inline int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return CGH_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? CGH_ENOMEM : CGH_ECUDA;
}

inline cudaEvent_t take_event(cgh_ctx *ctx)
{
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Brackets the launches made in its scope: an NVTX range named for the kernel (always; it costs nothing
// without a tool attached), and with CGH_OPT_PROFILE events on the context's stream.
class ProfileScope {
  public:
    ProfileScope(cgh_ctx *ctx, const char *name, int launches, cudaStream_t s = nullptr)
        : ctx_(ctx), name_(name), launches_(launches), stream_(s ? s : ctx->stream)
    {
        nvtxRangePushA(name);
        if (ctx_->profile && (start_ = take_event(ctx_))) cudaEventRecord(start_, stream_);
    }
    ~ProfileScope()
    {
        nvtxRangePop();
        if (!start_) return;
        cudaEvent_t stop = take_event(ctx_);
        if (!stop) return;
        cudaEventRecord(stop, stream_);
        ctx_->pending.push_back({name_, launches_, start_, stop});
    }

  private:
    cgh_ctx *ctx_;
    const char *name_;
    int launches_;
    cudaStream_t stream_;
    cudaEvent_t start_ = nullptr;
};

// The side stream and events of the factor/GEMM pipeline, created on first use.
inline int ensure_side_stream(cgh_ctx *ctx)
{
    if (ctx->side_stream) return CGH_OK;
    if (cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ctx->side_stream = nullptr;
        return CGH_ECUDA;
    }
    for (cudaEvent_t *ev : {&ctx->ev_ready, &ctx->ev_fact[0], &ctx->ev_fact[1], &ctx->ev_gemm[0], &ctx->ev_gemm[1]})
        if (cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return CGH_ECUDA;
        }
    return CGH_OK;
}

// frac(turns) in 2^-64 turn: the double's fraction in two 32-bit halves, so
// that all of its bits survive.
inline unsigned long long turns_fixed64(double turns)
{
    const double f = turns - std::floor(turns);             // [0, 1)
    const double hi = std::floor(std::ldexp(f, 32));
    const double lo = std::ldexp(std::ldexp(f, 32) - hi, 32);   // exact, [0, 2^32)
    return ((unsigned long long)hi << 32) + (unsigned long long)std::llround(lo);
}

// The context's plane-wave reference in fixed point: kx = p sin_x / lambda and
// ky = p sin_y / lambda turns per pixel, phi0 = phase0 / (2 pi) turns.
inline cgh::PhaseRef phase_ref(const cgh_ctx *ctx)
{
    cgh::PhaseRef r;
    r.kx = turns_fixed64(ctx->pitch * ctx->ref_sx / ctx->lambda);
    r.ky = turns_fixed64(ctx->pitch * ctx->ref_sy / ctx->lambda);
    const unsigned long long p0 = turns_fixed64(ctx->ref_phase0 / 6.283185307179586476925286766559);
    r.phi0 = (uint32_t)((p0 >> 32) + ((p0 >> 31) & 1ull));
    r.piston = ctx->phase_model != CGH_PHASE_FRESNEL ? 1u : 0u;
    return r;
}

inline bool piston_on(const cgh_ctx *ctx)
{
    return ctx->phase_model != CGH_PHASE_FRESNEL;   // Eq. 2 with its first term, and Eq. 1
}

// What the point preparation stores in aux.x for the context's phase terms:
// the piston, a zero piston slot (reference phase only), or the second
// difference of the plain recurrence.
inline int aux_mode(const cgh_ctx *ctx)
{
    if (piston_on(ctx)) return cgh::kAuxPiston;
    return phase_ref(ctx).any() ? cgh::kAuxZero : cgh::kAuxSecondDiff;
}

inline int64_t padded_points(int64_t n)
{
    return (n + kPointTile - 1) / kPointTile * kPointTile;
}


// Pipeline entry points (api.cu).
int run_direct(cgh_ctx *ctx, bool sfu, int width, int height, double pitch, double lambda, const float *d_xyz,
               const float *d_amp, int64_t n, float *d_out);
int run_gemm(cgh_ctx *ctx, int form, int width, int height, double pitch, double lambda, const float *d_xyz,
             const float *d_amp, int64_t n, float *d_out);
int compute_hologram(cgh_ctx *ctx, int width, int height, double pitch, double lambda, const float *d_xyz,
                     const float *d_amp, int64_t n, float *d_out);
int factor_mode(int form);
int resolve_form(cgh_ctx *ctx, int width, int height, int64_t n);
int run_batch(cgh_ctx *ctx, const cgh_instance *inst, int n_inst);
int batch_forms(const cgh_ctx *ctx, int *forms, int max_entries);
int run_single_persistent(cgh_ctx *ctx, int form, const cgh_instance &inst);
int run_wave(cgh_ctx *ctx, int form, const float *d_xyz, const float *d_amp, int64_t n, float *d_out);
int run_spherical(cgh_ctx *ctx, int width, int height, double pitch, double lambda, const float *d_xyz,
                  const float *d_amp, int64_t n, int planes, float *d_out);

}  // namespace cgh
