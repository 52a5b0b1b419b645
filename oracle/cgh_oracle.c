/*
 * FP64 CPU oracle for the point-cloud Fresnel hologram.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's compute path may link,
 * load or call this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA path, and it uses different arithmetic on purpose:
 * double-precision phases reduced in turns and libm cos/sin, where the GPU
 * uses 64-bit fixed-point turns and single precision.
 *
 * What it computes (the plain definition):
 *
 *   Eq. 2 (Fresnel approximation of the spherical wave of Eq. 1) and Eq. 5
 *   (amplitude CGH after dropping |O|^2, |R|^2 and the constant 2 A_r), with
 *   the per-point piston 2 pi z_j / lambda and the reference phase phi_r left
 *   out, and with hologram pixels (m, n) and point positions (x_j, y_j) in
 *   pixel units of pitch p:
 *
 *     I(m, n) = sum_j A_j cos(pi p^2 / (lambda z_j) * ((m - x_j)^2 + (n - y_j)^2))
 *
 *   which is written here as cos(2 pi t) with t = c_j r^2 turns and
 *   c_j = p^2 / (2 lambda z_j) turns per px^2 (Section 2.2 writes the same
 *   constant as P_j = 1/(2 lambda z_j) in metres).  t is reduced by
 *   subtracting the nearest integer before the cosine.
 *
 *   The complex object wave O(m, n) = sum_j A_j exp(i 2 pi t) of Eq. 2 (same
 *   restriction) is given too, for the kinoform of Eq. 3.
 *
 *   The separable factors: with alpha = 2 pi c_j (m - x_j)^2 and
 *   beta = 2 pi c_j (n - y_j)^2 the phase is alpha + beta, so
 *   cos(alpha + beta) = cos(alpha) cos(beta) - sin(alpha) sin(beta).  The
 *   factor matrices P[n][2j] = cos beta, P[n][2j+1] = sin beta,
 *   Q[m][2j] = A_j cos alpha, Q[m][2j+1] = -A_j sin alpha give I = P Q^T.
 *
 *   The 8-bit quantiser of an amplitude hologram (min/max rule); the paper
 *   only prints the phase rule of its listings (Section 4.1:
 *   holo = (uchar)(255/(2 pi) psi)), the min/max form is this library's reading
 *   for amplitude holograms.  It is specified in single precision with every
 *   product and difference rounded separately, so that it can be reproduced
 *   bit for bit; build this file with -ffp-contract=off.
 *
 * Pixels are stored row-major, out[n * width + m] (Section 4.1, adr = j + WIDTH i).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <float.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* c_j = p^2 / (2 lambda z_j), turns per square pixel, from the float inputs promoted to double. */
static double *turn_coefficients(double pitch, double lambda, const float *xyz, int64_t n)
{
    double *c = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!c) return NULL;
    for (int64_t j = 0; j < n; ++j) {
        double z = (double)xyz[3 * j + 2];
        c[j] = (pitch * pitch) / (2.0 * lambda * z);
    }
    return c;
}

/* 2 pi times the distance of t from its nearest integer, in [-pi, pi]. */
static double reduced_angle(double t)
{
    return TWO_PI * (t - rint(t));
}

/* One pixel of Eq. 5 (restricted form): sum_j A_j cos(2 pi c_j r^2). */
static double pixel_amplitude(double m, double n_row, const float *xyz, const float *amp,
                              const double *c, int64_t npts)
{
    double acc = 0.0;
    for (int64_t j = 0; j < npts; ++j) {
        double dx = m - (double)xyz[3 * j + 0];
        double dy = n_row - (double)xyz[3 * j + 1];
        double r2 = dx * dx + dy * dy;
        acc += (double)amp[j] * cos(reduced_angle(c[j] * r2));
    }
    return acc;
}

/*
 * I over the window rows [row0, row0+rows) x cols [col0, col0+cols) of the
 * hologram; out is [rows][cols] row-major.  Returns 0, or -1 on bad arguments.
 */
int oracle_field_window(double pitch, double lambda, const float *xyz, const float *amp, int64_t npts,
                        int row0, int rows, int col0, int cols, double *out)
{
    if (rows < 0 || cols < 0 || npts < 0 || !out) return -1;
    double *c = turn_coefficients(pitch, lambda, xyz, npts);
    if (!c) return -1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < rows; ++r) {
        for (int q = 0; q < cols; ++q) {
            out[(int64_t)r * cols + q] =
                pixel_amplitude((double)(col0 + q), (double)(row0 + r), xyz, amp, c, npts);
        }
    }
    free(c);
    return 0;
}

/* I at npix scattered pixels (pm[i], pn[i]) = (column, row). */
int oracle_field_points(double pitch, double lambda, const float *xyz, const float *amp, int64_t npts,
                        const int32_t *pm, const int32_t *pn, int64_t npix, double *out)
{
    if (npix < 0 || npts < 0 || !out) return -1;
    double *c = turn_coefficients(pitch, lambda, xyz, npts);
    if (!c) return -1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < npix; ++i)
        out[i] = pixel_amplitude((double)pm[i], (double)pn[i], xyz, amp, c, npts);
    free(c);
    return 0;
}

/* Complex object wave of Eq. 2 (restricted form) over a window: re + i im. */
int oracle_wave_window(double pitch, double lambda, const float *xyz, const float *amp, int64_t npts,
                       int row0, int rows, int col0, int cols, double *re, double *im)
{
    if (rows < 0 || cols < 0 || npts < 0 || !re || !im) return -1;
    double *c = turn_coefficients(pitch, lambda, xyz, npts);
    if (!c) return -1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < rows; ++r) {
        for (int q = 0; q < cols; ++q) {
            double sr = 0.0, si = 0.0;
            for (int64_t j = 0; j < npts; ++j) {
                double dx = (double)(col0 + q) - (double)xyz[3 * j + 0];
                double dy = (double)(row0 + r) - (double)xyz[3 * j + 1];
                double a = reduced_angle(c[j] * (dx * dx + dy * dy));
                sr += (double)amp[j] * cos(a);
                si += (double)amp[j] * sin(a);
            }
            re[(int64_t)r * cols + q] = sr;
            im[(int64_t)r * cols + q] = si;
        }
    }
    free(c);
    return 0;
}

/*
 * Phase models beyond the restricted form (Section 2.1), in turns, for the
 * widened entry points:
 *
 *   model 0  Eq. 2 / Eq. 5 without the piston:  t = r^2 / (2 lambda z_j)
 *   model 1  Eq. 2 / Eq. 5 with the piston:     t = (z_j + r^2 / (2 z_j)) / lambda
 *   model 2  Eq. 1 (exact spherical wave):      t = sqrt(r^2 + z_j^2) / lambda
 *
 * with r^2 = p^2 ((m - x_j)^2 + (n - y_j)^2) in square metres.  The reference
 * wave R = A_r exp(i phi_r) of Eq. 4 is a plane wave,
 *   phi_r(x_h, y_h) = 2 pi / lambda (x_h sin_x + y_h sin_y) + phase0,
 * x_h = m p, y_h = n p, and enters every term as the "+ phi_r" of Eq. 5:
 *   I(m, n) = sum_j A_j cos(2 pi t_j + phi_r),
 *   O(m, n) = sum_j A_j exp(i (2 pi t_j + phi_r)).
 * Each phase is reduced in turns (t - rint(t)) before cos/sin; t is up to
 * about 2e6 turns, so double precision leaves ~1e-10 turn.
 */
static double model_turn(int model, double pitch, double lambda, double m, double n_row, const float *p)
{
    const double dx = (m - (double)p[0]) * pitch;
    const double dy = (n_row - (double)p[1]) * pitch;
    const double z = (double)p[2];
    const double r2 = dx * dx + dy * dy;
    if (model == 2) return sqrt(r2 + z * z) / lambda;
    const double t = r2 / (2.0 * lambda * z);
    return model == 1 ? t + z / lambda : t;
}

static int model_sum(int model, double pitch, double lambda, double sin_x, double sin_y, double phase0,
                     const float *xyz, const float *amp, int64_t npts, double m, double n_row,
                     double *re, double *im)
{
    const double ref = (m * pitch * sin_x + n_row * pitch * sin_y) / lambda + phase0 / TWO_PI;   /* turns */
    double sr = 0.0, si = 0.0;
    for (int64_t j = 0; j < npts; ++j) {
        double t = model_turn(model, pitch, lambda, m, n_row, xyz + 3 * j);
        t = (t - rint(t)) + (ref - rint(ref));
        const double a = reduced_angle(t);
        sr += (double)amp[j] * cos(a);
        si += (double)amp[j] * sin(a);
    }
    *re = sr;
    if (im) *im = si;
    return 0;
}

/*
 * Field (re) and, when im is not NULL, the complex wave's imaginary part over
 * a window, for phase model 0, 1 or 2 and the plane-wave reference above.
 */
int oracle_model_window(int model, double pitch, double lambda, double sin_x, double sin_y, double phase0,
                        const float *xyz, const float *amp, int64_t npts, int row0, int rows, int col0, int cols,
                        double *re, double *im)
{
    if (model < 0 || model > 2 || rows < 0 || cols < 0 || npts < 0 || !re) return -1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < rows; ++r)
        for (int q = 0; q < cols; ++q) {
            const int64_t k = (int64_t)r * cols + q;
            model_sum(model, pitch, lambda, sin_x, sin_y, phase0, xyz, amp, npts, (double)(col0 + q),
                      (double)(row0 + r), &re[k], im ? &im[k] : NULL);
        }
    return 0;
}

/* The same at npix scattered pixels (pm[i], pn[i]) = (column, row). */
int oracle_model_points(int model, double pitch, double lambda, double sin_x, double sin_y, double phase0,
                        const float *xyz, const float *amp, int64_t npts, const int32_t *pm, const int32_t *pn,
                        int64_t npix, double *re, double *im)
{
    if (model < 0 || model > 2 || npix < 0 || npts < 0 || !re) return -1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < npix; ++i)
        model_sum(model, pitch, lambda, sin_x, sin_y, phase0, xyz, amp, npts, (double)pm[i], (double)pn[i],
                  &re[i], im ? &im[i] : NULL);
    return 0;
}

/*
 * Fresnel diffraction, Eq. 10, by its definition on the pixel grid: the input
 * plane u (height x width, pitch p) is propagated by z (metres, either sign)
 * onto a plane of the same grid,
 *   O(m, n) = exp(i 2 pi z / lambda) / (i lambda z) * p^2
 *             * sum_{m', n'} u(m', n') exp(i pi p^2 ((m - m')^2 + (n - n')^2) / (lambda z)),
 * the integral over the input plane as a sum of cells of area p^2 (the output
 * is the linear convolution, cropped to the input's extent).  The chirp's
 * phase is c ((m - m')^2 + (n - n')^2) turns with c = p^2 / (2 lambda z),
 * reduced in turns; out at npix scattered pixels (pm[i], pn[i]).
 */
int oracle_fresnel_points(int width, int height, double pitch, double lambda, double z, const double *in_re,
                          const double *in_im, const int32_t *pm, const int32_t *pn, int64_t npix, double *out_re,
                          double *out_im)
{
    if (width < 1 || height < 1 || npix < 0 || z == 0.0 || !in_re || !in_im || !out_re || !out_im) return -1;
    const double c = pitch * pitch / (2.0 * lambda * z);
    const double zt = z / lambda;
    const double a0 = TWO_PI * (zt - rint(zt));
    /* exp(i a0) / (i lambda z) * p^2 = exp(i a0) * (-i) * p^2 / (lambda z) */
    const double s = pitch * pitch / (lambda * z);
    const double pre_re = s * sin(a0), pre_im = -s * cos(a0);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < npix; ++i) {
        double sr = 0.0, si = 0.0;
        for (int n2 = 0; n2 < height; ++n2) {
            const double dy = (double)pn[i] - (double)n2;
            for (int m2 = 0; m2 < width; ++m2) {
                const double dx = (double)pm[i] - (double)m2;
                const double a = reduced_angle(c * (dx * dx + dy * dy));
                const double hr = cos(a), hi = sin(a);
                const double ur = in_re[(int64_t)n2 * width + m2], ui = in_im[(int64_t)n2 * width + m2];
                sr += ur * hr - ui * hi;
                si += ur * hi + ui * hr;
            }
        }
        out_re[i] = pre_re * sr - pre_im * si;
        out_im[i] = pre_re * si + pre_im * sr;
    }
    return 0;
}

/*
 * The window of the wavefront-recording method (Section 2.3): the light of a
 * point at distance d = z_j - z_wrp behind the virtual plane that can reach
 * the hologram within the grid's largest diffraction angle, sin(theta) =
 * lambda / (2 p), crosses the plane within radius d tan(theta).  In pixels,
 * w = d s / sqrt(1 - s^2) / p with s = lambda / (2 p), and the window holds the
 * pixels with (m - x_j)^2 + (n - y_j)^2 <= floor(w^2).  Each operation is
 * rounded on its own (double), so that any IEEE implementation draws the
 * same integer boundary.
 */
static double wrp_window2(double pitch, double lambda, double d)
{
    volatile double s = lambda / (2.0 * pitch);
    volatile double s2 = s * s;
    volatile double one_m = 1.0 - s2;
    volatile double den = sqrt(one_m);
    volatile double ds = d * s;
    volatile double t = ds / den;
    volatile double w = t / pitch;
    volatile double w2 = w * w;
    return floor(w2);
}

/*
 * WRP step 1 (Section 2.3): the complex amplitude recorded on the virtual
 * plane at distance z_wrp from the hologram, each point summed over its window
 * only, with phase model 0 or 1 of model_turn (Eq. 2 without or with the
 * piston) at the point's distance d_j = z_j - z_wrp > 0 from the plane:
 *   u(m, n) = sum_{j: r2 <= W2_j} A_j exp(i 2 pi t_j(d_j)).
 * Returns -1 if a point is not behind the plane (d_j <= 0).
 */
int oracle_wrp_record(int model, double pitch, double lambda, double z_wrp, const float *xyz, const float *amp,
                      int64_t npts, int row0, int rows, int col0, int cols, double *re, double *im)
{
    if (model < 0 || model > 1 || rows < 0 || cols < 0 || npts < 0 || !re || !im) return -1;
    for (int64_t j = 0; j < npts; ++j)
        if (!((double)xyz[3 * j + 2] - z_wrp > 0.0)) return -1;
    /* the window of each point, once */
    double *w2 = (double *)malloc(sizeof(double) * (size_t)(npts > 0 ? npts : 1));
    if (!w2) return -1;
    for (int64_t j = 0; j < npts; ++j) w2[j] = wrp_window2(pitch, lambda, (double)xyz[3 * j + 2] - z_wrp);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < rows; ++r)
        for (int q = 0; q < cols; ++q) {
            const double m = (double)(col0 + q), n_row = (double)(row0 + r);
            double sr = 0.0, si = 0.0;
            for (int64_t j = 0; j < npts; ++j) {
                const double d = (double)xyz[3 * j + 2] - z_wrp;
                const double dx = m - (double)xyz[3 * j + 0], dy = n_row - (double)xyz[3 * j + 1];
                if (dx * dx + dy * dy > w2[j]) continue;
                const double r2 = (dx * dx + dy * dy) * pitch * pitch;
                double t = r2 / (2.0 * lambda * d);
                if (model == 1) t += d / lambda;
                const double a = reduced_angle(t);
                sr += (double)amp[j] * cos(a);
                si += (double)amp[j] * sin(a);
            }
            re[(int64_t)r * cols + q] = sr;
            im[(int64_t)r * cols + q] = si;
        }
    free(w2);
    return 0;
}

/*
 * Separable factors: P is [height][2 npts], Q is [width][2 npts] (row-major),
 * with the interleaving described in the header comment.
 */
int oracle_factors(int width, int height, double pitch, double lambda, const float *xyz,
                   const float *amp, int64_t npts, double *P, double *Q)
{
    if (width < 0 || height < 0 || npts < 0 || !P || !Q) return -1;
    double *c = turn_coefficients(pitch, lambda, xyz, npts);
    if (!c) return -1;
    #pragma omp parallel for
    for (int n = 0; n < height; ++n) {
        for (int64_t j = 0; j < npts; ++j) {
            double dy = (double)n - (double)xyz[3 * j + 1];
            double b = reduced_angle(c[j] * dy * dy);
            P[(int64_t)n * 2 * npts + 2 * j] = cos(b);
            P[(int64_t)n * 2 * npts + 2 * j + 1] = sin(b);
        }
    }
    #pragma omp parallel for
    for (int m = 0; m < width; ++m) {
        for (int64_t j = 0; j < npts; ++j) {
            double dx = (double)m - (double)xyz[3 * j + 0];
            double a = reduced_angle(c[j] * dx * dx);
            Q[(int64_t)m * 2 * npts + 2 * j] = (double)amp[j] * cos(a);
            Q[(int64_t)m * 2 * npts + 2 * j + 1] = -(double)amp[j] * sin(a);
        }
    }
    free(c);
    return 0;
}

/*
 * Min/max 8-bit quantiser of an amplitude hologram.
 *   lo = min F, hi = max F (exact, order independent; NaN entries ignored);
 *   if hi == lo (or no finite range) every output is 0;
 *   s  = the smallest float >= 255 / ((double)hi - (double)lo), capped at FLT_MAX;
 *   q  = floor((v - lo) * s) in float with each operation rounded to nearest,
 *        then 255 if q >= 255, q if q >= 0, else 0 (NaN -> 0).
 * The upward rounding of s makes hi map to 255; lo maps to 0.
 * lohi (optional) receives {lo, hi, s}.
 */
int oracle_quantize8(const float *field, int64_t n, uint8_t *out, float *lohi)
{
    if (n < 0 || (n > 0 && (!field || !out))) return -1;
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        float v = field[i];
        if (v < lo) lo = v;
        if (v > hi) hi = v;
    }
    float s = 0.0f;
    int degenerate = !(hi > lo);
    if (!degenerate) {
        double range = (double)hi - (double)lo;
        double sd = 255.0 / range;
        if (sd > (double)FLT_MAX) {
            s = FLT_MAX;
        } else {
            s = (float)sd;
            if ((double)s < sd) s = nextafterf(s, INFINITY);
            if (isinf(s)) s = FLT_MAX;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        if (degenerate) { out[i] = 0; continue; }
        volatile float d = field[i] - lo;   /* rounded on its own */
        volatile float x = d * s;           /* rounded on its own */
        float f = floorf(x);
        out[i] = (f >= 255.0f) ? (uint8_t)255 : ((f >= 0.0f) ? (uint8_t)f : (uint8_t)0);
    }
    if (lohi) { lohi[0] = lo; lohi[1] = hi; lohi[2] = s; }
    return 0;
}

/*
 * Kinoform (phase-only hologram) of a complex field, Eq. 3: the argument
 * psi = atan2(im, re), taken in [0, 2 pi) by adding 2 pi to negative values as
 * the listings of Section 4.1 do, stored as floor(255 psi / (2 pi)) (at most
 * 255).  Computed in double from double inputs (the definition); NaN -> 0.
 */
int oracle_kinoform8(const double *re, const double *im, int64_t n, uint8_t *out)
{
    if (n < 0 || (n > 0 && (!re || !im || !out))) return -1;
    for (int64_t i = 0; i < n; ++i) {
        double psi = atan2(im[i], re[i]);
        if (psi < 0.0) psi += TWO_PI;
        double q = floor(255.0 * psi / TWO_PI);
        out[i] = (q >= 255.0) ? (uint8_t)255 : ((q >= 0.0) ? (uint8_t)q : (uint8_t)0);
    }
    return 0;
}
