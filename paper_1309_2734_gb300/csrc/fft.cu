// f3: the FFTs of Fresnel diffraction (Eq. 10), hand-written for the
// zero-padded linear convolution.
//
// The padded grid is Ly x Lx (powers of two >= 2H - 1, 2W - 1; at most 16384).
// Forward 2-D transform of the H x W input, product with the chirp's
// spectrum, inverse transform, crop:
//   rows     Lx-point FFT of the H nonzero rows only, the input planes read
//            straight into shared memory (the zero padding is never stored);
//   columns  Ly = L1 L2 four-step: pass A, L1-point FFTs over the rows
//            L2 a + b (rows >= H are zero: not loaded); pass B, L2-point FFTs
//            over the contiguous rows L2 c + b, which leaves the spectrum in
//            the scrambled order ky = c + L1 d at row L2 c + d.  Any fixed
//            order serves a convolution, so the chirp's spectrum is kept in
//            that order, and forward pass B, the product and inverse pass B
//            are ONE pass (the middle kernel), twiddles e^{-2 pi i c b / Ly}
//            included; inverse pass A writes only the rows < H.  Columns of
//            256 .. 2048 points instead take ONE pass over strips of 8 to 32
//            whole columns in shared memory (forward transform of the rows
//            < H, product with the spectrum in natural order, inverse, rows
//            < H stored), so the plane crosses HBM once each way; longer
//            columns do not fit at that strip width (64-byte row segments),
//            and narrower strips measured slower than the four-step passes;
//   rows     inverse Lx-point FFT of those H rows, only the first W columns
//            written, into the output planes.
// Every transform is a Stockham autosort FFT in shared memory (the
// formulation of Govindaraju et al., SC 2008: per stage, radix-R butterflies
// over elements M/R apart, twiddles e^{-2 pi i r (j mod Ns) / (Ns R)}, results
// at (j / Ns) Ns R + j mod Ns + r Ns), radix 16 (and one stage of 8, 4 or 2):
// each thread holds 16 values per stage; twiddles come from a table of
// e^{-2 pi i k / L} built in double on the host (the column passes copy the
// entries they use into shared memory).  The transform lengths of display-size
// planes (rows of 2048 .. 16384 points, columns of 32 .. 128) are compiled with
// their geometry as constants, and there the first stage reads its values
// straight from global memory and the last stage writes straight to it, so
// shared memory carries the values only between stages; other lengths take the
// run-time form, which stages whole tiles through shared memory.
#include "device_util.cuh"
#include "host_util.h"
#include "kernels.h"

namespace cgh {

namespace {

// Asynchronous global -> shared copies (no register staging: a whole tile in flight at once).
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// e^{-2 pi i k / 16}, k = 0..7 (cos(pi/8), sin(pi/8), 1/sqrt(2))
constexpr float kC1 = 0.923879532511286756f, kS1 = 0.382683432365089772f, kC2 = 0.707106781186547524f;
__device__ __forceinline__ float2 w16(int k)
{
    switch (k & 7) {
    case 0: return make_float2(1.0f, 0.0f);
    case 1: return make_float2(kC1, -kS1);
    case 2: return make_float2(kC2, -kC2);
    case 3: return make_float2(kS1, -kC1);
    case 4: return make_float2(0.0f, -1.0f);
    case 5: return make_float2(-kS1, -kC1);
    case 6: return make_float2(-kC2, -kC2);
    default: return make_float2(-kC1, -kS1);
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 conj_if(float2 a, bool c)
{
    return c ? make_float2(a.x, -a.y) : a;
}

__host__ __device__ constexpr int rev_bits(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// v * e^{-+2 pi i idx / 16} for a compile-time idx: no product for 1, a swap
// for -i, two for the odd multiples of pi/4 (IEEE rules keep x * 0 + y * 1
// from folding on its own).
__device__ __forceinline__ float2 tw16_mul(float2 v, int idx, bool inv)
{
    switch (idx & 15) {
    case 0: return v;
    case 4: return inv ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    case 8: return make_float2(-v.x, -v.y);
    case 12: return inv ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
    case 2: return inv ? make_float2((v.x - v.y) * kC2, (v.x + v.y) * kC2)
                       : make_float2((v.x + v.y) * kC2, (v.y - v.x) * kC2);
    case 6: return inv ? make_float2(-(v.x + v.y) * kC2, (v.x - v.y) * kC2)
                       : make_float2((v.y - v.x) * kC2, -(v.x + v.y) * kC2);
    default: return cmul(v, conj_if(w16(idx), inv));
    }
}

// y_k = sum_r v_r e^{-+2 pi i r k / R} in registers (radix-2 Cooley-Tukey, natural order out).
template <int R, bool INV>
__device__ __forceinline__ void dft_regs(float2 *v)
{
    constexpr int bits = R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1));
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int j = rev_bits(i, bits);
        if (i < j) {
            const float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
#pragma unroll
    for (int half = 1; half < R; half *= 2) {
#pragma unroll
        for (int k0 = 0; k0 < R; k0 += 2 * half) {
#pragma unroll
            for (int k = 0; k < half; ++k) {
                const float2 a = v[k0 + k], b = tw16_mul(v[k0 + k + half], k * (16 / (2 * half)), INV);
                v[k0 + k] = make_float2(a.x + b.x, a.y + b.y);
                v[k0 + k + half] = make_float2(a.x - b.x, a.y - b.y);
            }
        }
    }
}

enum { kLayoutRows = 0, kLayoutCols = 1, kLayoutStrip = 2 };

// The strip layout (whole columns of a narrow strip, 2^LQ columns): element e of column q at
// ((e + e / 16) << LQ) + q -- the columns interleaved, one gap per 16 elements against the bank conflicts of a
// radix-16 stage's strided stores.
template <int LQ>
__device__ __forceinline__ int strip_addr(int e, int q)
{
    return ((e + (e >> 4)) << LQ) + q;
}

__device__ __forceinline__ int ilog2(int v)
{
    return 31 - __clz(v);
}

// Shared-memory address of element e of sequence q.  Rows: sequences of M
// contiguous values, one float2 of padding per 32 (against bank conflicts of
// the strided stores); columns: element e of column q at e * stride + q.
template <int LAYOUT>
__device__ __forceinline__ int saddr(int e, int q, int M, int stride)
{
    if (LAYOUT == kLayoutRows) return q * (M + (M >> 5)) + e + (e >> 5);
    return e * stride + q;
}

// e^{-2 pi i r k / (Ns R)} for r = 1..R-1 from three table values (k, 4k and 8k
// steps) and at most two products each: w_r = w_(r mod 4) w_(r - r mod 4).
template <int R>
__device__ __forceinline__ void stage_twiddles(float2 *w, const float2 *tw, int idx1, bool inv)
{
    w[0] = make_float2(1.0f, 0.0f);
    if (R == 1) return;
    w[1] = conj_if(tw[idx1], inv);
    if (R == 2) return;
    w[2] = cmul(w[1], w[1]);
    w[3] = cmul(w[2], w[1]);
    if (R == 4) return;
    w[4] = conj_if(tw[4 * idx1], inv);
#pragma unroll
    for (int r = 5; r < 8; ++r) w[r] = cmul(w[4], w[r - 4]);
    if (R == 8) return;
    w[8] = conj_if(tw[8 * idx1], inv);
    w[12] = cmul(w[8], w[4]);
#pragma unroll
    for (int r = 9; r < 16; ++r)
        if (r != 12) w[r] = cmul(w[r & 12], w[r & 3]);
}

// One Stockham stage of radix R over nseq sequences of length M (Ns: size of
// the sub-transforms done so far); all sizes powers of two (lm = log2 M, lq =
// log2 nseq, ls = log2 Ns, lt = log2 of the table stride).  Each thread takes
// 16 / R butterflies.
template <int R, bool INV, int LAYOUT>
__device__ __forceinline__ void stockham_stage(float2 *s, int lm, int lq, int stride, int ls, const float2 *tw,
                                               int lt)
{
    constexpr int PER = 16 / R;
    constexpr int LR = R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1));
    const int T = blockDim.x;
    const int M = 1 << lm, nseq = 1 << lq;
    const int lspan = lm - LR, span = 1 << lspan;   // butterflies per sequence
    float2 v[16];
    int jj[PER], qq[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int w = threadIdx.x + u * T;
        int q, j;
        if (LAYOUT == kLayoutCols) {
            q = w & (nseq - 1);   // neighbouring threads: neighbouring columns
            j = w >> lq;
        } else {
            j = w & (span - 1);
            q = w >> lspan;
        }
        jj[u] = j;
        qq[u] = q;
        const bool live = q < nseq && j < span;
#pragma unroll
        for (int r = 0; r < R; ++r)
            v[u * R + r] = live ? s[saddr<LAYOUT>(j + (r << lspan), q, M, stride)] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = jj[u], q = qq[u];
        if (q >= nseq || j >= span) continue;
        const int k = j & ((1 << ls) - 1);
        if (ls > 0) {
            float2 w[R];
            stage_twiddles<R>(w, tw, (k << (lm - ls - LR)) << lt, INV);   // e^{-2 pi i k / (Ns R)}
#pragma unroll
            for (int r = 1; r < R; ++r) v[u * R + r] = cmul(v[u * R + r], w[r]);
        }
        dft_regs<R, INV>(&v[u * R]);
        const int base = ((j >> ls) << (ls + LR)) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) s[saddr<LAYOUT>(base + (r << ls), q, M, stride)] = v[u * R + r];
    }
    __syncthreads();
}

// nseq transforms of length M (power of two) in shared memory; tw[k * tws] = e^{-2 pi i k / M}.
template <bool INV, int LAYOUT>
__device__ void smem_fft(float2 *s, int M, int nseq, int stride, const float2 *tw, int tws)
{
    const int lm = ilog2(M), lq = ilog2(nseq), lt = ilog2(tws);
    int ls = 0;
    while (ls + 4 <= lm) {
        stockham_stage<16, INV, LAYOUT>(s, lm, lq, stride, ls, tw, lt);
        ls += 4;
    }
    const int rest = lm - ls;
    if (rest == 3) stockham_stage<8, INV, LAYOUT>(s, lm, lq, stride, ls, tw, lt);
    else if (rest == 2) stockham_stage<4, INV, LAYOUT>(s, lm, lq, stride, ls, tw, lt);
    else if (rest == 1) stockham_stage<2, INV, LAYOUT>(s, lm, lq, stride, ls, tw, lt);
}

// The same stages with the geometry known at compile time (LM = log2 M,
// LQ = log2 nseq, LS = log2 Ns; the CTA has exactly M nseq / 16 threads, so
// every butterfly slot is live): the index arithmetic folds into shifts and
// immediate offsets.  Rows layout: for spans of at least 32 values the padding
// term of an element r spans on is (j >> 5) + r (span / 32).
template <int LAYOUT, int M, int STRIDE>
__device__ __forceinline__ int saddr_ct(int e, int q)
{
    if (LAYOUT == kLayoutRows) return q * (M + (M >> 5)) + e + (e >> 5);
    return e * STRIDE + q;
}

template <int R, bool INV, int LAYOUT, int LM, int LQ, int LS>
__device__ __forceinline__ void stockham_stage_ct(float2 *s, const float2 *tw)
{
    constexpr int PER = 16 / R;
    constexpr int LR = R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1));
    constexpr int M = 1 << LM, NSEQ = 1 << LQ, T = (M << LQ) / 16;
    constexpr int LSPAN = LM - LR, SPAN = 1 << LSPAN;
    constexpr int STRIDE = NSEQ + 1;
    float2 v[16];
    int jj[PER], qq[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int w = threadIdx.x + u * T;
        int q, j;
        if (LAYOUT == kLayoutCols) {
            q = w & (NSEQ - 1);
            j = w >> LQ;
        } else {
            j = w & (SPAN - 1);
            q = w >> LSPAN;
        }
        jj[u] = j;
        qq[u] = q;
        if (LAYOUT == kLayoutRows && LSPAN >= 5) {
            const int base = q * (M + (M >> 5)) + j + (j >> 5);
#pragma unroll
            for (int r = 0; r < R; ++r) v[u * R + r] = s[base + r * (SPAN + (SPAN >> 5))];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[u * R + r] = s[saddr_ct<LAYOUT, M, STRIDE>(j + (r << LSPAN), q)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = jj[u], q = qq[u];
        const int k = j & ((1 << LS) - 1);
        if (LS > 0) {
            float2 w[R];
            stage_twiddles<R>(w, tw, k << (LM - LS - LR), INV);   // e^{-2 pi i k / (Ns R)}
#pragma unroll
            for (int r = 1; r < R; ++r) v[u * R + r] = cmul(v[u * R + r], w[r]);
        }
        dft_regs<R, INV>(&v[u * R]);
        const int base = ((j >> LS) << (LS + LR)) + k;
        if (LAYOUT == kLayoutRows && LS >= 5) {
            const int b0 = q * (M + (M >> 5)) + base + (base >> 5);
#pragma unroll
            for (int r = 0; r < R; ++r) s[b0 + r * ((1 << LS) + (1 << (LS - 5)))] = v[u * R + r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) s[saddr_ct<LAYOUT, M, STRIDE>(base + (r << LS), q)] = v[u * R + r];
        }
    }
    __syncthreads();
}

template <bool INV, int LAYOUT, int LM, int LQ, int LS>
__device__ __forceinline__ void smem_fft_ct(float2 *s, const float2 *tw)
{
    if constexpr (LS + 4 <= LM) {
        stockham_stage_ct<16, INV, LAYOUT, LM, LQ, LS>(s, tw);
        smem_fft_ct<INV, LAYOUT, LM, LQ, LS + 4>(s, tw);
    } else if constexpr (LM - LS == 3) {
        stockham_stage_ct<8, INV, LAYOUT, LM, LQ, LS>(s, tw);
    } else if constexpr (LM - LS == 2) {
        stockham_stage_ct<4, INV, LAYOUT, LM, LQ, LS>(s, tw);
    } else if constexpr (LM - LS == 1) {
        stockham_stage_ct<2, INV, LAYOUT, LM, LQ, LS>(s, tw);
    }
}

// Row transforms of the sizes the display-size planes use, at compile time; the rest at run time
// (tw[k] = e^{-2 pi i k / M}).
template <bool INV>
__device__ __forceinline__ void rows_fft(float2 *s, int M, int nseq, const float2 *tw)
{
    const int T = blockDim.x;   // the compile-time forms assume exactly M nseq / 16 threads
    if (M == 8192 && nseq == 1 && T == 512) smem_fft_ct<INV, kLayoutRows, 13, 0, 0>(s, tw);
    else if (M == 16384 && nseq == 1 && T == 1024) smem_fft_ct<INV, kLayoutRows, 14, 0, 0>(s, tw);
    else if (M == 4096 && nseq == 1 && T == 256) smem_fft_ct<INV, kLayoutRows, 12, 0, 0>(s, tw);
    else if (M == 2048 && nseq == 2 && T == 256) smem_fft_ct<INV, kLayoutRows, 11, 1, 0>(s, tw);
    else smem_fft<INV, kLayoutRows>(s, M, nseq, 0, tw, 1);
}

// Column transforms (M points over nseq columns, stride nseq + 1), likewise.
template <bool INV>
__device__ __forceinline__ void cols_fft(float2 *s, int M, int nseq, int stride, const float2 *tw)
{
    const bool t256 = blockDim.x == 256, s1 = stride == nseq + 1;
    if (M == 128 && nseq == 32 && t256 && s1) smem_fft_ct<INV, kLayoutCols, 7, 5, 0>(s, tw);
    else if (M == 64 && nseq == 64 && t256 && s1) smem_fft_ct<INV, kLayoutCols, 6, 6, 0>(s, tw);
    else if (M == 32 && nseq == 128 && t256 && s1) smem_fft_ct<INV, kLayoutCols, 5, 7, 0>(s, tw);
    else smem_fft<INV, kLayoutCols>(s, M, nseq, stride, tw, 1);
}

enum { kRowExpand = 0, kRowInPlace = 1, kRowCrop = 2, kRowPadRows = 3 };

// Transforms of compile-time length whose first stage reads its values from,
// and whose last stage writes them to, an IO object instead of shared memory
// (the element a thread holds in either is j + r M / R, so a warp's accesses to
// global memory stay contiguous: rows j, columns q): shared memory carries only
// the values between stages.  IO supplies load(q, e) and store(q, e, v) for
// sequence q, element e.
template <int R, bool INV, int LAYOUT, int LM, int LQ, int LS, bool FIRST, bool LAST, class IO>
__device__ __forceinline__ void stockham_stage_io(float2 *s, const float2 *tw, const IO &io)
{
    constexpr int PER = 16 / R;
    constexpr int LR = R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1));
    constexpr int M = 1 << LM, NSEQ = 1 << LQ, T = (M << LQ) / 16;
    constexpr int LSPAN = LM - LR, SPAN = 1 << LSPAN;
    constexpr int STRIDE = NSEQ + 1;   // columns layout
    static_assert(LAYOUT != kLayoutRows || LSPAN >= 5, "row spans of at least 32 values");
    static_assert(LAYOUT != kLayoutStrip || (LSPAN >= 4 && (LS == 0 ? R == 16 : LS >= 4)),
                  "strip spans of at least 16 values, radix 16 from the start");
    float2 v[16];
    int jj[PER], qq[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int w = threadIdx.x + u * T;
        int q, j;
        if (LAYOUT != kLayoutRows) {
            q = w & (NSEQ - 1);
            j = w >> LQ;
        } else {
            j = w & (SPAN - 1);
            q = w >> LSPAN;
        }
        jj[u] = j;
        qq[u] = q;
        if (FIRST) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[u * R + r] = io.load(q, j + r * SPAN);
        } else if (LAYOUT == kLayoutStrip) {   // SPAN is a multiple of 16: the gaps advance by SPAN / 16 per r
            const int b0 = strip_addr<LQ>(j, q);
#pragma unroll
            for (int r = 0; r < R; ++r) v[u * R + r] = s[b0 + r * ((SPAN + (SPAN >> 4)) << LQ)];
        } else if (LAYOUT == kLayoutCols) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[u * R + r] = s[(j + r * SPAN) * STRIDE + q];
        } else {
            const int base = q * (M + (M >> 5)) + j + (j >> 5);
#pragma unroll
            for (int r = 0; r < R; ++r) v[u * R + r] = s[base + r * (SPAN + (SPAN >> 5))];
        }
    }
    if (!FIRST) __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = jj[u], q = qq[u];
        const int k = j & ((1 << LS) - 1);
        if (LS > 0) {
            float2 w[R];
            stage_twiddles<R>(w, tw, k << (LM - LS - LR), INV);
#pragma unroll
            for (int r = 1; r < R; ++r) v[u * R + r] = cmul(v[u * R + r], w[r]);
        }
        dft_regs<R, INV>(&v[u * R]);
        const int base = ((j >> LS) << (LS + LR)) + k;
        if (LAST) {   // LS + LR = LM: base = j, the outputs are j + r 2^LS = j + r SPAN
#pragma unroll
            for (int r = 0; r < R; ++r) io.store(q, j + r * SPAN, v[u * R + r]);
        } else if (LAYOUT == kLayoutStrip) {   // LS = 0 (base = 16 j, r < 16) or a multiple of 4
            const int b0 = strip_addr<LQ>(base, q);
            constexpr int step = LS == 0 ? (1 << LQ) : (((1 << LS) + (1 << (LS >= 4 ? LS - 4 : 0))) << LQ);
#pragma unroll
            for (int r = 0; r < R; ++r) s[b0 + r * step] = v[u * R + r];
        } else if (LAYOUT == kLayoutCols) {
#pragma unroll
            for (int r = 0; r < R; ++r) s[(base + (r << LS)) * STRIDE + q] = v[u * R + r];
        } else if (LS >= 5) {
            const int b0 = q * (M + (M >> 5)) + base + (base >> 5);
#pragma unroll
            for (int r = 0; r < R; ++r) s[b0 + r * ((1 << LS) + (1 << (LS >= 5 ? LS - 5 : 0)))] = v[u * R + r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int e = base + (r << LS);
                s[q * (M + (M >> 5)) + e + (e >> 5)] = v[u * R + r];
            }
        }
    }
    if (!LAST) __syncthreads();
}

// IN_IO: the first stage reads io (else shared memory, as left by the caller); OUT_IO: the last stage writes io
// (else shared memory, natural order).  A last stage writing io does not end with a barrier.
template <bool INV, int LAYOUT, int LM, int LQ, bool IN_IO, bool OUT_IO, int LS, class IO>
__device__ __forceinline__ void fft_io(float2 *s, const float2 *tw, const IO &io)
{
    constexpr bool F = IN_IO && LS == 0;
    if constexpr (LS + 4 < LM) {
        stockham_stage_io<16, INV, LAYOUT, LM, LQ, LS, F, false>(s, tw, io);
        fft_io<INV, LAYOUT, LM, LQ, IN_IO, OUT_IO, LS + 4>(s, tw, io);
    } else if constexpr (LS + 4 == LM) {
        stockham_stage_io<16, INV, LAYOUT, LM, LQ, LS, F, OUT_IO>(s, tw, io);
    } else if constexpr (LM - LS == 3) {
        stockham_stage_io<8, INV, LAYOUT, LM, LQ, LS, F, OUT_IO>(s, tw, io);
    } else if constexpr (LM - LS == 2) {
        stockham_stage_io<4, INV, LAYOUT, LM, LQ, LS, F, OUT_IO>(s, tw, io);
    } else if constexpr (LM - LS == 1) {
        stockham_stage_io<2, INV, LAYOUT, LM, LQ, LS, F, OUT_IO>(s, tw, io);
    }
}

template <bool INV, int LM, int LQ, int LS, class IO>
__device__ __forceinline__ void rows_fft_io(float2 *s, const float2 *tw, const IO &io)
{
    fft_io<INV, kLayoutRows, LM, LQ, true, true, LS>(s, tw, io);
}

// Global sources and destinations of the row kernels (row q of the CTA is y0 + q).
template <int MODE>
struct RowIO {
    const float *in;
    float2 *pad;
    float *out;
    long long plane;
    int y0, rows, W, Lx;
    __device__ __forceinline__ float2 load(int q, int x) const
    {
        const int y = y0 + q;
        if (y >= rows || ((MODE == kRowExpand || MODE == kRowPadRows) && x >= W)) return make_float2(0.0f, 0.0f);
        if (MODE == kRowExpand) return make_float2(in[(long long)y * W + x], in[plane + (long long)y * W + x]);
        return pad[(long long)y * Lx + x];
    }
    __device__ __forceinline__ void store(int q, int x, float2 v) const
    {
        const int y = y0 + q;
        if (y >= rows) return;
        if (MODE == kRowCrop) {
            if (x < W) {
                out[(long long)y * W + x] = v.x;
                out[plane + (long long)y * W + x] = v.y;
            }
        } else {
            pad[(long long)y * Lx + x] = v;
        }
    }
};

// The row kernel's transform when its length has a compile-time form: true if done.
template <int MODE>
__device__ __forceinline__ bool rows_fft_direct(float2 *s, int Lx, int nseq, const float2 *tw, const RowIO<MODE> &io)
{
    constexpr bool INV = MODE == kRowCrop;
    const int T = blockDim.x;
    if (Lx == 8192 && nseq == 1 && T == 512) rows_fft_io<INV, 13, 0, 0>(s, tw, io);
    else if (Lx == 16384 && nseq == 1 && T == 1024) rows_fft_io<INV, 14, 0, 0>(s, tw, io);
    else if (Lx == 4096 && nseq == 1 && T == 256) rows_fft_io<INV, 12, 0, 0>(s, tw, io);
    else if (Lx == 2048 && nseq == 2 && T == 256) rows_fft_io<INV, 11, 1, 0>(s, tw, io);
    else return false;
    return true;
}

// Row transforms: nseq rows of length Lx per CTA.
//   kRowExpand:  rows y < H from the input planes [2][H][W] (zeros beyond W), forward, into pad;
//   kRowPadRows: rows y < H of pad, columns < W (zeros beyond), forward, in place;
//   kRowInPlace: rows of pad, forward, in place (the chirp, all Ly rows);
//   kRowCrop:    rows y < H of pad, inverse, columns < W into the output planes.
template <int MODE>
__global__ void __launch_bounds__(1024) fft_rows_kernel(const float *__restrict__ in, float2 *__restrict__ pad, float *__restrict__ out,
                                int H, int W, int Lx, int rows, int nseq, const float2 *__restrict__ twx)
{
    extern __shared__ float2 sm[];
    const int y0 = blockIdx.x * nseq;
    const int T = blockDim.x;
    const long long plane = (long long)H * W;
    if (rows_fft_direct<MODE>(sm, Lx, nseq, twx, RowIO<MODE>{in, pad, out, plane, y0, rows, W, Lx})) return;
    for (int q = 0; q < nseq; ++q) {
        const int y = y0 + q;
        for (int x = threadIdx.x; x < Lx; x += T) {
            float2 *d = &sm[saddr<kLayoutRows>(x, q, Lx, 0)];
            const bool live = y < rows && (MODE == kRowInPlace || MODE == kRowCrop || x < W);
            if (!live) {
                *d = make_float2(0.0f, 0.0f);
            } else if (MODE == kRowExpand) {
                cp_async4(&d->x, in + (long long)y * W + x);
                cp_async4(&d->y, in + plane + (long long)y * W + x);
            } else {
                cp_async8(d, pad + (long long)y * Lx + x);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    rows_fft<MODE == kRowCrop>(sm, Lx, nseq, twx);
    for (int q = 0; q < nseq; ++q) {
        const int y = y0 + q;
        if (y >= rows) break;
        if (MODE == kRowCrop) {
            for (int x = threadIdx.x; x < W; x += T) {
                const float2 v = sm[saddr<kLayoutRows>(x, q, Lx, 0)];
                out[(long long)y * W + x] = v.x;
                out[plane + (long long)y * W + x] = v.y;
            }
        } else {
            for (int x = threadIdx.x; x < Lx; x += T) pad[(long long)y * Lx + x] = sm[saddr<kLayoutRows>(x, q, Lx, 0)];
        }
    }
}

// Column transform lengths with a compile-time form (length L over sw columns, 256 threads).
__host__ __device__ inline bool cols_ct(int L, int sw)
{
    return (L == 128 && sw == 32) || (L == 64 && sw == 64) || (L == 32 && sw == 128);
}

template <bool INV, bool IN_IO, bool OUT_IO, class IO>
__device__ __forceinline__ void cols_fft_direct(float2 *s, int L, int sw, const float2 *tw, const IO &io)
{
    if (L == 128 && sw == 32) fft_io<INV, kLayoutCols, 7, 5, IN_IO, OUT_IO, 0>(s, tw, io);
    else if (L == 64 && sw == 64) fft_io<INV, kLayoutCols, 6, 6, IN_IO, OUT_IO, 0>(s, tw, io);
    else fft_io<INV, kLayoutCols, 5, 7, IN_IO, OUT_IO, 0>(s, tw, io);
}

// Column pass A's global side: sequence q is column x0 + q, element a is row L2 a + b.
struct ColsAIO {
    float2 *pad;
    int Lx, L2, b, x0, nz_rows, keep_rows;
    __device__ __forceinline__ float2 load(int q, int a) const
    {
        const int row = L2 * a + b;
        return row < nz_rows ? pad[(long long)row * Lx + x0 + q] : make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ void store(int q, int a, float2 v) const
    {
        const int row = L2 * a + b;
        if (row < keep_rows) pad[(long long)row * Lx + x0 + q] = v;
    }
};

// Column pass B, forward: in, rows L2 c + b times the four-step twiddle; out, the product with the spectrum into
// shared memory (natural order) -- or, building the spectrum itself (spec == nullptr), straight to pad.
struct ColsBFwdIO {
    float2 *pad;
    const float2 *spec;
    float2 *s;
    const float2 *t4;
    int Lx, L2, c, x0, stride;
    __device__ __forceinline__ float2 load(int q, int b) const
    {
        return cmul(pad[(long long)(L2 * c + b) * Lx + x0 + q], t4[b]);
    }
    __device__ __forceinline__ void store(int q, int d, float2 v) const
    {
        const long long g = (long long)(L2 * c + d) * Lx + x0 + q;
        if (spec != nullptr) s[d * stride + q] = cmul(v, spec[g]);
        else pad[g] = v;
    }
};

// Column pass B, inverse: out, rows L2 c + b times the conjugate four-step twiddle.
struct ColsBInvIO {
    float2 *pad;
    const float2 *t4;
    int Lx, L2, c, x0;
    __device__ __forceinline__ float2 load(int, int) const { return make_float2(0.0f, 0.0f); }
    __device__ __forceinline__ void store(int q, int b, float2 v) const
    {
        const float2 t = t4[b];
        pad[(long long)(L2 * c + b) * Lx + x0 + q] = cmul(v, make_float2(t.x, -t.y));
    }
};

// Column pass A: for each b < L2 and strip of sw columns, L1-point transforms
// over the rows L2 a + b.  Forward: rows >= nz_rows are zero (not loaded), all
// outputs stored at rows L2 c + b.  Inverse: outputs a stored at rows L2 a + b
// only below keep_rows.  (All sizes powers of two.)
template <bool INV>
__global__ void __launch_bounds__(256, 4) fft_cols_a_kernel(float2 *__restrict__ pad, int Lx, int L1, int L2, int sw, int nz_rows,
                                  int keep_rows, const float2 *__restrict__ twy)
{
    extern __shared__ float2 sm[];
    const int lsw = ilog2(sw);
    const int lstrips = ilog2(Lx) - lsw;
    const int b = blockIdx.x >> lstrips, x0 = (blockIdx.x & ((1 << lstrips) - 1)) << lsw;
    const int stride = sw + 1;
    const int n = L1 << lsw;
    float2 *tw = sm + L1 * stride;   // e^{-2 pi i k / L1} = twy[k L2], k < L1, in shared memory
    if (cols_ct(L1, sw) && blockDim.x == 256) {   // first and last stages on global memory
        for (int k = threadIdx.x; k < L1; k += blockDim.x) tw[k] = twy[k * L2];
        __syncthreads();
        cols_fft_direct<INV, true, true>(sm, L1, sw, tw, ColsAIO{pad, Lx, L2, b, x0, nz_rows, keep_rows});
        return;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int a = i >> lsw, c = i & (sw - 1);
        const int row = L2 * a + b;
        if (row < nz_rows) cp_async8(&sm[a * stride + c], pad + (long long)row * Lx + x0 + c);
        else sm[a * stride + c] = make_float2(0.0f, 0.0f);
    }
    for (int k = threadIdx.x; k < L1; k += blockDim.x) tw[k] = twy[k * L2];
    cp_async_wait_all();
    __syncthreads();
    cols_fft<INV>(sm, L1, sw, stride, tw);
#pragma unroll 4
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int a = i >> lsw, c = i & (sw - 1);
        const int row = L2 * a + b;
        if (row < keep_rows) pad[(long long)row * Lx + x0 + c] = sm[a * stride + c];
    }
}

// Column pass B over the rows L2 c + b (b < L2) of each strip, with the
// four-step twiddle e^{-2 pi i c b / Ly}.  spec == nullptr: forward only, the
// result (the spectrum in scrambled order) stored.  Otherwise: forward,
// product with spec (same order, its tile loaded together with the data),
// inverse, conjugate twiddle: the middle of the convolution in one pass.
__global__ void __launch_bounds__(256, 4) fft_cols_b_kernel(float2 *__restrict__ pad, const float2 *__restrict__ spec, int Lx, int L1, int L2,
                                  int sw, const float2 *__restrict__ twy)
{
    extern __shared__ float2 sm[];
    const int lsw = ilog2(sw);
    const int lstrips = ilog2(Lx) - lsw;
    const int c = blockIdx.x >> lstrips, x0 = (blockIdx.x & ((1 << lstrips) - 1)) << lsw;
    const int stride = sw + 1;
    const int n = L2 << lsw;
    if (cols_ct(L2, sw) && blockDim.x == 256) {   // first and last stages on global memory: one tile, no spectrum tile
        float2 *tw = sm + L2 * stride, *t4 = tw + L2;
        for (int k = threadIdx.x; k < L2; k += blockDim.x) {
            tw[k] = twy[k * L1];
            t4[k] = twy[c * k];
        }
        __syncthreads();
        cols_fft_direct<false, true, true>(sm, L2, sw, tw, ColsBFwdIO{pad, spec, sm, t4, Lx, L2, c, x0, stride});
        if (spec == nullptr) return;
        __syncthreads();   // the products are in shared memory
        cols_fft_direct<true, false, true>(sm, L2, sw, tw, ColsBInvIO{pad, t4, Lx, L2, c, x0});
        return;
    }
    float2 *sp = sm + L2 * stride;   // the spectrum's tile
    // in shared memory: e^{-2 pi i k / L2} = twy[k L1] and the four-step twiddles e^{-2 pi i c b / Ly} = twy[c b]
    float2 *tw = sm + (spec != nullptr ? 2 : 1) * L2 * stride, *t4 = tw + L2;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int b = i >> lsw, q = i & (sw - 1);
        const long long g = (long long)(L2 * c + b) * Lx + x0 + q;
        cp_async8(&sm[b * stride + q], pad + g);
        if (spec != nullptr) cp_async8(&sp[b * stride + q], spec + g);
    }
    for (int k = threadIdx.x; k < L2; k += blockDim.x) {
        tw[k] = twy[k * L1];
        t4[k] = twy[c * k];
    }
    cp_async_wait_all();
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {   // the four-step twiddle
        const int b = i >> lsw, q = i & (sw - 1);
        sm[b * stride + q] = cmul(sm[b * stride + q], t4[b]);
    }
    __syncthreads();
    cols_fft<false>(sm, L2, sw, stride, tw);
    if (spec == nullptr) {
#pragma unroll 4
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int d = i >> lsw, q = i & (sw - 1);
            pad[(long long)(L2 * c + d) * Lx + x0 + q] = sm[d * stride + q];
        }
        return;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int d = i >> lsw, q = i & (sw - 1);
        sm[d * stride + q] = cmul(sm[d * stride + q], sp[d * stride + q]);
    }
    __syncthreads();
    cols_fft<true>(sm, L2, sw, stride, tw);
#pragma unroll 4
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int b = i >> lsw, q = i & (sw - 1);
        const float2 t = t4[b];
        pad[(long long)(L2 * c + b) * Lx + x0 + q] = cmul(sm[b * stride + q], make_float2(t.x, -t.y));
    }
}

// The fused column pass's global side: sequence q is column x0 + q, element e is row e (natural order).  Loads
// read the rows below nz_rows (the rest are zero).  Stores: with spec, the product with the spectrum into shared
// memory (the input of the inverse transform); without, the rows below keep_rows into pad.
template <int LQ>
struct StripIO {
    float2 *pad;
    const float2 *spec;
    float2 *s;
    int Lx, x0, nz_rows, keep_rows;
    __device__ __forceinline__ float2 load(int q, int e) const
    {
        return e < nz_rows ? pad[e * Lx + x0 + q] : make_float2(0.0f, 0.0f);   // offsets below 2^27
    }
    __device__ __forceinline__ void store(int q, int e, float2 v) const
    {
        const int g = e * Lx + x0 + q;
        if (spec != nullptr) s[strip_addr<LQ>(e, q)] = cmul(v, spec[g]);
        else if (e < keep_rows) pad[g] = v;
    }
};

// The columns in one pass, where a whole column fits in shared memory: per strip of 2^LQ columns, the forward
// Ly-point transform (Ly = 2^LM) of the rows below nz_rows, the product with the spectrum (natural order) as the
// last forward stage stores, the inverse transform, and the rows below keep_rows stored -- the plane crosses
// HBM once each way instead of three times.  spec == nullptr: the forward transform alone, every row below
// keep_rows stored (the chirp's spectrum).  2^(LM + LQ - 4) threads, each holding 16 values per stage.
template <int LM, int LQ>
__global__ void __launch_bounds__(1 << (LM + LQ - 4), 1024 >> (LM + LQ - 4))
    fft_cols_full_kernel(float2 *__restrict__ pad, const float2 *__restrict__ spec, int Lx, int nz_rows,
                         int keep_rows, const float2 *__restrict__ twy)
{
    extern __shared__ float2 sm[];
    constexpr int T = 1 << (LM + LQ - 4);
    const int x0 = blockIdx.x << LQ;
    const StripIO<LQ> io{pad, nullptr, sm, Lx, x0, nz_rows, keep_rows};
    if (spec == nullptr) {
        fft_io<false, kLayoutStrip, LM, LQ, true, true, 0>(sm, twy, io);
        return;
    }
    fft_io<false, kLayoutStrip, LM, LQ, true, false, 0>(sm, twy, io);   // natural order in shared memory
#pragma unroll 4
    for (int i = threadIdx.x; i < (1 << (LM + LQ)); i += T) {
        const int q = i & ((1 << LQ) - 1), e = i >> LQ;
        float2 &v = sm[strip_addr<LQ>(e, q)];
        v = cmul(v, spec[e * Lx + x0 + q]);
    }
    __syncthreads();
    fft_io<true, kLayoutStrip, LM, LQ, false, true, 0>(sm, twy, io);
}

// The chirp on the Ly x Lx grid, h(k, l) = pre exp(i 2 pi C (k'^2 + l'^2) / 2^64) (k' = k or k - Ly, the signed
// offset; likewise l'), as the product of its separable factors: a(l) = exp(i 2 pi C l'^2 / 2^64) for the thread's
// kChirpCols columns, computed once, and pre a(k) for each of the block's kChirpRows rows -- a complex product per
// entry in place of a sine and cosine (the turns of the two factors add to the joint turn within 2^-31; each factor
// is an accurate single-precision sine and cosine, the product adds about two units of rounding).
constexpr int kChirpCols = 8, kChirpRows = 64;

__device__ __forceinline__ float2 chirp_factor(unsigned long long C, int k, int L)
{
    const long long kk = k <= L / 2 ? k : k - L;
    const uint32_t t = (uint32_t)((C * (unsigned long long)(kk * kk)) >> 32);
    float s, c;
    sincospif((float)(int)t * (1.0f / 2147483648.0f), &s, &c);
    return make_float2(c, s);
}

__global__ void chirp_grid_kernel(float2 *__restrict__ h, int Ly, int Lx, unsigned long long C, float pre_re,
                                  float pre_im)
{
    const int l0 = blockIdx.x * blockDim.x * kChirpCols + threadIdx.x;
    float2 a[kChirpCols];
#pragma unroll
    for (int j = 0; j < kChirpCols; ++j) {
        const int l = l0 + j * (int)blockDim.x;
        a[j] = l < Lx ? chirp_factor(C, l, Lx) : make_float2(0.0f, 0.0f);
    }
    const int k1 = min(Ly, (int)(blockIdx.y + 1) * kChirpRows);
    for (int k = blockIdx.y * kChirpRows; k < k1; ++k) {
        const float2 b = cmul(chirp_factor(C, k, Ly), make_float2(pre_re, pre_im));
#pragma unroll
        for (int j = 0; j < kChirpCols; ++j) {
            const int l = l0 + j * (int)blockDim.x;
            if (l < Lx) h[(long long)k * Lx + l] = cmul(b, a[j]);
        }
    }
}

int threads_for(int work)
{
    int t = work / 16;   // 16 values per thread per stage
    if (t < 32) t = 32;
    if (t > 1024) t = 1024;
    return t;
}

}  // namespace

FftGrid fft_grid(int H, int W)
{
    auto p2 = [](int n) {
        int l = 1;
        while (l < n) l *= 2;
        return l;
    };
    FftGrid g;
    g.Ly = p2(2 * H - 1);
    g.Lx = p2(2 * W - 1);
    int lg = 0;
    while ((1 << lg) < g.Ly) ++lg;
    g.L1 = 1 << ((lg + 1) / 2);
    g.L2 = g.Ly / g.L1;
    g.ok = g.Lx <= kFftMaxLen && g.Ly <= kFftMaxLen;
    return g;
}

static int rows_per_cta(int Lx)
{
    int n = 4096 / Lx;   // at least 256 threads for short rows
    return n < 1 ? 1 : n;
}

static int strip_width(int Lx, int L)
{
    int sw = 4096 / (L > 0 ? L : 1);   // L x sw values per tile: 32 KB
    if (sw < 32) sw = 32;
    if (sw > Lx) sw = Lx;
    return sw;
}

static size_t rows_smem(int Lx, int nseq)
{
    return (size_t)nseq * (Lx + (Lx >> 5)) * sizeof(float2);
}

static cudaError_t configure_rows(size_t bytes)
{
    static size_t done = 0;
    if (bytes <= 48 * 1024 || bytes <= done) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (auto fn : {(const void *)fft_rows_kernel<kRowExpand>, (const void *)fft_rows_kernel<kRowInPlace>,
                    (const void *)fft_rows_kernel<kRowCrop>, (const void *)fft_rows_kernel<kRowPadRows>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done = bytes;
    return e;
}

// Column passes: the data tile(s) of L x (sw + 1) values and the twiddle tables in shared memory.
static size_t cols_a_smem(const FftGrid &g, int swa)
{
    return ((size_t)g.L1 * (swa + 1) + g.L1) * sizeof(float2);
}

static size_t cols_b_smem(const FftGrid &g, int swb, bool product)
{
    const int tiles = product && !cols_ct(g.L2, swb) ? 2 : 1;   // the compile-time form reads the spectrum directly
    return ((size_t)tiles * g.L2 * (swb + 1) + 2 * g.L2) * sizeof(float2);
}

static cudaError_t configure_cols(const FftGrid &g)
{
    static size_t done_a = 0, done_b = 0;
    const size_t a = cols_a_smem(g, strip_width(g.Lx, g.L1)), b = cols_b_smem(g, strip_width(g.Lx, g.L2), true);
    cudaError_t e = cudaSuccess;
    if (a > 48 * 1024 && a > done_a) {
        for (auto fn : {(const void *)fft_cols_a_kernel<false>, (const void *)fft_cols_a_kernel<true>})
            if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a);
        if (e == cudaSuccess) done_a = a;
    }
    if (e == cudaSuccess && b > 48 * 1024 && b > done_b) {   // the product pass holds two tiles
        e = cudaFuncSetAttribute(fft_cols_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
        if (e == cudaSuccess) done_b = b;
    }
    return e;
}

// The fused column pass's strip width (log2) for the grid, or -1 where the four-step passes serve: columns of
// 256 .. 2048 points, strips of 8 or more columns (64-byte row segments); 512 or 1024 threads per strip.
static int cols_full_lq(const FftGrid &g)
{
    int lq = -1;
    switch (g.Ly) {
    case 2048: lq = 3; break;   // 1024 threads
    case 1024: lq = 3; break;   // 512 threads
    case 512: lq = 4; break;    // 512 threads
    case 256: lq = 5; break;    // 512 threads
    default: break;
    }
    return lq >= 0 && g.Lx >= (1 << lq) ? lq : -1;
}

template <int LM, int LQ>
static cudaError_t launch_cols_full_as(const FftGrid &g, float2 *pad, const float2 *spec, int nz_rows, int keep_rows,
                                       const float2 *twy, cudaStream_t s)
{
    constexpr int M = 1 << LM;
    constexpr size_t bytes = (size_t)((M + M / 16) << LQ) * sizeof(float2);
    static PerDeviceOnce configured;
    const cudaError_t e = configured.run([&] {
        return cudaFuncSetAttribute(fft_cols_full_kernel<LM, LQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)bytes);
    });
    if (e != cudaSuccess) return e;
    fft_cols_full_kernel<LM, LQ><<<g.Lx >> LQ, 1 << (LM + LQ - 4), bytes, s>>>(pad, spec, g.Lx, nz_rows, keep_rows, twy);
    return cudaGetLastError();
}

static cudaError_t launch_cols_full(const FftGrid &g, float2 *pad, const float2 *spec, int nz_rows, int keep_rows,
                                    const float2 *twy, cudaStream_t s)
{
    const int lq = cols_full_lq(g);
#define CGH_COLS_FULL(LMV, LQV) \
    if (g.Ly == (1 << LMV) && lq == LQV) return launch_cols_full_as<LMV, LQV>(g, pad, spec, nz_rows, keep_rows, twy, s);
    CGH_COLS_FULL(11, 3)
    CGH_COLS_FULL(10, 3)
    CGH_COLS_FULL(9, 4)
    CGH_COLS_FULL(8, 5)
#undef CGH_COLS_FULL
    return cudaErrorInvalidValue;
}

cudaError_t launch_fft_chirp_spectrum(const FftGrid &g, float2 *spec, unsigned long long C, double pre_re,
                                      double pre_im, const float2 *twx, const float2 *twy, cudaStream_t s)
{
    chirp_grid_kernel<<<dim3((g.Lx + 256 * kChirpCols - 1) / (256 * kChirpCols), (g.Ly + kChirpRows - 1) / kChirpRows),
                        256, 0, s>>>(spec, g.Ly, g.Lx, C, (float)pre_re, (float)pre_im);
    const int nseq = rows_per_cta(g.Lx);
    const size_t rs = rows_smem(g.Lx, nseq);
    cudaError_t e = configure_rows(rs);
    if (e != cudaSuccess) return e;
    fft_rows_kernel<kRowInPlace><<<(g.Ly + nseq - 1) / nseq, threads_for(nseq * g.Lx), rs, s>>>(
        nullptr, spec, nullptr, 0, 0, g.Lx, g.Ly, nseq, twx);
    if (cols_full_lq(g) >= 0) return launch_cols_full(g, spec, nullptr, g.Ly, g.Ly, twy, s);
    const int swa = strip_width(g.Lx, g.L1), swb = strip_width(g.Lx, g.L2);
    e = configure_cols(g);
    if (e != cudaSuccess) return e;
    fft_cols_a_kernel<false><<<g.L2 * (g.Lx / swa), threads_for(g.L1 * swa), cols_a_smem(g, swa), s>>>(
        spec, g.Lx, g.L1, g.L2, swa, g.Ly, g.Ly, twy);
    fft_cols_b_kernel<<<g.L1 * (g.Lx / swb), threads_for(g.L2 * swb), cols_b_smem(g, swb, false), s>>>(
        spec, nullptr, g.Lx, g.L1, g.L2, swb, twy);
    return cudaGetLastError();
}

cudaError_t launch_fft_convolve(const FftGrid &g, const float *in, int H, int W, float2 *pad, const float2 *spec,
                                const float2 *twx, const float2 *twy, float *out, cudaStream_t s)
{
    const int nseq = rows_per_cta(g.Lx);
    const size_t rs = rows_smem(g.Lx, nseq);
    cudaError_t e = configure_rows(rs);
    if (e != cudaSuccess) return e;
    if (in != nullptr)
        fft_rows_kernel<kRowExpand><<<(H + nseq - 1) / nseq, threads_for(nseq * g.Lx), rs, s>>>(in, pad, nullptr, H, W,
                                                                                             g.Lx, H, nseq, twx);
    else
        fft_rows_kernel<kRowPadRows><<<(H + nseq - 1) / nseq, threads_for(nseq * g.Lx), rs, s>>>(nullptr, pad, nullptr,
                                                                                              H, W, g.Lx, H, nseq, twx);
    if (cols_full_lq(g) >= 0) {
        e = launch_cols_full(g, pad, spec, H, H, twy, s);
        if (e != cudaSuccess) return e;
        fft_rows_kernel<kRowCrop><<<(H + nseq - 1) / nseq, threads_for(nseq * g.Lx), rs, s>>>(nullptr, pad, out, H, W,
                                                                                           g.Lx, H, nseq, twx);
        return cudaGetLastError();
    }
    const int swa = strip_width(g.Lx, g.L1), swb = strip_width(g.Lx, g.L2);
    const size_t sa = cols_a_smem(g, swa), sb = cols_b_smem(g, swb, true);
    e = configure_cols(g);
    if (e != cudaSuccess) return e;
    fft_cols_a_kernel<false><<<g.L2 * (g.Lx / swa), threads_for(g.L1 * swa), sa, s>>>(pad, g.Lx, g.L1, g.L2, swa, H,
                                                                                     g.Ly, twy);
    fft_cols_b_kernel<<<g.L1 * (g.Lx / swb), threads_for(g.L2 * swb), sb, s>>>(pad, spec, g.Lx, g.L1, g.L2, swb, twy);
    fft_cols_a_kernel<true><<<g.L2 * (g.Lx / swa), threads_for(g.L1 * swa), sa, s>>>(pad, g.Lx, g.L1, g.L2, swa, g.Ly,
                                                                                    H, twy);
    fft_rows_kernel<kRowCrop><<<(H + nseq - 1) / nseq, threads_for(nseq * g.Lx), rs, s>>>(nullptr, pad, out, H, W,
                                                                                       g.Lx, H, nseq, twx);
    return cudaGetLastError();
}

}  // namespace cgh
