/*
 * wv_oracle.c -- TEST INFRASTRUCTURE, not part of the decoder library.
 *
 * Plain, slow reference lifting transforms used only by the tests, the smoke
 * check and the benchmark's CPU-baseline leg (the lines of a 2D level may be
 * shared out among host threads with OpenMP; the arithmetic of a line is the
 * same).  Shares no code with the CUDA library.
 *
 * Method (Groth et al., "Wavelet-Based Fast Decoding of 360 deg Videos"):
 *   Sec. 3.1, Eq. 1: frame-wise 2D fast wavelet transform, l levels, with the
 *     CDF 9/7 wavelet (the irreversible JPEG2000 wavelet).
 *   Sec. 2.2: the LeGall-Tabatabai 5/3 wavelet, JPEG2000's reversible integer
 *     wavelet, named as the lossless alternative.
 *
 * Readings where the paper is silent:
 *   - lifting factorisation of CDF 9/7 by Daubechies & Sweldens with constants
 *     alpha, beta, gamma, delta and K; low band scaled by 1/K, high band by K
 *     (analysis low-pass DC gain 1, high-pass Nyquist gain 2, JPEG2000 style);
 *   - 5/3: d[n] = x[2n+1] - floor((x[2n]+x[2n+2])/2),
 *          s[n] = x[2n]   + floor((d[n-1]+d[n]+2)/4);
 *   - whole-sample symmetric extension at both ends of every line;
 *   - 2D analysis per level: columns (vertical) then rows (horizontal);
 *     synthesis in the reverse order; Mallat layout in place, level 1 finest.
 * Frame sides must be divisible by 2^levels.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double ALPHA = -1.586134342059924;
static const double BETA = -0.052980118572961;
static const double GAMMA = 0.882911075530934;
static const double DELTA = 0.443506852043971;
static const double KAPPA = 1.230174104914001;

/* whole-sample symmetric extension: ... x2 x1 | x0 x1 ... x(n-1) | x(n-2) ... */
static long reflect(long i, long n)
{
    if (n == 1) return 0;
    for (;;) {
        if (i < 0) i = -i;
        else if (i >= n) i = 2 * (n - 1) - i;
        else return i;
    }
}

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b) != 0 && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

/* one lifting step on an interleaved line: y[i] += c*(y[i-1]+y[i+1]) for all
 * i of the given parity; the neighbours have the other parity and are read
 * through the symmetric extension. */
static void lift97(double *y, long n, int parity, double c)
{
    for (long i = parity; i < n; i += 2)
        y[i] += c * (y[reflect(i - 1, n)] + y[reflect(i + 1, n)]);
}

/* analysis of one line of n (even) samples: out[0..n/2) = s, out[n/2..n) = d */
static void fwd97_line(const double *x, double *out, long n, double *y)
{
    memcpy(y, x, (size_t)n * sizeof(double));
    lift97(y, n, 1, ALPHA);
    lift97(y, n, 0, BETA);
    lift97(y, n, 1, GAMMA);
    lift97(y, n, 0, DELTA);
    for (long k = 0; k < n / 2; ++k) {
        out[k] = y[2 * k] / KAPPA;
        out[n / 2 + k] = y[2 * k + 1] * KAPPA;
    }
}

/* synthesis of one line: in[0..n/2) = s, in[n/2..n) = d -> out samples */
static void inv97_line(const double *in, double *out, long n, double *y)
{
    for (long k = 0; k < n / 2; ++k) {
        y[2 * k] = in[k] * KAPPA;
        y[2 * k + 1] = in[n / 2 + k] / KAPPA;
    }
    lift97(y, n, 0, -DELTA);
    lift97(y, n, 1, -GAMMA);
    lift97(y, n, 0, -BETA);
    lift97(y, n, 1, -ALPHA);
    memcpy(out, y, (size_t)n * sizeof(double));
}

static void fwd53_line(const int64_t *x, int64_t *out, long n, int64_t *y)
{
    memcpy(y, x, (size_t)n * sizeof(int64_t));
    for (long i = 1; i < n; i += 2)
        y[i] -= floor_div(y[reflect(i - 1, n)] + y[reflect(i + 1, n)], 2);
    for (long i = 0; i < n; i += 2)
        y[i] += floor_div(y[reflect(i - 1, n)] + y[reflect(i + 1, n)] + 2, 4);
    for (long k = 0; k < n / 2; ++k) {
        out[k] = y[2 * k];
        out[n / 2 + k] = y[2 * k + 1];
    }
}

static void inv53_line(const int64_t *in, int64_t *out, long n, int64_t *y)
{
    for (long k = 0; k < n / 2; ++k) {
        y[2 * k] = in[k];
        y[2 * k + 1] = in[n / 2 + k];
    }
    for (long i = 0; i < n; i += 2)
        y[i] -= floor_div(y[reflect(i - 1, n)] + y[reflect(i + 1, n)] + 2, 4);
    for (long i = 1; i < n; i += 2)
        y[i] += floor_div(y[reflect(i - 1, n)] + y[reflect(i + 1, n)], 2);
    memcpy(out, y, (size_t)n * sizeof(int64_t));
}

/* ---- exported 1D entry points (used by the filter-bank pins) ---- */

void or_fwd97_1d(const double *x, double *out, long n)
{
    double *y = malloc((size_t)n * sizeof(double));
    fwd97_line(x, out, n, y);
    free(y);
}

void or_inv97_1d(const double *in, double *out, long n)
{
    double *y = malloc((size_t)n * sizeof(double));
    inv97_line(in, out, n, y);
    free(y);
}

void or_fwd53_1d(const int64_t *x, int64_t *out, long n)
{
    int64_t *y = malloc((size_t)n * sizeof(int64_t));
    fwd53_line(x, out, n, y);
    free(y);
}

void or_inv53_1d(const int64_t *in, int64_t *out, long n)
{
    int64_t *y = malloc((size_t)n * sizeof(int64_t));
    inv53_line(in, out, n, y);
    free(y);
}

/* ---- 2D multi-level transforms on a w x h row-major image, in place ----
 *
 * The rows (columns) of one level are independent lines; with OpenMP they are
 * shared out among the host's threads (or_set_threads), each thread using its
 * own line buffers.  The arithmetic per line is the same either way. */

static int thread_id(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

static int thread_count(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads the 2D transforms use (1 when built without OpenMP). */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return thread_count();
}

int or_fwd2d_97(double *img, long w, long h, int levels)
{
    long m = (w > h ? w : h);
    double *s = malloc((size_t)thread_count() * 3 * (size_t)m * sizeof(double));
    if (!s) return -1;
    for (int l = 0; l < levels; ++l) {
        long cw = w >> l, ch = h >> l;
#pragma omp parallel for schedule(static)
        for (long c = 0; c < cw; ++c) {           /* vertical analysis */
            double *a = s + (size_t)thread_id() * 3 * m, *b = a + m, *y = b + m;
            for (long r = 0; r < ch; ++r) a[r] = img[r * w + c];
            fwd97_line(a, b, ch, y);
            for (long r = 0; r < ch; ++r) img[r * w + c] = b[r];
        }
#pragma omp parallel for schedule(static)
        for (long r = 0; r < ch; ++r) {           /* horizontal analysis */
            double *b = s + (size_t)thread_id() * 3 * m, *y = b + m;
            fwd97_line(img + r * w, b, cw, y);
            memcpy(img + r * w, b, (size_t)cw * sizeof(double));
        }
    }
    free(s);
    return 0;
}

int or_inv2d_97(double *img, long w, long h, int levels)
{
    long m = (w > h ? w : h);
    double *s = malloc((size_t)thread_count() * 3 * (size_t)m * sizeof(double));
    if (!s) return -1;
    for (int l = levels - 1; l >= 0; --l) {
        long cw = w >> l, ch = h >> l;
#pragma omp parallel for schedule(static)
        for (long r = 0; r < ch; ++r) {           /* horizontal synthesis */
            double *b = s + (size_t)thread_id() * 3 * m, *y = b + m;
            inv97_line(img + r * w, b, cw, y);
            memcpy(img + r * w, b, (size_t)cw * sizeof(double));
        }
#pragma omp parallel for schedule(static)
        for (long c = 0; c < cw; ++c) {           /* vertical synthesis */
            double *a = s + (size_t)thread_id() * 3 * m, *b = a + m, *y = b + m;
            for (long r = 0; r < ch; ++r) a[r] = img[r * w + c];
            inv97_line(a, b, ch, y);
            for (long r = 0; r < ch; ++r) img[r * w + c] = b[r];
        }
    }
    free(s);
    return 0;
}

int or_fwd2d_53(int64_t *img, long w, long h, int levels)
{
    long m = (w > h ? w : h);
    int64_t *s = malloc((size_t)thread_count() * 3 * (size_t)m * sizeof(int64_t));
    if (!s) return -1;
    for (int l = 0; l < levels; ++l) {
        long cw = w >> l, ch = h >> l;
#pragma omp parallel for schedule(static)
        for (long c = 0; c < cw; ++c) {
            int64_t *a = s + (size_t)thread_id() * 3 * m, *b = a + m, *y = b + m;
            for (long r = 0; r < ch; ++r) a[r] = img[r * w + c];
            fwd53_line(a, b, ch, y);
            for (long r = 0; r < ch; ++r) img[r * w + c] = b[r];
        }
#pragma omp parallel for schedule(static)
        for (long r = 0; r < ch; ++r) {
            int64_t *b = s + (size_t)thread_id() * 3 * m, *y = b + m;
            fwd53_line(img + r * w, b, cw, y);
            memcpy(img + r * w, b, (size_t)cw * sizeof(int64_t));
        }
    }
    free(s);
    return 0;
}

int or_inv2d_53(int64_t *img, long w, long h, int levels)
{
    long m = (w > h ? w : h);
    int64_t *s = malloc((size_t)thread_count() * 3 * (size_t)m * sizeof(int64_t));
    if (!s) return -1;
    for (int l = levels - 1; l >= 0; --l) {
        long cw = w >> l, ch = h >> l;
#pragma omp parallel for schedule(static)
        for (long r = 0; r < ch; ++r) {
            int64_t *b = s + (size_t)thread_id() * 3 * m, *y = b + m;
            inv53_line(img + r * w, b, cw, y);
            memcpy(img + r * w, b, (size_t)cw * sizeof(int64_t));
        }
#pragma omp parallel for schedule(static)
        for (long c = 0; c < cw; ++c) {
            int64_t *a = s + (size_t)thread_id() * 3 * m, *b = a + m, *y = b + m;
            for (long r = 0; r < ch; ++r) a[r] = img[r * w + c];
            inv53_line(a, b, ch, y);
            for (long r = 0; r < ch; ++r) img[r * w + c] = b[r];
        }
    }
    free(s);
    return 0;
}
