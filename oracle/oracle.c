/*
 * FP64 CPU oracle for the batched 1-D complex-to-complex DFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * Every routine works on interleaved complex doubles (re, im), signal-major:
 * signal b, element i lives at x[2*(b*n + i)] (re) and x[2*(b*n + i) + 1] (im).
 *
 * What each routine follows (Pascuzzi & Goli, SYCL-FFT, Sec. 3):
 *   oracle_dft_naive   - the definitions, Eq. (dft) (forward, omega_N = e^{-2 pi i/N})
 *                        and Eq. (idft) (inverse: sign of the exponent flipped,
 *                        normalised by 1/N), summed directly in O(N^2).
 *   oracle_fft_radix2  - the recursive radix-2 decimation in time of Eq. (radix2):
 *                        X_k = E_k + w^k O_k, X_{k+N/2} = E_k - w^k O_k, with E
 *                        and O the DFTs of the even and odd samples.
 *   oracle_grad_weighted_power
 *                      - gradient of L = sum_k |W_k X_k|^2, X = DFT(x), in the
 *                        PyTorch convention dL/dRe + i dL/dIm.  L is a real
 *                        quadratic form X^H A X with A = diag(|W|^2), so
 *                        grad_x = 2 F^H (|W|^2 .* F x), F^H being the
 *                        unnormalised transform with the opposite sign.
 *
 * Readings where the paper is garbled: Eq. (idft) is read as
 * x_n = (1/N) sum_k X_k omega_N^{-kn}; Eq. (radix2) is read as the standard
 * even/odd split with omega_N^{2nk} and omega_N^{(2n+1)k}.
 *
 * Pins (tests run without a GPU): closed forms (delta, single tone, the
 * paper's ramp f(x) = x), linearity, Parseval, the inverse round trip, shift
 * and modulation theorems, conjugate symmetry for real input, naive ==
 * recursive by brute force for every N <= 64, the radix-2 and split-radix
 * identities of Sec. 3.1 rebuilt from sub-DFTs, agreement with an independent
 * library FFT, and central finite differences for the gradient.
 *
 * Mutation hooks: building with -DORACLE_MUTANT=k plants mistake k (a wrong
 * sign, a dropped factor, a shifted index ...).  Tests build those variants
 * and check that at least one pin fails for each; the default build has none.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------------- */
/* Eq. (dft) / Eq. (idft): direct summation.                                 */
/* ------------------------------------------------------------------------- */

/*
 * One signal.  The phase of omega_N^{kn} depends only on (k*n) mod N, so the
 * product is reduced in integers first and the root of unity is taken from a
 * per-call table of cos/sin(2*pi*m/N), m < N.  That keeps every angle small
 * and every term exact to libm's accuracy.
 */
static void dft_naive_one(const double* x, double* y, int64_t n, double sign,
                          double scale, const double* c, const double* s) {
    for (int64_t k = 0; k < n; ++k) {
        double acc_re = 0.0, acc_im = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t m = (k * i) % n;
#if ORACLE_MUTANT == 3
            m = (k * i + 1) % n; /* planted: shifted phase index */
#endif
            double wr = c[m];
            double wi = sign * s[m];
            double xr = x[2 * i], xi = x[2 * i + 1];
            acc_re += xr * wr - xi * wi;
            acc_im += xr * wi + xi * wr;
        }
        y[2 * k] = acc_re * scale;
        y[2 * k + 1] = acc_im * scale;
    }
}

/*
 * inverse = 0: Eq. (dft).  inverse = 1: Eq. (idft), with the 1/N factor when
 * normalize != 0 and without it (the plain adjoint F^H) when normalize == 0.
 * x and y must not overlap.  Returns 0, or -1 on bad arguments / no memory.
 */
int oracle_dft_naive(const double* x, double* y, int64_t n, int64_t batch,
                     int inverse, int normalize) {
    if (n < 1 || batch < 0 || !x || !y) return -1;
    double* c = (double*)malloc(sizeof(double) * (size_t)n);
    double* s = (double*)malloc(sizeof(double) * (size_t)n);
    if (!c || !s) { free(c); free(s); return -1; }
    for (int64_t m = 0; m < n; ++m) {
        double a = TWO_PI * (double)m / (double)n;
        c[m] = cos(a);
        s[m] = sin(a);
    }
    /* forward: omega_N^{m} = cos(2 pi m/N) - i sin(2 pi m/N) */
    double sign = inverse ? 1.0 : -1.0;
    double scale = (inverse && normalize) ? 1.0 / (double)n : 1.0;
#if ORACLE_MUTANT == 2
    scale = 1.0; /* planted: inverse loses its 1/N */
#endif
    for (int64_t b = 0; b < batch; ++b)
        dft_naive_one(x + 2 * b * n, y + 2 * b * n, n, sign, scale, c, s);
    free(c);
    free(s);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Eq. (radix2): recursive radix-2 decimation in time.                       */
/* ------------------------------------------------------------------------- */

/*
 * y[0..n) <- DFT_n of the samples x[0], x[stride], x[2 stride], ...
 * E (even samples) lands in y[0..n/2), O (odd samples) in y[n/2..n); the
 * butterfly then combines them in place.
 */
static void fft_rec(const double* x, int64_t stride, int64_t n, double* y,
                    double sign) {
    if (n == 1) {
        y[0] = x[0];
        y[1] = x[1];
        return;
    }
    int64_t h = n / 2;
#if ORACLE_MUTANT == 4
    /* planted: even and odd halves swapped */
    fft_rec(x + 2 * stride, 2 * stride, h, y, sign);
    fft_rec(x, 2 * stride, h, y + 2 * h, sign);
#else
    fft_rec(x, 2 * stride, h, y, sign);                  /* E_k */
    fft_rec(x + 2 * stride, 2 * stride, h, y + 2 * h, sign); /* O_k */
#endif
    for (int64_t k = 0; k < h; ++k) {
        double a = TWO_PI * (double)k / (double)n;
        double wr = cos(a);
        double wi = sign * sin(a);
#if ORACLE_MUTANT == 1
        wi = -wi; /* planted: twiddle of the wrong sign */
#endif
#if ORACLE_MUTANT == 5
        wr = 1.0; wi = 0.0; /* planted: twiddle dropped */
#endif
        double er = y[2 * k], ei = y[2 * k + 1];
        double orr = y[2 * (k + h)], oi = y[2 * (k + h) + 1];
        double tr = orr * wr - oi * wi; /* w^k O_k */
        double ti = orr * wi + oi * wr;
        y[2 * k] = er + tr;
        y[2 * k + 1] = ei + ti;
        y[2 * (k + h)] = er - tr;
        y[2 * (k + h) + 1] = ei - ti;
    }
}

static int is_pow2(int64_t n) { return n >= 1 && (n & (n - 1)) == 0; }

typedef struct {
    const double* x;
    double* y;
    int64_t n, b0, b1;
    double sign, scale;
} rec_job;

static void* rec_worker(void* arg) {
    rec_job* j = (rec_job*)arg;
    for (int64_t b = j->b0; b < j->b1; ++b) {
        double* yb = j->y + 2 * b * j->n;
        fft_rec(j->x + 2 * b * j->n, 1, j->n, yb, j->sign);
        if (j->scale != 1.0)
            for (int64_t i = 0; i < 2 * j->n; ++i) yb[i] *= j->scale;
    }
    return NULL;
}

/*
 * Batched recursive radix-2 FFT over `threads` POSIX threads (signals split
 * into contiguous ranges; threads <= 1 runs inline).  n must be a power of
 * two.  Direction and normalisation as in oracle_dft_naive.  Returns 0 or -1.
 */
int oracle_fft_radix2(const double* x, double* y, int64_t n, int64_t batch,
                      int inverse, int normalize, int threads) {
    if (!is_pow2(n) || batch < 0 || !x || !y) return -1;
    double sign = inverse ? 1.0 : -1.0;
    double scale = (inverse && normalize) ? 1.0 / (double)n : 1.0;
#if ORACLE_MUTANT == 2
    scale = 1.0;
#endif
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if ((int64_t)threads > batch) threads = (int)(batch > 0 ? batch : 1);
    rec_job jobs[256];
    pthread_t tids[256];
    int64_t per = batch / threads, extra = batch % threads, start = 0;
    for (int t = 0; t < threads; ++t) {
        int64_t cnt = per + (t < extra ? 1 : 0);
        jobs[t].x = x; jobs[t].y = y; jobs[t].n = n;
        jobs[t].b0 = start; jobs[t].b1 = start + cnt;
        jobs[t].sign = sign; jobs[t].scale = scale;
        start += cnt;
    }
    if (threads == 1) {
        rec_worker(&jobs[0]);
        return 0;
    }
    int started[256];
    for (int t = 0; t < threads; ++t) {
        started[t] = pthread_create(&tids[t], NULL, rec_worker, &jobs[t]) == 0;
        if (!started[t]) rec_worker(&jobs[t]); /* no thread: do the range here */
    }
    for (int t = 0; t < threads; ++t)
        if (started[t]) pthread_join(tids[t], NULL);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gradient of the weighted spectral power.                                   */
/* ------------------------------------------------------------------------- */

/*
 * L = sum_b sum_k |W[b,k] X[b,k]|^2 with X = DFT(x) (Eq. (dft)).
 * grad[b] = 2 * F^H( |W[b]|^2 .* X[b] ), F^H the unnormalised inverse
 * (Eq. (idft) without 1/N).  Also returns L (summed over the batch) in *loss
 * when loss != NULL.  Returns 0 or -1.
 */
int oracle_grad_weighted_power(const double* x, const double* w, double* grad,
                               double* loss, int64_t n, int64_t batch,
                               int threads) {
    if (!is_pow2(n) || batch < 0 || !x || !w || !grad) return -1;
    size_t bytes = sizeof(double) * 2 * (size_t)n * (size_t)batch;
    double* X = (double*)malloc(bytes > 0 ? bytes : 1);
    if (!X) return -1;
    if (oracle_fft_radix2(x, X, n, batch, 0, 0, threads) != 0) { free(X); return -1; }
    double total = 0.0;
    for (int64_t i = 0; i < n * batch; ++i) {
        double a2 = w[2 * i] * w[2 * i] + w[2 * i + 1] * w[2 * i + 1];
        double p = X[2 * i] * X[2 * i] + X[2 * i + 1] * X[2 * i + 1];
        total += a2 * p;
        double f = 2.0 * a2;
#if ORACLE_MUTANT == 6
        f = a2; /* planted: factor 2 of the Wirtinger gradient dropped */
#endif
        X[2 * i] *= f;
        X[2 * i + 1] *= f;
#if ORACLE_MUTANT == 7
        X[2 * i + 1] = -X[2 * i + 1]; /* planted: stray conjugation */
#endif
    }
    int rc = oracle_fft_radix2(X, grad, n, batch, 1, 0, threads);
    if (loss) *loss = total;
    free(X);
    return rc;
}

/* Build identification, so tests can tell the planted variants apart. */
int oracle_mutant_id(void) { return ORACLE_MUTANT; }
