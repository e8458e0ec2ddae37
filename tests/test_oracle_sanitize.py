"""The C oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU).

A small C driver links oracle/oracle.c built with both sanitizers and calls
every entry point over a range of lengths, batch sizes (including 0) and
thread counts, plus the argument checks; it also cross-checks the radix-2
routine against the naive DFT.  Any out-of-bounds access, leak, or undefined
operation fails the test.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "oracle.c")

DRIVER = r"""
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int oracle_dft_naive(const double* x, double* y, int64_t n, int64_t batch, int inverse, int normalize);
int oracle_fft_radix2(const double* x, double* y, int64_t n, int64_t batch, int inverse, int normalize,
                      int threads);
int oracle_grad_weighted_power(const double* x, const double* w, double* grad, double* loss, int64_t n,
                               int64_t batch, int threads);

static double lcg(uint64_t* s) {
    *s = *s * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(*s >> 11) / 9007199254740992.0 * 2.0 - 1.0;
}

int main(void) {
    uint64_t seed = 12345;
    int bad = 0;
    for (int64_t n = 1; n <= 2048; n *= 2) {
        for (int64_t batch = 0; batch <= 3; ++batch) {
            size_t len = (size_t)(2 * n * batch);
            double* x = malloc(len * sizeof(double) + 1);
            double* a = malloc(len * sizeof(double) + 1);
            double* b = malloc(len * sizeof(double) + 1);
            double* w = malloc(len * sizeof(double) + 1);
            for (size_t i = 0; i < len; ++i) { x[i] = lcg(&seed); w[i] = lcg(&seed); }
            for (int inv = 0; inv < 2; ++inv) {
                for (int threads = 1; threads <= 3; threads += 2) {
                    bad |= oracle_fft_radix2(x, a, n, batch, inv, 1, threads) != 0;
                    if (n <= 256) {
                        bad |= oracle_dft_naive(x, b, n, batch, inv, 1) != 0;
                        for (size_t i = 0; i < len; ++i)
                            if (fabs(a[i] - b[i]) > 1e-9 * (double)n) bad |= 1;
                    }
                }
            }
            double loss = 0.0;
            bad |= oracle_grad_weighted_power(x, w, a, &loss, n, batch, 3) != 0;
            bad |= oracle_grad_weighted_power(x, w, a, NULL, n, batch, 1) != 0;
            free(x); free(a); free(b); free(w);
        }
    }
    /* naive DFT on lengths that are not powers of two */
    for (int64_t n = 3; n <= 17; n += 2) {
        double x[2 * 17 * 2], y[2 * 17 * 2];
        for (int i = 0; i < 2 * 17 * 2; ++i) x[i] = lcg(&seed);
        bad |= oracle_dft_naive(x, y, n, 2, 0, 1) != 0;
    }
    /* argument checks */
    double z[4] = {0, 0, 0, 0};
    bad |= oracle_fft_radix2(z, z + 2, 3, 1, 0, 1, 1) != -1;
    bad |= oracle_fft_radix2(NULL, z, 2, 1, 0, 1, 1) != -1;
    bad |= oracle_dft_naive(z, z, 0, 1, 0, 1) != -1;
    bad |= oracle_grad_weighted_power(z, NULL, z, NULL, 2, 1, 1) != -1;
    printf("%s\n", bad ? "FAIL" : "OK");
    return bad;
}
"""


def test_oracle_is_clean_under_sanitizers(tmp_path):
    drv = tmp_path / "drv.c"
    drv.write_text(DRIVER)
    exe = tmp_path / "drv"
    cmd = ["gcc", "-std=c99", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-DORACLE_MUTANT=0", ORACLE_C, str(drv), "-o", str(exe),
           "-lm", "-pthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and ("asan" in r.stderr.lower() or "ubsan" in r.stderr.lower()):
        pytest.skip("the compiler's sanitizer runtimes are not installed")
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout + out.stderr[-4000:]
    assert "runtime error" not in out.stderr and "AddressSanitizer" not in out.stderr, out.stderr[-4000:]
