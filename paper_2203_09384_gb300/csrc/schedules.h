// Radix schedules per transform length: the analogue of the paper's host-side
// `stage_sizes` array and work-group factor (Sec. 4), fixed at compile time so
// that every stage's register array has a static size.
//
// Generic Stockham kernel, one row per log2(N):
//   X(log2N, E = complex elements per thread, S = signals per block,
//     R0, R1, R2, R3 = stage radices first to last, 0 = no stage)
// Threads per block = S * N / E.  The first radix R0 = E/2 (and the last, where
// listed) lets a thread own two neighbouring butterflies, so its HBM accesses
// are 128-bit; an index model on the host checked every exchange below for
// shared-memory bank conflicts under the XOR swizzle of fft_device.cuh.
#pragma once

#define GBFFT_SCHEDULES(X)            \
    X(5, 16, 128, 8, 4, 0, 0)         \
    X(6, 16, 64, 8, 8, 0, 0)          \
    X(7, 16, 32, 8, 16, 0, 0)         \
    X(8, 16, 16, 16, 16, 0, 0)        \
    X(9, 16, 8, 8, 8, 8, 0)           \
    X(10, 16, 2, 8, 16, 8, 0)         \
    X(11, 16, 1, 8, 16, 16, 0)

// N = 2..16: one thread per signal, whole transform in registers.
#define GBFFT_SMALL_SCHEDULES(X) X(1) X(2) X(3) X(4)

#define GBFFT_MIN_LOG2N 1
#define GBFFT_MAX_LOG2N 11
