// Radix schedules per transform length: the analogue of the paper's host-side
// `stage_sizes` array and work-group factor (Sec. 4), fixed at compile time so
// that every stage's register array has a static size.  Several candidate
// schedules ("variants") may exist per length; plans use variant 0 unless the
// caller or the autotuner picks another.
//
// Generic Stockham kernel rows:
//   GX(log2N, variant, E = complex elements per thread, S = signals per block,
//      R0, R1, R2, R3 = stage radices first to last (0 = no stage),
//      MINB = minimum resident blocks per SM requested from the compiler,
//      PIPE = 0: stage 0 loads straight from HBM into registers;
//             D >= 2: a ring of D shared-memory tiles filled by bulk-copy
//             (TMA) prefetch, D-1 tiles ahead of the one being transformed,
//      TC = 0: FP32 butterflies; 1 / 2: every radix-16 stage runs as a dense
//           16 x 16 complex product on FP16 / BF16 tensor cores (tcgen05),
//           FP32 accumulation (FP16: a power-of-two prescale per butterfly
//           row; BF16 shares FP32's exponent range and needs none); 5 / 6:
//           as 1 / 2 for the last radix-16 stage only,
//      XB = exchange buffers: 0 = automatic, 1 = one buffer and two barriers
//           per exchange (less shared memory, more resident blocks),
//           -1 = none: with PIPE >= 2, every exchange reuses the ring slot
//           the tile arrived in; -2 = as -1, and the tensor-core A operand
//           lives in that slot too; -3 = as -1, with the A operand in TMEM;
//           3 = none: the exchange of a two-stage N = R x R row with E = R is
//           a transpose by warp shuffles; -5 = as -1, with the signals of a
//           tile placed every N + T elements of the slot (one bulk copy per
//           signal), so that stage 0 reads them without bank conflicts,
//      CH = cache hints: bit 0 plain loads, bit 1 plain stores (else
//           evict-first); the defaults are the measured best per length)
// Threads per block = S * N / E.  Stage 0 with R0 = E/2 (and the last stage,
// where its radix is E/2 or less) lets a thread own neighbouring butterflies,
// so its HBM accesses are 128-bit.  tests/test_bank_model.py replays the
// shared-memory exchanges of every row under the XOR swizzle of
// fft_device.cuh and counts their bank conflicts (64-bit accesses resolve per
// half-warp); tests/test_stockham_model.py replays every row's index mapping
// on the CPU and checks that it computes the DFT.
//
// One-thread-per-signal rows (N <= 32): SX(log2N, variant, warps per block,
// 32-signal groups per warp tile, cache hints as CH above).
#pragma once

#define GBFFT_GENERIC_SCHEDULES(GX)                   \
    GX(5, 1, 16, 128, 8, 4, 0, 0, 1, 0, 0, 0, 0) \
    GX(6, 0, 16, 32, 8, 8, 0, 0, 4, 2, 0, -5, 2) \
    GX(6, 2, 8, 32, 8, 8, 0, 0, 1, 0, 0, 3, 0) \
    GX(6, 3, 8, 32, 8, 8, 0, 0, 1, 0, 0, 0, 0) \
    GX(7, 0, 16, 16, 8, 16, 0, 0, 4, 2, 0, -5, 2) \
    GX(7, 1, 16, 16, 8, 16, 0, 0, 3, 2, 1, 0, 0) \
    GX(7, 2, 16, 16, 8, 16, 0, 0, 3, 2, 2, 0, 0) \
    GX(7, 3, 16, 32, 8, 16, 0, 0, 2, 0, 1, 0, 0) \
    GX(7, 4, 16, 32, 8, 16, 0, 0, 2, 0, 2, 0, 0) \
    GX(8, 17, 16, 16, 16, 16, 0, 0, 1, 0, 0, 0, 2) \
    GX(8, 7, 16, 8, 16, 16, 0, 0, 3, 2, 1, 0, 0) \
    GX(8, 8, 16, 8, 16, 16, 0, 0, 3, 2, 2, 0, 0) \
    GX(8, 3, 16, 16, 16, 16, 0, 0, 1, 0, 1, 0, 0) \
    GX(8, 4, 16, 16, 16, 16, 0, 0, 1, 0, 2, 0, 0) \
    GX(8, 9, 16, 16, 16, 16, 0, 0, 1, 0, 1, 0, 2) \
    GX(8, 10, 16, 16, 16, 16, 0, 0, 1, 0, 2, 0, 2) \
    GX(8, 11, 16, 8, 16, 16, 0, 0, 3, 2, 1, 0, 2) \
    GX(8, 2, 16, 8, 16, 16, 0, 0, 3, 2, 2, 0, 2) \
    GX(8, 1, 16, 8, 16, 16, 0, 0, 3, 2, 5, 0, 2) \
    GX(8, 12, 16, 8, 16, 16, 0, 0, 3, 2, 6, 0, 2) \
    GX(8, 13, 16, 16, 16, 16, 0, 0, 1, 0, 0, 3, 2) \
    GX(8, 14, 16, 8, 16, 16, 0, 0, 3, 2, 0, 0, 2) \
    GX(8, 15, 16, 8, 16, 16, 0, 0, 4, 2, 0, -1, 2) \
    GX(8, 16, 16, 8, 16, 16, 0, 0, 5, 2, 0, -1, 2) \
    GX(8, 0, 16, 16, 16, 16, 0, 0, 2, 2, 0, -1, 2) \
    GX(9, 0, 16, 8, 8, 8, 8, 0, 2, 0, 0, 0, 3) \
    GX(9, 1, 16, 8, 8, 8, 8, 0, 1, 0, 0, 0, 0) \
    GX(10, 0, 16, 2, 8, 16, 8, 0, 2, 2, 0, 0, 2) \
    GX(10, 1, 16, 2, 8, 16, 8, 0, 1, 0, 0, 0, 0) \
    GX(10, 2, 16, 2, 8, 16, 8, 0, 4, 0, 0, 0, 0) \
    GX(10, 3, 16, 2, 8, 16, 8, 0, 2, 3, 0, 0, 0) \
    GX(10, 4, 16, 2, 8, 16, 8, 0, 5, 2, 1, -3, 0) \
    GX(10, 5, 16, 2, 8, 16, 8, 0, 5, 2, 2, -3, 0) \
    GX(10, 6, 16, 2, 8, 16, 8, 0, 2, 2, 1, 0, 0) \
    GX(10, 7, 16, 2, 8, 16, 8, 0, 2, 2, 2, 0, 0) \
    GX(10, 10, 16, 2, 8, 16, 8, 0, 5, 2, 0, -1, 2) \
    GX(10, 11, 16, 2, 8, 16, 8, 0, 5, 2, 1, -2, 0) \
    GX(10, 12, 16, 2, 8, 16, 8, 0, 5, 2, 2, -2, 0) \
    GX(10, 13, 16, 2, 8, 16, 8, 0, 4, 2, 1, 1, 0) \
    GX(10, 14, 16, 2, 8, 16, 8, 0, 4, 2, 2, 1, 0) \
    GX(11, 0, 16, 1, 8, 16, 16, 0, 4, 2, 0, -1, 2) \
    GX(11, 1, 16, 1, 8, 16, 16, 0, 1, 0, 0, 0, 0) \
    GX(11, 2, 16, 1, 8, 16, 16, 0, 2, 3, 0, 0, 0) \
    GX(11, 3, 16, 2, 8, 16, 16, 0, 1, 2, 0, 0, 0) \
    GX(11, 15, 16, 1, 8, 16, 16, 0, 5, 2, 1, -3, 0) \
    GX(11, 16, 16, 1, 8, 16, 16, 0, 5, 2, 2, -3, 0) \
    GX(11, 6, 16, 1, 8, 16, 16, 0, 3, 2, 1, 0, 0) \
    GX(11, 7, 16, 1, 8, 16, 16, 0, 3, 2, 2, 0, 0) \
    GX(11, 10, 16, 1, 8, 16, 16, 0, 3, 2, 0, 0, 2) \
    GX(11, 11, 16, 1, 8, 16, 16, 0, 5, 2, 1, -2, 0) \
    GX(11, 12, 16, 1, 8, 16, 16, 0, 5, 2, 2, -2, 0) \
    GX(11, 13, 16, 1, 8, 16, 16, 0, 4, 2, 1, 1, 0) \
    GX(11, 14, 16, 1, 8, 16, 16, 0, 4, 2, 2, 1, 0) \
    GX(11, 4, 16, 1, 8, 16, 16, 0, 5, 2, 1, -3, 2) \
    GX(11, 5, 16, 1, 8, 16, 16, 0, 5, 2, 2, -3, 2) \
    GX(11, 17, 16, 1, 8, 16, 16, 0, 5, 2, 5, -3, 2) \
    GX(11, 18, 16, 1, 8, 16, 16, 0, 5, 2, 6, -3, 2) \
    GX(11, 19, 16, 1, 8, 16, 16, 0, 5, 2, 0, -1, 2) \
    GX(6, 4, 16, 64, 8, 8, 0, 0, 1, 0, 0, 0, 0) \
    GX(7, 6, 16, 32, 8, 16, 0, 0, 1, 0, 0, 0, 2)

#define GBFFT_SMALL_SCHEDULES(SX) \
    SX(1, 0, 8, 1, 3)                \
    SX(1, 1, 8, 2, 0)                \
    SX(2, 0, 4, 8, 2)                \
    SX(2, 1, 8, 1, 0)                \
    SX(2, 2, 8, 4, 2)                \
    SX(2, 3, 16, 2, 2)               \
    SX(3, 0, 8, 4, 0)                \
    SX(3, 1, 8, 1, 0)                \
    SX(3, 2, 4, 4, 0)                \
    SX(4, 0, 4, 2, 2)                \
    SX(4, 1, 8, 1, 0)                \
    SX(4, 2, 8, 2, 0)                \
    SX(5, 0, 2, 2, 0)                \
    SX(5, 2, 4, 1, 0)

// complex32-storage rows (FFT_C32): CX(log2N, variant, E, S, R0..R3, MINB,
// PIPE, XB) as in GX, the Stockham kernel with binary16 loads/stores and
// per-signal exponents, FP32 arithmetic; PIPE >= 2 stages the binary16 tiles
// through a bulk-copy ring.  A length's first complex32 row is its default;
// for N <= 32 that is the one-thread-per-signal SCX row further down.
#define GBFFT_C32_SCHEDULES(CX)                   \
    CX(1, 3, 2, 256, 2, 0, 0, 0, 1, 0, 0)        \
    CX(2, 5, 2, 128, 2, 2, 0, 0, 1, 0, 0)        \
    CX(3, 4, 4, 128, 2, 4, 0, 0, 1, 0, 0)        \
    CX(4, 4, 8, 128, 4, 4, 0, 0, 1, 0, 0)        \
    CX(5, 4, 16, 128, 8, 4, 0, 0, 1, 0, 0)       \
    CX(6, 1, 16, 64, 8, 8, 0, 0, 1, 0, 0)        \
    CX(7, 5, 16, 32, 8, 16, 0, 0, 1, 0, 0)       \
    CX(8, 18, 16, 16, 16, 16, 0, 0, 3, 2, 1)      \
    CX(8, 6, 16, 16, 16, 16, 0, 0, 1, 0, 0)      \
    CX(9, 2, 16, 8, 8, 8, 8, 0, 2, 0, 0)         \
    CX(10, 8, 16, 2, 8, 16, 8, 0, 2, 3, 0)       \
    CX(10, 9, 16, 2, 8, 16, 8, 0, 2, 0, 0)       \
    CX(11, 8, 16, 1, 8, 16, 16, 0, 3, 3, 0)      \
    CX(11, 9, 16, 1, 8, 16, 16, 0, 3, 0, 0)      \
    CX(8, 5, 16, 8, 16, 16, 0, 0, 5, 2, 1)

// complex32 one-thread-per-signal rows (N <= 32): SCX(log2N, variant, warps
// per block, 32-signal groups per warp tile, cache hints)
#define GBFFT_C32_SMALL_SCHEDULES(SCX) \
    SCX(1, 2, 8, 4, 0)                  \
    SCX(2, 4, 4, 8, 0)                  \
    SCX(3, 3, 8, 4, 0)                  \
    SCX(4, 3, 4, 4, 0)                  \
    SCX(5, 3, 4, 2, 0)

#define GBFFT_MIN_LOG2N 1
#define GBFFT_MAX_LOG2N 11
#define GBFFT_MAX_VARIANTS 31  // FFT_FLAG_VARIANT(k) holds k = 0..30
