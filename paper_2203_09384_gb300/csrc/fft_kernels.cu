// Kernel instantiations for one transform length, selected at compile time by
// -DGBFFT_LOG2N=<1..11>.  The build compiles this file once per length, in
// parallel, and links the objects with the host plan code.
#include "fft_device.cuh"
#include "registry.h"
#include "schedules.h"
#include "../../include/gbfft.h"

#ifndef GBFFT_LOG2N
#error "compile with -DGBFFT_LOG2N=<log2 of the transform length>"
#endif

namespace gbfft {

// Twiddle table of a generic schedule: for each stage s >= 1 with radix R and
// Ns = R_0 * ... * R_{s-1}, entry tw_off(s) + (r - 1) * Ns + m holds
// omega_{Ns*R}^{m*r} for r = 1..R-1, m = 0..Ns-1 (laid out so that threads
// with consecutive butterflies read consecutive entries).
template <class C>
static void fill_generic_twiddles(float* host) {
    for (int s = 1; s < C::M; ++s) {
        const int R = C::radix(s), Ns = C::ns(s);
        for (int r = 1; r < R; ++r)
            for (int m = 0; m < Ns; ++m) {
                const int64_t idx = C::tw_off(s) + (int64_t)(r - 1) * Ns + m;
                fft_twiddle_fp32((int64_t)Ns * R, (int64_t)m * r, host + 2 * idx);
            }
    }
}

[[maybe_unused]] static void fill_nothing(float*) {}

template <class C>
static KernelEntry generic_entry(int variant) {
    KernelEntry e{};
    e.log2n = C::LOG2N;
    e.variant = variant;
    e.kind = C::PIPE ? KernelKind::Ring : KernelKind::Direct;
    e.elems_per_thread = C::E;
    e.signals_per_block = C::S;
    e.threads_per_block = C::NT;
    e.smem_bytes = C::kSmemBytes;
    e.num_stages = C::M;
    for (int s = 0; s < 4; ++s) e.radix[s] = C::radix(s);
    e.min_blocks = C::MINB;
    e.pipeline = C::PIPE;
    e.tc = C::TC;
    e.tc_stages = C::kTcStages;
    e.tmem_cols = C::TC ? C::kTcCols : 0;
    e.twiddles = C::kTwiddles;
    if constexpr (C::kInRing) {
        e.kernel_fwd = reinterpret_cast<const void*>(&fft_stockham_slot_ring_kernel<C, false>);
        e.kernel_inv = reinterpret_cast<const void*>(&fft_stockham_slot_ring_kernel<C, true>);
    } else if constexpr (C::PIPE > 0) {
        e.kernel_fwd = reinterpret_cast<const void*>(&fft_stockham_ring_kernel<C, false>);
        e.kernel_inv = reinterpret_cast<const void*>(&fft_stockham_ring_kernel<C, true>);
    } else {
        e.kernel_fwd = reinterpret_cast<const void*>(&fft_stockham_kernel<C, false>);
        e.kernel_inv = reinterpret_cast<const void*>(&fft_stockham_kernel<C, true>);
    }
    e.fill_twiddles = &fill_generic_twiddles<C>;
    return e;
}

template <class C>
static KernelEntry c32_entry(int variant) {
    KernelEntry e = generic_entry<C>(variant);
    e.kind = KernelKind::C32;
    e.smem_bytes = C32Smem<C>::kBytes;
    if constexpr (C::PIPE > 0) {
        e.kernel_fwd = reinterpret_cast<const void*>(&fft_stockham_c32_ring_kernel<C, false>);
        e.kernel_inv = reinterpret_cast<const void*>(&fft_stockham_c32_ring_kernel<C, true>);
    } else {
        e.kernel_fwd = reinterpret_cast<const void*>(&fft_stockham_c32_kernel<C, false>);
        e.kernel_inv = reinterpret_cast<const void*>(&fft_stockham_c32_kernel<C, true>);
    }
    return e;
}

template <class SC>
static KernelEntry small_c32_entry(int variant) {
    KernelEntry e{};
    e.log2n = 0;
    while ((1 << e.log2n) < SC::N) ++e.log2n;
    e.variant = variant;
    e.kind = KernelKind::C32;
    e.elems_per_thread = SC::N;
    e.signals_per_block = 32 * SC::UNROLL * SC::WARPS_PER_BLOCK;
    e.threads_per_block = SC::NT;
    e.smem_bytes = SC::kSmemBytes;
    e.num_stages = 1;
    e.radix[0] = SC::N;
    e.min_blocks = 1;
    e.twiddles = 0;
    e.kernel_fwd = reinterpret_cast<const void*>(&fft_small_c32_kernel<SC, false>);
    e.kernel_inv = reinterpret_cast<const void*>(&fft_small_c32_kernel<SC, true>);
    e.fill_twiddles = &fill_nothing;
    return e;
}

template <class SC>
static KernelEntry small_entry(int variant) {
    KernelEntry e{};
    e.log2n = 0;
    while ((1 << e.log2n) < SC::N) ++e.log2n;
    e.variant = variant;
    e.kind = KernelKind::Small;
    e.elems_per_thread = SC::N;
    e.signals_per_block = 32 * SC::UNROLL * SC::WARPS_PER_BLOCK;
    e.threads_per_block = SC::NT;
    e.smem_bytes = SC::kSmemBytes;
    e.num_stages = 1;
    e.radix[0] = SC::N;
    e.min_blocks = 1;
    e.pipeline = 0;
    e.tc = 0;
    e.tmem_cols = 0;
    e.twiddles = 0;
    e.kernel_fwd = reinterpret_cast<const void*>(&fft_small_kernel<SC, false>);
    e.kernel_inv = reinterpret_cast<const void*>(&fft_small_kernel<SC, true>);
    e.fill_twiddles = &fill_nothing;
    return e;
}

}  // namespace gbfft

// GBFFT_ONLY_<L>(...) keeps its argument only in the build for length 2^L, so
// each translation unit instantiates just its own length's kernels.
#if GBFFT_LOG2N == 1
#define GBFFT_ONLY_1(...) __VA_ARGS__
#else
#define GBFFT_ONLY_1(...)
#endif
#if GBFFT_LOG2N == 2
#define GBFFT_ONLY_2(...) __VA_ARGS__
#else
#define GBFFT_ONLY_2(...)
#endif
#if GBFFT_LOG2N == 3
#define GBFFT_ONLY_3(...) __VA_ARGS__
#else
#define GBFFT_ONLY_3(...)
#endif
#if GBFFT_LOG2N == 4
#define GBFFT_ONLY_4(...) __VA_ARGS__
#else
#define GBFFT_ONLY_4(...)
#endif
#if GBFFT_LOG2N == 5
#define GBFFT_ONLY_5(...) __VA_ARGS__
#else
#define GBFFT_ONLY_5(...)
#endif
#if GBFFT_LOG2N == 6
#define GBFFT_ONLY_6(...) __VA_ARGS__
#else
#define GBFFT_ONLY_6(...)
#endif
#if GBFFT_LOG2N == 7
#define GBFFT_ONLY_7(...) __VA_ARGS__
#else
#define GBFFT_ONLY_7(...)
#endif
#if GBFFT_LOG2N == 8
#define GBFFT_ONLY_8(...) __VA_ARGS__
#else
#define GBFFT_ONLY_8(...)
#endif
#if GBFFT_LOG2N == 9
#define GBFFT_ONLY_9(...) __VA_ARGS__
#else
#define GBFFT_ONLY_9(...)
#endif
#if GBFFT_LOG2N == 10
#define GBFFT_ONLY_10(...) __VA_ARGS__
#else
#define GBFFT_ONLY_10(...)
#endif
#if GBFFT_LOG2N == 11
#define GBFFT_ONLY_11(...) __VA_ARGS__
#else
#define GBFFT_ONLY_11(...)
#endif

#define GBFFT_ENTRIES_FN2(L) gbfft_entries_##L
#define GBFFT_ENTRIES_FN(L) GBFFT_ENTRIES_FN2(L)

int GBFFT_ENTRIES_FN(GBFFT_LOG2N)(gbfft::KernelEntry* out, int max) {
    using namespace gbfft;
    int count = 0;
    auto put = [&](const KernelEntry& e) {
        if (e.variant >= 0 && e.variant < max) {
            out[e.variant] = e;
            if (e.variant + 1 > count) count = e.variant + 1;
        }
    };
#define GBFFT_GX(L, V, E, S, R0, R1, R2, R3, MINB, PIPE, TC, XB, CH) \
    GBFFT_ONLY_##L(put(generic_entry<Cfg<L, E, S, R0, R1, R2, R3, MINB, PIPE, TC, XB, CH>>(V));)
    GBFFT_GENERIC_SCHEDULES(GBFFT_GX)
#undef GBFFT_GX
#define GBFFT_SX(L, V, W, U, CH) GBFFT_ONLY_##L(put(small_entry<SmallCfg<L, W, U, CH>>(V));)
    GBFFT_SMALL_SCHEDULES(GBFFT_SX)
#undef GBFFT_SX
#define GBFFT_CX(L, V, E, S, R0, R1, R2, R3, MINB, PIPE, XB) \
    GBFFT_ONLY_##L(put(c32_entry<Cfg<L, E, S, R0, R1, R2, R3, MINB, PIPE, 0, XB, 0>>(V));)
    GBFFT_C32_SCHEDULES(GBFFT_CX)
#undef GBFFT_CX
#define GBFFT_SCX(L, V, W, U, CH) GBFFT_ONLY_##L(put(small_c32_entry<SmallC32Cfg<L, W, U, CH>>(V));)
    GBFFT_C32_SMALL_SCHEDULES(GBFFT_SCX)
#undef GBFFT_SCX
    return count;
}
