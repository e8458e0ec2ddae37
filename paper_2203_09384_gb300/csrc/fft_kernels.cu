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

template <int L>
struct Sched;

#define GBFFT_GENERIC_SCHED(L, E, S, R0, R1, R2, R3)  \
    template <>                                       \
    struct Sched<L> {                                 \
        using type = Cfg<L, E, S, R0, R1, R2, R3>;    \
        static constexpr bool small = false;          \
    };
GBFFT_SCHEDULES(GBFFT_GENERIC_SCHED)
#undef GBFFT_GENERIC_SCHED

#define GBFFT_SMALL_SCHED(L)                   \
    template <>                                \
    struct Sched<L> {                          \
        using type = SmallCfg<L>;              \
        static constexpr bool small = true;    \
    };
GBFFT_SMALL_SCHEDULES(GBFFT_SMALL_SCHED)
#undef GBFFT_SMALL_SCHED

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

static void fill_nothing(float*) {}

template <int L>
static KernelEntry make_entry() {
    using SC = Sched<L>;
    using C = typename SC::type;
    KernelEntry e{};
    e.log2n = L;
    e.small = SC::small;
    if constexpr (SC::small) {
        e.elems_per_thread = C::N;
        e.signals_per_block = 32 * kSmallWarps;
        e.threads_per_block = C::NT;
        e.smem_bytes = C::kSmemBytes;
        e.num_stages = 1;
        e.radix[0] = C::N;
        e.twiddles = 0;
        e.signals_per_warp_tile = 32;
        e.kernel_fwd = reinterpret_cast<const void*>(&fft_small_kernel<L, false>);
        e.kernel_inv = reinterpret_cast<const void*>(&fft_small_kernel<L, true>);
        e.fill_twiddles = &fill_nothing;
    } else {
        e.elems_per_thread = C::E;
        e.signals_per_block = C::S;
        e.threads_per_block = C::NT;
        e.smem_bytes = C::kSmemElems * (int)sizeof(float2);
        e.num_stages = C::M;
        for (int s = 0; s < 4; ++s) e.radix[s] = C::radix(s);
        e.twiddles = C::kTwiddles;
        e.signals_per_warp_tile = 0;
        e.kernel_fwd = reinterpret_cast<const void*>(&fft_stockham_kernel<C, false>);
        e.kernel_inv = reinterpret_cast<const void*>(&fft_stockham_kernel<C, true>);
        e.fill_twiddles = &fill_generic_twiddles<C>;
    }
    return e;
}

}  // namespace gbfft

#define GBFFT_ENTRY_FN2(L) gbfft_entry_##L
#define GBFFT_ENTRY_FN(L) GBFFT_ENTRY_FN2(L)

gbfft::KernelEntry GBFFT_ENTRY_FN(GBFFT_LOG2N)() { return gbfft::make_entry<GBFFT_LOG2N>(); }
