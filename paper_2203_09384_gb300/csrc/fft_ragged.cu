// Ragged batches: signals of mixed power-of-two lengths, packed back to back
// with an offset table, transformed by ONE persistent launch.
//
// Plan time (host): signals are bucketed by length; every bucket is cut into
// tiles of S_N signals (the same per-length schedules as the uniform path,
// re-shaped so that every length runs in a 256-thread block), and the tiles
// become a device work list ordered from the longest length down (variant 9:
// the lengths up to 128 first, then the rest longest first).
//
// Ten variants are compiled.  Bit 0 of variants 0..3 picks the schedule
// set: set 0 keeps 16 complex elements per thread for N >= 32 (fewest
// exchanges), set 1 keeps 8 (fewer registers, more resident blocks, finer
// tiles).  Bit 1 picks how blocks get work: 0 = a shared counter (one
// atomicAdd per item; fft_execute clears it with a memset node first), 1 =
// static round robin with the next item's descriptor prefetched.  Variant 4
// runs set 1 with a bulk-copy (TMA) ring that keeps the next item's signals in
// flight.  Variants 5..9 run set 0 in ring slots that a producer warp fills
// (exchanges inside the slot): 5 with 256 compute threads and 2 slots, 6 with
// 128 compute threads and 2 slots, 7 with 128 and 3 slots, 8 as 6 with
// registers capped at 80, 9 (the default) the kernel of 8 with the lengths up
// to 128 first in the work list.
// A tile whose signals lie back to back (runs of one length in the input)
// is marked at plan time: its threads compute their offsets instead of
// loading them, and the bulk-copy variants fetch a tile of short signals in
// 2 KB copies rather than one copy per signal.  The producer variants place
// the signals of any other tile of N = 4..128 with a gap in the ring slot, so
// that stage 0 reads them without shared-memory bank conflicts (slot_pad).
// Variants 4..9 wait on mbarriers, with the same bounded waits, error word
// and stall test mode as the uniform ring kernels.  Every step is
// stream-ordered, so an execute can be captured in a CUDA graph.  The
// autotuner picks a variant per workload.
#include <cuda_runtime.h>

#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "../../include/gbfft.h"
#include "fft_device.cuh"
#include "registry.h"
#include "schedules.h"

namespace gbfft {

struct RaggedItem {
    int log2n;
    int count;     // signals in this tile (<= S of the length's schedule)
    int first;     // index of the tile's first signal in the bucketed offset list
    int contig;    // 1: the tile's signals lie back to back from off0, so one
                   // bulk copy fetches the tile and no offset is loaded
    int64_t off0;  // element offset of that first signal (= sig_off[first]): a
                   // single-signal tile needs no second, dependent load
};

struct RaggedArgs {
    const float2* in;
    float2* out;
    const RaggedItem* items;
    int n_items;
    int scale_mode;  // 0: none, 1: times 1/N of each signal's length
    const int64_t* sig_off;
    const float2* tw;
    int tw_off[GBFFT_MAX_LOG2N + 1];
    unsigned int* counter;
    int* err;          // device error word (bounded waits of the prefetch ring)
    uint64_t wait_ns;  // limit of each such wait
    int stall;         // failure-detection test mode: the bulk-copy variants issue no copy
};

// per-variant, per-length schedules; every one has 256 threads per block
template <int V, int L>
struct RCfg;
#define GBFFT_RCFG(V, L, E, S, R0, R1, R2, R3)          \
    template <>                                        \
    struct RCfg<V, L> {                                \
        using type = Cfg<L, E, S, R0, R1, R2, R3, 1, 0>; \
        static_assert(type::NT == 256, "ragged tiles use 256 threads"); \
    };
// variant 0: E = 16 for N >= 32
GBFFT_RCFG(0, 1, 2, 256, 2, 0, 0, 0)
GBFFT_RCFG(0, 2, 2, 128, 2, 2, 0, 0)
GBFFT_RCFG(0, 3, 4, 128, 2, 4, 0, 0)
GBFFT_RCFG(0, 4, 8, 128, 4, 4, 0, 0)
GBFFT_RCFG(0, 5, 16, 128, 8, 4, 0, 0)
GBFFT_RCFG(0, 6, 16, 64, 8, 8, 0, 0)
GBFFT_RCFG(0, 7, 16, 32, 8, 16, 0, 0)
GBFFT_RCFG(0, 8, 16, 16, 16, 16, 0, 0)
GBFFT_RCFG(0, 9, 16, 8, 8, 8, 8, 0)
GBFFT_RCFG(0, 10, 16, 4, 8, 16, 8, 0)
GBFFT_RCFG(0, 11, 16, 2, 8, 16, 16, 0)
// variant 1: E = 8 for N >= 16
GBFFT_RCFG(1, 1, 2, 256, 2, 0, 0, 0)
GBFFT_RCFG(1, 2, 2, 128, 2, 2, 0, 0)
GBFFT_RCFG(1, 3, 4, 128, 2, 4, 0, 0)
GBFFT_RCFG(1, 4, 8, 128, 4, 4, 0, 0)
GBFFT_RCFG(1, 5, 8, 64, 4, 8, 0, 0)
GBFFT_RCFG(1, 6, 8, 32, 8, 8, 0, 0)
GBFFT_RCFG(1, 7, 8, 16, 4, 4, 8, 0)
GBFFT_RCFG(1, 8, 8, 8, 4, 8, 8, 0)
GBFFT_RCFG(1, 9, 8, 4, 8, 8, 8, 0)
GBFFT_RCFG(1, 10, 8, 2, 4, 4, 8, 8)
GBFFT_RCFG(1, 11, 8, 1, 4, 8, 8, 8)
#undef GBFFT_RCFG

// variants 0..3: bit 0 schedule set, bit 1 work distribution; variant 4: the
// schedule set 1 shapes fed by a bulk-copy (TMA) prefetch ring; variants 5..8:
// set 0 shapes in ring slots filled by a producer warp (5: 256 compute threads
// and 2 slots; 6 / 7: 128 compute threads, half the signals per tile, 2 / 3
// slots, 4 resident blocks per SM; 8: as 6 with registers capped at 80;
// 9: as 8, short lengths first in the work list)
constexpr int kRaggedVariants = 10;
constexpr int kRingVariant = 4;
constexpr int kFirstProducerVariant = 5;
constexpr int kDefaultRaggedVariant = 9;  // measured fastest on the mixed-length workload
constexpr int kShortFirstVariant = 9;     // variant 8's kernel, short lengths first in the work list
constexpr int kShortMaxLog2n = 7;  // measured: up to 128 first beats up to 32 or 64 on the mix
// the variant ragged plans use when the caller names none (process-wide; the
// autotuner's cached choice is applied through fft_set_default_ragged_variant)
std::atomic<int> g_default_ragged_variant{kDefaultRaggedVariant};
__host__ __device__ constexpr bool is_producer_variant(int v) { return v >= kFirstProducerVariant; }

// the ring variant's per-length schedules: set 1 with a 2-slot ring
template <int L>
struct RingCfg {
    using B = typename RCfg<1, L>::type;
    using type = Cfg<L, B::E, B::S, B::radix(0), B::radix(1), B::radix(2), B::radix(3), 3, 2>;
};
constexpr int kRingTile = 2048;  // complex elements per item (S * N) at most
// a back-to-back tile of signals shorter than this is fetched in copies of
// this many elements (2 KB) instead of one copy per signal; longer signals
// keep one copy each (measured: the per-signal form is faster there, all
// N = 256 30.5 us against 32.1 us with the span form, both one copy per signal)
constexpr int kSpanChunk = 256;
constexpr int kRaggedThreads = 256;

// the producer variants' per-length schedules for NTC compute threads: set 0
// radices and elements per thread, NTC / 256 of its signals per tile, stage 0
// read from the ring slot and every exchange inside it (XB = -1); CH = 2
// stores plainly (not evict-first), as the uniform defaults of N >= 128 do
template <int NTC, int L, int CH = 0>
struct SlotCfg {
    using B = typename RCfg<0, L>::type;
    using type = Cfg<L, B::E, B::S * NTC / kRaggedThreads, B::radix(0), B::radix(1), B::radix(2), B::radix(3), 2, 2,
                     0, -1, CH>;
    static_assert(type::NT == NTC, "one tile per compute group");
};
template <int NTC, int MINB>
struct SlotShape {
    // complex elements of a ring slot: a tile (S * N <= NTC * 16) plus the
    // stage-0 padding of scattered short signals (S * T = NTC, see slot_pad)
    static constexpr int kTile = NTC * 17;
    static constexpr int kThreads = NTC + 32;     // compute threads + the producer warp
    static constexpr int kMinBlocks = MINB;       // resident blocks per SM asked of the compiler
};
template <int V>
struct RaggedMinBlocks {
    static constexpr int value = V == 0 ? 2 : 3;
};

template <int V0>
constexpr int ragged_smem_bytes() {
    constexpr int V = V0 & 1;
    int m = 0;
#define GBFFT_RSMEM(L) m = m > RCfg<V, L>::type::kSmemElems * 8 ? m : RCfg<V, L>::type::kSmemElems * 8;
    GBFFT_RSMEM(1) GBFFT_RSMEM(2) GBFFT_RSMEM(3) GBFFT_RSMEM(4) GBFFT_RSMEM(5) GBFFT_RSMEM(6)
    GBFFT_RSMEM(7) GBFFT_RSMEM(8) GBFFT_RSMEM(9) GBFFT_RSMEM(10) GBFFT_RSMEM(11)
#undef GBFFT_RSMEM
    return m;
}

// Offset of this thread's signal in work item w (0 when the thread has none).
template <class C>
__device__ __forceinline__ int64_t ragged_offset(const RaggedArgs& a, const RaggedItem& w) {
    const int sl = threadIdx.x / C::T;
    if (sl >= w.count) return 0;
    return sl == 0 || w.contig ? w.off0 + ((int64_t)sl << C::LOG2N) : a.sig_off[w.first + sl];
}

template <class C, bool INV>
__device__ __forceinline__ void ragged_tile(const RaggedArgs& a, const RaggedItem& w, float2* smem, int64_t off) {
    const int tid = threadIdx.x;
    const int sl = tid / C::T;
    const int t = tid % C::T;
    const bool active = sl < w.count;
    const float2* tw = a.tw + a.tw_off[C::LOG2N];
    const float scale = a.scale_mode ? 1.0f / (float)C::N : 1.0f;
    int buf = 0;
    TcCtx tc;  // FP32 butterflies only
    float2 v[C::E];
    load_first<C, INV>(v, a.in + off, t, active);
    twist_and_dft<C, 0>(v, t, tw, tc);
    rest_stages<C, 1>(v, smem, buf, sl * C::N, t, tw, tc);
    store_last<C, INV>(v, a.out + off, t, active, scale);
}

template <int V>
__device__ __forceinline__ int64_t ragged_offset_for(const RaggedArgs& a, const RaggedItem& w) {
    switch (w.log2n) {
#define GBFFT_ROFF(L) \
    case L: return ragged_offset<typename RCfg<V, L>::type>(a, w);
        GBFFT_ROFF(1) GBFFT_ROFF(2) GBFFT_ROFF(3) GBFFT_ROFF(4) GBFFT_ROFF(5) GBFFT_ROFF(6)
        GBFFT_ROFF(7) GBFFT_ROFF(8) GBFFT_ROFF(9) GBFFT_ROFF(10) GBFFT_ROFF(11)
#undef GBFFT_ROFF
        default: return 0;
    }
}

template <int V, bool INV>
__device__ __forceinline__ void ragged_dispatch(const RaggedArgs& a, const RaggedItem& w, float2* smem, int64_t off) {
    switch (w.log2n) {
#define GBFFT_RCASE(L) \
    case L: ragged_tile<typename RCfg<V, L>::type, INV>(a, w, smem, off); break;
        GBFFT_RCASE(1) GBFFT_RCASE(2) GBFFT_RCASE(3) GBFFT_RCASE(4) GBFFT_RCASE(5) GBFFT_RCASE(6)
        GBFFT_RCASE(7) GBFFT_RCASE(8) GBFFT_RCASE(9) GBFFT_RCASE(10) GBFFT_RCASE(11)
#undef GBFFT_RCASE
        default: break;
    }
}

// Variant bit 1 selects how blocks get work: 0 = the shared counter (each
// block takes the next item with one atomicAdd), 1 = static round robin
// (block b takes items b, b + grid, ...) with the next item's descriptor and
// this thread's signal offset loaded while the current item is transformed,
// so the data loads of an item start without a chain of dependent reads.
template <int V, bool INV>
__global__ void __launch_bounds__(kRaggedThreads, RaggedMinBlocks<V & 1>::value) fft_ragged_kernel(RaggedArgs a) {
    pdl_enter();
    constexpr int S = V & 1;  // schedule set
    extern __shared__ __align__(16) float2 smem[];
    dbg_set_err(a.err);
    if constexpr ((V >> 1) == 0) {
        __shared__ int s_item;
        for (;;) {
            if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
            __syncthreads();
            const int it = s_item;
            __syncthreads();  // everyone has read s_item before the next fetch
            if (it >= a.n_items) break;
            const RaggedItem w = a.items[it];
            ragged_dispatch<S, INV>(a, w, smem, ragged_offset_for<S>(a, w));
        }
    } else {
        int it = blockIdx.x;
        if (it >= a.n_items) return;
        RaggedItem w = a.items[it];
        int64_t off = ragged_offset_for<S>(a, w);
        for (;;) {
            const int nx = it + (int)gridDim.x;
            RaggedItem wn{};
            int64_t offn = 0;
            if (nx < a.n_items) {  // prefetch the next item's descriptor and offset
                wn = a.items[nx];
                offn = ragged_offset_for<S>(a, wn);
            }
            ragged_dispatch<S, INV>(a, w, smem, off);
            if (nx >= a.n_items) break;
            __syncthreads();  // the next item may reuse shared memory differently
            it = nx;
            w = wn;
            off = offn;
        }
    }
}

// Warp 0 copies every signal of item `it` into ring slot `slot`: one bulk copy
// per signal (contiguous in HBM), all completing on the slot's mbarrier.
__device__ __forceinline__ void ragged_issue(const RaggedArgs& a, float2* slot_base, uint64_t* bar, int it) {
    const int lane = threadIdx.x & 31;
    const RaggedItem w = a.items[it];
    const int n = 1 << w.log2n;
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(w.count * n * 8));
    __syncwarp();
    if (w.contig && n < kSpanChunk) {
        const int total = w.count * n;
        for (int j = lane * kSpanChunk; j < total; j += 32 * kSpanChunk)
            bulk_copy_g2s(slot_base + j, a.in + w.off0 + j, (uint32_t)(min(kSpanChunk, total - j) * 8), bar);
        return;
    }
    for (int k = lane; k < w.count; k += 32)
        bulk_copy_g2s(slot_base + k * n, a.in + (k == 0 ? w.off0 : a.sig_off[w.first + k]), (uint32_t)(n * 8), bar);
}

template <class C, bool INV>
__device__ __forceinline__ void ragged_ring_tile(const RaggedArgs& a, const RaggedItem& w, float2* xbuf,
                                                 const float2* slot_base, int64_t off, bool dead,
                                                 float2* refill_base, uint64_t* refill_bar, int refill_it) {
    const int tid = threadIdx.x;
    const int sl = tid / C::T;
    const int t = tid % C::T;
    const bool active = sl < w.count && !dead;
    const float2* tw = a.tw + a.tw_off[C::LOG2N];
    const float scale = a.scale_mode ? 1.0f / (float)C::N : 1.0f;
    TcCtx tc;
    float2 v[C::E];
    gather_tile<C, INV>(v, slot_base, sl * C::N, t);
    __syncthreads();  // every thread has read the slot: refill it
    if (tid < 32 && refill_it >= 0) {
        fence_proxy_async_smem();
        ragged_issue(a, refill_base, refill_bar, refill_it);
    }
    int buf = 0;
    twist_and_dft<C, 0>(v, t, tw, tc);
    rest_stages<C, 1>(v, xbuf, buf, sl * C::N, t, tw, tc);
    store_last<C, INV>(v, a.out + off, t, active, scale);
}

// Static round robin over the work list; warp 0 keeps the next item's
// signals in flight into the other ring slot while the current one runs.
template <bool INV>
__global__ void __launch_bounds__(kRaggedThreads, 3) fft_ragged_ring_kernel(RaggedArgs a) {
    pdl_enter();
    extern __shared__ __align__(16) float2 smem[];
    float2* xbuf = smem;                   // 2 exchange buffers
    float2* ring = smem + 2 * kRingTile;   // 2 ring slots
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + 2 * kRingTile);
    const int tid = threadIdx.x;
    const int grid = (int)gridDim.x;
    dbg_set_err(a.err);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    RingInFlight inflight;  // thread 0's view of warp 0's copies in flight
    // stall != 0 is the failure-detection test mode: nothing is issued, so the
    // first wait of every block runs out, records FFT_ERR_TIMEOUT, and the
    // block finishes its items without waiting or storing
    if (tid < 32 && !a.stall) {
        for (int d = 0; d < 2; ++d) {
            const int it = (int)blockIdx.x + d * grid;
            if (it < a.n_items) {
                ragged_issue(a, ring + d * kRingTile, &bars[d], it);
                inflight.issued(d, 0);
            }
        }
    }
    bool dead = false;
    int k = 0;
    for (int it = blockIdx.x; it < a.n_items; it += grid, ++k) {
        const int slot = k & 1;
        const uint32_t parity = (uint32_t)((k >> 1) & 1);
        if (!dead) {
            if (mbar_wait_bounded(&bars[slot], parity, a.wait_ns)) {
                inflight.completed(slot);
            } else {
                dead = true;
                atomicCAS(a.err, 0, kErrTimeout);
            }
        }
        const RaggedItem w = a.items[it];
        const int nx = it + 2 * grid;
        // warp 0 issues the refill together (one lane sets the byte count,
        // all lanes copy), so it decides once: no refill if any lane gave up
        const bool wdead = __any_sync(0xffffffffu, dead);
        const int refill = (nx < a.n_items && !wdead) ? nx : -1;
        if (refill >= 0) inflight.issued(slot, (uint32_t)(((k + 2) >> 1) & 1));
        switch (w.log2n) {
#define GBFFT_RRING(L)                                                                                        \
    case L: {                                                                                                 \
        using C = typename RingCfg<L>::type;                                                                  \
        ragged_ring_tile<C, INV>(a, w, xbuf, ring + slot * kRingTile, ragged_offset<C>(a, w), dead,           \
                                 ring + slot * kRingTile, &bars[slot], refill);                               \
        break;                                                                                                \
    }
            GBFFT_RRING(1) GBFFT_RRING(2) GBFFT_RRING(3) GBFFT_RRING(4) GBFFT_RRING(5) GBFFT_RRING(6)
            GBFFT_RRING(7) GBFFT_RRING(8) GBFFT_RRING(9) GBFFT_RRING(10) GBFFT_RRING(11)
#undef GBFFT_RRING
            default: break;
        }
        __syncthreads();  // the next item reuses shared memory with another shape
    }
    if (tid == 0) inflight.drain(bars, a.wait_ns);  // copies in flight after a wait gave up
}

// ---------------------------------------------------------------------------
// Variant 5: a producer warp and ring slots.  Block = 256 compute threads plus
// one producer warp.  The producer walks the block's items (round robin) and,
// once the compute threads have released a slot (its `empty` mbarrier), copies
// the next item's signals into it with one bulk copy per signal, completing on
// the slot's `full` mbarrier.  The compute threads wait on `full`, read stage
// 0 from the slot, exchange inside it (one named barrier per signal over the
// threads of a signal, or a warp sync when a signal stays in one warp), release
// the slot after the last exchange and store the result from registers.  The dependent
// descriptor and offset loads of the next item are the producer's alone, so
// they never stall the compute threads.  Every wait is bounded.
// ---------------------------------------------------------------------------
// Exchange barrier of one signal: its slot region is touched by its own T
// threads only, so a signal within one warp needs a warp sync, and a signal
// spanning warps syncs its T threads on a named barrier of its own; barrier 0
// stays the block's.  Warps are not synchronised between items, so one warp
// group may already run a later item (another length, other signal
// boundaries) while another is still exchanging in an earlier one.  A barrier
// must never see arrivals with two thread counts at once, so every signal
// width T has its own range of barrier numbers: signal group g (warps
// g*T/32 .. (g+1)*T/32 - 1) of width T uses bar_base(T) + g.  A number is then
// only ever used by the same warps with the same count, whatever the order of
// the items, and consecutive uses by those warps follow one another.
//
// The barrier number is an immediate (one branch per signal group of the
// block), so the compiler reserves only the barriers a kernel can name (1..3
// for 128 compute threads, 1..6 for 256).  A number held in a register would
// reserve all 16, and the SM's barrier supply would then cap the resident
// blocks below what registers and shared memory allow.
template <int NT, int T>
constexpr int bar_base() {
    int base = 1;
    for (int t = 64; t < T; t *= 2) base += NT / t;
    return base;
}

template <int T, int BASE, int G, int NG>
__device__ __forceinline__ void signal_bar(int g) {
    if constexpr (G < NG) {
        if (g == G) {
            asm volatile("bar.sync %0, %1;" ::"n"(BASE + G), "n"(T) : "memory");
        } else {
            signal_bar<T, BASE, G + 1, NG>(g);
        }
    }
}

template <class C>
__device__ __forceinline__ void slot_sync() {
    if constexpr (C::T <= 32) {
        __syncwarp();
    } else {
        static_assert(C::T % 32 == 0 && bar_base<C::NT, C::T>() + C::NT / C::T <= 16, "whole warps; barriers 1..15");
        constexpr int kWarps = C::T / 32;  // warps per signal
        signal_bar<C::T, bar_base<C::NT, C::T>(), 0, C::NT / C::T>(((int)threadIdx.x >> 5) / kWarps);
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <class C, int s>
__device__ __forceinline__ void slot_stages(float2 (&v)[C::E], float2* b, int sb, int t, const float2* __restrict__ tw,
                                            TcCtx& tc) {
    if constexpr (s < C::M) {
        slot_sync<C>();  // every reader of b (the tile, or stage s-1's gather) is done
        scatter<C, s - 1>(v, b, sb, t);
        slot_sync<C>();
        gather<C, s>(v, b, sb, t);
        twist_and_dft<C, s>(v, t, tw, tc);
        slot_stages<C, s + 1>(v, b, sb, t, tw, tc);
    }
}

// Stage-0 padding in the ring slot.  Stage 0 reads a tile as the bulk copies
// wrote it, without a swizzle: with signals of N = 4..128 packed every N
// elements, the threads of a half-warp (several signals, T threads each) hit
// the same few banks (2-8 way, CPU bank model).  So the producer places the
// signals of a tile of scattered signals (one copy per signal anyway) every
// N + T elements: consecutive signals then start T bank slots apart and
// stage 0 reads without conflicts.  The exchanges after it use the dense
// layout again, behind a barrier of all compute threads.  Back-to-back tiles
// keep the dense layout and their 2 KB copies; N = 2 has one stage.
template <class C>
constexpr int slot_pad_of() {
    return C::LOG2N >= 2 && C::LOG2N <= 7 ? C::T : 0;
}
template <int NTC>
__device__ __forceinline__ int slot_pad(int log2n) {
    switch (log2n) {
#define GBFFT_SPAD(L) \
    case L: return slot_pad_of<typename SlotCfg<NTC, L>::type>();
        GBFFT_SPAD(2) GBFFT_SPAD(3) GBFFT_SPAD(4) GBFFT_SPAD(5) GBFFT_SPAD(6) GBFFT_SPAD(7)
#undef GBFFT_SPAD
        default: return 0;
    }
}

// stage-0 inputs of this thread's signal, which starts at element `sb` of the
// slot (sl * N packed, sl * (N + T) padded); conjugated for the inverse
template <class C, bool INV>
__device__ __forceinline__ void slot_gather0(float2 (&v)[C::E], const float2* tile, int sb, int t) {
    constexpr int R = C::radix(0);
    constexpr int K = C::E / R;
    constexpr int stride = C::N / R;
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const int j = bfly<C, 0>(t, c);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!dbg_ok(sb + j + r * stride < C::NT * 17)) continue;
            const float2 x = tile[sb + j + r * stride];
            v[c * R + r] = INV ? conj2(x) : x;
        }
    }
}

template <class C, bool INV>
__device__ __forceinline__ void slot_tile(const RaggedArgs& a, const RaggedItem& w, float2* slot, uint64_t* empty,
                                          int64_t off, bool dead) {
    static_assert(C::S * C::N <= C::NT * 16, "a tile must fit a ring slot");
    static_assert(C::S * (C::N + slot_pad_of<C>()) <= C::NT * 17, "a padded tile must fit a ring slot");
    const int tid = threadIdx.x;
    const int sl = tid / C::T;
    const int t = tid % C::T;
    const bool active = sl < w.count && !dead;
    const float2* tw = a.tw + a.tw_off[C::LOG2N];
    const float scale = a.scale_mode ? 1.0f / (float)C::N : 1.0f;
    TcCtx tc;  // FP32 butterflies only
    float2 v[C::E];
    constexpr int kPad = slot_pad_of<C>();
    const bool padded = kPad != 0 && !w.contig && w.count > 1;  // the same for every compute thread
    slot_gather0<C, INV>(v, slot, sl * (C::N + (padded ? kPad : 0)), t);
    twist_and_dft<C, 0>(v, t, tw, tc);
    if constexpr (kPad != 0) {
        // the dense exchanges below overwrite other signals' padded inputs:
        // every compute thread must have read its own first
        if (padded) asm volatile("bar.sync %0, %1;" ::"n"(bar_base<C::NT, 2 * C::NT>()), "n"(C::NT) : "memory");
    }
    slot_stages<C, 1>(v, slot, sl * C::N, t, tw, tc);
    // this thread is done with the slot: order its shared-memory accesses
    // before the producer's next copy into it; once the whole warp is, one
    // lane releases the slot for the warp (the barrier counts warps)
    fence_proxy_async_smem();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(empty);
    store_last<C, INV>(v, a.out + off, t, active, scale);
}

template <int NTC>
__device__ __forceinline__ int64_t slot_offset_for(const RaggedArgs& a, const RaggedItem& w) {
    switch (w.log2n) {
#define GBFFT_SOFF(L) \
    case L: return ragged_offset<typename SlotCfg<NTC, L>::type>(a, w);
        GBFFT_SOFF(1) GBFFT_SOFF(2) GBFFT_SOFF(3) GBFFT_SOFF(4) GBFFT_SOFF(5) GBFFT_SOFF(6)
        GBFFT_SOFF(7) GBFFT_SOFF(8) GBFFT_SOFF(9) GBFFT_SOFF(10) GBFFT_SOFF(11)
#undef GBFFT_SOFF
        default: return 0;
    }
}

// The producer warp.  Lane 0 sets each fill's byte count; every lane copies
// signals lane, lane + 32, ...  The next item's descriptor is loaded before
// the wait for a free slot, so its latency hides behind that wait, and a
// tile's first signal comes with its own offset (RaggedItem::off0), so a
// single-signal tile costs one global load before its copy, not two.  Before
// it exits, lane 0 waits (bounded) for the copies it issued last, so none
// lands after the block is gone even when the compute threads gave up.
template <int NTC, int SLOTS, int MINB>
__device__ __forceinline__ void slot_produce(const RaggedArgs& a, float2* ring, uint64_t* full, uint64_t* empty) {
    constexpr int kSlots = SLOTS;
    constexpr int kSlotTile = SlotShape<NTC, MINB>::kTile;
    const int lane = threadIdx.x & 31;
    RingInFlight inflight;  // lane 0
    // failure-detection test mode: copy nothing, so the compute threads' first
    // wait runs out and they finish their items without waiting or storing
    if (a.stall) return;
    int it = blockIdx.x;
    if (it >= a.n_items) return;
    RaggedItem w = a.items[it];
    for (int k = 0;; ++k) {
        const int slot = k % kSlots;
        const int nx = it + (int)gridDim.x;
        RaggedItem wn{};
        if (nx < a.n_items) wn = a.items[nx];  // in flight during the wait below
        if (k >= kSlots) {  // the compute threads must have released the slot's previous item
            bool ok = true;
            if (lane == 0) {
                ok = mbar_wait_bounded(&empty[slot], (uint32_t)((k / kSlots - 1) & 1), a.wait_ns);
                if (ok) inflight.completed(slot);  // that item's copy was consumed
                else atomicCAS(a.err, 0, kErrTimeout);
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
        }
        const int n = 1 << w.log2n;
        float2* dst = ring + slot * kSlotTile;
        if (lane == 0) {
            mbar_arrive_expect_tx(&full[slot], (uint32_t)(w.count * n * 8));
            inflight.issued(slot, (uint32_t)((k / kSlots) & 1));
        }
        __syncwarp();
        if (w.contig && n < kSpanChunk) {  // one span of short signals: copies of kSpanChunk elements
            const int total = w.count * n;
            for (int j = lane * kSpanChunk; j < total; j += 32 * kSpanChunk)
                bulk_copy_g2s(dst + j, a.in + w.off0 + j, (uint32_t)(min(kSpanChunk, total - j) * 8), &full[slot]);
        } else {
            // scattered signals, one copy each, every n + pad elements (slot_pad)
            const int pitch = n + (w.count > 1 ? slot_pad<NTC>(w.log2n) : 0);
            for (int j = lane; j < w.count; j += 32)
                bulk_copy_g2s(dst + j * pitch, a.in + (j == 0 ? w.off0 : a.sig_off[w.first + j]), (uint32_t)(n * 8),
                              &full[slot]);
        }
        if (nx >= a.n_items) break;
        it = nx;
        w = wn;
    }
    if (lane == 0) inflight.drain(full, a.wait_ns);
}

// The body of the producer-warp kernels; the __global__ wrappers below differ
// only in how they bound registers.
template <int NTC, int SLOTS, int MINB, int CH, bool INV>
__device__ __forceinline__ void ragged_slot_body(const RaggedArgs& a) {
    constexpr int kSlots = SLOTS;
    constexpr int kSlotTile = SlotShape<NTC, MINB>::kTile;
    extern __shared__ __align__(16) float2 smem[];
    float2* ring = smem;  // kSlots slots of kSlotTile elements
    uint64_t* full = reinterpret_cast<uint64_t*>(ring + kSlots * kSlotTile);
    uint64_t* empty = full + kSlots;
    const int tid = threadIdx.x;
    const int grid = (int)gridDim.x;
    dbg_set_err(a.err);
    if (tid == 0) {
        for (int d = 0; d < kSlots; ++d) {
            mbar_init(&full[d], 1);
            mbar_init(&empty[d], NTC / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();  // the last barrier of all NTC + 32 threads
    if (tid >= NTC) {
        slot_produce<NTC, SLOTS, MINB>(a, ring, full, empty);
        return;
    }
    int it = blockIdx.x;
    if (it >= a.n_items) return;
    RaggedItem w = a.items[it];
    int64_t off = slot_offset_for<NTC>(a, w);
    bool dead = false;
    for (int k = 0;; ++k) {
        const int nx = it + grid;
        RaggedItem wn{};
        int64_t offn = 0;
        if (nx < a.n_items) {  // the next item's descriptor and this thread's offset, ahead of time
            wn = a.items[nx];
            offn = slot_offset_for<NTC>(a, wn);
        }
        const int slot = k % kSlots;
        if (!dead && !mbar_wait_bounded(&full[slot], (uint32_t)((k / kSlots) & 1), a.wait_ns)) {
            dead = true;
            atomicCAS(a.err, 0, kErrTimeout);
        }
        switch (w.log2n) {
#define GBFFT_SCASE(L)                                                                                       \
    case L:                                                                                                  \
        slot_tile<typename SlotCfg<NTC, L, CH>::type, INV>(a, w, ring + slot * kSlotTile, &empty[slot], off, dead); \
        break;
            GBFFT_SCASE(1) GBFFT_SCASE(2) GBFFT_SCASE(3) GBFFT_SCASE(4) GBFFT_SCASE(5) GBFFT_SCASE(6)
            GBFFT_SCASE(7) GBFFT_SCASE(8) GBFFT_SCASE(9) GBFFT_SCASE(10) GBFFT_SCASE(11)
#undef GBFFT_SCASE
            default: break;
        }
        if (nx >= a.n_items) break;
        it = nx;
        w = wn;
        off = offn;
    }
}

// Residency asked as a minimum of MINB blocks per SM (the compiler then
// picks the register budget).
template <int NTC, int SLOTS, int MINB, bool INV>
__global__ void __launch_bounds__(SlotShape<NTC, MINB>::kThreads, SlotShape<NTC, MINB>::kMinBlocks)
    fft_ragged_slot_kernel(RaggedArgs a) {
    pdl_enter();
    ragged_slot_body<NTC, SLOTS, MINB, 0, INV>(a);
}

// Registers capped at REGS per thread directly.  (Registers are allocated per
// SM sub-partition, 4 x 16K, a warp at a time: at 80 registers 4 blocks of 5
// warps fit per SM, 5 would need 72 or fewer.  Measured: a 72-register form,
// with the next item loaded late to avoid spills, ran 5 blocks per SM and was
// no faster.)
template <int NTC, int SLOTS, int REGS, int CH, bool INV>
__global__ void __maxnreg__(REGS) fft_ragged_slot_kernel_capped(RaggedArgs a) {
    pdl_enter();
    ragged_slot_body<NTC, SLOTS, 5, CH, INV>(a);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

template <int V0>
struct RaggedHost {
    // V0 & 1 is the schedule set; variants 2 and 3 use only kernel()
    static int signals_per_tile(int L) {
        constexpr int V = V0 & 1;
        switch (L) {
#define GBFFT_RS(L) \
    case L: return RCfg<V, L>::type::S;
            GBFFT_RS(1) GBFFT_RS(2) GBFFT_RS(3) GBFFT_RS(4) GBFFT_RS(5) GBFFT_RS(6)
            GBFFT_RS(7) GBFFT_RS(8) GBFFT_RS(9) GBFFT_RS(10) GBFFT_RS(11)
#undef GBFFT_RS
        }
        return 0;
    }
    // twiddle table of length 2^L's schedule (same layout as the uniform path)
    static int twiddles(int L) {
        constexpr int V = V0 & 1;
        switch (L) {
#define GBFFT_RT(L) \
    case L: return RCfg<V, L>::type::kTwiddles;
            GBFFT_RT(1) GBFFT_RT(2) GBFFT_RT(3) GBFFT_RT(4) GBFFT_RT(5) GBFFT_RT(6)
            GBFFT_RT(7) GBFFT_RT(8) GBFFT_RT(9) GBFFT_RT(10) GBFFT_RT(11)
#undef GBFFT_RT
        }
        return 0;
    }
    template <class C>
    static void fill(float* host) {
        for (int s = 1; s < C::M; ++s) {
            const int R = C::radix(s), Ns = C::ns(s);
            for (int r = 1; r < R; ++r)
                for (int m = 0; m < Ns; ++m) {
                    const int64_t idx = C::tw_off(s) + (int64_t)(r - 1) * Ns + m;
                    fft_twiddle_fp32((int64_t)Ns * R, (int64_t)m * r, host + 2 * idx);
                }
        }
    }
    static void fill_twiddles(int L, float* host) {
        constexpr int V = V0 & 1;
        switch (L) {
#define GBFFT_RF(L) \
    case L: fill<typename RCfg<V, L>::type>(host); break;
            GBFFT_RF(1) GBFFT_RF(2) GBFFT_RF(3) GBFFT_RF(4) GBFFT_RF(5) GBFFT_RF(6)
            GBFFT_RF(7) GBFFT_RF(8) GBFFT_RF(9) GBFFT_RF(10) GBFFT_RF(11)
#undef GBFFT_RF
        }
    }
    static const void* kernel(bool inv) {
        return inv ? reinterpret_cast<const void*>(&fft_ragged_kernel<V0, true>)
                   : reinterpret_cast<const void*>(&fft_ragged_kernel<V0, false>);
    }
};

// The schedule set a variant's kernel runs: bit 0 of variants 0..3; the ring
// variant runs set 1.  Work list, tile sizes and twiddle tables must follow it.
int schedule_set(int v) { return v == kRingVariant ? 1 : is_producer_variant(v) ? 0 : (v & 1); }
// compute threads per block of a producer variant (0 for the others) and its ring slots
int producer_group(int v) { return v == 5 ? 256 : is_producer_variant(v) ? 128 : 0; }
int producer_slots(int v) { return v == 7 ? 3 : 2; }
int ragged_threads(int v) { return is_producer_variant(v) ? producer_group(v) + 32 : kRaggedThreads; }

int signals_per_tile(int v, int L) {
    const int s = schedule_set(v) == 0 ? RaggedHost<0>::signals_per_tile(L) : RaggedHost<1>::signals_per_tile(L);
    return is_producer_variant(v) ? s * producer_group(v) / kRaggedThreads : s;  // as SlotCfg<NTC, L>
}
int twiddle_count(int v, int L) {
    return schedule_set(v) == 0 ? RaggedHost<0>::twiddles(L) : RaggedHost<1>::twiddles(L);
}
void fill_twiddles(int v, int L, float* host) {
    if (schedule_set(v) == 0)
        RaggedHost<0>::fill_twiddles(L, host);
    else
        RaggedHost<1>::fill_twiddles(L, host);
}
const void* ragged_kernel(int v, bool inv) {
    switch (v) {
        case 0: return RaggedHost<0>::kernel(inv);
        case 1: return RaggedHost<1>::kernel(inv);
        case 2: return RaggedHost<2>::kernel(inv);
        case 3: return RaggedHost<3>::kernel(inv);
        case 5:
            return inv ? reinterpret_cast<const void*>(&fft_ragged_slot_kernel<256, 2, 2, true>)
                       : reinterpret_cast<const void*>(&fft_ragged_slot_kernel<256, 2, 2, false>);
        case 6:
            return inv ? reinterpret_cast<const void*>(&fft_ragged_slot_kernel<128, 2, 4, true>)
                       : reinterpret_cast<const void*>(&fft_ragged_slot_kernel<128, 2, 4, false>);
        case 7:
            return inv ? reinterpret_cast<const void*>(&fft_ragged_slot_kernel<128, 3, 4, true>)
                       : reinterpret_cast<const void*>(&fft_ragged_slot_kernel<128, 3, 4, false>);
        case 8:
        case 9:
            return inv ? reinterpret_cast<const void*>(&fft_ragged_slot_kernel_capped<128, 2, 80, 0, true>)
                       : reinterpret_cast<const void*>(&fft_ragged_slot_kernel_capped<128, 2, 80, 0, false>);
        default:
            return inv ? reinterpret_cast<const void*>(&fft_ragged_ring_kernel<true>)
                       : reinterpret_cast<const void*>(&fft_ragged_ring_kernel<false>);
    }
}
int ragged_smem(int v) {
    if (v == kRingVariant) return 4 * kRingTile * (int)sizeof(float2) + 16;
    if (is_producer_variant(v)) return producer_slots(v) * producer_group(v) * 17 * (int)sizeof(float2) + 2 * producer_slots(v) * 8;
    return schedule_set(v) == 0 ? ragged_smem_bytes<0>() : ragged_smem_bytes<1>();
}

}  // namespace

struct RaggedState {
    int variant = 0;
    bool inverse = false;
    int scale_mode = 0;
    int64_t count = 0;
    int64_t begin = 0, end = 0;  // element range covered by the signals
    int n_items = 0;
    int64_t grid = 0;
    int smem = 0;
    void* dmem = nullptr;
    RaggedArgs args{};
    int bucket_signals[GBFFT_MAX_LOG2N + 1] = {};
};

int ragged_variant_count() { return kRaggedVariants; }

bool ragged_set_default_variant(int v) {
    if (v < 0 || v >= kRaggedVariants) return false;
    g_default_ragged_variant.store(v);
    return true;
}

int ragged_get_default_variant() { return g_default_ragged_variant.load(); }

void ragged_set_wait_limit(RaggedState* st, uint64_t ns) { st->args.wait_ns = ns; }

bool ragged_waits_on_device(const RaggedState* st) { return st->variant >= kRingVariant; }

fft_status_t ragged_create(const int64_t* offsets, int64_t count, int direction, uint32_t flags,
                           RaggedState** out, int64_t* grid_out) {
    if (count < 0 || (count > 0 && !offsets)) return FFT_ERR_INVALID_VALUE;
    if (count > (int64_t)1 << 31) return FFT_ERR_INVALID_VALUE;
    int variant = (int)((flags & FFT_FLAG_VARIANT_MASK) >> 8) - 1;
    if (variant < 0) variant = g_default_ragged_variant.load();
    if (variant >= kRaggedVariants) return FFT_ERR_INVALID_VALUE;
    if (offsets && (offsets[0] < 0 || (offsets[0] & 1))) return FFT_ERR_MISALIGNED;
    std::vector<std::vector<int64_t>> buckets(GBFFT_MAX_LOG2N + 1);
    for (int64_t i = 0; i < count; ++i) {
        const int64_t n = offsets[i + 1] - offsets[i];
        if (n < 2 || n > 2048 || (n & (n - 1)) != 0) return FFT_ERR_INVALID_SIZE;
        int L = 0;
        while ((int64_t(1) << L) < n) ++L;
        buckets[L].push_back(offsets[i]);
    }
    RaggedState* st = new (std::nothrow) RaggedState();
    if (!st) return FFT_ERR_ALLOC;
    st->variant = variant;
    st->inverse = direction == FFT_INVERSE;
    st->scale_mode = st->inverse ? !(flags & FFT_FLAG_UNNORMALIZED) : (flags & FFT_FLAG_SCALE_FORWARD) != 0;
    st->count = count;
    st->begin = count > 0 ? offsets[0] : 0;
    st->end = count > 0 ? offsets[count] : 0;

    // work list and the bucketed offsets.  Longest length first, so that the
    // last items, which run while the machine drains, are short; variant 9
    // takes the lengths up to 128 (tiles of many short signals, one bulk copy
    // each) first instead, then the rest longest first, so the final items
    // are the N = 256 tiles (8 signals each).  (The named barriers of the producer
    // variants allow any order, see slot_sync.)
    std::vector<int> order;
    const bool short_first = variant >= kShortFirstVariant;
    if (short_first)
        for (int L = GBFFT_MIN_LOG2N; L <= kShortMaxLog2n; ++L) order.push_back(L);
    for (int L = GBFFT_MAX_LOG2N; L >= GBFFT_MIN_LOG2N; --L)
        if (!short_first || L > kShortMaxLog2n) order.push_back(L);
    std::vector<RaggedItem> items;
    std::vector<int64_t> sig;
    sig.reserve((size_t)count);
    int tw_total = 0;
    int tw_off[GBFFT_MAX_LOG2N + 1] = {};
    for (const int L : order) {
        st->bucket_signals[L] = (int)buckets[L].size();
        if (buckets[L].empty()) continue;
        tw_off[L] = tw_total;
        tw_total += twiddle_count(variant, L);
        const int S = signals_per_tile(variant, L);
        // a tile must fit the kernel
        if (S < 1 || (variant == kRingVariant && (int64_t)S << L > kRingTile) ||
            (is_producer_variant(variant) && (int64_t)S << L > (int64_t)producer_group(variant) * 16)) {
            delete st;
            return FFT_ERR_UNSUPPORTED;
        }
        for (size_t k = 0; k < buckets[L].size(); k += S) {
            RaggedItem it;
            it.log2n = L;
            it.count = (int)std::min<size_t>(S, buckets[L].size() - k);
            it.first = (int)(sig.size() + k);
            it.off0 = buckets[L][k];
            it.contig = 1;
            for (int j = 1; j < it.count; ++j)
                if (buckets[L][k + j] != it.off0 + ((int64_t)j << L)) it.contig = 0;
            items.push_back(it);
        }
        sig.insert(sig.end(), buckets[L].begin(), buckets[L].end());
    }
    st->n_items = (int)items.size();

    // one device allocation: counter | items | offsets | twiddles
    const size_t off_items = 256;
    const size_t off_sig = off_items + ((items.size() * sizeof(RaggedItem) + 255) / 256) * 256;
    const size_t off_tw = off_sig + ((sig.size() * sizeof(int64_t) + 255) / 256) * 256;
    const size_t bytes = off_tw + (size_t)tw_total * sizeof(float2) + 16;
    if (plan_malloc(&st->dmem, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete st;
        return FFT_ERR_ALLOC;
    }
    std::vector<unsigned char> host(bytes, 0);
    if (!items.empty()) memcpy(host.data() + off_items, items.data(), items.size() * sizeof(RaggedItem));
    if (!sig.empty()) memcpy(host.data() + off_sig, sig.data(), sig.size() * sizeof(int64_t));
    for (int L = GBFFT_MIN_LOG2N; L <= GBFFT_MAX_LOG2N; ++L)
        if (!buckets[L].empty() && twiddle_count(variant, L) > 0)
            fill_twiddles(variant, L, reinterpret_cast<float*>(host.data() + off_tw) + 2 * tw_off[L]);
    if (cudaMemcpy(st->dmem, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(st->dmem);
        delete st;
        return FFT_ERR_CUDA;
    }
    char* base = static_cast<char*>(st->dmem);
    st->args.counter = reinterpret_cast<unsigned int*>(base);
    st->args.items = reinterpret_cast<const RaggedItem*>(base + off_items);
    st->args.n_items = st->n_items;
    st->args.sig_off = reinterpret_cast<const int64_t*>(base + off_sig);
    st->args.tw = reinterpret_cast<const float2*>(base + off_tw);
    for (int L = 0; L <= GBFFT_MAX_LOG2N; ++L) st->args.tw_off[L] = tw_off[L];
    st->args.scale_mode = st->scale_mode;
    st->args.err = reinterpret_cast<int*>(base + 16);
    st->args.wait_ns = 4000000000ull;
    st->args.stall = (flags & FFT_FLAG_TEST_STALL) ? 1 : 0;

    // launch shape: persistent, every SM filled
    const void* k = ragged_kernel(variant, st->inverse);
    st->smem = ragged_smem(variant);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        (st->smem > 48 * 1024 &&
         cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, st->smem) != cudaSuccess) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, ragged_threads(variant), st->smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        cudaFree(st->dmem);
        delete st;
        return FFT_ERR_CUDA;
    }
    const int64_t resident = (int64_t)sms * per_sm;
    st->grid = st->n_items < resident ? st->n_items : resident;
    if (st->grid < 1) st->grid = 1;
    *out = st;
    *grid_out = st->grid;
    return FFT_OK;
}

fft_status_t ragged_execute(RaggedState* st, const void* in, void* out, void* stream) {
    if (st->count == 0) return FFT_OK;
    if (!in || !out) return FFT_ERR_INVALID_VALUE;
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return FFT_ERR_MISALIGNED;
    const uintptr_t lo = 8 * (uintptr_t)st->begin, hi = 8 * (uintptr_t)st->end;
    const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
    if (a != b && a + lo < b + hi && b + lo < a + hi) return FFT_ERR_OVERLAP;
    cudaStream_t s = (cudaStream_t)stream;
    // only the work-counter variants (bit 1 clear, not the ring) read the counter
    const bool uses_counter = st->variant < kRingVariant && ((st->variant >> 1) & 1) == 0;
    if (uses_counter && cudaMemsetAsync(st->args.counter, 0, sizeof(unsigned int), s) != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_CUDA;
    }
    RaggedArgs args = st->args;
    args.in = static_cast<const float2*>(in);
    args.out = static_cast<float2*>(out);
    void* kargs[] = {&args};
    if (launch_kernel(ragged_kernel(st->variant, st->inverse), (unsigned)st->grid,
                      (unsigned)ragged_threads(st->variant), kargs, (size_t)st->smem, s,
                      st->end - st->begin) != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_CUDA;
    }
    return FFT_OK;
}

void ragged_info(const RaggedState* st, fft_plan_info_t* info) {
    info->batch = st->count;
    info->variant = st->variant;
    info->threads_per_block = ragged_threads(st->variant);
    info->smem_bytes = st->smem;
    info->grid = st->grid;
    info->kernel_kind = 3;
    info->num_stages = 0;
    info->elems_per_thread = schedule_set(st->variant) == 0 ? 16 : 8;
    info->work_items = st->n_items;
}

int* ragged_error_word(RaggedState* st) { return st->args.err; }

void ragged_destroy(RaggedState* st) {
    if (!st) return;
    if (st->dmem) cudaFree(st->dmem);
    delete st;
}

}  // namespace gbfft
