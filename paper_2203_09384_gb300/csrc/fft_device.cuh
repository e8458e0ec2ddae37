// Device code of the batched FP32 C2C power-of-two FFT (sm_103a).
//
// The transform is Eq. (dft) of Pascuzzi & Goli (Sec. 3); the inverse,
// Eq. (idft), is taken as conj(DFT(conj(x))) times 1/N, so one forward
// butterfly set and one twiddle table serve both directions.
//
// Algorithm: Stockham autosort decimation in time, mixed radix 2/4/8/16
// (Sec. 3.1 radix-2 split generalised to the higher radices the paper's
// Sec. 4 lists).  With stage radices R_0..R_{M-1} and Ns = R_0*...*R_{s-1},
// stage s performs N/R butterflies; butterfly j
//   reads   a_r = x[j + r*N/R]                                (r < R)
//   twists  a_r *= omega_{Ns*R}^{(j mod Ns)*r}
//   applies the R-point DFT  b_q = sum_r a_r omega_R^{rq}
//   writes  y[(j div Ns)*Ns*R + (j mod Ns) + q*Ns] = b_q      (q < R)
// and the last stage leaves the result in natural order (no bit reversal).
//
// GB300 mapping: each thread keeps E complex elements in registers and runs
// E/R butterflies per stage.  Stage 0 reads straight from HBM and the last
// stage writes straight to HBM, with 128-bit accesses whenever a thread owns
// two neighbouring butterflies; stages exchange through shared memory with an
// XOR swizzle (conflict free for N = 128, 256, 1024, 2048; 1.25x the minimum
// wavefronts at N = 512 and 1.5x at N = 32 and 64, where HBM still bounds the
// kernel).  A persistent grid-stride loop walks tiles of S signals.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace gbfft {

// ---------------------------------------------------------------------------
// complex helpers (float2 = interleaved complex64)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// (x + iy) * (-i) = y - ix
__device__ __forceinline__ float2 mul_neg_i(float2 a) { return make_float2(a.y, -a.x); }
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

// Roots of unity used inside the radix-8 and radix-16 butterflies:
// cos(pi/4), cos(pi/8), sin(pi/8).
constexpr float kSqrtHalf = 0.70710678118654752440f;
constexpr float kCos8 = 0.92387953251128675613f;
constexpr float kSin8 = 0.38268343236508977173f;

// omega_8 * a = sqrt(1/2) (1 - i) a
__device__ __forceinline__ float2 mul_w8_1(float2 a) {
    return make_float2(kSqrtHalf * (a.x + a.y), kSqrtHalf * (a.y - a.x));
}
// omega_8^3 * a = sqrt(1/2) (-1 - i) a
__device__ __forceinline__ float2 mul_w8_3(float2 a) {
    return make_float2(kSqrtHalf * (a.y - a.x), -kSqrtHalf * (a.x + a.y));
}

// ---------------------------------------------------------------------------
// R-point DFTs in registers, in place, natural order in and out:
// v[q] <- sum_r v[r] omega_R^{rq}, omega_R = e^{-2 pi i / R}.
// ---------------------------------------------------------------------------
template <int R>
struct Dft;

template <>
struct Dft<1> {
    static __device__ __forceinline__ void run(float2*) {}
};

template <>
struct Dft<2> {
    static __device__ __forceinline__ void run(float2* v) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <>
struct Dft<4> {
    static __device__ __forceinline__ void run(float2* v) {
        float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        float2 s13 = cadd(v[1], v[3]), d13 = mul_neg_i(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <>
struct Dft<8> {
    // radix-2 split (Eq. (radix2)) over two 4-point DFTs
    static __device__ __forceinline__ void run(float2* v) {
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4>::run(e);
        Dft<4>::run(o);
        o[1] = mul_w8_1(o[1]);
        o[2] = mul_neg_i(o[2]);
        o[3] = mul_w8_3(o[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 4] = csub(e[k], o[k]);
        }
    }
};

template <>
struct Dft<16> {
    // 4 x 4: input index r1 + 4 r2, output index k2 + 4 k1.
    static __device__ __forceinline__ void run(float2* v) {
        float2 y[4][4];
#pragma unroll
        for (int r1 = 0; r1 < 4; ++r1) {
            y[r1][0] = v[r1];
            y[r1][1] = v[r1 + 4];
            y[r1][2] = v[r1 + 8];
            y[r1][3] = v[r1 + 12];
            Dft<4>::run(y[r1]);
        }
        // twiddles omega_16^{r1 k2}
        y[1][1] = cmul(y[1][1], make_float2(kCos8, -kSin8));         // ^1
        y[1][2] = mul_w8_1(y[1][2]);                                 // ^2
        y[1][3] = cmul(y[1][3], make_float2(kSin8, -kCos8));         // ^3
        y[2][1] = mul_w8_1(y[2][1]);                                 // ^2
        y[2][2] = mul_neg_i(y[2][2]);                                // ^4
        y[2][3] = mul_w8_3(y[2][3]);                                 // ^6
        y[3][1] = cmul(y[3][1], make_float2(kSin8, -kCos8));         // ^3
        y[3][2] = mul_w8_3(y[3][2]);                                 // ^6
        y[3][3] = cmul(y[3][3], make_float2(-kCos8, kSin8));         // ^9
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            float2 z[4] = {y[0][k2], y[1][k2], y[2][k2], y[3][k2]};
            Dft<4>::run(z);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) v[k2 + 4 * k1] = z[k1];
        }
    }
};

// cos and sin of pi/16 and 3 pi/16 for the radix-32 butterfly
constexpr float kCos16 = 0.98078528040323044913f;
constexpr float kSin16 = 0.19509032201612826785f;
constexpr float kCos316 = 0.83146961230254523708f;
constexpr float kSin316 = 0.55557023301960222474f;

template <>
struct Dft<32> {
    // radix-2 split (Eq. (radix2)) over two 16-point DFTs; omega_32^k, k < 16
    static __device__ __forceinline__ void run(float2* v) {
        float2 e[16], o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        Dft<16>::run(e);
        Dft<16>::run(o);
        o[1] = cmul(o[1], make_float2(kCos16, -kSin16));
        o[2] = cmul(o[2], make_float2(kCos8, -kSin8));
        o[3] = cmul(o[3], make_float2(kCos316, -kSin316));
        o[4] = mul_w8_1(o[4]);
        o[5] = cmul(o[5], make_float2(kSin316, -kCos316));
        o[6] = cmul(o[6], make_float2(kSin8, -kCos8));
        o[7] = cmul(o[7], make_float2(kSin16, -kCos16));
        o[8] = mul_neg_i(o[8]);
        o[9] = cmul(o[9], make_float2(-kSin16, -kCos16));
        o[10] = cmul(o[10], make_float2(-kSin8, -kCos8));
        o[11] = cmul(o[11], make_float2(-kSin316, -kCos316));
        o[12] = mul_w8_3(o[12]);
        o[13] = cmul(o[13], make_float2(-kCos316, -kSin316));
        o[14] = cmul(o[14], make_float2(-kCos8, -kSin8));
        o[15] = cmul(o[15], make_float2(-kCos16, -kSin16));
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 16] = csub(e[k], o[k]);
        }
    }
};

// ---------------------------------------------------------------------------
// memory helpers: streaming (evict-first) 64/128-bit global accesses
// ---------------------------------------------------------------------------
// Cache hint per schedule (CH): bit 0 set = plain loads instead of
// evict-first (.cs) loads, bit 1 set = plain stores instead of .cs stores.
// Which is faster depends on the length (measured, see the schedule table).
template <int CH>
__device__ __forceinline__ float4 ld_stream4(const float2* p) {
    if constexpr (CH & 1) {
        return *reinterpret_cast<const float4*>(p);
    } else {
        return __ldcs(reinterpret_cast<const float4*>(p));
    }
}
template <int CH>
__device__ __forceinline__ float2 ld_stream2(const float2* p) {
    if constexpr (CH & 1) {
        return *p;
    } else {
        return __ldcs(p);
    }
}
template <int CH>
__device__ __forceinline__ void st_stream4(float2* p, float2 a, float2 b) {
    if constexpr (CH & 2) {
        *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
    } else {
        __stcs(reinterpret_cast<float4*>(p), make_float4(a.x, a.y, b.x, b.y));
    }
}
template <int CH>
__device__ __forceinline__ void st_stream2(float2* p, float2 a) {
    if constexpr (CH & 2) {
        *p = a;
    } else {
        __stcs(p, a);
    }
}
template <int CH>
__device__ __forceinline__ float4 ld_stream4v(const float4* p) {
    if constexpr (CH & 1) {
        return *p;
    } else {
        return __ldcs(p);
    }
}
template <int CH>
__device__ __forceinline__ void st_stream4v(float4* p, float4 a) {
    if constexpr (CH & 2) {
        *p = a;
    } else {
        __stcs(p, a);
    }
}

// Shared-memory swizzle at 8-byte granularity: the 16 elements (128 B) of row
// `row = a >> 4` are XOR-permuted by the row index, for transforms of length
// N = 32 and 64 by row ^ (row >> 2).  By the row alone their exchanges
// (signals starting every 2 or 4 rows) take 1.5x the conflict-free
// wavefronts; with row >> 2 folded in none conflicts.  The other lengths keep
// the cheaper form (measured, the folded one cost the N = 2048 ring kernel
// 1.4 points); their defaults model at 1.0x, except N = 512 (1.25x) and the
// exchanges of the N = 128 padded in-ring default (1.33x).
// tests/test_bank_model.py replays every schedule's exchanges under it and
// counts the wavefronts (64-bit accesses resolve per half-warp), in agreement
// with ncu.
template <int N>
__device__ __forceinline__ int swz8(int a) {
    const int row = a >> 4;
    if constexpr (N == 32 || N == 64) {
        return a ^ ((row ^ (row >> 2)) & 15);
    } else {
        return a ^ (row & 15);
    }
}
// Same idea at 16-byte granularity: the 8 float4 slots of row `row = a >> 3`
// XOR-permuted by the row index, for N = 32 by row ^ (row >> 3) (by the row
// alone, the one-thread-per-signal reads of 32-point signals, 16 slots apart,
// meet 1.5x conflicts; the shorter lengths are conflict free either way).
template <int N>
__device__ __forceinline__ int swz16(int a) {
    const int row = a >> 3;
    if constexpr (N == 32) {
        return a ^ ((row ^ (row >> 3)) & 7);
    } else {
        return a ^ (row & 7);
    }
}

// Programmatic dependent launch.  Every kernel here starts with pdl_enter():
// it lets the next kernel of its stream launch at once (so that its blocks
// are scheduled while this grid drains, instead of after it), then waits
// until the previous kernel of the stream has completed and its memory is
// visible, before touching any buffer.  Both steps are no-ops for a kernel
// launched without programmatic stream serialization.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Bulk copy (TMA, non-tensor form) and mbarrier primitives, inline PTX
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier generic-proxy shared accesses before later
// async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy; completion is signalled on `bar` as tx bytes.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// try_wait with a suspend-time hint: the thread sleeps until the phase
// completes or about hint_ns pass, instead of polling (a polling warp takes
// issue slots from the warps that have work)
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
constexpr uint32_t kSuspendHintNs = 100000;  // 100 us: also the timeout check granularity

// Wait for phase `parity` of `bar` to complete, giving up after limit_ns of
// wall time.  Returns false on timeout (the caller records the error).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait_suspend(bar, parity, kSuspendHintNs)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

// status code written to the plan's error word by a wait that gave up
constexpr int kErrTimeout = 8;
// status code written by a failed device-side check of a GBFFT_DEBUG build
constexpr int kErrDeviceCheck = 9;

// ---------------------------------------------------------------------------
// GBFFT_DEBUG builds (a separate library, for tests): every shared-memory
// exchange index, stage-0 tile read, global element index and twiddle index
// is checked against its buffer; a failed check records FFT_ERR_DEVICE_CHECK
// in the plan's error word (first error wins) and the access is skipped, so
// nothing faults.  And every exchange slot a thread reads is poisoned with NaN
// right after the read: each slot is read once per stage, so a slot the next
// scatter fails to write reaches the output as NaN.  The plan's error word
// reaches the helpers through a block-wide pointer each kernel sets first.
// Release builds compile all of this away.
// ---------------------------------------------------------------------------
#ifdef GBFFT_DEBUG
__shared__ int* g_dbg_err;
__device__ __forceinline__ void dbg_set_err(int* err) {
    if (threadIdx.x == 0) g_dbg_err = err;
    __syncthreads();
}
__device__ __forceinline__ bool dbg_ok(bool cond) {
    if (!cond && g_dbg_err) atomicCAS(g_dbg_err, 0, kErrDeviceCheck);
    return cond;
}
#define GBFFT_DBG_ONLY(...) __VA_ARGS__
#else
__device__ __forceinline__ void dbg_set_err(int*) {}
__device__ __forceinline__ constexpr bool dbg_ok(bool) { return true; }
#define GBFFT_DBG_ONLY(...)
#endif

// Bulk copies that thread 0 issued into ring slots and has not yet seen
// complete (at most one per slot).  A block whose wait gave up stops waiting
// and finishes its loop; before it exits, thread 0 waits (bounded) for these,
// so that no copy lands in shared memory after the block is gone.
struct RingInFlight {
    uint32_t pending = 0;  // bit d: slot d's latest copy not yet seen complete
    uint32_t parity = 0;   // bit d: mbarrier phase parity of that copy
    __device__ __forceinline__ void issued(int d, uint32_t phase_parity) {
        pending |= 1u << d;
        parity = (parity & ~(1u << d)) | ((phase_parity & 1u) << d);
    }
    __device__ __forceinline__ void completed(int d) { pending &= ~(1u << d); }
    __device__ __forceinline__ void drain(uint64_t* bars, uint64_t limit_ns) {
        for (int d = 0; pending != 0 && d < 32; ++d) {
            if (pending & (1u << d)) {
                mbar_wait_bounded(&bars[d], (parity >> d) & 1u, limit_ns);
                pending &= ~(1u << d);
            }
        }
    }
};

// ---------------------------------------------------------------------------
// Compile-time schedule
// ---------------------------------------------------------------------------
template <int LOG2N_, int E_, int S_, int R0, int R1, int R2, int R3, int MINB_ = 1, int PIPE_ = 0, int TC_ = 0,
          int XB_ = 0, int CH_ = 0>
struct Cfg {
    static constexpr int CH = CH_;  // cache hints of the HBM loads / stores
    static constexpr int LOG2N = LOG2N_;
    static constexpr int N = 1 << LOG2N_;
    static constexpr int E = E_;          // complex elements per thread
    static constexpr int S = S_;          // signals per tile (per block)
    static constexpr int T = N / E;       // threads per signal
    static constexpr int NT = T * S;      // threads per block
    static constexpr int MINB = MINB_;    // min resident blocks per SM (launch bounds)
    static constexpr int PIPE = PIPE_;    // 0: direct loads; D: bulk-copy ring of D tiles
    static constexpr int M = (R0 > 0) + (R1 > 0) + (R2 > 0) + (R3 > 0);
    // a signal never spans warps, so exchanges need only warp syncs (the
    // bulk-copy ring refills after a block-wide barrier, so it uses those)
    static constexpr bool kWarpLocal = T <= 32 && PIPE_ == 0;
    // XB = -1 / -2 (bulk-copy ring only): no exchange buffer of its own; every
    // exchange reuses the ring slot the tile arrived in, which is refilled
    // once the next tile's first barrier shows the block is done with it.
    // With -2 the tensor-core A operand lives in that slot too (one more
    // barrier per tensor-core stage, 8 KiB less per block).  Less shared
    // memory, more resident blocks.
    static constexpr bool kInRing = XB_ < 0;
    static constexpr bool kAInRing = XB_ == -2;
    // XB = -3: exchanges in the ring slot and the tensor-core A operand in
    // TMEM (written with tcgen05.st, 16 columns after the accumulators)
    static constexpr bool kAInTmem = XB_ == -3;
    // XB = -5: as -1, with the tile's signals placed every N + T elements of
    // the ring slot (one bulk copy per signal, issued by the lanes of warp 0):
    // stage 0, which reads the slot as the copies wrote it, then meets no
    // bank conflicts (packed, the signals all start on the same banks); the
    // exchanges use the dense layout behind the barrier that follows stage 0
    static constexpr bool kPadSlot = XB_ == -5;
    // exchange buffers: one suffices when a signal stays in one warp; across
    // warps two let one barrier per exchange do (XB = 1 forces one buffer and
    // a second barrier, halving the shared memory of the exchange)
    // XB = 3: no shared memory at all; the one exchange of a two-stage
    // schedule N = R x R with E = R (R lanes per signal) is an R x R transpose
    // across those lanes done with warp shuffles (shuffle_transpose)
    static constexpr bool kShuffle = XB_ == 3;
    static constexpr int kBuffers = kInRing ? 1 : kShuffle ? 0 : XB_ ? XB_ : (kWarpLocal ? 1 : 2);
    static constexpr int kSmemElems = kInRing ? 0 : kBuffers * S * N;  // exchange buffers
    static constexpr int kSlotPad = kPadSlot ? T : 0;             // elements between signals in a slot
    static constexpr int kSlotElems = S * (N + kSlotPad);         // one ring slot
    static constexpr int kRingElems = PIPE * kSlotElems;          // prefetch ring
    // 0: FP32 butterflies; 1 / 2: radix-16 stages on FP16 / BF16 tensor cores;
    // + 4: only the last radix-16 stage on tensor cores (one MMA round trip
    // per tile), the others in FP32
    static constexpr int TC = TC_ & 3;
    static constexpr bool kTcLastOnly = (TC_ & 4) != 0;
    static constexpr int kLast16 = R3 == 16 ? 3 : R2 == 16 ? 2 : R1 == 16 ? 1 : R0 == 16 ? 0 : -1;
    static constexpr int kTcTiles = NT / 128;  // 128-row MMA tiles per radix-16 stage
    // TMEM columns: FP32 accumulators (32 per tile), plus 16 for an A operand
    // kept in TMEM, rounded up to the allocation granularity
    static constexpr int kTcCols = kAInTmem ? 64 : 32 * kTcTiles;
    static constexpr int kTcACol = 32 * kTcTiles;  // first A column (kAInTmem)
    // radix-16 stages on the tensor cores
    static constexpr int kTcStages =
        !TC ? 0 : kTcLastOnly ? (kLast16 >= 0 ? 1 : 0) : (R0 == 16) + (R1 == 16) + (R2 == 16) + (R3 == 16);
    // FP16 dynamic range: a signal spanning warps is scaled once per tile by
    // its own power of two (measured faster there); a signal within one warp
    // scales each butterfly row before its conversion.  BF16: no scale.
    static constexpr bool kTcSignalScale = TC == 1 && T > 32;
    static constexpr bool kTcRowScale = TC == 1 && T <= 32;
    static constexpr int kTcOffset = (((kSmemElems + kRingElems) * 8 + 8 * PIPE) + 127) / 128 * 128;
    // A operand (kTcTiles x 8 KiB, unless it lives in the ring slot), B (2 KiB),
    // the MMA-completion mbarrier and the TMEM address slot
    static constexpr int kTcABytes = (kAInRing || kAInTmem) ? 0 : kTcTiles * 8192;
    static constexpr int kTcBytes = TC ? kTcABytes + 2048 + 128 : 0;
    static constexpr int kSmemBytes = TC ? kTcOffset + kTcBytes : (kSmemElems + kRingElems) * 8 + 8 * PIPE;
    __host__ __device__ static constexpr int radix(int s) {
        return s == 0 ? R0 : s == 1 ? R1 : s == 2 ? R2 : R3;
    }
    // stage s runs on the tensor cores
    __host__ __device__ static constexpr bool tc_stage(int s) {
        return TC != 0 && E == 16 && radix(s) == 16 && (!kTcLastOnly || s == kLast16);
    }
    // Ns of stage s: product of the radices before it
    __host__ __device__ static constexpr int ns(int s) {
        int p = 1;
        for (int i = 0; i < s; ++i) p *= radix(i);
        return p;
    }
    // offset of stage s's twiddles: (R_i - 1) * Ns_i entries for each i in [1, s)
    __host__ __device__ static constexpr int tw_off(int s) {
        int o = 0;
        for (int i = 1; i < s; ++i) o += (radix(i) - 1) * ns(i);
        return o;
    }
    static constexpr int kTwiddles = tw_off(M);
    static_assert(N % E == 0, "E must divide N");
    static_assert(ns(M) == N, "radices must multiply to N");
    static_assert(M >= 1, "at least one stage");
    static_assert(E % R0 == 0 && E % (R1 ? R1 : 1) == 0 && E % (R2 ? R2 : 1) == 0 && E % (R3 ? R3 : 1) == 0,
                  "every radix must divide E");
    static_assert(32 % T == 0 || T % 32 == 0, "T must tile warps");
    static_assert(PIPE == 0 || PIPE >= 2, "the bulk-copy ring needs at least two slots");
    static_assert(!kInRing || PIPE >= 2, "exchanges in the ring slot need the bulk-copy ring");
    static_assert(!kShuffle || (M == 2 && R0 == R1 && E == R0 && T == E && T <= 32 && PIPE == 0 && TC_ == 0),
                  "shuffle exchange: two stages N = R x R, one butterfly of R per thread, R lanes per signal");
    static_assert(!kAInRing || TC == 0 || kTcTiles * 8192 <= S * N * 8, "the A operand must fit in a ring slot");
    static_assert(!kAInTmem || TC == 0 || kTcTiles == 1, "A in TMEM: one 128-row tile per block");
    static_assert(!kPadSlot || (TC_ == 0 && (N + T) % 2 == 0),
                  "padded slots: FP32, every signal on a 16-byte boundary");
    // a signal spanning warps finds its maximum through shared memory after a
    // block barrier, so its first stage cannot be a tensor-core one
    static_assert(!kTcSignalScale || (R0 != 16 && PIPE >= 2 && NT <= 256),
                  "FP16 per-signal scale: signals spanning warps only in ring kernels");
    static_assert(TC == 0 || (E == 16 && NT % 128 == 0 && (kTcCols == 32 || kTcCols == 64 || kTcCols == 128)),
                  "tensor-core radix-16 stages need one 16-point butterfly per thread and 128-row tiles");
};

// ---------------------------------------------------------------------------
// Tensor-core radix-16 stage (tcgen05, FP16 or BF16 operands, FP32 in TMEM)
//
// A batch of 16-point DFTs Y = F X is one real matrix product: row m of A is
// one butterfly's inputs [Re x_0..15, Im x_0..15] (K = 32), and the 32 x 32
// real form of F (stored N x K) gives row m of D = [Re y_0..15, Im y_0..15]:
//   Re y_q = sum_r  c_qr Re x_r + s_qr Im x_r,   Im y_q = sum_r -s_qr Re x_r + c_qr Im x_r,
// with c_qr + i s_qr = e^{+2 pi i qr/16} (so F_qr = c_qr - i s_qr).  A block of
// 128 threads is one M = 128 tile: each thread writes its own row, one thread
// issues the MMA (two K = 16 steps), and after tcgen05.ld each thread holds its
// own butterfly's 16 outputs again.  Operands are in the canonical K-major
// layout without swizzle: 8-row x 16-byte core matrices, 128 B apart along K
// (leading byte offset) and 512 B apart along M/N (stride byte offset).
//
// Dynamic range: BF16 shares FP32's exponent range and a power-of-two scale
// commutes with its rounding, so BF16 operands are converted unscaled.  FP16
// operands are scaled by powers of two: per butterfly row when a signal stays
// in one warp (see tc_dft16), per signal when it spans warps (tc_norm_begin);
// both give each row at least the precision a per-signal scale gives it.
// ---------------------------------------------------------------------------
struct TcCtx {
    uint32_t tmem = 0;   // TMEM base address of the accumulators
    uint32_t phase = 0;  // parity of the next MMA-completion phase
    unsigned char* a = nullptr;
    unsigned char* b = nullptr;
    uint64_t* bar = nullptr;
    int* err = nullptr;
    uint64_t wait_ns = 0;
    int mma_pending = -1;  // thread 0: parity of an MMA phase it gave up waiting for
    int e = 0;             // FP16: the current tile's signal exponent (data scaled by 2^-e)
    float* red = nullptr;  // FP16: per-warp signal maxima (signals spanning warps)
    bool dead = false;     // a bounded wait gave up: stop waiting, issue nothing, finish
    bool stall = false;    // failure-detection test mode: issue no MMA
};

__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
    d |= (uint64_t)(128 >> 4) << 16;                    // leading byte offset: next core matrix along K
    d |= (uint64_t)(512 >> 4) << 32;                    // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                             // descriptor version
    return d;                                           // layout 0: no swizzle
}

template <int TC>
__device__ __forceinline__ uint32_t umma_idesc() {
    constexpr uint32_t fmt = TC == 2 ? 1u : 0u;  // operand type: 0 FP16, 1 BF16
    return (1u << 4)               // accumulate in FP32
           | (fmt << 7) | (fmt << 10)  // A and B type (same type for both)
           | ((32u >> 3) << 17)    // N = 32
           | ((128u >> 4) << 24);  // M = 128; A and B K-major, no negation
}

template <int TC>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    if constexpr (TC == 2) {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}

template <int TC>
__device__ __forceinline__ uint16_t to_bits(float x) {
    if constexpr (TC == 2) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    } else {
        return __half_as_ushort(__float2half_rn(x));
    }
}

// cos and sin of 2 pi m / 16 from the butterfly constants
__device__ __forceinline__ float2 cs16(int m) {
    const float c[5] = {1.0f, kCos8, kSqrtHalf, kSin8, 0.0f};  // cos(2 pi k/16), k = 0..4
    m &= 15;
    const int q = m >> 2, k = m & 3;  // angle = q * pi/2 + k * pi/8
    float cc = c[k], ss = c[4 - k];   // cos, sin of k * pi/8
    switch (q) {
        case 0: return make_float2(cc, ss);
        case 1: return make_float2(-ss, cc);
        case 2: return make_float2(-cc, -ss);
        default: return make_float2(ss, -cc);
    }
}

template <class C>
__device__ __forceinline__ void tc_setup(TcCtx& tc, unsigned char* base, int* err, uint64_t wait_ns) {
    tc.a = base;  // XB = -2 schedules point this at the tile's slot before each use
    tc.b = base + C::kTcABytes;
    tc.bar = reinterpret_cast<uint64_t*>(tc.b + 2048);
    uint32_t* slot = reinterpret_cast<uint32_t*>(tc.b + 2048 + 8);
    tc.red = reinterpret_cast<float*>(tc.b + 2048 + 16);  // NT / 32 <= 8 floats
    tc.err = err;
    tc.wait_ns = wait_ns;
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(C::kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(tc.bar, 1);
        fence_mbar_init();
    }
    // B = real form of F, N x K (K-major)
    for (int i = threadIdx.x; i < 32 * 32; i += C::NT) {
        const int n = i >> 5, k = i & 31;
        const int q = n & 15, r = k & 15;
        const float2 w = cs16(q * r);
        float val;
        if (n < 16) val = k < 16 ? w.x : w.y;  // Re y: c, s
        else val = k < 16 ? -w.y : w.x;        // Im y: -s, c
        if (C::kTcSignalScale) val *= 0.0625f;  // F / 16 (exact): no stage grows the data
        *reinterpret_cast<uint16_t*>(tc.b + (n >> 3) * 512 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) =
            to_bits<C::TC>(val);
    }
    fence_proxy_async_smem();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tc.tmem = *slot;
}

template <class C>
__device__ __forceinline__ void tc_teardown(TcCtx& tc) {
    // an MMA whose completion thread 0 gave up on may still write TMEM: wait
    // for it (bounded) before the columns are freed
    if (threadIdx.x == 0 && tc.mma_pending >= 0) mbar_wait_bounded(tc.bar, (uint32_t)tc.mma_pending, tc.wait_ns);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem), "r"(C::kTcCols)
                     : "memory");
    }
}

// 2^k as a float, k in [-126, 127]
__device__ __forceinline__ float exp2i(int k) { return __uint_as_float((uint32_t)(127 + k) << 23); }

// e with mx = m 2^e, m in [1/2, 1), read off the biased exponent field
// (mx >= 0); clamped to [-120, 126] so that 2^-e and 2^e are normal floats
// (zero and subnormal maxima take -120: any power-of-two scale is exact for
// them).
__device__ __forceinline__ int pow2_exponent(float mx) {
    const int e = (int)(__float_as_uint(mx) >> 23) - 126;
    return e < -120 ? -120 : (e > 126 ? 126 : e);
}

// Every thread of the block calls this with its own butterfly's 16 inputs
// and gets back F x, or F x / 16 when the signal was scaled as a whole
// (kTcSignalScale: B holds F / 16, see tc_norm_begin).  With kTcRowScale the
// row is scaled here by its own power of two 2^-e (exact) before the FP16
// conversion, which keeps every operand in [-1, 1) whatever the signal's
// magnitude, and the FP32 accumulators are multiplied by 2^e after the
// read-back.
template <class C>
__device__ __forceinline__ void tc_dft16(float2* v, TcCtx& tc) {
    const int tid = threadIdx.x;
    const int row = tid & 127;
    float up = 1.0f;
    if constexpr (C::kTcRowScale) {
        float mx = 0.0f;
#pragma unroll
        for (int i = 0; i < 16; ++i) mx = fmaxf(mx, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
        const int e = pow2_exponent(mx);
        const float down = exp2i(-e);
        up = exp2i(e);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = make_float2(v[i].x * down, v[i].y * down);
    }
    // XB = -2 writes A over the slot the inputs were just gathered from:
    // every thread must be done reading it
    if constexpr (C::kAInRing) __syncthreads();
    if constexpr (C::kAInTmem) {
        // row `row` of A in TMEM lane `row`: 16 columns of two 16-bit K values
        // each, K order Re x_0..15, Im x_0..15 (as in the shared-memory layout)
        uint32_t q[16];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            q[i] = pack2<C::TC>(v[2 * i].x, v[2 * i + 1].x);
            q[8 + i] = pack2<C::TC>(v[2 * i].y, v[2 * i + 1].y);
        }
        const uint32_t ta = tc.tmem + ((uint32_t)(((tid >> 5) & 3) * 32) << 16) + C::kTcACol;
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
                ta),
            "r"(q[0]), "r"(q[1]), "r"(q[2]), "r"(q[3]), "r"(q[4]), "r"(q[5]), "r"(q[6]), "r"(q[7]), "r"(q[8]),
            "r"(q[9]), "r"(q[10]), "r"(q[11]), "r"(q[12]), "r"(q[13]), "r"(q[14]), "r"(q[15])
            : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    } else {
        unsigned char* arow = tc.a + (tid >> 7) * 8192 + (row >> 3) * 512 + (row & 7) * 16;
#pragma unroll
        for (int c = 0; c < 4; ++c) {  // K chunk c: Re x_0..7, Re x_8..15, Im x_0..7, Im x_8..15
            const int o = (c & 1) * 8;
            uint4 q;
            if (c < 2) {
                q.x = pack2<C::TC>(v[o + 0].x, v[o + 1].x);
                q.y = pack2<C::TC>(v[o + 2].x, v[o + 3].x);
                q.z = pack2<C::TC>(v[o + 4].x, v[o + 5].x);
                q.w = pack2<C::TC>(v[o + 6].x, v[o + 7].x);
            } else {
                q.x = pack2<C::TC>(v[o + 0].y, v[o + 1].y);
                q.y = pack2<C::TC>(v[o + 2].y, v[o + 3].y);
                q.z = pack2<C::TC>(v[o + 4].y, v[o + 5].y);
                q.w = pack2<C::TC>(v[o + 6].y, v[o + 7].y);
            }
            *reinterpret_cast<uint4*>(arow + c * 128) = q;
        }
        fence_proxy_async_smem();  // make the rows visible to the tensor core
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool issuer = tid == 0 && !tc.stall && !tc.dead;
    if (issuer) {
        const uint32_t idesc = umma_idesc<C::TC>();
        const uint32_t b0 = smem_u32(tc.b);
        if constexpr (C::kAInTmem) {
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {  // K = 16 per step: 8 A columns
                const uint64_t db = umma_smem_desc(b0 + ks * 256);
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tc.tmem),
                    "r"(tc.tmem + C::kTcACol + 8 * ks), "l"(db), "r"(idesc), "r"(ks)
                    : "memory");
            }
        } else {
            const uint32_t a0 = smem_u32(tc.a);
#pragma unroll
            for (int t = 0; t < C::kTcTiles; ++t) {
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t da = umma_smem_desc(a0 + t * 8192 + ks * 256);
                    const uint64_t db = umma_smem_desc(b0 + ks * 256);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tc.tmem + 32 * t),
                        "l"(da), "l"(db), "r"(idesc), "r"(ks)
                        : "memory");
                }
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(tc.bar))
                     : "memory");
    }
    if (!tc.dead && !mbar_wait_bounded(tc.bar, tc.phase, tc.wait_ns)) {
        tc.dead = true;
        if (issuer) tc.mma_pending = (int)tc.phase;
        atomicCAS(tc.err, 0, kErrTimeout);
    }
    tc.phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int warp = tid >> 5;
    const uint32_t taddr = tc.tmem + ((uint32_t)((warp & 3) * 32) << 16) + 32 * (warp >> 2);
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        v[q] = make_float2(__uint_as_float(r[q]), __uint_as_float(r[16 + q]));
        if constexpr (C::kTcRowScale) v[q] = make_float2(v[q].x * up, v[q].y * up);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// FP16 tensor-core stages of signals spanning warps (kTcSignalScale):
// per-signal power-of-two normalisation.  Before its first stage a signal is
// multiplied by 2^-e, e taken from the largest |Re|, |Im| over the whole
// signal, so that component lies in [1/2, 1); with
// B = F / 16 no tensor-core stage can grow the largest modulus
// (|F x|_inf <= 16 |x|_inf) and the FP32 radix-8 stages and twiddles grow it
// by at most 8, so every FP16 operand stays below 8 sqrt(2).  The store
// multiplies by 2^(e + 4k) for k tensor-core stages.  All factors are powers
// of two, so they commute with the FP16 rounding (normal range).
template <class C>
__device__ __forceinline__ void tc_scale(float2 (&v)[C::E], int e) {
    const float down = exp2i(-e);
#pragma unroll
    for (int i = 0; i < C::E; ++i) v[i] = make_float2(v[i].x * down, v[i].y * down);
}

// Step 1, right after a tile's stage-0 inputs are in registers (every thread
// of the block calls it): each warp's maximum with one redux (non-negative
// floats order like their bit patterns), published for step 2.
template <class C>
__device__ __forceinline__ void tc_norm_begin(float2 (&v)[C::E], TcCtx& tc) {
    if constexpr (C::kTcSignalScale) {
        float m = 0.0f;
#pragma unroll
        for (int i = 0; i < C::E; ++i) m = fmaxf(m, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
        m = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m)));
        if ((threadIdx.x & 31) == 0) tc.red[threadIdx.x >> 5] = m;
    }
}

// Step 2: after the block barrier that follows step 1 and before the next
// one, read the signal's warp maxima and scale v.
template <class C>
__device__ __forceinline__ void tc_norm_end(float2 (&v)[C::E], TcCtx& tc) {
    if constexpr (C::kTcSignalScale) {
        constexpr int W = C::T / 32;  // warps per signal
        const float* r = tc.red + (threadIdx.x / C::T) * W;
        float m = r[0];
#pragma unroll
        for (int i = 1; i < W; ++i) m = fmaxf(m, r[i]);
        tc.e = pow2_exponent(m);
        tc_scale<C>(v, tc.e);
    }
}

// The factor the last stage's outputs are stored with: `scale`, times
// 2^(e + 4k) for a signal scaled as a whole; the rare excess beyond the
// normal float range is applied to v here first.
template <class C>
__device__ __forceinline__ float tc_store_factor(float2 (&v)[C::E], const TcCtx& tc, float scale) {
    if constexpr (!C::kTcSignalScale) {
        return scale;
    } else {
        int ex = tc.e + 4 * C::kTcStages;  // in [-120, 126 + 16]
        if (ex > 120) {
            const float hi = exp2i(ex - 120);
#pragma unroll
            for (int i = 0; i < C::E; ++i) v[i] = make_float2(v[i].x * hi, v[i].y * hi);
            ex = 120;
        }
        return scale * exp2i(ex);
    }
}

// Butterfly handled by thread t in slot c of stage s.  The first and the last
// stage give a thread neighbouring butterflies (vectorised HBM access); the
// middle stages interleave threads (coalesced exchanges).
template <class C, int s>
__device__ __forceinline__ int bfly(int t, int c) {
    constexpr int K = C::E / C::radix(s);
    // with the bulk-copy ring, stage 0 reads shared memory: interleave threads
    if constexpr ((s == 0 && C::PIPE == 0) || s == C::M - 1) {
        return K * t + c;
    } else {
        return t + C::T * c;
    }
}

template <class C, int s>
__device__ __forceinline__ void twist_and_dft(float2 (&v)[C::E], int t, const float2* __restrict__ tw, TcCtx& tc) {
    constexpr int R = C::radix(s);
    constexpr int K = C::E / R;
    constexpr int Ns = C::ns(s);
#pragma unroll
    for (int c = 0; c < K; ++c) {
        if constexpr (s > 0) {
            const int j = bfly<C, s>(t, c);
            const float2* twp = tw + C::tw_off(s) + (j & (Ns - 1));
#pragma unroll
            for (int r = 1; r < R; ++r) {
                if (!dbg_ok(C::tw_off(s) + (j & (Ns - 1)) + (r - 1) * Ns < C::kTwiddles)) continue;
                v[c * R + r] = cmul(v[c * R + r], __ldg(twp + (r - 1) * Ns));
            }
        }
        if constexpr (C::tc_stage(s) && K == 1) {
            tc_dft16<C>(&v[0], tc);
        } else {
            Dft<R>::run(&v[c * R]);
        }
    }
}

// stage s outputs -> shared memory (signal base `sb` within the block's buffer)
template <class C, int s>
__device__ __forceinline__ void scatter(const float2 (&v)[C::E], float2* buf, int sb, int t) {
    constexpr int R = C::radix(s);
    constexpr int K = C::E / R;
    constexpr int Ns = C::ns(s);
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const int j = bfly<C, s>(t, c);
        const int base = sb + (j / Ns) * (Ns * R) + (j & (Ns - 1));
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (!dbg_ok(base + q * Ns >= 0 && base + q * Ns < C::S * C::N)) continue;
            buf[swz8<C::N>(base + q * Ns)] = v[c * R + q];
        }
    }
}

// shared memory -> stage s inputs (GBFFT_DEBUG: each slot poisoned once read)
template <class C, int s>
__device__ __forceinline__ void gather(float2 (&v)[C::E], float2* buf, int sb, int t) {
    constexpr int R = C::radix(s);
    constexpr int K = C::E / R;
    constexpr int stride = C::N / R;
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const int j = bfly<C, s>(t, c);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int a = sb + j + r * stride;
            if (!dbg_ok(a >= 0 && a < C::S * C::N)) continue;
            v[c * R + r] = buf[swz8<C::N>(a)];
            GBFFT_DBG_ONLY(buf[swz8<C::N>(a)] = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));)
        }
    }
}

// stage 0 inputs straight from HBM
template <class C, bool INV>
__device__ __forceinline__ void load_first(float2 (&v)[C::E], const float2* src, int t, bool active) {
    constexpr int R = C::radix(0);
    constexpr int K = C::E / R;
    constexpr int stride = C::N / R;
    if (!active) {
#pragma unroll
        for (int i = 0; i < C::E; ++i) v[i] = make_float2(0.f, 0.f);
        return;
    }
    if constexpr (K >= 2) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int c = 0; c < K; c += 2) {
                if (!dbg_ok(K * t + c + r * stride + 1 < C::N)) continue;
                float4 f = ld_stream4<C::CH>(src + K * t + c + r * stride);
                v[c * R + r] = make_float2(f.x, f.y);
                v[(c + 1) * R + r] = make_float2(f.z, f.w);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!dbg_ok(t + r * stride < C::N)) continue;
            v[r] = ld_stream2<C::CH>(src + t + r * stride);
        }
    }
    if constexpr (INV) {
#pragma unroll
        for (int i = 0; i < C::E; ++i) v[i].y = -v[i].y;
    }
}

// last-stage outputs straight to HBM (natural order)
template <class C, bool INV>
__device__ __forceinline__ void store_last(float2 (&v)[C::E], float2* dst, int t, bool active, float scale) {
    constexpr int R = C::radix(C::M - 1);
    constexpr int K = C::E / R;
    constexpr int stride = C::N / R;
    if (!active) return;
    if (scale != 1.0f) {
#pragma unroll
        for (int i = 0; i < C::E; ++i) v[i] = make_float2(v[i].x * scale, (INV ? -v[i].y : v[i].y) * scale);
    } else if constexpr (INV) {
#pragma unroll
        for (int i = 0; i < C::E; ++i) v[i].y = -v[i].y;
    }
    if constexpr (K >= 2) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
#pragma unroll
            for (int c = 0; c < K; c += 2) {
                if (!dbg_ok(K * t + c + q * stride + 1 < C::N)) continue;
                st_stream4<C::CH>(dst + K * t + c + q * stride, v[c * R + q], v[(c + 1) * R + q]);
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (!dbg_ok(t + q * stride < C::N)) continue;
            st_stream2<C::CH>(dst + t + q * stride, v[q]);
        }
    }
}

template <class C>
__device__ __forceinline__ void exchange_barrier() {
    if constexpr (C::kWarpLocal) {
        __syncwarp();
    } else {
        __syncthreads();
    }
}

// The exchange of a two-stage N = R x R schedule (kShuffle) by warp shuffles.
// Thread t of a signal's R lanes holds row t of an R x R matrix (its stage-0
// butterfly's outputs, v[q] = b_q of butterfly t) and needs column t (v[r] =
// b_t of butterfly r, the Stockham read y[t + R r]).  For each lane bit b
// (R/2 down to 1) the two lanes t and t ^ b swap the off-diagonal halves of
// their 2b x 2b block: the lane with bit b clear keeps v[q] and sends v[q|b],
// the lane with bit b set keeps v[q|b] and sends v[q], for every q with bit b
// clear; after log2 R rounds every element sits at its transposed place.
// Register indices are compile-time; the lane's choice is a select.
template <class C>
__device__ __forceinline__ void shuffle_transpose(float2 (&v)[C::E]) {
    constexpr int R = C::E;
    const int t = (int)threadIdx.x & (R - 1);  // R lanes per signal, aligned within the warp
#pragma unroll
    for (int b = R / 2; b >= 1; b >>= 1) {
        const bool hi = (t & b) != 0;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (q & b) continue;
            const int q1 = q | b;
            const float2 send = hi ? v[q] : v[q1];
            float2 got;
            got.x = __shfl_xor_sync(0xffffffffu, send.x, b);
            got.y = __shfl_xor_sync(0xffffffffu, send.y, b);
            if (hi) {
                v[q] = got;
            } else {
                v[q1] = got;
            }
        }
    }
}

// stages 1..M-1: exchange through shared memory (or, for kShuffle, warp
// shuffles), then butterflies
template <class C, int s>
__device__ __forceinline__ void rest_stages(float2 (&v)[C::E], float2* smem, int& buf, int sb, int t,
                                            const float2* __restrict__ tw, TcCtx& tc) {
    if constexpr (s < C::M && C::kShuffle) {
        shuffle_transpose<C>(v);
        twist_and_dft<C, s>(v, t, tw, tc);
    } else if constexpr (s < C::M) {
        float2* b = smem + buf * (C::S * C::N);
        if constexpr (C::kBuffers == 1) {  // previous readers of b are done
            if constexpr (C::kWarpLocal) {
                __syncwarp();
            } else {
                __syncthreads();
            }
        }
        scatter<C, s - 1>(v, b, sb, t);
        exchange_barrier<C>();
        gather<C, s>(v, b, sb, t);
        if constexpr (C::kBuffers == 2) buf ^= 1;
        twist_and_dft<C, s>(v, t, tw, tc);
        rest_stages<C, s + 1>(v, smem, buf, sb, t, tw, tc);
    }
}

// The generic kernel: N = 32..2048.
template <class C, bool INV>
__global__ void __launch_bounds__(C::NT, C::MINB)
    fft_stockham_kernel(const float2* in, float2* out, int64_t batch, const float2* __restrict__ tw, float scale,
                        int* err, uint64_t wait_ns, int stall) {
    pdl_enter();
    extern __shared__ __align__(16) float2 smem[];
    const int tid = threadIdx.x;
    const int sl = tid / C::T;
    const int t = tid % C::T;
    const int sb = sl * C::N;
    const int64_t ntiles = (batch + C::S - 1) / C::S;
    dbg_set_err(err);
    TcCtx tc;
    if constexpr (C::TC != 0) tc_setup<C>(tc, reinterpret_cast<unsigned char*>(smem) + C::kTcOffset, err, wait_ns);
    tc.stall = stall != 0;
    int buf = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t sig = tile * C::S + sl;
        const bool active = sig < batch;
        const int64_t base = sig * C::N;
        float2 v[C::E];
        load_first<C, INV>(v, in + base, t, active);
        twist_and_dft<C, 0>(v, t, tw, tc);
        rest_stages<C, 1>(v, smem, buf, sb, t, tw, tc);
        store_last<C, INV>(v, out + base, t, active && !tc.dead, scale);
    }
    if constexpr (C::TC != 0) tc_teardown<C>(tc);
}

// stage-0 inputs from a dense tile in shared memory (the bulk-copy ring)
template <class C, bool INV>
__device__ __forceinline__ void gather_tile(float2 (&v)[C::E], const float2* tile, int sb, int t) {
    constexpr int R = C::radix(0);
    constexpr int K = C::E / R;
    constexpr int stride = C::N / R;
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const int j = bfly<C, 0>(t, c);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!dbg_ok(sb + j + r * stride < C::kSlotElems)) continue;
            float2 a = tile[sb + j + r * stride];
            v[c * R + r] = INV ? conj2(a) : a;
        }
    }
}

// The generic kernel with a bulk-copy (TMA) prefetch ring: thread 0 keeps
// PIPE tiles in flight from HBM into shared memory, each completion tracked by
// an mbarrier's transaction count, so HBM latency is hidden by copies in
// flight rather than by registers.  A ring slot is refilled as soon as the
// first exchange barrier shows every thread has read it.  Waits are bounded:
// on timeout the kernel records FFT_ERR_TIMEOUT, stops waiting and finishes.
template <class C, bool INV>
__global__ void __launch_bounds__(C::NT, C::MINB)
    fft_stockham_ring_kernel(const float2* in, float2* out, int64_t batch, const float2* __restrict__ tw,
                             float scale, int* err, uint64_t wait_ns, int stall) {
    pdl_enter();
    constexpr int D = C::PIPE;
    constexpr int TILE = C::S * C::N;
    extern __shared__ __align__(16) float2 smem[];
    float2* ring = smem + C::kSmemElems;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + D * TILE);
    const int tid = threadIdx.x;
    const int sl = tid / C::T;
    const int t = tid % C::T;
    const int sb = sl * C::N;
    const int64_t ntiles = (batch + C::S - 1) / C::S;
    dbg_set_err(err);

    RingInFlight inflight;  // thread 0's copies in flight
    // copy the tile of the block's iteration `j` into slot j mod D (thread 0 only)
    auto issue = [&](int64_t j) {
        const int slot = (int)(j % D);
        const int64_t tile = blockIdx.x + j * gridDim.x;
        const int64_t first = tile * C::S;
        const int64_t left = batch - first;
        const uint32_t bytes = (uint32_t)((left < C::S ? left : C::S) * C::N * 8);
        mbar_arrive_expect_tx(&bars[slot], bytes);
        bulk_copy_g2s(ring + slot * TILE, in + first * C::N, bytes, &bars[slot]);
        inflight.issued(slot, (uint32_t)((j / D) & 1));
    };
    if (tid == 0) {
        for (int d = 0; d < D; ++d) mbar_init(&bars[d], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // stall != 0 is the failure-detection test mode: nothing is issued, so
    // every wait below runs out, records FFT_ERR_TIMEOUT and the kernel ends
    if (tid == 0 && !stall) {
        for (int d = 0; d < D; ++d)
            if (blockIdx.x + (int64_t)d * gridDim.x < ntiles) issue(d);
    }
    TcCtx tc;
    if constexpr (C::TC != 0) tc_setup<C>(tc, reinterpret_cast<unsigned char*>(smem) + C::kTcOffset, err, wait_ns);
    tc.stall = stall != 0;
    bool dead = false;
    if (stall) {  // wait for a phase nothing will complete: must give up after wait_ns
        if (!mbar_wait_bounded(&bars[0], 0, wait_ns)) atomicCAS(err, 0, kErrTimeout);
        dead = true;
    }
    int buf = 0;
    int64_t it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int slot = (int)(it % D);
        const uint32_t parity = (uint32_t)((it / D) & 1);
        if (!dead) {
            if (mbar_wait_bounded(&bars[slot], parity, wait_ns)) {
                inflight.completed(slot);
            } else {
                dead = true;
                atomicCAS(err, 0, kErrTimeout);
            }
        }
        const int64_t sig = tile * C::S + sl;
        float2 v[C::E];
        gather_tile<C, INV>(v, ring + slot * TILE, sb, t);
        tc_norm_begin<C>(v, tc);
        twist_and_dft<C, 0>(v, t, tw, tc);
        float2* b = smem + buf * TILE;
        if constexpr (C::kBuffers == 1) __syncthreads();  // previous readers of b are done
        scatter<C, 0>(v, b, sb, t);
        __syncthreads();  // every thread is done with ring[slot]
        if (tid == 0 && !dead && !stall) {
            if (tile + (int64_t)D * gridDim.x < ntiles) {
                fence_proxy_async_smem();
                issue(it + D);
            }
        }
        gather<C, 1>(v, b, sb, t);
        tc_norm_end<C>(v, tc);  // signals spanning warps: maxima published before the barrier
        if constexpr (C::kBuffers == 2) buf ^= 1;
        twist_and_dft<C, 1>(v, t, tw, tc);
        rest_stages<C, 2>(v, smem, buf, sb, t, tw, tc);
        const bool active = sig < batch && !dead && !tc.dead;
        const float f = tc_store_factor<C>(v, tc, scale);
        store_last<C, INV>(v, out + sig * C::N, t, active, f);
    }
    if (tid == 0) inflight.drain(bars, wait_ns);  // copies in flight after a wait gave up
    if constexpr (C::TC != 0) tc_teardown<C>(tc);
}

// Stages 1..M-1 of an in-ring schedule: every exchange goes through the one
// ring slot `b` that holds the tile.  Before a scatter, the block must be done
// reading `b`: after an FP32 stage that takes a barrier; after a tensor-core
// stage it is already so (every thread passed the barrier before the MMA
// after its gather, and the MMA's reads of A ended before its completion
// wait returned).
template <class C, int s>
__device__ __forceinline__ void rest_stages_in_ring(float2 (&v)[C::E], float2* b, int sb, int t,
                                                    const float2* __restrict__ tw, TcCtx& tc) {
    if constexpr (s < C::M) {
        constexpr bool prev_tc = C::tc_stage(s - 1);
        if constexpr (!prev_tc) __syncthreads();
        scatter<C, s - 1>(v, b, sb, t);
        __syncthreads();
        gather<C, s>(v, b, sb, t);
        twist_and_dft<C, s>(v, t, tw, tc);
        rest_stages_in_ring<C, s + 1>(v, b, sb, t, tw, tc);
    }
}

// The bulk-copy ring kernel without exchange buffers of its own (XB = -1):
// a tile arrives in ring slot k by bulk copy (TMA), stage 0 reads it from
// there, and every later exchange (and the tensor-core A operand) reuses slot
// k.  Slot k is refilled at the first barrier of the next tile, when every
// thread is done with it, so the ring runs D-1 tiles ahead.  Shared memory is
// the ring alone (plus the tensor-core B operand), so more blocks fit per SM.
// Waits are bounded as in fft_stockham_ring_kernel.
template <class C, bool INV>
__global__ void __launch_bounds__(C::NT, C::MINB)
    fft_stockham_slot_ring_kernel(const float2* in, float2* out, int64_t batch, const float2* __restrict__ tw,
                                  float scale, int* err, uint64_t wait_ns, int stall) {
    pdl_enter();
    static_assert(C::kInRing, "in-ring schedules only");
    constexpr int D = C::PIPE;
    constexpr int TILE = C::kSlotElems;
    extern __shared__ __align__(16) float2 smem[];
    float2* ring = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + D * TILE);
    const int tid = threadIdx.x;
    const int sl = tid / C::T;
    const int t = tid % C::T;
    const int sb = sl * C::N;
    const int64_t ntiles = (batch + C::S - 1) / C::S;
    dbg_set_err(err);

    RingInFlight inflight;  // thread 0's copies in flight
    // copy the tile of the block's iteration `j` into slot j mod D: thread 0
    // with one copy, or (padded slots) the lanes of warp 0 with one copy per
    // signal after lane 0 has set the byte count
    constexpr int kIssuers = C::kPadSlot ? 32 : 1;
    auto issue = [&](int64_t j) {
        const int slot = (int)(j % D);
        const int64_t tile = blockIdx.x + j * gridDim.x;
        const int64_t first = tile * C::S;
        const int64_t left = batch - first;
        const int nsig = (int)(left < C::S ? left : C::S);
        const uint32_t bytes = (uint32_t)(nsig * C::N * 8);
        if constexpr (C::kPadSlot) {
            const int lane = threadIdx.x & 31;
            if (lane == 0) {
                mbar_arrive_expect_tx(&bars[slot], bytes);
                inflight.issued(slot, (uint32_t)((j / D) & 1));
            }
            __syncwarp();
            for (int q = lane; q < nsig; q += 32)
                bulk_copy_g2s(ring + slot * TILE + q * (C::N + C::kSlotPad), in + (first + q) * C::N,
                              (uint32_t)(C::N * 8), &bars[slot]);
        } else {
            mbar_arrive_expect_tx(&bars[slot], bytes);
            bulk_copy_g2s(ring + slot * TILE, in + first * C::N, bytes, &bars[slot]);
            inflight.issued(slot, (uint32_t)((j / D) & 1));
        }
    };
    if (tid == 0) {
        for (int d = 0; d < D; ++d) mbar_init(&bars[d], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // stall != 0 is the failure-detection test mode: nothing is issued, so
    // every wait below runs out, records FFT_ERR_TIMEOUT and the kernel ends
    if (tid < kIssuers && !stall) {
        for (int d = 0; d < D; ++d)
            if (blockIdx.x + (int64_t)d * gridDim.x < ntiles) issue(d);
    }
    TcCtx tc;
    if constexpr (C::TC != 0) tc_setup<C>(tc, reinterpret_cast<unsigned char*>(smem) + C::kTcOffset, err, wait_ns);
    tc.stall = stall != 0;
    bool dead = false;
    if (stall) {  // wait for a phase nothing will complete: must give up after wait_ns
        if (!mbar_wait_bounded(&bars[0], 0, wait_ns)) atomicCAS(err, 0, kErrTimeout);
        dead = true;
    }
    int64_t it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int slot = (int)(it % D);
        const uint32_t parity = (uint32_t)((it / D) & 1);
        if (!dead) {
            if (mbar_wait_bounded(&bars[slot], parity, wait_ns)) {
                inflight.completed(slot);
            } else {
                dead = true;
                atomicCAS(err, 0, kErrTimeout);
            }
        }
        float2* b = ring + slot * TILE;
        if constexpr (C::kAInRing) tc.a = reinterpret_cast<unsigned char*>(b);
        const int64_t sig = tile * C::S + sl;
        float2 v[C::E];
        gather_tile<C, INV>(v, b, sl * (C::N + C::kSlotPad), t);
        tc_norm_begin<C>(v, tc);
        twist_and_dft<C, 0>(v, t, tw, tc);
        // order this thread's generic accesses of the previous tile's slot
        // before the bulk copy that refills it, then one barrier: every thread
        // is done with that slot and has read this tile's stage-0 inputs
        // (padded slots: before the dense exchanges overwrite them)
        fence_proxy_async_smem();
        __syncthreads();
        if (tid < kIssuers && it > 0 && !stall) {
            bool go = !dead;
            if constexpr (C::kPadSlot) go = __shfl_sync(0xffffffffu, go, 0);  // warp 0 follows lane 0
            if (go && tile + (int64_t)(D - 1) * gridDim.x < ntiles) issue(it - 1 + D);
        }
        tc_norm_end<C>(v, tc);  // signals spanning warps: maxima published before the barrier
        scatter<C, 0>(v, b, sb, t);
        __syncthreads();
        gather<C, 1>(v, b, sb, t);
        twist_and_dft<C, 1>(v, t, tw, tc);
        rest_stages_in_ring<C, 2>(v, b, sb, t, tw, tc);
        const bool active = sig < batch && !dead && !tc.dead;
        const float f = tc_store_factor<C>(v, tc, scale);
        store_last<C, INV>(v, out + sig * C::N, t, active, f);
    }
    if (tid == 0) inflight.drain(bars, wait_ns);  // copies in flight after a wait gave up
    if constexpr (C::TC != 0) tc_teardown<C>(tc);
}

// ---------------------------------------------------------------------------
// N = 2..32: one thread owns a whole signal.  Each warp stages a contiguous
// tile of 32 signals through shared memory with coalesced 128-bit copies, so
// HBM sees fully used sectors while each thread reads its own signal.
// ---------------------------------------------------------------------------
template <int LOG2N, int WARPS, int U = 1, int CH_ = 0>
struct SmallCfg {
    static constexpr int CH = CH_;  // cache hints of the HBM loads / stores
    static constexpr int N = 1 << LOG2N;
    static constexpr int H = N / 2;  // float4 slots per signal
    static constexpr int WARPS_PER_BLOCK = WARPS;
    static constexpr int UNROLL = U;  // 32-signal groups a warp keeps in flight per iteration
    static constexpr int NT = 32 * WARPS;
    static constexpr int kSmemBytes = WARPS * 32 * U * H * 16;
};

// One warp tile = 32*U consecutive signals (contiguous in HBM): loaded with
// coalesced 128-bit copies into the warp's shared-memory slab, then each lane
// transforms U signals of its own, then the slab is stored back the same way.
template <class SC, bool INV>
__global__ void __launch_bounds__(SC::NT) fft_small_kernel(const float2* in, float2* out, int64_t batch,
                                                           float scale) {
    pdl_enter();
    constexpr int N = SC::N, H = SC::H, W = SC::WARPS_PER_BLOCK, U = SC::UNROLL;
    constexpr int TS = 32 * U;  // signals per warp tile
    extern __shared__ __align__(16) float4 smem4[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* sm = smem4 + warp * (TS * H);
    const int64_t wtiles = (batch + TS - 1) / TS;
    for (int64_t wt = (int64_t)blockIdx.x * W + warp; wt < wtiles; wt += (int64_t)gridDim.x * W) {
        const int64_t first = wt * TS;
        const int64_t left = batch - first;
        const int valid4 = (int)((left < TS ? left : TS) * H);
        const float4* src = reinterpret_cast<const float4*>(in + first * N);
        float4* dst = reinterpret_cast<float4*>(out + first * N);
#pragma unroll
        for (int i = 0; i < U * H; ++i) {
            const int p = lane + 32 * i;
            if (p < valid4) sm[swz16<SC::N>(p)] = ld_stream4v<SC::CH>(src + p);
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int sig = u * 32 + lane;
            float2 v[N];
#pragma unroll
            for (int i = 0; i < H; ++i) {
                float4 f = sm[swz16<SC::N>(sig * H + i)];
                v[2 * i] = make_float2(f.x, INV ? -f.y : f.y);
                v[2 * i + 1] = make_float2(f.z, INV ? -f.w : f.w);
            }
            Dft<N>::run(v);
#pragma unroll
            for (int i = 0; i < N; ++i) v[i] = make_float2(v[i].x * scale, (INV ? -v[i].y : v[i].y) * scale);
#pragma unroll
            for (int i = 0; i < H; ++i)
                sm[swz16<SC::N>(sig * H + i)] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < U * H; ++i) {
            const int p = lane + 32 * i;
            if (p < valid4) st_stream4v<SC::CH>(dst + p, sm[swz16<SC::N>(p)]);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// complex32 storage: each element is two IEEE binary16 (re, im) and signal b
// carries a power-of-two exponent, value = stored * 2^exp[b].  The transform
// is linear, so the kernels transform the stored values themselves in FP32
// (|stored| < 2^16, at most N * 2^16 after the transform) and fold the input
// exponent and the 1/N normalisation into the output exponent; one
// power-of-two multiply per component puts each signal's largest output
// component in [2^14, 2^15).
// ---------------------------------------------------------------------------
// binary16 pairs moved as 32-bit words
__device__ __forceinline__ __half2 bits_h2(float x) {
    __half2 h;
    memcpy(&h, &x, 4);
    return h;
}
__device__ __forceinline__ float h2_bits(__half2 h) {
    float x;
    memcpy(&x, &h, 4);
    return x;
}

struct C32Out {
    int e;       // output exponent
    float mult;  // stored output = transform of stored input * mult
};

// m = largest |component| of the signal's unscaled FP32 transform; the
// values carry 2^(ein + ls) (input exponent, log2 of the normalisation).
__device__ __forceinline__ C32Out c32_out_scale(float m, int ein, int ls) {
    if (!(m > 0.0f) || !(m <= 3.0e38f)) return {0, 1.0f};  // zero (or non-finite) signal
    int f = 0;
    frexpf(m, &f);  // m = g 2^f, g in [0.5, 1)
    int e = ein + ls + f - 15;
    e = e < -128 ? -128 : (e > 127 ? 127 : e);  // int8: stored values under/overflow past this
    int k = ein + ls - e;                       // 15 - f unless e was clamped
    k = k < -126 ? -126 : (k > 127 ? 127 : k);
    return {e, __int_as_float((k + 127) << 23)};  // 2^k, a normal binary32
}

// log2 of the power-of-two normalisation factor (1, 1/N)
__device__ __forceinline__ int log2_pow2(float scale) {
    int x = 0;
    frexpf(scale, &x);
    return x - 1;
}

template <class C, bool INV>
__device__ __forceinline__ void load_first_c32(float2 (&v)[C::E], const __half2* src, int t, bool active) {
    constexpr int R = C::radix(0);
    constexpr int K = C::E / R;
    constexpr int stride = C::N / R;
    if (!active) {
#pragma unroll
        for (int i = 0; i < C::E; ++i) v[i] = make_float2(0.f, 0.f);
        return;
    }
    if constexpr (K >= 2) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int c = 0; c < K; c += 2) {
                const float2 raw = __ldcs(reinterpret_cast<const float2*>(src + K * t + c + r * stride));
                v[c * R + r] = __half22float2(bits_h2(raw.x));
                v[(c + 1) * R + r] = __half22float2(bits_h2(raw.y));
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = __half22float2(src[t + r * stride]);
    }
    if constexpr (INV) {
#pragma unroll
        for (int i = 0; i < C::E; ++i) v[i].y = -v[i].y;
    }
}

// Largest |component| of the thread's signal (every thread of the block calls it).
template <class C>
__device__ __forceinline__ float c32_signal_max(const float2 (&v)[C::E], float* red) {
    float m = 0.0f;
#pragma unroll
    for (int i = 0; i < C::E; ++i) m = fmaxf(m, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
    if constexpr (C::T <= 32) {
#pragma unroll
        for (int o = 1; o < C::T; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    } else {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const int warp = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) red[warp] = m;
        __syncthreads();
        constexpr int W = C::T / 32;
        const int w0 = (warp / W) * W;
        m = 0.0f;
#pragma unroll
        for (int w = 0; w < W; ++w) m = fmaxf(m, red[w0 + w]);
    }
    return m;
}

template <class C, bool INV>
__device__ __forceinline__ void store_last_c32(const float2 (&v)[C::E], __half2* dst, int8_t* exp_out, int t,
                                               bool active, C32Out o) {
    constexpr int R = C::radix(C::M - 1);
    constexpr int K = C::E / R;
    constexpr int stride = C::N / R;
    if (!active) return;
    if (t == 0) *exp_out = (int8_t)o.e;
    const float my = INV ? -o.mult : o.mult;
    if constexpr (K >= 2) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
#pragma unroll
            for (int c = 0; c < K; c += 2) {
                const float2 raw =
                    make_float2(h2_bits(__floats2half2_rn(v[c * R + q].x * o.mult, v[c * R + q].y * my)),
                                h2_bits(__floats2half2_rn(v[(c + 1) * R + q].x * o.mult, v[(c + 1) * R + q].y * my)));
                __stcs(reinterpret_cast<float2*>(dst + K * t + c + q * stride), raw);
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < R; ++q) dst[t + q * stride] = __floats2half2_rn(v[q].x * o.mult, v[q].y * my);
    }
}

// Shared memory of the complex32 kernels: FP32 exchange buffers, then (ring
// variants) PIPE binary16 tiles and their mbarriers, then per-warp maxima.
template <class C>
struct C32Smem {
    static constexpr int kRingOffset = C::kSmemElems * 8;
    static constexpr int kBarOffset = kRingOffset + C::PIPE * C::S * C::N * 4;
    static constexpr int kRedOffset = kBarOffset + C::PIPE * 8;
    static constexpr int kBytes = kRedOffset + 128;
};

// Direct loads.  err / wait_ns / stall are accepted so that all complex32
// kernels share one argument list; nothing here waits.
template <class C, bool INV>
__global__ void __launch_bounds__(C::NT, C::MINB)
    fft_stockham_c32_kernel(const __half2* in, const int8_t* in_exp, __half2* out, int8_t* out_exp, int64_t batch,
                            const float2* __restrict__ tw, float scale, int* err, uint64_t wait_ns, int stall) {
    pdl_enter();
    extern __shared__ __align__(16) float2 smem[];
    float* red = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(smem) + C32Smem<C>::kRedOffset);
    const int tid = threadIdx.x;
    const int sl = tid / C::T;
    const int t = tid % C::T;
    const int sb = sl * C::N;
    const int ls = log2_pow2(scale);
    const int64_t ntiles = (batch + C::S - 1) / C::S;
    dbg_set_err(err);
    TcCtx tc;  // FP32 butterflies only
    int buf = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t sig = tile * C::S + sl;
        const bool active = sig < batch;
        const int64_t base = sig * C::N;
        const int ein = active ? (int)in_exp[sig] : 0;
        float2 v[C::E];
        load_first_c32<C, INV>(v, in + base, t, active);
        twist_and_dft<C, 0>(v, t, tw, tc);
        rest_stages<C, 1>(v, smem, buf, sb, t, tw, tc);
        const C32Out o = c32_out_scale(c32_signal_max<C>(v, red), ein, ls);
        store_last_c32<C, INV>(v, out + base, out_exp + sig, t, active, o);
    }
}

// stage-0 inputs of a complex32 signal from its binary16 tile in shared memory
template <class C, bool INV>
__device__ __forceinline__ void gather_tile_c32(float2 (&v)[C::E], const __half2* tile, int sb, int t) {
    constexpr int R = C::radix(0);
    constexpr int K = C::E / R;
    constexpr int stride = C::N / R;
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const int j = bfly<C, 0>(t, c);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 a = __half22float2(tile[sb + j + r * stride]);
            v[c * R + r] = INV ? conj2(a) : a;
        }
    }
}

// complex32 with the bulk-copy ring: thread 0 keeps PIPE binary16 tiles in
// flight as in fft_stockham_ring_kernel, with the same bounded waits and
// error word.
template <class C, bool INV>
__global__ void __launch_bounds__(C::NT, C::MINB)
    fft_stockham_c32_ring_kernel(const __half2* in, const int8_t* in_exp, __half2* out, int8_t* out_exp,
                                 int64_t batch, const float2* __restrict__ tw, float scale, int* err,
                                 uint64_t wait_ns, int stall) {
    pdl_enter();
    constexpr int D = C::PIPE;
    constexpr int TILE = C::S * C::N;
    using SM = C32Smem<C>;
    extern __shared__ __align__(16) float2 smem[];
    unsigned char* base8 = reinterpret_cast<unsigned char*>(smem);
    __half2* ring = reinterpret_cast<__half2*>(base8 + SM::kRingOffset);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base8 + SM::kBarOffset);
    float* red = reinterpret_cast<float*>(base8 + SM::kRedOffset);
    const int tid = threadIdx.x;
    const int sl = tid / C::T;
    const int t = tid % C::T;
    const int sb = sl * C::N;
    const int ls = log2_pow2(scale);
    const int64_t ntiles = (batch + C::S - 1) / C::S;
    dbg_set_err(err);

    RingInFlight inflight;  // thread 0's copies in flight
    // copy the tile of the block's iteration `j` into slot j mod D (thread 0 only)
    auto issue = [&](int64_t j) {
        const int slot = (int)(j % D);
        const int64_t tile = blockIdx.x + j * gridDim.x;
        const int64_t first = tile * C::S;
        const int64_t left = batch - first;
        const uint32_t bytes = (uint32_t)((left < C::S ? left : C::S) * C::N * 4);
        mbar_arrive_expect_tx(&bars[slot], bytes);
        bulk_copy_g2s(ring + slot * TILE, in + first * C::N, bytes, &bars[slot]);
        inflight.issued(slot, (uint32_t)((j / D) & 1));
    };
    if (tid == 0) {
        for (int d = 0; d < D; ++d) mbar_init(&bars[d], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0 && !stall) {
        for (int d = 0; d < D; ++d)
            if (blockIdx.x + (int64_t)d * gridDim.x < ntiles) issue(d);
    }
    TcCtx tc;  // FP32 butterflies only
    bool dead = false;
    if (stall) {  // failure-detection test mode, as in fft_stockham_ring_kernel
        if (!mbar_wait_bounded(&bars[0], 0, wait_ns)) atomicCAS(err, 0, kErrTimeout);
        dead = true;
    }
    int buf = 0;
    int64_t it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int slot = (int)(it % D);
        const uint32_t parity = (uint32_t)((it / D) & 1);
        const int64_t sig = tile * C::S + sl;
        const bool in_range = sig < batch;
        const int ein = in_range ? (int)in_exp[sig] : 0;
        if (!dead) {
            if (mbar_wait_bounded(&bars[slot], parity, wait_ns)) {
                inflight.completed(slot);
            } else {
                dead = true;
                atomicCAS(err, 0, kErrTimeout);
            }
        }
        float2 v[C::E];
        gather_tile_c32<C, INV>(v, ring + slot * TILE, sb, t);
        twist_and_dft<C, 0>(v, t, tw, tc);
        float2* b = smem + buf * TILE;
        if constexpr (C::kBuffers == 1) __syncthreads();  // previous readers of b are done
        scatter<C, 0>(v, b, sb, t);
        __syncthreads();  // every thread is done with ring[slot]
        if (tid == 0 && !dead && !stall) {
            if (tile + (int64_t)D * gridDim.x < ntiles) {
                fence_proxy_async_smem();
                issue(it + D);
            }
        }
        gather<C, 1>(v, b, sb, t);
        if constexpr (C::kBuffers == 2) buf ^= 1;
        twist_and_dft<C, 1>(v, t, tw, tc);
        rest_stages<C, 2>(v, smem, buf, sb, t, tw, tc);
        const C32Out o = c32_out_scale(c32_signal_max<C>(v, red), ein, ls);
        store_last_c32<C, INV>(v, out + sig * C::N, out_exp + sig, t, in_range && !dead, o);
    }
    if (tid == 0) inflight.drain(bars, wait_ns);  // copies in flight after a wait gave up
}

// complex32, N = 2..32: one thread owns a whole signal, as in
// fft_small_kernel.  A warp tile of 32*U signals moves between HBM and the
// warp's shared-memory slab in 128-bit pieces (4 elements each); each lane
// finds its own signal's exponent without any exchange.
template <class SC, bool INV>
__global__ void __launch_bounds__(SC::NT)
    fft_small_c32_kernel(const __half2* in, const int8_t* in_exp, __half2* out, int8_t* out_exp, int64_t batch,
                         const float2* __restrict__ tw, float scale, int* err, uint64_t wait_ns, int stall) {
    pdl_enter();
    constexpr int N = SC::N, W = SC::WARPS_PER_BLOCK, U = SC::UNROLL;
    constexpr int TS = 32 * U;         // signals per warp tile
    constexpr int P = TS * N / 4;      // 128-bit pieces per warp tile
    extern __shared__ __align__(16) float4 smem4[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* sm = smem4 + warp * P;
    const int ls = log2_pow2(scale);
    const int64_t wtiles = (batch + TS - 1) / TS;
    for (int64_t wt = (int64_t)blockIdx.x * W + warp; wt < wtiles; wt += (int64_t)gridDim.x * W) {
        const int64_t first = wt * TS;
        const int64_t left = batch - first;
        const int nsig = (int)(left < TS ? left : TS);
        const int valid_e = nsig * N;          // binary16 pairs in this tile
        const int full = valid_e / 4;          // whole 128-bit pieces
        const float4* src = reinterpret_cast<const float4*>(in + first * N);
        float4* dst = reinterpret_cast<float4*>(out + first * N);
#pragma unroll
        for (int i = 0; i < (P + 31) / 32; ++i) {
            const int p = lane + 32 * i;
            if (p < full) sm[swz16<N>(p)] = ld_stream4v<SC::CH>(src + p);
        }
        if (N == 2 && lane == 0 && (valid_e & 3))  // odd signal count: the last signal is half a piece
            reinterpret_cast<float2*>(sm + swz16<N>(full))[0] =
                *reinterpret_cast<const float2*>(in + first * N + 4 * full);
        __syncwarp();
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int sg = u * 32 + lane;
            const bool act = sg < nsig;
            const int ein = act ? (int)in_exp[first + sg] : 0;
            float2 v[N];
            if constexpr (N >= 4) {
#pragma unroll
                for (int i = 0; i < N / 4; ++i) {
                    const float4 f = sm[swz16<N>(sg * (N / 4) + i)];
                    v[4 * i + 0] = __half22float2(bits_h2(f.x));
                    v[4 * i + 1] = __half22float2(bits_h2(f.y));
                    v[4 * i + 2] = __half22float2(bits_h2(f.z));
                    v[4 * i + 3] = __half22float2(bits_h2(f.w));
                }
            } else {
                const float2 f = reinterpret_cast<const float2*>(sm + swz16<N>(sg >> 1))[sg & 1];
                v[0] = __half22float2(bits_h2(f.x));
                v[1] = __half22float2(bits_h2(f.y));
            }
            if constexpr (INV) {
#pragma unroll
                for (int i = 0; i < N; ++i) v[i].y = -v[i].y;
            }
            Dft<N>::run(v);
            float m = 0.0f;
#pragma unroll
            for (int i = 0; i < N; ++i) m = fmaxf(m, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
            const C32Out o = c32_out_scale(m, ein, ls);
            const float my = INV ? -o.mult : o.mult;
            float hw[N];  // binary16 pairs as 32-bit words
#pragma unroll
            for (int i = 0; i < N; ++i) hw[i] = h2_bits(__floats2half2_rn(v[i].x * o.mult, v[i].y * my));
            if constexpr (N >= 4) {
#pragma unroll
                for (int i = 0; i < N / 4; ++i)
                    sm[swz16<N>(sg * (N / 4) + i)] = make_float4(hw[4 * i], hw[4 * i + 1], hw[4 * i + 2], hw[4 * i + 3]);
            } else {
                reinterpret_cast<float2*>(sm + swz16<N>(sg >> 1))[sg & 1] = make_float2(hw[0], hw[1]);
            }
            if (act) out_exp[first + sg] = (int8_t)o.e;
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < (P + 31) / 32; ++i) {
            const int p = lane + 32 * i;
            if (p < full) st_stream4v<SC::CH>(dst + p, sm[swz16<N>(p)]);
        }
        if (N == 2 && lane == 0 && (valid_e & 3))
            *reinterpret_cast<float2*>(out + first * N + 4 * full) = reinterpret_cast<const float2*>(sm + swz16<N>(full))[0];
        __syncwarp();
    }
}

template <int LOG2N, int WARPS, int U = 1, int CH_ = 0>
struct SmallC32Cfg : SmallCfg<LOG2N, WARPS, U, CH_> {
    static constexpr int kSmemBytes = WARPS * 32 * U * (1 << LOG2N) * 4;
};

}  // namespace gbfft
