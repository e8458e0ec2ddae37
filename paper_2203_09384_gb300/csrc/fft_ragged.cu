// Ragged batches: signals of mixed power-of-two lengths, packed back to back
// with an offset table, transformed by ONE persistent launch.
//
// Plan time (host): signals are bucketed by length; every bucket is cut into
// tiles of S_N signals (the same per-length schedules as the uniform path,
// re-shaped so that every length runs in a 256-thread block), and the tiles
// become a device work list ordered from the longest length down.  Execute:
// a memset node clears the work counter, then the kernel's blocks pull work
// items with one atomicAdd each until the list is exhausted.  Both steps are
// stream-ordered, so the pair can be captured in a CUDA graph.
//
// Two schedule variants are compiled: V0 keeps 16 complex elements per thread
// for N >= 32 (fewest exchanges), V1 keeps 8 (fewer registers, more resident
// blocks, finer tiles).  The autotuner picks between them per workload.
#include <cuda_runtime.h>

#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/gbfft.h"
#include "fft_device.cuh"
#include "registry.h"
#include "schedules.h"

namespace gbfft {

struct RaggedItem {
    int log2n;
    int count;  // signals in this tile (<= S of the length's schedule)
    int first;  // index of the tile's first signal in the bucketed offset list
    int pad;
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

constexpr int kRaggedVariants = 2;
constexpr int kRaggedThreads = 256;
template <int V>
struct RaggedMinBlocks {
    static constexpr int value = V == 0 ? 2 : 3;
};

template <int V>
constexpr int ragged_smem_bytes() {
    int m = 0;
#define GBFFT_RSMEM(L) m = m > RCfg<V, L>::type::kSmemElems * 8 ? m : RCfg<V, L>::type::kSmemElems * 8;
    GBFFT_RSMEM(1) GBFFT_RSMEM(2) GBFFT_RSMEM(3) GBFFT_RSMEM(4) GBFFT_RSMEM(5) GBFFT_RSMEM(6)
    GBFFT_RSMEM(7) GBFFT_RSMEM(8) GBFFT_RSMEM(9) GBFFT_RSMEM(10) GBFFT_RSMEM(11)
#undef GBFFT_RSMEM
    return m;
}

template <class C, bool INV>
__device__ __forceinline__ void ragged_tile(const RaggedArgs& a, const RaggedItem& w, float2* smem) {
    const int tid = threadIdx.x;
    const int sl = tid / C::T;
    const int t = tid % C::T;
    const bool active = sl < w.count;
    const int64_t off = active ? a.sig_off[w.first + sl] : 0;
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

template <int V, bool INV>
__global__ void __launch_bounds__(kRaggedThreads, RaggedMinBlocks<V>::value) fft_ragged_kernel(RaggedArgs a) {
    extern __shared__ __align__(16) float2 smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();  // everyone has read s_item before the next fetch
        if (it >= a.n_items) break;
        const RaggedItem w = a.items[it];
        switch (w.log2n) {
#define GBFFT_RCASE(L) \
    case L: ragged_tile<typename RCfg<V, L>::type, INV>(a, w, smem); break;
            GBFFT_RCASE(1) GBFFT_RCASE(2) GBFFT_RCASE(3) GBFFT_RCASE(4) GBFFT_RCASE(5) GBFFT_RCASE(6)
            GBFFT_RCASE(7) GBFFT_RCASE(8) GBFFT_RCASE(9) GBFFT_RCASE(10) GBFFT_RCASE(11)
#undef GBFFT_RCASE
            default: break;
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

template <int V>
struct RaggedHost {
    static int signals_per_tile(int L) {
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
        switch (L) {
#define GBFFT_RF(L) \
    case L: fill<typename RCfg<V, L>::type>(host); break;
            GBFFT_RF(1) GBFFT_RF(2) GBFFT_RF(3) GBFFT_RF(4) GBFFT_RF(5) GBFFT_RF(6)
            GBFFT_RF(7) GBFFT_RF(8) GBFFT_RF(9) GBFFT_RF(10) GBFFT_RF(11)
#undef GBFFT_RF
        }
    }
    static const void* kernel(bool inv) {
        return inv ? reinterpret_cast<const void*>(&fft_ragged_kernel<V, true>)
                   : reinterpret_cast<const void*>(&fft_ragged_kernel<V, false>);
    }
};

int signals_per_tile(int v, int L) { return v == 0 ? RaggedHost<0>::signals_per_tile(L) : RaggedHost<1>::signals_per_tile(L); }
int twiddle_count(int v, int L) { return v == 0 ? RaggedHost<0>::twiddles(L) : RaggedHost<1>::twiddles(L); }
void fill_twiddles(int v, int L, float* host) {
    if (v == 0)
        RaggedHost<0>::fill_twiddles(L, host);
    else
        RaggedHost<1>::fill_twiddles(L, host);
}
const void* ragged_kernel(int v, bool inv) { return v == 0 ? RaggedHost<0>::kernel(inv) : RaggedHost<1>::kernel(inv); }
int ragged_smem(int v) { return v == 0 ? ragged_smem_bytes<0>() : ragged_smem_bytes<1>(); }

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

fft_status_t ragged_create(const int64_t* offsets, int64_t count, int direction, uint32_t flags,
                           RaggedState** out, int64_t* grid_out) {
    if (count < 0 || (count > 0 && !offsets)) return FFT_ERR_INVALID_VALUE;
    if (count > (int64_t)1 << 31) return FFT_ERR_INVALID_VALUE;
    int variant = (int)((flags & FFT_FLAG_VARIANT_MASK) >> 8) - 1;
    if (variant < 0) variant = 0;
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

    // work list (longest length first) and the bucketed offsets
    std::vector<RaggedItem> items;
    std::vector<int64_t> sig;
    sig.reserve((size_t)count);
    int tw_total = 0;
    int tw_off[GBFFT_MAX_LOG2N + 1] = {};
    for (int L = GBFFT_MAX_LOG2N; L >= GBFFT_MIN_LOG2N; --L) {
        st->bucket_signals[L] = (int)buckets[L].size();
        if (buckets[L].empty()) continue;
        tw_off[L] = tw_total;
        tw_total += twiddle_count(variant, L);
        const int S = signals_per_tile(variant, L);
        for (size_t k = 0; k < buckets[L].size(); k += S) {
            RaggedItem it;
            it.log2n = L;
            it.count = (int)std::min<size_t>(S, buckets[L].size() - k);
            it.first = (int)(sig.size() + k);
            it.pad = 0;
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
    if (cudaMalloc(&st->dmem, bytes) != cudaSuccess) {
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

    // launch shape: persistent, every SM filled
    const void* k = ragged_kernel(variant, st->inverse);
    st->smem = ragged_smem(variant);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        (st->smem > 48 * 1024 &&
         cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, st->smem) != cudaSuccess) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kRaggedThreads, st->smem) != cudaSuccess ||
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
    if (cudaMemsetAsync(st->args.counter, 0, sizeof(unsigned int), s) != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_CUDA;
    }
    RaggedArgs args = st->args;
    args.in = static_cast<const float2*>(in);
    args.out = static_cast<float2*>(out);
    void* kargs[] = {&args};
    if (cudaLaunchKernel(ragged_kernel(st->variant, st->inverse), dim3((unsigned)st->grid), dim3(kRaggedThreads),
                         kargs, (size_t)st->smem, s) != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_CUDA;
    }
    return FFT_OK;
}

void ragged_info(const RaggedState* st, fft_plan_info_t* info) {
    info->batch = st->count;
    info->variant = st->variant;
    info->threads_per_block = kRaggedThreads;
    info->smem_bytes = st->smem;
    info->grid = st->grid;
    info->kernel_kind = 3;
    info->num_stages = 0;
    info->elems_per_thread = st->variant == 0 ? 16 : 8;
    info->work_items = st->n_items;
}

void ragged_destroy(RaggedState* st) {
    if (!st) return;
    if (st->dmem) cudaFree(st->dmem);
    delete st;
}

}  // namespace gbfft
