// Host side of the C-ABI: argument validation, plan construction (radix
// schedule lookup, FP64 twiddle generation rounded to FP32, launch shape),
// asynchronous execution and error reporting.  See include/gbfft.h.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>

#include "../../include/gbfft.h"
#include "registry.h"
#include "schedules.h"

GBFFT_DECLARE_ENTRIES(1)
GBFFT_DECLARE_ENTRIES(2)
GBFFT_DECLARE_ENTRIES(3)
GBFFT_DECLARE_ENTRIES(4)
GBFFT_DECLARE_ENTRIES(5)
GBFFT_DECLARE_ENTRIES(6)
GBFFT_DECLARE_ENTRIES(7)
GBFFT_DECLARE_ENTRIES(8)
GBFFT_DECLARE_ENTRIES(9)
GBFFT_DECLARE_ENTRIES(10)
GBFFT_DECLARE_ENTRIES(11)

namespace {

using gbfft::KernelEntry;
using gbfft::KernelKind;

struct LengthVariants {
    KernelEntry v[GBFFT_MAX_VARIANTS];
    int count = 0;
    std::atomic<int> preferred{0};  // variant new plans use unless told otherwise
};

LengthVariants* registry() {
    static LengthVariants table[GBFFT_MAX_LOG2N + 1];
    static std::once_flag once;
    std::call_once(once, [] {
        table[1].count = gbfft_entries_1(table[1].v, GBFFT_MAX_VARIANTS);
        table[2].count = gbfft_entries_2(table[2].v, GBFFT_MAX_VARIANTS);
        table[3].count = gbfft_entries_3(table[3].v, GBFFT_MAX_VARIANTS);
        table[4].count = gbfft_entries_4(table[4].v, GBFFT_MAX_VARIANTS);
        table[5].count = gbfft_entries_5(table[5].v, GBFFT_MAX_VARIANTS);
        table[6].count = gbfft_entries_6(table[6].v, GBFFT_MAX_VARIANTS);
        table[7].count = gbfft_entries_7(table[7].v, GBFFT_MAX_VARIANTS);
        table[8].count = gbfft_entries_8(table[8].v, GBFFT_MAX_VARIANTS);
        table[9].count = gbfft_entries_9(table[9].v, GBFFT_MAX_VARIANTS);
        table[10].count = gbfft_entries_10(table[10].v, GBFFT_MAX_VARIANTS);
        table[11].count = gbfft_entries_11(table[11].v, GBFFT_MAX_VARIANTS);
    });
    return table;
}

int ilog2(int64_t n) {
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return l;
}

// Resident blocks per SM from registers, shared memory and threads alone.
// The occupancy API returns 1 for every kernel that allocates tensor memory
// (TMEM); measured on GB300, such kernels do run several blocks per SM, so
// for them the limit is worked out here and then capped by TMEM capacity.
int occupancy_without_tmem(const void* kernel, int threads, int smem_bytes, int dev) {
    cudaFuncAttributes fa;
    int regs_sm = 0, smem_sm = 0, thr_sm = 0, blk_sm = 0, smem_reserved = 0;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int warps = (threads + 31) / 32;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // allocated per warp in 256-register units
    int by_regs = regs_warp > 0 ? regs_sm / (regs_warp * warps) : blk_sm;
    int by_smem = smem_sm / ((int)fa.sharedSizeBytes + smem_bytes + smem_reserved);
    int by_thr = thr_sm / threads;
    int n = by_regs < by_smem ? by_regs : by_smem;
    n = n < by_thr ? n : by_thr;
    return n < blk_sm ? n : blk_sm;
}

constexpr uint32_t kKnownFlags =
    FFT_FLAG_UNNORMALIZED | FFT_FLAG_SCALE_FORWARD | FFT_FLAG_VARIANT_MASK | FFT_FLAG_TEST_STALL |
    FFT_FLAG_HOST_STAGING;
constexpr uint64_t kDefaultWaitNs = 4000000000ull;  // bounded device waits: 4 s

}  // namespace

namespace gbfft {
namespace {
thread_local int t_plan_allocs = 0;
}
void begin_plan_allocs() { t_plan_allocs = 0; }
cudaError_t launch_kernel(const void* kernel, unsigned grid, unsigned block, void** args, size_t smem,
                          cudaStream_t stream, int64_t elems) {
    if (elems < kPdlMinElems) return cudaLaunchKernel(kernel, dim3(grid), dim3(block), args, smem, stream);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, kernel, args);
}

cudaError_t plan_malloc(void** ptr, size_t bytes) {
    ++t_plan_allocs;
    const char* fail = getenv("GBFFT_TEST_FAIL_ALLOC");
    if (fail && atoi(fail) == t_plan_allocs) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

// Registry lookup for other host translation units: the kernel entry of
// `variant` (or of the length's current default when variant < 0), or NULL.
const KernelEntry* lookup_entry(int log2n, int variant) {
    if (log2n < GBFFT_MIN_LOG2N || log2n > GBFFT_MAX_LOG2N) return nullptr;
    LengthVariants* lv = &registry()[log2n];
    if (variant < 0) variant = lv->preferred.load();
    if (variant >= lv->count || !lv->v[variant].kernel_fwd) return nullptr;
    return &lv->v[variant];
}
}  // namespace gbfft

struct gbfft_plan {
    int64_t n = 0, batch = 0;
    int log2n = 0, direction = 0, dtype = 0;
    uint32_t flags = 0;
    int device = -1;
    int sm_count = 0;
    const KernelEntry* entry = nullptr;
    const void* kernel = nullptr;
    float* d_twiddles = nullptr;  // interleaved complex64
    int* d_error = nullptr;
    int64_t grid = 0;
    float scale = 1.0f;
    uint64_t wait_ns = kDefaultWaitNs;
    int64_t resident = 0;                  // blocks that fit on the device at once
    gbfft::RaggedState* ragged = nullptr;  // set for mixed-length plans
    // host-buffer pipeline (FFT_FLAG_HOST_STAGING): device chunk buffers,
    // one stream each, and the events that tie them to the caller's stream
    int stages = 0;
    int64_t chunk_signals = 0;
    float2* d_stage = nullptr;
    cudaStream_t stage_stream[3] = {};
    cudaEvent_t stage_done[3] = {};
    cudaEvent_t stage_start = nullptr;
};

namespace {

// One launch of the plan's kernel over `batch` signals (any batch up to the
// plan's), grid sized for that batch.
fft_status_t launch_plain(gbfft_plan* p, const float2* in2, float2* out2, int64_t batch, cudaStream_t stream) {
    const KernelEntry* e = p->entry;
    const int64_t tiles = (batch + e->signals_per_block - 1) / e->signals_per_block;
    const int64_t grid = tiles < p->resident ? tiles : p->resident;
    const float2* tw = (const float2*)p->d_twiddles;
    float scale = p->scale;
    int* err = p->d_error;
    uint64_t wait_ns = p->wait_ns;
    cudaError_t ce;
    if (e->kind == KernelKind::Small) {
        void* args[] = {&in2, &out2, &batch, &scale};
        ce = gbfft::launch_kernel(p->kernel, (unsigned)grid, (unsigned)e->threads_per_block, args,
                                  (size_t)e->smem_bytes, stream, batch * p->n);
    } else {
        int stall = (p->flags & FFT_FLAG_TEST_STALL) ? 1 : 0;
        void* args[] = {&in2, &out2, &batch, &tw, &scale, &err, &wait_ns, &stall};
        ce = gbfft::launch_kernel(p->kernel, (unsigned)grid, (unsigned)e->threads_per_block, args,
                                  (size_t)e->smem_bytes, stream, batch * p->n);
    }
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_CUDA;
    }
    return FFT_OK;
}

void release_staging(gbfft_plan* p) {
    for (int i = 0; i < 3; ++i) {
        if (p->stage_stream[i]) cudaStreamDestroy(p->stage_stream[i]);
        if (p->stage_done[i]) cudaEventDestroy(p->stage_done[i]);
        p->stage_stream[i] = nullptr;
        p->stage_done[i] = nullptr;
    }
    if (p->stage_start) cudaEventDestroy(p->stage_start);
    if (p->d_stage) cudaFree(p->d_stage);
    p->stage_start = nullptr;
    p->d_stage = nullptr;
    p->stages = 0;
}

// Chunk buffers for fft_execute_host: three of about 64 MiB each (whole tiles
// of signals), transformed in place.
fft_status_t create_staging(gbfft_plan* p) {
    const int64_t sig_bytes = p->n * 8;
    const int64_t S = p->entry->signals_per_block;
    int64_t chunk = (int64_t(64) << 20) / sig_bytes;
    chunk = chunk / S * S;
    if (chunk < S) chunk = S;
    if (chunk > p->batch) chunk = p->batch;
    if (chunk < 1) chunk = 1;
    p->chunk_signals = chunk;
    p->stages = 3;
    if (gbfft::plan_malloc(reinterpret_cast<void**>(&p->d_stage), (size_t)(3 * chunk * sig_bytes)) != cudaSuccess) {
        cudaGetLastError();
        p->d_stage = nullptr;
        p->stages = 0;
        return FFT_ERR_ALLOC;
    }
    for (int i = 0; i < 3; ++i) {
        if (cudaStreamCreateWithFlags(&p->stage_stream[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->stage_done[i], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            release_staging(p);
            return FFT_ERR_CUDA;
        }
    }
    if (cudaEventCreateWithFlags(&p->stage_start, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        release_staging(p);
        return FFT_ERR_CUDA;
    }
    return FFT_OK;
}

}  // namespace

extern "C" {

const char* fft_version(void) { return "0.1.0"; }

const char* fft_status_string(fft_status_t s) {
    switch (s) {
        case FFT_OK: return "success";
        case FFT_ERR_INVALID_SIZE: return "transform length must be a power of two in [2, 2048]";
        case FFT_ERR_INVALID_VALUE: return "invalid argument";
        case FFT_ERR_MISALIGNED: return "input and output must be 16-byte aligned";
        case FFT_ERR_OVERLAP: return "input and output overlap without being the same buffer";
        case FFT_ERR_ALLOC: return "allocation failed";
        case FFT_ERR_CUDA: return "CUDA runtime error";
        case FFT_ERR_UNSUPPORTED: return "unsupported by this build";
        case FFT_ERR_TIMEOUT: return "device-side wait timed out";
        case FFT_ERR_DEVICE_CHECK: return "device-side check failed";
        case FFT_ERR_NO_DEVICE: return "no usable CUDA device (sm_103 required)";
        case FFT_ERR_NOALLOC_LIMIT:
            return "request needs more scratch than fft_execute_noalloc's static device array holds";
    }
    return "unknown status";
}

void fft_twiddle_fp32(int64_t m, int64_t k, float* out) {
    // omega_m^k = exp(-2 pi i k / m).  Reduce k to [0, m), split the angle
    // into a quadrant q (a factor (-i)^q, exact) and alpha in [0, pi/2),
    // folded to [0, pi/4] so libm sees small arguments.
    if (m <= 0) {
        out[0] = 1.0f;
        out[1] = 0.0f;
        return;
    }
    k %= m;
    if (k < 0) k += m;
    const int64_t q = (4 * k) / m;      // quadrant 0..3
    const int64_t r = 4 * k - q * m;    // alpha = (pi/2) * r / m, r in [0, m)
    const double half_pi = 1.57079632679489661923;
    double c, s;
    if (2 * r <= m) {
        const double a = half_pi * (double)r / (double)m;
        c = cos(a);
        s = sin(a);
    } else {
        const double b = half_pi * (double)(m - r) / (double)m;  // pi/2 - alpha
        c = sin(b);
        s = cos(b);
    }
    // e^{-i alpha} = (c, -s); times (-i)^q
    double re, im;
    switch (q) {
        case 0: re = c; im = -s; break;
        case 1: re = -s; im = -c; break;
        case 2: re = -c; im = s; break;
        default: re = s; im = c; break;
    }
    out[0] = (float)re;
    out[1] = (float)im;
}

fft_status_t fft_validate(int64_t n, int64_t batch, int direction, int dtype, uint32_t flags) {
    if (n < 2 || n > 2048 || (n & (n - 1)) != 0) return FFT_ERR_INVALID_SIZE;
    if (batch < 0) return FFT_ERR_INVALID_VALUE;
    if (batch > INT64_MAX / (16 * n)) return FFT_ERR_INVALID_VALUE;  // byte count must fit
    if (direction != FFT_FORWARD && direction != FFT_INVERSE) return FFT_ERR_INVALID_VALUE;
    if (dtype != FFT_C64 && dtype != FFT_C64_TC_F16 && dtype != FFT_C64_TC_BF16 && dtype != FFT_C32)
        return FFT_ERR_INVALID_VALUE;
    if (flags & ~kKnownFlags) return FFT_ERR_INVALID_VALUE;
    if (dtype == FFT_C32 && (flags & FFT_FLAG_HOST_STAGING)) return FFT_ERR_UNSUPPORTED;
    return FFT_OK;
}

fft_status_t fft_plan_create_ex(int64_t n, int64_t batch, int direction, int dtype, uint32_t flags,
                                fft_plan_t* plan) {
    if (!plan) return FFT_ERR_INVALID_VALUE;
    gbfft::begin_plan_allocs();
    fft_status_t st = fft_validate(n, batch, direction, dtype, flags);
    if (st != FFT_OK) return st;

    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return FFT_ERR_NO_DEVICE;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFT_ERR_NO_DEVICE;
    int major = 0, minor = 0, sms = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FFT_ERR_CUDA;
    if (major != 10 || minor != 3) return FFT_ERR_NO_DEVICE;

    const int log2n = ilog2(n);
    LengthVariants* lv = &registry()[log2n];
    const int want_tc = dtype == FFT_C64_TC_F16 ? 1 : dtype == FFT_C64_TC_BF16 ? 2 : 0;
    const bool want_c32 = dtype == FFT_C32;
    int variant = (int)((flags & FFT_FLAG_VARIANT_MASK) >> 8) - 1;
    if (variant < 0) {
        // FP32: the length's default.  Tensor-core types: the first variant of
        // that type; lengths without a radix-16 tensor-core schedule run FP32.
        // complex32 storage: the first complex32 variant.
        variant = lv->preferred.load();
        for (int v = 0; v < lv->count && (want_tc || want_c32); ++v) {
            const KernelEntry& c = lv->v[v];
            if (c.kernel_fwd && ((want_c32 && c.kind == KernelKind::C32) || (want_tc && c.tc == want_tc))) {
                variant = v;
                break;
            }
        }
    }
    if (variant >= lv->count || !lv->v[variant].kernel_fwd) return FFT_ERR_INVALID_VALUE;
    if (lv->v[variant].tc != 0 && lv->v[variant].tc != want_tc) return FFT_ERR_INVALID_VALUE;
    if ((lv->v[variant].kind == KernelKind::C32) != want_c32) return FFT_ERR_INVALID_VALUE;
    const KernelEntry* e = &lv->v[variant];
    gbfft_plan* p = new (std::nothrow) gbfft_plan();
    if (!p) return FFT_ERR_ALLOC;
    p->n = n;
    p->batch = batch;
    p->log2n = log2n;
    p->direction = direction;
    p->dtype = dtype;
    p->flags = flags;
    p->device = dev;
    p->sm_count = sms;
    p->entry = e;
    p->kernel = direction == FFT_INVERSE ? e->kernel_inv : e->kernel_fwd;
    const bool scaled = direction == FFT_INVERSE ? !(flags & FFT_FLAG_UNNORMALIZED)
                                                 : (flags & FFT_FLAG_SCALE_FORWARD) != 0;
    p->scale = scaled ? 1.0f / (float)n : 1.0f;  // a power of two: exact

    // twiddle table (+ error word) in one allocation
    const size_t tw_bytes = (size_t)e->twiddles * 2 * sizeof(float);
    const size_t alloc = tw_bytes + 256;
    void* dmem = nullptr;
    if (gbfft::plan_malloc(&dmem, alloc) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return FFT_ERR_ALLOC;
    }
    p->d_twiddles = (float*)dmem;
    p->d_error = (int*)((char*)dmem + tw_bytes);
    if (e->twiddles > 0) {
        float* host = (float*)malloc(tw_bytes);
        if (!host) {
            cudaFree(dmem);
            delete p;
            return FFT_ERR_ALLOC;
        }
        e->fill_twiddles(host);
        cudaError_t ce = cudaMemcpy(p->d_twiddles, host, tw_bytes, cudaMemcpyHostToDevice);
        free(host);
        if (ce != cudaSuccess) {
            cudaFree(dmem);
            delete p;
            return FFT_ERR_CUDA;
        }
    }
    if (cudaMemset(p->d_error, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(dmem);
        delete p;
        return FFT_ERR_CUDA;
    }

    // launch shape: persistent grid, enough resident blocks to fill every SM
    if (e->smem_bytes > 48 * 1024) {
        if (cudaFuncSetAttribute(p->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, e->smem_bytes) !=
            cudaSuccess) {
            cudaFree(dmem);
            delete p;
            return FFT_ERR_CUDA;
        }
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->kernel, e->threads_per_block,
                                                      e->smem_bytes) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        cudaFree(dmem);
        delete p;
        return FFT_ERR_CUDA;
    }
    const int64_t tiles = (batch + e->signals_per_block - 1) / e->signals_per_block;
    if (e->tmem_cols > 0) per_sm = occupancy_without_tmem(p->kernel, e->threads_per_block, e->smem_bytes, dev);
    if (e->tmem_cols > 0 && per_sm * e->tmem_cols > 512) {
        // every resident block holds its TMEM columns for its whole life; more
        // than 512 per SM would leave a block waiting for columns forever
        per_sm = 512 / e->tmem_cols;
    }
    if (per_sm < 1) {
        cudaFree(dmem);
        delete p;
        return FFT_ERR_UNSUPPORTED;
    }
    const int64_t resident = (int64_t)sms * per_sm;
    p->resident = resident;
    p->grid = tiles < resident ? tiles : resident;
    if ((flags & FFT_FLAG_HOST_STAGING) && batch > 0) {
        fft_status_t sst = create_staging(p);
        if (sst != FFT_OK) {
            cudaFree(dmem);
            delete p;
            return sst;
        }
    }
    *plan = p;
    return FFT_OK;
}

int fft_ragged_variant_count(void) { return gbfft::ragged_variant_count(); }

fft_status_t fft_plan_create_ragged(const int64_t* offsets_host, int64_t count, int direction, int dtype,
                                    uint32_t flags, fft_plan_t* plan) {
    if (!plan) return FFT_ERR_INVALID_VALUE;
    gbfft::begin_plan_allocs();
    if (direction != FFT_FORWARD && direction != FFT_INVERSE) return FFT_ERR_INVALID_VALUE;
    if (dtype != FFT_C64 && dtype != FFT_C64_TC_F16 && dtype != FFT_C64_TC_BF16 && dtype != FFT_C32)
        return FFT_ERR_INVALID_VALUE;
    if (flags & ~kKnownFlags) return FFT_ERR_INVALID_VALUE;
    if (dtype != FFT_C64) return FFT_ERR_UNSUPPORTED;
    if (count < 0 || (count > 0 && !offsets_host)) return FFT_ERR_INVALID_VALUE;
    int ndev = 0, dev = 0, major = 0, minor = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return FFT_ERR_NO_DEVICE;
    }
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
        return FFT_ERR_CUDA;
    if (major != 10 || minor != 3) return FFT_ERR_NO_DEVICE;
    gbfft_plan* p = new (std::nothrow) gbfft_plan();
    if (!p) return FFT_ERR_ALLOC;
    int64_t grid = 0;
    fft_status_t st = gbfft::ragged_create(offsets_host, count, direction, flags, &p->ragged, &grid);
    if (st != FFT_OK) {
        delete p;
        return st;
    }
    p->batch = count;
    p->direction = direction;
    p->dtype = dtype;
    p->flags = flags;
    p->device = dev;
    p->grid = grid;
    p->d_error = gbfft::ragged_error_word(p->ragged);
    *plan = p;
    return FFT_OK;
}

fft_status_t fft_plan_create(int64_t n, int64_t batch, int direction, int dtype, fft_plan_t* plan) {
    return fft_plan_create_ex(n, batch, direction, dtype, 0u, plan);
}

fft_status_t fft_execute_c32(fft_plan_t p, const void* in, const int8_t* in_exp, void* out, int8_t* out_exp,
                             void* stream) {
    if (!p || p->ragged || !p->entry || p->entry->kind != KernelKind::C32) return FFT_ERR_INVALID_VALUE;
    if (p->batch == 0) return FFT_OK;
    if (!in || !out || !in_exp || !out_exp) return FFT_ERR_INVALID_VALUE;
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return FFT_ERR_MISALIGNED;
    const uintptr_t bytes = (uintptr_t)(p->n * p->batch * 4);
    const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
    if (a != b && a < b + bytes && b < a + bytes) return FFT_ERR_OVERLAP;
    const uintptr_t ea = (uintptr_t)in_exp, eb = (uintptr_t)out_exp, eb_n = (uintptr_t)p->batch;
    if (ea != eb && ea < eb + eb_n && eb < ea + eb_n) return FFT_ERR_OVERLAP;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return FFT_ERR_INVALID_VALUE;
    const KernelEntry* e = p->entry;
    int64_t batch = p->batch;
    const void* in2 = in;
    void* out2 = out;
    const float2* tw = (const float2*)p->d_twiddles;
    float scale = p->scale;
    int* err = p->d_error;
    uint64_t wait_ns = p->wait_ns;
    int stall = (p->flags & FFT_FLAG_TEST_STALL) ? 1 : 0;
    void* args[] = {&in2, &in_exp, &out2, &out_exp, &batch, &tw, &scale, &err, &wait_ns, &stall};
    if (gbfft::launch_kernel(p->kernel, (unsigned)p->grid, (unsigned)e->threads_per_block, args,
                             (size_t)e->smem_bytes, (cudaStream_t)stream, batch * p->n) != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_CUDA;
    }
    return FFT_OK;
}

fft_status_t fft_execute(fft_plan_t p, const void* in, void* out, void* stream) {
    if (!p) return FFT_ERR_INVALID_VALUE;
    if (p->entry && p->entry->kind == KernelKind::C32) return FFT_ERR_INVALID_VALUE;  // fft_execute_c32
    if (p->ragged) {
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return FFT_ERR_INVALID_VALUE;
        return gbfft::ragged_execute(p->ragged, in, out, stream);
    }
    if (p->batch == 0) return FFT_OK;
    if (!in || !out) return FFT_ERR_INVALID_VALUE;
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return FFT_ERR_MISALIGNED;
    const uintptr_t bytes = (uintptr_t)(p->n * p->batch * 8);
    const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
    if (a != b && a < b + bytes && b < a + bytes) return FFT_ERR_OVERLAP;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return FFT_ERR_INVALID_VALUE;

    return launch_plain(p, (const float2*)in, (float2*)out, p->batch, (cudaStream_t)stream);
}

fft_status_t fft_execute_host(fft_plan_t p, const void* in_host, void* out_host, void* stream) {
    if (!p || p->ragged || p->entry->kind == KernelKind::C32) return FFT_ERR_INVALID_VALUE;
    if (p->batch == 0) return FFT_OK;
    if (!p->stages) return FFT_ERR_INVALID_VALUE;  // plan made without FFT_FLAG_HOST_STAGING
    if (!in_host || !out_host) return FFT_ERR_INVALID_VALUE;
    const uintptr_t bytes = (uintptr_t)(p->n * p->batch * 8);
    const uintptr_t a = (uintptr_t)in_host, b = (uintptr_t)out_host;
    if (a != b && a < b + bytes && b < a + bytes) return FFT_ERR_OVERLAP;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return FFT_ERR_INVALID_VALUE;
    cudaStream_t user = (cudaStream_t)stream;
    // the pipeline starts after the caller's earlier work ...
    if (cudaEventRecord(p->stage_start, user) != cudaSuccess) goto cuda_fail;
    for (int i = 0; i < p->stages; ++i)
        if (cudaStreamWaitEvent(p->stage_stream[i], p->stage_start, 0) != cudaSuccess) goto cuda_fail;
    {
        const int64_t sig_bytes = p->n * 8;
        const char* src = static_cast<const char*>(in_host);
        char* dst = static_cast<char*>(out_host);
        int64_t k = 0;
        for (int64_t first = 0; first < p->batch; first += p->chunk_signals, ++k) {
            const int i = (int)(k % p->stages);
            const int64_t nsig = p->batch - first < p->chunk_signals ? p->batch - first : p->chunk_signals;
            const size_t nbytes = (size_t)(nsig * sig_bytes);
            float2* buf = p->d_stage + (size_t)i * p->chunk_signals * p->n;
            cudaStream_t s = p->stage_stream[i];
            // in one stream a chunk's copy in, transform and copy out stay in
            // order; the three streams overlap both copy directions and kernels
            if (cudaMemcpyAsync(buf, src + first * sig_bytes, nbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
                goto cuda_fail;
            fft_status_t st = launch_plain(p, buf, buf, nsig, s);
            if (st != FFT_OK) return st;
            if (cudaMemcpyAsync(dst + first * sig_bytes, buf, nbytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
                goto cuda_fail;
        }
    }
    // ... and the caller's stream resumes once every chunk is back on the host
    for (int i = 0; i < p->stages; ++i) {
        if (cudaEventRecord(p->stage_done[i], p->stage_stream[i]) != cudaSuccess ||
            cudaStreamWaitEvent(user, p->stage_done[i], 0) != cudaSuccess)
            goto cuda_fail;
    }
    return FFT_OK;
cuda_fail:
    cudaGetLastError();
    return FFT_ERR_CUDA;
}

fft_status_t fft_plan_get_error(fft_plan_t p) {
    if (!p) return FFT_ERR_INVALID_VALUE;
    // Wait for every stream of the plan's device, non-blocking ones included
    // (a plain cudaMemcpy would wait for the legacy stream only), then read
    // and clear the word while no kernel of this device can be writing it.
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_CUDA;
    }
    fft_status_t st = FFT_OK;
    if (prev != p->device && cudaSetDevice(p->device) != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_CUDA;
    }
    int word = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        st = FFT_ERR_CUDA;
    } else if (p->d_error) {
        if (cudaMemcpy(&word, p->d_error, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            st = FFT_ERR_CUDA;
        } else if (word != 0) {
            const int zero = 0;
            if (cudaMemcpy(p->d_error, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) st = FFT_ERR_CUDA;
        }
    }
    if (st != FFT_OK) cudaGetLastError();
    if (prev != p->device) cudaSetDevice(prev);
    return st != FFT_OK ? st : (fft_status_t)word;
}

fft_status_t fft_plan_destroy(fft_plan_t p) {
    if (!p) return FFT_OK;
    fft_status_t st = FFT_OK;
    if (p->d_twiddles && cudaFree(p->d_twiddles) != cudaSuccess) st = FFT_ERR_CUDA;
    release_staging(p);
    gbfft::ragged_destroy(p->ragged);
    delete p;
    return st;
}

fft_status_t fft_plan_get_info(fft_plan_t p, fft_plan_info_t* info) {
    if (!p || !info) return FFT_ERR_INVALID_VALUE;
    memset(info, 0, sizeof(*info));
    if (p->ragged) {
        info->direction = p->direction;
        info->dtype = p->dtype;
        info->flags = p->flags;
        gbfft::ragged_info(p->ragged, info);
        return FFT_OK;
    }
    const KernelEntry* e = p->entry;
    info->n = p->n;
    info->batch = p->batch;
    info->direction = p->direction;
    info->dtype = p->dtype;
    info->flags = p->flags;
    info->elems_per_thread = e->elems_per_thread;
    info->signals_per_block = e->signals_per_block;
    info->threads_per_block = e->threads_per_block;
    info->num_stages = e->num_stages;
    info->variant = e->variant;
    info->pipeline = e->pipeline;
    info->min_blocks = e->min_blocks;
    info->kernel_kind = (int)e->kind;
    info->tc = e->tc;
    info->tc_stages = e->tc_stages;
    for (int s = 0; s < e->num_stages && s < 4; ++s) info->radix[s] = e->radix[s];
    info->grid = p->grid;
    info->smem_bytes = e->smem_bytes;
    info->twiddle_count = e->twiddles;
    return FFT_OK;
}

int fft_variant_count(int64_t n) {
    if (n < 2 || n > 2048 || (n & (n - 1)) != 0) return 0;
    return registry()[ilog2(n)].count;
}

fft_status_t fft_set_default_variant(int64_t n, int variant) {
    if (n < 2 || n > 2048 || (n & (n - 1)) != 0) return FFT_ERR_INVALID_SIZE;
    LengthVariants* lv = &registry()[ilog2(n)];
    if (variant < 0 || variant >= lv->count || !lv->v[variant].kernel_fwd || lv->v[variant].tc != 0 ||
        lv->v[variant].kind == KernelKind::C32)
        return FFT_ERR_INVALID_VALUE;
    lv->preferred.store(variant);
    return FFT_OK;
}

int fft_variant_dtype(int64_t n, int variant) {
    if (n < 2 || n > 2048 || (n & (n - 1)) != 0) return -1;
    LengthVariants* lv = &registry()[ilog2(n)];
    if (variant < 0 || variant >= lv->count || !lv->v[variant].kernel_fwd) return -1;
    if (lv->v[variant].kind == KernelKind::C32) return FFT_C32;
    const int tc = lv->v[variant].tc;
    return tc == 1 ? FFT_C64_TC_F16 : tc == 2 ? FFT_C64_TC_BF16 : FFT_C64;
}

int fft_get_default_variant(int64_t n) {
    if (n < 2 || n > 2048 || (n & (n - 1)) != 0) return -1;
    return registry()[ilog2(n)].preferred.load();
}

fft_status_t fft_plan_set_wait_limit(fft_plan_t p, uint64_t nanoseconds) {
    if (!p || nanoseconds == 0) return FFT_ERR_INVALID_VALUE;
    if (p->ragged) {
        gbfft::ragged_set_wait_limit(p->ragged, nanoseconds);
        return FFT_OK;
    }
    p->wait_ns = nanoseconds;
    return FFT_OK;
}

fft_status_t fft_set_default_ragged_variant(int variant) {
    return gbfft::ragged_set_default_variant(variant) ? FFT_OK : FFT_ERR_INVALID_VALUE;
}

int fft_get_default_ragged_variant(void) { return gbfft::ragged_get_default_variant(); }

fft_status_t fft_plan_get_twiddles(fft_plan_t p, void* host_out, int64_t count) {
    if (!p || (!host_out && count > 0) || p->ragged) return FFT_ERR_INVALID_VALUE;
    if (count != p->entry->twiddles) return FFT_ERR_INVALID_VALUE;
    if (count == 0) return FFT_OK;
    if (cudaMemcpy(host_out, p->d_twiddles, (size_t)count * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return FFT_ERR_CUDA;
    return FFT_OK;
}

}  // extern "C"
