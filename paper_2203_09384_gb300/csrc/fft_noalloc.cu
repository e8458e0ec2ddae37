// fft_execute_noalloc: the batched transform without a plan and without any
// device allocation.
//
// Some callers cannot call cudaMalloc: a serving process that hands all free
// device memory to its own caching allocator at start-up and must not take
// more afterwards, code running where an allocation's implicit device-wide
// synchronisation is not acceptable (cudaMalloc/cudaFree can stall every
// stream), or a caller that simply has no plan object to keep.  The plan path
// allocates its twiddle table and error word with cudaMalloc; this entry point
// keeps both in one file-scope static __device__ array instead, which the
// CUDA runtime reserves when the library's module loads on a device and which
// stays reserved on every device that loaded it until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents, so each call first rewrites the twiddles its length needs and
// clears the error word (one small kernel on the caller's stream), then runs
// the same FFT kernel the plan path runs, pointed at the static array.  Calls
// that overlap on one GPU (for instance on two streams) race on that array;
// each device has its own copy, so calls on different devices do not.
#include <cuda_runtime.h>

#include <stdint.h>

#include <mutex>

#include "../../include/gbfft.h"
#include "registry.h"
#include "schedules.h"

namespace {

// Stated maximum: 4096 complex64 twiddles (32 KiB) plus one 256-byte slot for
// the error word.  The largest table any compiled schedule needs is the
// N = 2048 one, 2040 entries.
constexpr int kNoAllocTwiddles = 4096;
constexpr int kNoAllocSlots = kNoAllocTwiddles + 32;  // + error word slot

static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocSlots];

constexpr int kMaxDevices = 64;

struct LaunchShape {
    int64_t per_sm = 0;  // resident blocks per SM for this kernel, 0 = not set up
};

struct DeviceState {
    bool ready = false;
    float2* scratch = nullptr;  // device address of g_noalloc_scratch on this device
    int sm_count = 0;
    LaunchShape shape[GBFFT_MAX_LOG2N + 1][GBFFT_MAX_VARIANTS][2];
};

DeviceState g_state[kMaxDevices];
std::mutex g_mutex;

// omega_m^k rounded to FP32 the way the plan path's host generator
// (fft_twiddle_fp32) does it: k reduced to [0, m), the angle split into a
// quadrant q (a factor (-i)^q, exact) and alpha in [0, pi/2), folded to
// [0, pi/4] so that cos and sin see small arguments, FP64 cos/sin, then one
// rounding to FP32.  The same steps on FP64 math give the same FP32 table as
// the plan path (the tests compare the two paths' outputs bit for bit for
// every compiled FP32 schedule).
__device__ float2 noalloc_twiddle(long long m, long long k) {
    k %= m;
    if (k < 0) k += m;
    const long long q = (4 * k) / m;
    const long long r = 4 * k - q * m;
    const double half_pi = 1.57079632679489661923;
    double c, s;
    if (2 * r <= m) {
        const double a = half_pi * (double)r / (double)m;
        c = cos(a);
        s = sin(a);
    } else {
        const double b = half_pi * (double)(m - r) / (double)m;
        c = sin(b);
        s = cos(b);
    }
    double re, im;
    switch (q) {
        case 0: re = c; im = -s; break;
        case 1: re = -s; im = -c; break;
        case 2: re = -c; im = s; break;
        default: re = s; im = c; break;
    }
    return make_float2((float)re, (float)im);
}

// Fill the first `count` twiddles of the schedule with radices r0..r3 (same
// layout as the plan path's table: stage s >= 1, entry off_s + (r-1)*Ns + m =
// omega_{Ns*R}^{m*r}) and clear the error word.
__global__ void noalloc_prepare(float2* scratch, int r0, int r1, int r2, int r3, int count) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx == 0) *reinterpret_cast<int*>(scratch + kNoAllocTwiddles) = 0;
    if (idx >= count) return;
    const int radix[4] = {r0, r1, r2, r3};
    int ns = radix[0], off = 0;
    for (int s = 1; s < 4 && radix[s] > 0; ++s) {
        const int R = radix[s];
        const int size = (R - 1) * ns;
        if (idx < off + size) {
            const int local = idx - off;
            const int r = local / ns + 1;
            const int m = local % ns;
            scratch[idx] = noalloc_twiddle((long long)ns * R, (long long)m * r);
            return;
        }
        off += size;
        ns *= R;
    }
}

int ilog2_exact(int64_t n) {
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return l;
}

// One-time set-up of the current device: the static array's device address
// (cudaGetSymbolAddress with this device current) and the SM count.
fft_status_t setup_device(int dev, DeviceState** out) {
    if (dev < 0 || dev >= kMaxDevices) return FFT_ERR_UNSUPPORTED;
    DeviceState* d = &g_state[dev];
    if (!d->ready) {
        int major = 0, minor = 0, sms = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return FFT_ERR_CUDA;
        }
        if (major != 10 || minor != 3) return FFT_ERR_NO_DEVICE;
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return FFT_ERR_CUDA;
        }
        d->scratch = static_cast<float2*>(ptr);
        d->sm_count = sms;
        d->ready = true;
    }
    *out = d;
    return FFT_OK;
}

// Launch shape of one kernel on this device, worked out once (occupancy query
// and, above 48 KiB, the dynamic shared-memory opt-in).
fft_status_t kernel_shape(DeviceState* d, const gbfft::KernelEntry* e, int inverse, int64_t* per_sm) {
    LaunchShape& ls = d->shape[e->log2n][e->variant][inverse];
    if (ls.per_sm == 0) {
        const void* k = inverse ? e->kernel_inv : e->kernel_fwd;
        if (e->smem_bytes > 48 * 1024 &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, e->smem_bytes) != cudaSuccess) {
            cudaGetLastError();
            return FFT_ERR_CUDA;
        }
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, e->threads_per_block, e->smem_bytes) !=
                cudaSuccess ||
            nb < 1) {
            cudaGetLastError();
            return FFT_ERR_CUDA;
        }
        ls.per_sm = nb;
    }
    *per_sm = ls.per_sm;
    return FFT_OK;
}

}  // namespace

extern "C" fft_status_t fft_execute_noalloc(int64_t n, int64_t batch, int direction, uint32_t flags,
                                            const void* in, void* out, void* stream) {
    // only the flags this call honours: normalisation and the schedule variant
    if (flags & ~(uint32_t)(FFT_FLAG_UNNORMALIZED | FFT_FLAG_SCALE_FORWARD | FFT_FLAG_VARIANT_MASK))
        return FFT_ERR_INVALID_VALUE;
    fft_status_t st = fft_validate(n, batch, direction, FFT_C64, flags);
    if (st != FFT_OK) return st;
    if (batch == 0) return FFT_OK;
    if (!in || !out) return FFT_ERR_INVALID_VALUE;
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return FFT_ERR_MISALIGNED;
    const uintptr_t bytes = (uintptr_t)(n * batch * 8);
    const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
    if (a != b && a < b + bytes && b < a + bytes) return FFT_ERR_OVERLAP;

    const int log2n = ilog2_exact(n);
    const int variant = (int)((flags & FFT_FLAG_VARIANT_MASK) >> 8) - 1;
    const gbfft::KernelEntry* e = gbfft::lookup_entry(log2n, variant);
    if (!e || e->tc != 0 || e->kind == gbfft::KernelKind::C32) return FFT_ERR_INVALID_VALUE;  // FP32, complex64 only
    if (e->twiddles > kNoAllocTwiddles) return FFT_ERR_NOALLOC_LIMIT;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_NO_DEVICE;
    }
    DeviceState* d = nullptr;
    int64_t per_sm = 0;
    const int inverse = direction == FFT_INVERSE;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        st = setup_device(dev, &d);
        if (st == FFT_OK) st = kernel_shape(d, e, inverse, &per_sm);
    }
    if (st != FFT_OK) return st;

    cudaStream_t s = (cudaStream_t)stream;
    // rewrite this length's twiddles and clear the error word
    const int count = e->twiddles;
    const int threads = 256;
    const int blocks = count > 0 ? (count + threads - 1) / threads : 1;
    noalloc_prepare<<<blocks, threads, 0, s>>>(d->scratch, e->radix[0], e->radix[1], e->radix[2], e->radix[3],
                                                count);
    if (cudaGetLastError() != cudaSuccess) return FFT_ERR_CUDA;

    const bool scaled = inverse ? !(flags & FFT_FLAG_UNNORMALIZED) : (flags & FFT_FLAG_SCALE_FORWARD) != 0;
    float scale = scaled ? 1.0f / (float)n : 1.0f;
    const int64_t tiles = (batch + e->signals_per_block - 1) / e->signals_per_block;
    const int64_t resident = (int64_t)d->sm_count * per_sm;
    const int64_t grid = tiles < resident ? tiles : resident;
    const float2* in2 = (const float2*)in;
    float2* out2 = (float2*)out;
    const float2* tw = d->scratch;
    int* err = reinterpret_cast<int*>(d->scratch + kNoAllocTwiddles);
    uint64_t wait_ns = 4000000000ull;
    const void* kernel = inverse ? e->kernel_inv : e->kernel_fwd;
    cudaError_t ce;
    if (e->kind == gbfft::KernelKind::Small) {
        void* args[] = {&in2, &out2, &batch, &scale};
        ce = cudaLaunchKernel(kernel, dim3((unsigned)grid), dim3(e->threads_per_block), args, (size_t)e->smem_bytes,
                              s);
    } else {
        int stall = 0;
        void* args[] = {&in2, &out2, &batch, &tw, &scale, &err, &wait_ns, &stall};
        ce = cudaLaunchKernel(kernel, dim3((unsigned)grid), dim3(e->threads_per_block), args, (size_t)e->smem_bytes,
                              s);
    }
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_CUDA;
    }
    return FFT_OK;
}
