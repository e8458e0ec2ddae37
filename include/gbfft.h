/*
 * gbfft - batched 1-D complex-to-complex power-of-two FFT for GB300 (sm_103a).
 *
 * The operation (Pascuzzi & Goli, "Benchmarking a Proof-of-Concept
 * Performance Portable SYCL-based FFT Library", Sec. 3, Eq. (dft) and
 * Eq. (idft)):
 *
 *   forward  X_k = sum_{n<N} x_n omega_N^{kn},          omega_N = e^{-2 pi i / N}
 *   inverse  x_n = (1/N) sum_{k<N} X_k omega_N^{-kn}
 *
 * applied independently to `batch` signals of length N, N a power of two with
 * 2 <= N <= 2048 (Sec. 4: single-precision C2C, lengths up to 2^11).  The
 * paper's problem statement is an FFT object built on the host from the length
 * (its radix schedule and work-group factor chosen a priori) and run on
 * device input/output buffers with a direction flag (Sec. 4, Listing 1); the
 * plan / execute / destroy calls below are that split.
 *
 * Data layout: complex64 = interleaved (re, im) float pairs, 8 bytes per
 * element.  Signal b occupies elements [b*N, (b+1)*N) of the buffer (batch
 * stride N, no padding).  Output is in natural order.
 *
 * Every call returns an fft_status_t.  Out-parameters are written only on
 * FFT_OK.  No call here aborts, prints, or throws.
 *
 * Test hook: with GBFFT_TEST_FAIL_ALLOC=k in the environment, the k-th device
 * allocation of each plan-creation call reports failure (FFT_ERR_ALLOC)
 * without allocating, so tests can take every allocation-failure path.
 */
#ifndef GBFFT_H
#define GBFFT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GBFFT_API __attribute__((visibility("default")))
#else
#define GBFFT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbfft_plan* fft_plan_t;

/* Direction (Sec. 4: SYCLFFT_FORWARD / SYCLFFT_INVERSE). */
enum {
    FFT_FORWARD = 0, /* Eq. (dft): exponent sign -1, no scaling                 */
    FFT_INVERSE = 1  /* Eq. (idft): exponent sign +1, times 1/N (unless flagged) */
};

/* Arithmetic / storage type.  Input and output are complex64 except FFT_C32. */
enum {
    FFT_C64 = 0,         /* FP32 arithmetic throughout                          */
    FFT_C64_TC_F16 = 1,  /* radix-16 stages on FP16 tensor cores, FP32 accumulate */
    FFT_C64_TC_BF16 = 2, /* radix-16 stages on BF16 tensor cores, FP32 accumulate */
    FFT_C32 = 3          /* complex32 STORAGE (two binary16 per element, with a
                            per-signal power-of-two exponent), FP32 arithmetic;
                            run with fft_execute_c32                           */
};

/* Plan flags (fft_plan_create_ex). */
enum {
    /* With FFT_INVERSE: skip the 1/N, giving the plain adjoint F^H of the
     * forward transform (used for the backward pass of autograd). */
    FFT_FLAG_UNNORMALIZED = 1u << 0,
    /* With FFT_FORWARD: multiply by 1/N, giving (1/N) F, the adjoint of the
     * normalised inverse (used for the backward pass of an inverse). */
    FFT_FLAG_SCALE_FORWARD = 1u << 1,
    /* Bits 8..12: 1 + the schedule variant to use, k = 0..30 (0 = the
     * length's default, see fft_set_default_variant).  Build them with
     * FFT_FLAG_VARIANT(k). */
    FFT_FLAG_VARIANT_MASK = 0x1Fu << 8,
    /* Test hook for failure detection: kernels with device-side waits (the
     * bulk-copy rings, the tensor-core stages, ragged variants 4 and up) issue
     * nothing, so their bounded waits run out after the plan's wait limit and
     * fft_plan_get_error reports FFT_ERR_TIMEOUT.  The output is not written.
     * Plans of kernels without device-side waits ignore it. */
    FFT_FLAG_TEST_STALL = 1u << 16,
    /* Give the plan device staging buffers (three chunks of about 64 MiB)
     * and three internal streams so that fft_execute_host can be used. */
    FFT_FLAG_HOST_STAGING = 1u << 17
};
#define FFT_FLAG_VARIANT(k) ((uint32_t)((k) + 1) << 8)

typedef enum {
    FFT_OK = 0,
    FFT_ERR_INVALID_SIZE = 1,  /* n not a power of two in [2, 2048]          */
    FFT_ERR_INVALID_VALUE = 2, /* batch < 0, unknown direction/dtype/flag,
                                  NULL plan or NULL data pointer              */
    FFT_ERR_MISALIGNED = 3,    /* in or out not 16-byte aligned               */
    FFT_ERR_OVERLAP = 4,       /* in and out overlap without being equal      */
    FFT_ERR_ALLOC = 5,         /* host or device allocation failed            */
    FFT_ERR_CUDA = 6,          /* a CUDA runtime call or kernel launch failed */
    FFT_ERR_UNSUPPORTED = 7,   /* valid request this build cannot run         */
    FFT_ERR_TIMEOUT = 8,       /* a device-side bounded wait gave up          */
    FFT_ERR_DEVICE_CHECK = 9,  /* a device-side bounds check of a GBFFT_DEBUG
                                  build failed (release builds never set it)  */
    FFT_ERR_NO_DEVICE = 10,    /* no CUDA device, or not an sm_103 device     */
    FFT_ERR_NOALLOC_LIMIT = 11 /* fft_execute_noalloc: the request needs more
                                  scratch than its static array holds         */
} fft_status_t;

/*
 * Create a plan for `batch` transforms of length `n` on the current CUDA
 * device.  Host work only (validation, radix schedule, twiddle table built in
 * FP64 and rounded to FP32, launch shape) plus one device allocation for the
 * twiddle table and the error word.  batch == 0 is valid (execute is a no-op).
 * Errors: FFT_ERR_INVALID_SIZE, FFT_ERR_INVALID_VALUE, FFT_ERR_ALLOC,
 * FFT_ERR_CUDA, FFT_ERR_NO_DEVICE, FFT_ERR_UNSUPPORTED.
 */
GBFFT_API fft_status_t fft_plan_create(int64_t n, int64_t batch, int direction, int dtype,
                             fft_plan_t* plan);

/*
 * Ragged batch: `count` signals of mixed power-of-two lengths packed back to
 * back.  offsets_host[0..count] (host memory, int64, read only during this
 * call) gives signal i the elements [offsets_host[i], offsets_host[i+1]) of the
 * buffers later passed to fft_execute; every length must be a power of two in
 * [2, 2048] and offsets_host[0] must be even (so every signal starts 16-byte
 * aligned).  The plan buckets the signals by length into tiles and uploads a
 * device work list; fft_execute then launches ONE persistent kernel whose
 * blocks take tiles from the list (graph-capturable).  Variants that share
 * the tiles through a work counter clear it first with a memset node; because
 * of that counter, a ragged plan must not be executed on two streams at once.
 * flags: FFT_FLAG_UNNORMALIZED, FFT_FLAG_SCALE_FORWARD, FFT_FLAG_TEST_STALL,
 * FFT_FLAG_VARIANT(k) with k < fft_ragged_variant_count() (without it: the
 * process-wide default of fft_set_default_ragged_variant, initially variant
 * 9: a producer warp filling ring slots for 128 compute threads per block,
 * four such blocks per SM, the lengths up to 128 first in the work list).
 * Errors: FFT_ERR_INVALID_SIZE (a length), FFT_ERR_INVALID_VALUE, FFT_ERR_MISALIGNED
 * (odd offsets_host[0]), FFT_ERR_ALLOC, FFT_ERR_CUDA, FFT_ERR_NO_DEVICE.
 */
GBFFT_API fft_status_t fft_plan_create_ragged(const int64_t* offsets_host, int64_t count, int direction,
                                              int dtype, uint32_t flags, fft_plan_t* plan);

/* Number of compiled schedule variants of the ragged kernel. */
GBFFT_API int fft_ragged_variant_count(void);

/*
 * The ragged variant that later fft_plan_create_ragged calls use when their
 * flags name none (process-wide; plans already made keep theirs).  The
 * autotuner applies its cached choice through this call.  Needs no GPU.
 * Errors: FFT_ERR_INVALID_VALUE when variant is not in
 * [0, fft_ragged_variant_count()).  fft_get_default_ragged_variant returns
 * the current choice.
 */
GBFFT_API fft_status_t fft_set_default_ragged_variant(int variant);
GBFFT_API int fft_get_default_ragged_variant(void);

/* As fft_plan_create, with FFT_FLAG_* bits in `flags`. */
GBFFT_API fft_status_t fft_plan_create_ex(int64_t n, int64_t batch, int direction, int dtype,
                                uint32_t flags, fft_plan_t* plan);

/*
 * Run the planned transform: read batch*n complex64 from device pointer `in`,
 * write batch*n complex64 to device pointer `out`, on CUDA stream `stream`
 * (a cudaStream_t; NULL means the legacy default stream).  Asynchronous: it
 * enqueues one kernel and returns; it never allocates or synchronises, so it
 * may be captured in a CUDA graph.  in == out (exact aliasing) is allowed;
 * any other overlap is rejected.  Both pointers must be 16-byte aligned.
 * The caller owns both buffers and must keep them alive until the stream has
 * run the kernel.  One plan may be executed concurrently on several streams.
 * A call of 2^22 elements or more is launched with programmatic stream
 * serialization: its kernel may be scheduled while the previous kernel of the
 * stream finishes, but it waits for that kernel to complete before it reads or
 * writes any buffer, so stream order holds as for a plain launch.
 * Errors: FFT_ERR_INVALID_VALUE, FFT_ERR_MISALIGNED, FFT_ERR_OVERLAP,
 * FFT_ERR_CUDA (launch failure, reported from cudaGetLastError).
 */
GBFFT_API fft_status_t fft_execute(fft_plan_t plan, const void* in, void* out, void* stream);

/*
 * The planned transform for complex32 storage (plan dtype FFT_C32): `in` and
 * `out` hold batch*n elements of two IEEE binary16 each (re, im; 4 bytes),
 * signal b meaning stored * 2^in_exp[b] (input) and stored * 2^out_exp[b]
 * (output).  in_exp / out_exp are device arrays of `batch` int8.  The
 * arithmetic is FP32; the call picks out_exp[b] so that the signal's largest
 * output component lands in [2^14, 2^15) (the binary16 range, full
 * precision).  Half the HBM bytes of complex64 for about 2^-11 relative
 * storage rounding.  Pointers 16-byte aligned (exponent arrays any
 * alignment); in == out allowed; asynchronous on `stream` like fft_execute.
 * Errors: FFT_ERR_INVALID_VALUE (NULL, or the plan is not FFT_C32),
 * FFT_ERR_MISALIGNED, FFT_ERR_OVERLAP, FFT_ERR_CUDA.
 */
GBFFT_API fft_status_t fft_execute_c32(fft_plan_t plan, const void* in, const int8_t* in_exp, void* out,
                                       int8_t* out_exp, void* stream);

/*
 * The planned transform on HOST buffers: batch*n complex64 read from
 * `in_host`, results written to `out_host` (equal, or not overlapping).  The
 * plan must have been made with FFT_FLAG_HOST_STAGING.  Work is split into
 * chunks of whole signals; each chunk is copied to one of the plan's device
 * buffers, transformed in place and copied back, the chunks round-robin over
 * the plan's three streams so that host-to-device copies, kernels and
 * device-to-host copies overlap.  Asynchronous with respect to the host: the
 * pipeline starts after work already enqueued on `stream` and `stream` waits
 * for its end (synchronise `stream` before reading out_host).  Host buffers
 * should be page-locked (cudaHostAlloc / cudaHostRegister); pageable memory
 * works but the copies then serialise.  One call at a time per plan.
 * Errors: FFT_ERR_INVALID_VALUE (no staging, NULL, ragged plan, wrong device),
 * FFT_ERR_OVERLAP, FFT_ERR_CUDA.
 */
GBFFT_API fft_status_t fft_execute_host(fft_plan_t plan, const void* in_host, void* out_host, void* stream);

/*
 * Read and clear the plan's device error word (FFT_OK when no device-side
 * check fired).  It first synchronises the plan's whole device
 * (cudaDeviceSynchronize with that device current, the caller's current
 * device restored afterwards), so work enqueued on any stream of that device
 * before the call, non-blocking streams included, has finished and the word
 * is final when it is read.  Call it after the work you want checked has been
 * enqueued, and not while a stream of that device is being captured into a
 * CUDA graph.  Returns FFT_ERR_CUDA if the synchronisation or the copy fails
 * (for example after an earlier kernel fault), else the word: FFT_OK or the
 * code a kernel recorded (FFT_ERR_TIMEOUT; in a GBFFT_DEBUG build also
 * FFT_ERR_DEVICE_CHECK).
 */
GBFFT_API fft_status_t fft_plan_get_error(fft_plan_t plan);

/* Release the plan and its device memory.  NULL is a no-op returning FFT_OK.
 * The caller must not destroy a plan whose kernels may still be running. */
GBFFT_API fft_status_t fft_plan_destroy(fft_plan_t plan);

/* Static English text for a status code (never NULL). */
GBFFT_API const char* fft_status_string(fft_status_t status);

/* Introspection, for tests and tuning. */
typedef struct {
    int64_t n, batch;
    int direction, dtype;
    uint32_t flags;
    int elems_per_thread;   /* registers' worth of complex elements per thread */
    int signals_per_block;  /* signals one thread block transforms per tile     */
    int threads_per_block;
    int num_stages;         /* radix stages, first to last                      */
    int radix[8];
    int variant;            /* schedule variant of this length in use           */
    int pipeline;           /* bulk-copy (TMA) prefetch ring depth, 0 = none     */
    int min_blocks;         /* launch-bounds residency hint                     */
    int kernel_kind;        /* 0 one thread per signal, 1 direct, 2 TMA ring,
                               3 ragged persistent work list, 4 complex32 I/O   */
    int64_t work_items;     /* ragged plans: tiles in the device work list      */
    int tc;                 /* radix-16 stages on tensor cores: 0 no (FP32),
                               1 FP16 operands, 2 BF16 operands                 */
    int64_t grid;           /* blocks launched (persistent grid-stride loop)    */
    int64_t smem_bytes;     /* dynamic shared memory per block                  */
    int64_t twiddle_count;  /* complex64 entries in the plan's twiddle table    */
    int tc_stages;          /* radix stages that run on tensor cores            */
} fft_plan_info_t;

GBFFT_API fft_status_t fft_plan_get_info(fft_plan_t plan, fft_plan_info_t* info);

/*
 * Schedule variants.  Each length has one or more compiled radix schedules /
 * launch shapes (the analogue of the paper's host-chosen stage_sizes and
 * work-group factor, Sec. 4).  fft_variant_count returns how many (0 for an
 * invalid length); fft_set_default_variant chooses the FP32 one later plans of
 * that length use (process-wide; the autotuner calls it); plans already made
 * keep theirs.  fft_get_default_variant returns the current choice or -1.
 */
GBFFT_API int fft_variant_count(int64_t n);
GBFFT_API fft_status_t fft_set_default_variant(int64_t n, int variant);
GBFFT_API int fft_get_default_variant(int64_t n);
/* The dtype (FFT_C64, FFT_C64_TC_F16, FFT_C64_TC_BF16 or FFT_C32) that variant k of
 * length n computes in, or -1 when there is no such variant.  Plans accept a
 * variant only with its own dtype. */
GBFFT_API int fft_variant_dtype(int64_t n, int variant);

/*
 * Wall-time limit for the device-side waits of this plan's kernels (the
 * bulk-copy prefetch rings, ragged variants 4 and up and the tensor-core MMA
 * completion wait on mbarriers).  A wait that runs out records FFT_ERR_TIMEOUT in the plan's
 * error word (see fft_plan_get_error); the block then stops waiting and
 * issuing, skips its stores and finishes, after waiting once more (with the
 * same limit) for copies or MMAs it had already issued.  Default 4 s.  0 is
 * rejected.
 */
GBFFT_API fft_status_t fft_plan_set_wait_limit(fft_plan_t plan, uint64_t nanoseconds);

/*
 * Copy the plan's FP32 twiddle table (twiddle_count complex64 entries) into
 * the host buffer `host_out`.  For tests of its accuracy and symmetry.
 */
GBFFT_API fft_status_t fft_plan_get_twiddles(fft_plan_t plan, void* host_out, int64_t count);

/*
 * Host-side twiddle generator used by every plan: omega_m^k for integer k,
 * computed in FP64 (libm cos/sin on an angle reduced to [0, pi/4] by the
 * symmetry of Sec. 3, Eq. (twiddle): omega^{k+m/4} = -i omega^k), then rounded to
 * nearest FP32.  Writes (re, im) into out[0], out[1].  Needs no GPU.
 */
GBFFT_API void fft_twiddle_fp32(int64_t m, int64_t k, float* out);

/*
 * Validate arguments the way fft_plan_create does, without touching a GPU.
 * Returns FFT_OK or the error code fft_plan_create would return for them.
 */
GBFFT_API fft_status_t fft_validate(int64_t n, int64_t batch, int direction, int dtype,
                          uint32_t flags);

/*
 * fft_execute_noalloc - the planned transform of fft_execute, for callers
 * that cannot allocate device memory.  (The paper has no counterpart: this
 * is an interface for library users, not part of the method.)
 *
 * Who needs it: a process that gives all free device memory to its own
 * caching allocator at start-up and may not take more afterwards, or code
 * that must not pay the implicit device-wide synchronisation that cudaMalloc
 * and cudaFree can cause.  This call makes no plan and calls no cudaMalloc,
 * cudaFree or other allocating routine.  Its scratch (the twiddle table of the
 * length and an error word) lives in a file-scope static __device__ array of
 * 4096 complex64 entries plus one 256-byte slot (about 33 KiB), which every
 * GPU that loads the library keeps reserved until the process exits.
 *
 * Arguments: n, batch, direction as for fft_plan_create (dtype is FFT_C64);
 * flags may hold FFT_FLAG_UNNORMALIZED, FFT_FLAG_SCALE_FORWARD and
 * FFT_FLAG_VARIANT(k) of an FP32 variant, any other bit is refused with
 * FFT_ERR_INVALID_VALUE; in/out/stream as for fft_execute (device pointers,
 * 16-byte aligned, equal or disjoint; the caller owns them).  The twiddle
 * table is generated on the device by the same steps as the plan path's
 * (quadrant fold, FP64 cos/sin, one rounding to FP32), and the same kernel
 * runs, so the result is bit-identical to fft_execute's for the same length,
 * direction, flags and variant (tested for every compiled FP32 schedule).
 *
 * Behaviour:
 *  - The first call on a device does a one-time set-up (it looks up the
 *    static array's device address with cudaGetSymbolAddress while that
 *    device is current); the first call for each length, direction and
 *    variant also queries its launch shape.  Make those first calls before
 *    any stream capture.
 *  - Every call enqueues two kernels on `stream`: one rewrites the shared
 *    array (this length's twiddles, error word cleared), one transforms.  All
 *    calls on a device share the array, which keeps the last call's
 *    contents, so calls that may overlap on the GPU (e.g. on two streams)
 *    race and must be serialised by the caller.
 *  - A request whose twiddle table would not fit the array returns
 *    FFT_ERR_NOALLOC_LIMIT (no compiled schedule needs more than 2040
 *    entries, so every valid length fits); invalid arguments return the
 *    codes fft_plan_create / fft_execute return; a failed launch returns
 *    FFT_ERR_CUDA.  Device-side wait timeouts are not reported by this call.
 */
GBFFT_API fft_status_t fft_execute_noalloc(int64_t n, int64_t batch, int direction, uint32_t flags,
                                           const void* in, void* out, void* stream);

/* Library version, "major.minor.patch". */
GBFFT_API const char* fft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBFFT_H */
