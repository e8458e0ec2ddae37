// Kernel registry shared by the per-length kernel translation units and the
// host plan code.  Each fft_kernels.cu build (one per log2 N) defines
// gbfft_entries_<log2N>(out, max) filling the launch facts of every schedule
// variant it compiled, variant 0 first.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbfft.h"

namespace gbfft {

enum class KernelKind : int { Small = 0, Direct = 1, Ring = 2, C32 = 4 };

struct KernelEntry {
    int log2n;
    int variant;
    KernelKind kind;
    int elems_per_thread;
    int signals_per_block;   // signals one block transforms per tile
    int threads_per_block;
    int smem_bytes;
    int num_stages;
    int radix[4];
    int min_blocks;          // launch-bounds hint
    int pipeline;            // bulk-copy ring depth (0 = none)
    int tc;                  // 0 FP32, 1 FP16 / 2 BF16 tensor-core radix-16 stages
    int tc_stages;           // stages that run on the tensor cores
    int tmem_cols;           // TMEM columns one block allocates (tensor-core variants)
    int twiddles;            // complex64 entries in the twiddle table
    const void* kernel_fwd;
    const void* kernel_inv;
    // Fill `host` (twiddles entries, interleaved re/im) with this schedule's table.
    void (*fill_twiddles)(float* host);
};

// Device allocation of plan creation (host).  Every plan-creation call starts
// its count with begin_plan_allocs(); with GBFFT_TEST_FAIL_ALLOC=k in the
// environment (a test hook for failure detection) the k-th allocation of the
// call reports failure without allocating, so the tests can take every
// allocation-failure path of plan creation.
void begin_plan_allocs();
cudaError_t plan_malloc(void** ptr, size_t bytes);
// Every kernel launch of the library.  A call that moves at least
// kPdlMinElems elements is launched with programmatic stream serialization,
// so that it may be scheduled while the previous kernel of the stream drains
// (each kernel waits for its predecessor before touching memory, pdl_enter);
// smaller calls are bound by the host's launch rate, where the extended
// launch only adds host time.
constexpr int64_t kPdlMinElems = int64_t(1) << 22;
cudaError_t launch_kernel(const void* kernel, unsigned grid, unsigned block, void** args, size_t smem,
                          cudaStream_t stream, int64_t elems);

// Registry lookup (host): the entry of `variant`, or of the length's current
// default when variant < 0; NULL when there is none.
const KernelEntry* lookup_entry(int log2n, int variant);

// Ragged (mixed-length) plans, implemented in fft_ragged.cu.
struct RaggedState;
int ragged_variant_count();
bool ragged_set_default_variant(int v);  // false when v is not a ragged variant
int ragged_get_default_variant();
void ragged_set_wait_limit(RaggedState* st, uint64_t ns);
bool ragged_waits_on_device(const RaggedState* st);  // the bulk-copy variants (4 and up)
fft_status_t ragged_create(const int64_t* offsets, int64_t count, int direction, uint32_t flags,
                           RaggedState** out, int64_t* grid_out);
fft_status_t ragged_execute(RaggedState* st, const void* in, void* out, void* stream);
void ragged_info(const RaggedState* st, fft_plan_info_t* info);
int* ragged_error_word(RaggedState* st);
void ragged_destroy(RaggedState* st);

}  // namespace gbfft

#define GBFFT_DECLARE_ENTRIES(L) int gbfft_entries_##L(gbfft::KernelEntry* out, int max);
