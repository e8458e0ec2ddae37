// Kernel registry shared by the per-length kernel translation units and the
// host plan code.  Each fft_kernels.cu build (one per log2 N) defines one
// gbfft_entry_<log2N>() returning the launch facts of its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbfft {

struct KernelEntry {
    int log2n;
    bool small;              // one thread per signal (N <= 16)
    int elems_per_thread;
    int signals_per_block;   // generic kernel: signals per tile
    int threads_per_block;
    int smem_bytes;
    int num_stages;
    int radix[4];
    int twiddles;            // complex64 entries in the twiddle table
    int signals_per_warp_tile;  // small kernel: signals per warp tile
    const void* kernel_fwd;
    const void* kernel_inv;
    // Fill `host` (twiddles entries, interleaved re/im) with this schedule's table.
    void (*fill_twiddles)(float* host);
};

}  // namespace gbfft

#define GBFFT_DECLARE_ENTRY(L) gbfft::KernelEntry gbfft_entry_##L();
