// Device primitives used by the plan and the output step: exclusive prefix
// sum (scan) and a stable LSD radix sort of (key, value) pairs, plus a small
// stream-ordered device buffer holder.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace bisim {

// Keep the memory that plans free in the device's default pool (release
// threshold: unlimited) instead of returning it to the driver at every
// synchronisation, so the next plan's allocations need no new mappings.
// Done once per device; other users of the default pool see the same pool.
int retain_pool_memory();

// Stream-ordered device allocation (cudaMallocAsync / cudaFreeAsync).
struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    DevMem() = default;
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
    ~DevMem() { release(); }
    int alloc(size_t nbytes, cudaStream_t stream) {
        release();
        st = stream;
        bytes = nbytes;
        if (nbytes == 0) nbytes = 16;
        cudaError_t e = cudaMallocAsync(&p, nbytes, stream);
        if (e != cudaSuccess) {
            p = nullptr;
            set_last_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
            return BISIM_ENOMEM;
        }
        return BISIM_OK;
    }
    void release() {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        bytes = 0;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

// out[i] = sum_{j<i} in[j] for i < n (in == out allowed). If total != NULL,
// *total (device) receives the sum of all n inputs. Temporary memory is
// allocated on the stream.
int scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                       cudaStream_t st);

// Stable LSD radix sort on the low `bits` bits of the keys, 8 bits per pass.
// keys/vals hold the input; keys_alt/vals_alt are scratch of the same size.
// On return *result_in_alt tells which pair of buffers holds the output.
template <typename K, typename V>
int radix_sort_pairs(K* keys, V* vals, K* keys_alt, V* vals_alt, int64_t n, int bits,
                     cudaStream_t st, bool* result_in_alt);

}  // namespace bisim
