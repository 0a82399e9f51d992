// Shared device helpers: cache-global loads for state that other CTAs
// mutate, the grid-wide barrier with a time limit, status bits, and host-side
// error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/bisim.h"

namespace bisim {

// Device status word bits (OR-ed by kernels, read by the host after a call).
enum : int {
    ST_INVALID = 1,   // an input entry out of range
    ST_TIMEOUT = 2,   // a grid barrier wait ran out
    ST_ROUNDS = 4,    // round cap exceeded
    ST_OVERFLOW = 8,  // an internal list exceeded its capacity
    ST_INTERNAL = 16  // an internal consistency check failed
};
constexpr int ST_ABORT_MASK = ST_TIMEOUT | ST_ROUNDS | ST_OVERFLOW | ST_INTERNAL;

constexpr int32_t NONE = 0x7fffffff;  // "no label" / +infinity for atomicMin

// ---------------------------------------------------------------- host side

void set_last_error(const std::string& s);

// Kernels launched on the calling host thread since the last reset (every
// launch site bumps it; the ABI reports it per plan / refine call).
extern thread_local long long g_launches;
#define BISIM_LAUNCHED() (++::bisim::g_launches)

#define BISIM_CUDA_TRY(...)                                                                   \
    do {                                                                                      \
        cudaError_t e__ = (__VA_ARGS__);                                                      \
        if (e__ != cudaSuccess) {                                                             \
            ::bisim::set_last_error(std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e__)); \
            return e__ == cudaErrorMemoryAllocation ? BISIM_ENOMEM : BISIM_ECUDA;         \
        }                                                                                 \
    } while (0)

#define BISIM_TRY(...)            \
    do {                          \
        int r__ = (__VA_ARGS__);  \
        if (r__ != BISIM_OK) return r__; \
    } while (0)

inline int status_to_code(int st) {
    if (st & ST_INVALID) return BISIM_EINVAL;
    if (st & ST_TIMEOUT) return BISIM_ETIMEOUT;
    if (st & ST_ROUNDS) return BISIM_EROUNDS;
    if (st & (ST_OVERFLOW | ST_INTERNAL)) return BISIM_ECUDA;
    return BISIM_OK;
}

inline int ceil_log2_u64(uint64_t x) {
    int b = 0;
    while (b < 64 && (uint64_t(1) << b) < x) b++;
    return b;
}

inline unsigned grid_for(int64_t work, int threads, unsigned cap = 152u * 32u) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return unsigned(g);
}

// -------------------------------------------------------------- device side

__device__ __forceinline__ int ldcg(const int* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned ldcg(const unsigned* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ldcg(const unsigned long long* p) { return __ldcg(p); }
__device__ __forceinline__ int4 ldcg(const int4* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned char ldcg(const unsigned char* p) {
    return (unsigned char)__ldcg((const char*)p);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Grid-wide barrier for a cooperative (co-resident) launch. The counter is
// monotonic and zeroed before the launch; every CTA adds one per barrier and
// waits until the counter reaches (barriers passed) x gridDim.x. Ordering:
// __syncthreads orders the CTA's writes before thread 0's arrive, a release
// add at GPU scope (cumulative, so it publishes them), and the acquire load
// that ends the wait, followed by __syncthreads, orders the other CTAs'
// writes before everything this CTA does next; no separate fences are needed.
// Every wait is bounded: after timeout_ns (measured with the global timer) or
// a spin cap, or when another CTA has raised an abort bit, the CTA gives up,
// records ST_TIMEOUT, and the caller returns. Returns false when the caller
// must stop.
struct GridBarrier {
    unsigned long long* counter;
    int* status;
    unsigned long long timeout_ns;
};

__device__ __forceinline__ bool grid_sync(const GridBarrier& gb, unsigned long long& target) {
    __shared__ int s_abort;
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        int ab = 0;
        red_release_add_u64(gb.counter, 1ull);
        unsigned long long t0 = 0;
        unsigned spins = 0;
        while (ld_acquire_u64(gb.counter) < target) {
            ++spins;
            if ((spins & 31u) == 0) {
                unsigned long long now = globaltimer_ns();
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > gb.timeout_ns || spins > (1u << 30)) {
                    atomicOr(gb.status, ST_TIMEOUT);
                    ab = 1;
                    break;
                }
                if (ldcg(gb.status) & ST_ABORT_MASK) {
                    ab = 1;
                    break;
                }
            }
        }
        s_abort = ab;
    }
    __syncthreads();
    return !s_abort;
}

// Block-wide reductions for blockDim.x a multiple of 32 (<= 1024).
__device__ __forceinline__ int block_reduce_min(int v, int* sh /* >= 32 ints */) {
    unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    v = __reduce_min_sync(0xffffffffu, v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    int r = (int)lane < nw ? sh[lane] : NONE;
    if (w == 0) r = __reduce_min_sync(0xffffffffu, r);
    __syncthreads();
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

}  // namespace bisim
