// Allocation-free canonical renumbering: the same result as the output step
// of bisim_refine (block ids numbered in order of their smallest state), for
// callers that cannot allocate device memory. All scratch lives in one
// file-scope __device__ array of fixed size; one cooperative kernel does the
// whole job with the grid barrier of common.cuh.
#include <mutex>

#include "common.cuh"

namespace {

using namespace bisim;

constexpr int32_t MAX_N = BISIM_NOALLOC_MAX_N;
constexpr int MAX_CTAS = 1024;
constexpr int THREADS = 512;
constexpr int MAX_DEVICES = 64;

struct NoAllocScratch {
    int32_t first[MAX_N];  // smallest state of each label
    int32_t rank[MAX_N];   // canonical id, stored at the smallest state of its block
    int32_t cta_count[MAX_CTAS];
    unsigned long long barrier;
    int status;
    int num_blocks;
};

// Shared by every call on this device; holds the last call's contents.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__global__ void __launch_bounds__(THREADS) k_canonical_noalloc(const int32_t* __restrict__ labels, int32_t n,
                                                               int32_t* out, NoAllocScratch* sc) {
    __shared__ int sh[32];
    __shared__ int s_base;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    GridBarrier gb;
    gb.counter = &sc->barrier;
    gb.status = &sc->status;
    gb.timeout_ns = 2000000000ull;
    unsigned long long tgt = 0;
    const int32_t chunk = (n + (int32_t)gridDim.x - 1) / (int32_t)gridDim.x;
    const int32_t lo = min(n, (int32_t)blockIdx.x * chunk);
    const int32_t hi = min(n, lo + chunk);
    // 1: reset and validate
    int bad = 0;
    for (int64_t i = gtid; i < n; i += gsz) {
        sc->first[i] = NONE;
        bad |= (unsigned)labels[i] >= (unsigned)n;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&sc->status, ST_INVALID);
    if (!grid_sync(gb, tgt)) return;
    if (ldcg(&sc->status) & ST_INVALID) return;  // every CTA sees the same word here
    // 2: smallest state per label
    for (int64_t i = gtid; i < n; i += gsz) atomicMin(&sc->first[labels[i]], (int32_t)i);
    if (!grid_sync(gb, tgt)) return;
    // 3: blocks whose smallest state lies in this CTA's chunk
    unsigned c = 0;
    for (int32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) c += ldcg(&sc->first[labels[i]]) == i;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (int)c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
        sc->cta_count[blockIdx.x] = t;
    }
    if (!grid_sync(gb, tgt)) return;
    // 4: ranks in state order
    if (threadIdx.x == 0) {
        int b = 0;
        for (unsigned j = 0; j < blockIdx.x; j++) b += ldcg(&sc->cta_count[j]);
        s_base = b;
        if (blockIdx.x == gridDim.x - 1) sc->num_blocks = b + ldcg(&sc->cta_count[blockIdx.x]);
    }
    __syncthreads();
    int base = s_base;
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    for (int32_t cb = lo; cb < hi; cb += blockDim.x) {
        const int32_t i = cb + threadIdx.x;
        const bool f = i < hi && ldcg(&sc->first[labels[i]]) == i;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        __syncthreads();
        if (lane == 0) sh[wid] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            const int v = sh[w];
            if (w < (int)wid) before += v;
            total += v;
        }
        if (f) sc->rank[i] = base + before + __popc(bal & lanemask_lt());
        base += total;
    }
    if (!grid_sync(gb, tgt)) return;
    // 5: canonical id of every state
    for (int64_t i = gtid; i < n; i += gsz) out[i] = ldcg(&sc->rank[ldcg(&sc->first[labels[i]])]);
}

std::mutex g_setup_mu;
NoAllocScratch* g_scratch_ptr[MAX_DEVICES];
int g_grid[MAX_DEVICES];

struct HostStatus {
    int status;
    int num_blocks;
};

}  // namespace

extern "C" int bisim_canonical_ids_noalloc(const int32_t* labels, int32_t n, int32_t* out_ids,
                                           int32_t* num_blocks_h, void* stream) {
    if (n < 0 || n > MAX_N) return BISIM_EINVAL;
    if (n == 0) {
        if (num_blocks_h) *num_blocks_h = 0;
        return BISIM_OK;
    }
    if (!labels || !out_ids) return BISIM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BISIM_ECUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return BISIM_ENOTSUP;
    NoAllocScratch* sc;
    int grid;
    {
        // once per device, with that device current: the host-side symbol is
        // only a stand-in, the kernel needs the device address
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_ptr[dev]) {
            NoAllocScratch* p = nullptr;
            if (cudaGetSymbolAddress((void**)&p, g_noalloc_scratch) != cudaSuccess || !p) return BISIM_ECUDA;
            int occ = 0, sms = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_canonical_noalloc, THREADS, 0) !=
                    cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || occ < 1)
                return BISIM_ECUDA;
            g_grid[dev] = sms * occ < MAX_CTAS ? sms * occ : MAX_CTAS;
            g_scratch_ptr[dev] = p;
        }
        sc = g_scratch_ptr[dev];
        grid = g_grid[dev];
    }
    const int64_t want = ((int64_t)n + THREADS - 1) / THREADS;
    if (want < grid) grid = (int)want;
    cudaStream_t st = (cudaStream_t)stream;
    // the barrier counter and the status word must start at zero
    if (cudaMemsetAsync(&sc->barrier, 0, sizeof(unsigned long long) + sizeof(int), st) != cudaSuccess)
        return BISIM_ECUDA;
    void* args[] = {(void*)&labels, (void*)&n, (void*)&out_ids, (void*)&sc};
    if (cudaLaunchCooperativeKernel((const void*)k_canonical_noalloc, dim3(grid), dim3(THREADS), args, 0, st) !=
        cudaSuccess)
        return BISIM_ECUDA;
    HostStatus hs{0, 0};
    if (cudaMemcpyAsync(&hs.status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&hs.num_blocks, &sc->num_blocks, sizeof(int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return BISIM_ECUDA;
    if (hs.status & ST_INVALID) return BISIM_EINVAL;
    if (hs.status & ST_TIMEOUT) return BISIM_ETIMEOUT;
    if (hs.status) return BISIM_ECUDA;
    if (num_blocks_h) *num_blocks_h = hs.num_blocks;
    return BISIM_OK;
}
