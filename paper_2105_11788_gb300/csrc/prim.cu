// Exclusive scan (reduce-then-scan over 2048-element tiles, recursive on the
// tile sums) and a stable LSD radix sort (8-bit digits; per pass a tile
// histogram, a scan of the digit-major histogram, and a stable scatter whose
// in-tile ranks come from warp match/ballot).
#include <mutex>

#include "prim.cuh"

namespace bisim {

int retain_pool_memory() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    BISIM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64 || done[dev]) return BISIM_OK;
    cudaMemPool_t pool;
    BISIM_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t threshold = UINT64_MAX;
    BISIM_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold));
    done[dev] = true;
    return BISIM_OK;
}

}  // namespace bisim

extern "C" {

int bisim_pool_usage(uint64_t* used, uint64_t* used_high, uint64_t* reserved) {
    int dev = 0;
    BISIM_CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    BISIM_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t v = 0;
    if (used) {
        BISIM_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v));
        *used = v;
    }
    if (used_high) {
        BISIM_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v));
        *used_high = v;
    }
    if (reserved) {
        BISIM_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v));
        *reserved = v;
    }
    return BISIM_OK;
}

int bisim_pool_reset_high(void) {
    int dev = 0;
    BISIM_CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    BISIM_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t zero = 0;
    BISIM_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    return BISIM_OK;
}

int bisim_pool_trim(uint64_t keep_bytes) {
    int dev = 0;
    BISIM_CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    BISIM_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    BISIM_CUDA_TRY(cudaDeviceSynchronize());
    BISIM_CUDA_TRY(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
    return BISIM_OK;
}

}  // extern "C"

namespace bisim {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* sh, uint32_t& total) {
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const unsigned nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < nw ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= (unsigned)o) t += y;
        }
        sh[lane] = t;
    }
    __syncthreads();
    uint32_t warp_prefix = w > 0 ? sh[w - 1] : 0u;
    total = sh[nw - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums) {
    __shared__ uint32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t idx = base + i;
        if (idx < n) s += in[idx];
    }
    s = __reduce_add_sync(0xffffffffu, s);
    if ((threadIdx.x & 31u) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = threadIdx.x < (SCAN_THREADS / 32) ? sh[threadIdx.x] : 0u;
        t = __reduce_add_sync(0xffffffffu, t);
        if (threadIdx.x == 0) sums[blockIdx.x] = t;
    }
}

__global__ void k_scan_tile(const uint32_t* in, uint32_t* out, int64_t n,
                            const uint32_t* __restrict__ tile_off, uint32_t* total) {
    __shared__ uint32_t tile[SCAN_TILE];
    __shared__ uint32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t idx = base + i;
        tile[i] = idx < n ? in[idx] : 0u;
    }
    __syncthreads();
    uint32_t loc[SCAN_ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        loc[j] = tile[threadIdx.x * SCAN_ITEMS + j];
        sum += loc[j];
    }
    uint32_t bt;
    uint32_t ex = block_excl_scan(sum, sh, bt);
    const uint32_t off = tile_off ? tile_off[blockIdx.x] : 0u;
    uint32_t run = off + ex;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        tile[threadIdx.x * SCAN_ITEMS + j] = run;
        run += loc[j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = tile[i];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = off + bt;
}

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_WTILE = 32 * RS_ITEMS;
constexpr int RS_TILE = RS_WARPS * RS_WTILE;

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const K* __restrict__ keys, int64_t n, int shift,
                                                         uint32_t* __restrict__ hist, int ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        int64_t idx = base + i;
        if (idx < n) atomicAdd(&h[(unsigned)(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

template <typename K, typename V>
__global__ void __launch_bounds__(RS_THREADS)
    k_rs_scatter(const K* __restrict__ kin, const V* __restrict__ vin, K* __restrict__ kout,
                 V* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ offs,
                 int ntiles) {
    __shared__ uint32_t wc[RS_WARPS][256];
    __shared__ uint32_t dbase[256];  // first tile-local position of each digit
    __shared__ uint32_t gbase[256];  // global position of the tile's first key of each digit
    extern __shared__ __align__(16) unsigned char stage[];  // tile in digit order: keys then values
    K* skey = reinterpret_cast<K*>(stage);
    V* sval = reinterpret_cast<V*>(stage + sizeof(K) * RS_TILE);
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wc[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    const int64_t base = tile0 + (int64_t)w * RS_WTILE;
    K kr[RS_ITEMS];
    V vr[RS_ITEMS];
    uint32_t lr[RS_ITEMS];
    // Keys of a warp are visited in index order (iteration-major, then lane),
    // so counting equal digits before each key gives a stable in-warp rank.
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        const int64_t idx = base + j * 32 + lane;
        const bool valid = idx < n;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        lr[j] = 0;
        if (valid) {
            K k = kin[idx];
            kr[j] = k;
            vr[j] = vin[idx];
            unsigned d = (unsigned)(k >> shift) & 255u;
            unsigned peers = __match_any_sync(vm, d);
            unsigned before = peers & lanemask_lt();
            uint32_t c = wc[w][d];
            lr[j] = c + __popc(before);
            __syncwarp(vm);
            if (before == 0) wc[w][d] = c + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit: warp offsets inside the digit, the digit's tile total, and
    // (block-wide exclusive scan over digits) its first tile-local position
    uint32_t dtot = 0;
    {
        const int d = threadIdx.x;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ww++) {
            uint32_t c = wc[ww][d];
            wc[ww][d] = dtot;
            dtot += c;
        }
        gbase[d] = offs[(int64_t)d * ntiles + blockIdx.x];
    }
    {
        __shared__ uint32_t wsum[RS_WARPS];
        uint32_t x = dtot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        uint32_t wpre = 0;
        for (unsigned ww = 0; ww < w; ww++) wpre += wsum[ww];
        dbase[threadIdx.x] = wpre + x - dtot;
    }
    __syncthreads();
    // stage the tile in digit order
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        const int64_t idx = base + j * 32 + lane;
        if (idx < n) {
            const unsigned d = (unsigned)(kr[j] >> shift) & 255u;
            const uint32_t pos = dbase[d] + wc[w][d] + lr[j];
            skey[pos] = kr[j];
            sval[pos] = vr[j];
        }
    }
    __syncthreads();
    // write runs of equal digits to consecutive global addresses
    const int cnt = (int)(n - tile0 < RS_TILE ? n - tile0 : RS_TILE);
    for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
        const K k = skey[i];
        const unsigned d = (unsigned)(k >> shift) & 255u;
        const uint32_t pos = gbase[d] + (uint32_t)i - dbase[d];
        kout[pos] = k;
        vout[pos] = sval[i];
    }
}

}  // namespace

int scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                       cudaStream_t st) {
    if (n <= 0) {
        if (total) BISIM_CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(uint32_t), st));
        return BISIM_OK;
    }
    const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles == 1) {
        k_scan_tile<<<1, SCAN_THREADS, 0, st>>>(in, out, n, nullptr, total);
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        return BISIM_OK;
    }
    DevMem sums;
    BISIM_TRY(sums.alloc(sizeof(uint32_t) * (size_t)ntiles, st));
    k_scan_reduce<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(in, n, sums.as<uint32_t>());
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    BISIM_TRY(scan_exclusive_u32(sums.as<uint32_t>(), sums.as<uint32_t>(), ntiles, nullptr, st));
    k_scan_tile<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(in, out, n, sums.as<uint32_t>(), total);
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    return BISIM_OK;
}

template <typename K, typename V>
int radix_sort_pairs(K* keys, V* vals, K* keys_alt, V* vals_alt, int64_t n, int bits,
                     cudaStream_t st, bool* result_in_alt) {
    *result_in_alt = false;
    if (n <= 1 || bits <= 0) return BISIM_OK;
    const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    DevMem hist;
    BISIM_TRY(hist.alloc(sizeof(uint32_t) * 256u * (size_t)ntiles, st));
    const size_t smem = (sizeof(K) + sizeof(V)) * RS_TILE;  // staging buffer of the scatter
    BISIM_CUDA_TRY(cudaFuncSetAttribute(k_rs_scatter<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    K* kin = keys;
    V* vin = vals;
    K* kout = keys_alt;
    V* vout = vals_alt;
    bool alt = false;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<K><<<ntiles, RS_THREADS, 0, st>>>(kin, n, shift, hist.as<uint32_t>(), ntiles);
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        BISIM_TRY(scan_exclusive_u32(hist.as<uint32_t>(), hist.as<uint32_t>(), 256ll * ntiles,
                                     nullptr, st));
        k_rs_scatter<K, V><<<ntiles, RS_THREADS, smem, st>>>(kin, vin, kout, vout, n, shift,
                                                             hist.as<uint32_t>(), ntiles);
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        K* tk = kin; kin = kout; kout = tk;
        V* tv = vin; vin = vout; vout = tv;
        alt = !alt;
    }
    *result_in_alt = alt;
    return BISIM_OK;
}

template int radix_sort_pairs<uint32_t, uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*,
                                                  int64_t, int, cudaStream_t, bool*);
template int radix_sort_pairs<uint64_t, uint32_t>(uint64_t*, uint32_t*, uint64_t*, uint32_t*,
                                                  int64_t, int, cudaStream_t, bool*);
template int radix_sort_pairs<uint32_t, uint64_t>(uint32_t*, uint64_t*, uint32_t*, uint64_t*,
                                                  int64_t, int, cudaStream_t, bool*);
template int radix_sort_pairs<uint64_t, uint64_t>(uint64_t*, uint64_t*, uint64_t*, uint64_t*,
                                                  int64_t, int, cudaStream_t, bool*);

}  // namespace bisim
