// Batches of LTSs: one plan over the disjoint union, one refinement launch
// with one CTA per LTS at a time, per-LTS canonical ids.
//
// The union keeps every LTS in its own contiguous range of states
// [state_off[i], state_off[i+1]); its initial partition puts different LTSs
// in different blocks, so no block ever spans two LTSs and the coarsest
// stable refinement of the union is the union of the LTSs' results. One sort,
// one incoming-transition CSR and one pass of preprocessing rounds (one per
// label that occurs in any LTS) serve the whole batch.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>

#include "plan.cuh"

using namespace bisim;

namespace {

constexpr int T = 256;

// index i of the range [off[i], off[i+1]) holding x (off non-decreasing)
__device__ __forceinline__ int find_range(const int64_t* __restrict__ off, int k, int64_t x) {
    int lo = 0, hi = k - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Element ranges of the LTSs (transitions or states), tile by tile: a tile
// of TILE consecutive elements looks up the ranges it meets once (thread 0,
// binary search) and keeps their offsets in shared memory; each element then
// finds its range there. A tile that meets more than TILE_RANGES ranges (many
// tiny or empty LTSs) searches the global offsets per element instead.
constexpr int TILE = 2048;
constexpr int TILE_RANGES = 64;

struct TileRanges {
    int l0, cnt;  // ranges l0 .. l0 + cnt - 1; cnt = 0: use the global offsets
    int64_t off[TILE_RANGES];
};

__device__ __forceinline__ void tile_ranges(const int64_t* __restrict__ off, int k, int64_t i0, int64_t i1,
                                            TileRanges& tr) {
    __syncthreads();  // the previous tile's lookups are done
    if (threadIdx.x == 0) {
        const int l0 = find_range(off, k, i0), l1 = find_range(off, k, i1 - 1);
        tr.l0 = l0;
        tr.cnt = l1 - l0 + 1 <= TILE_RANGES ? l1 - l0 + 1 : 0;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < tr.cnt; j += blockDim.x) tr.off[j] = off[tr.l0 + j];
    __syncthreads();
}

__device__ __forceinline__ int range_of(const int64_t* __restrict__ off, int k, const TileRanges& tr, int64_t i) {
    if (tr.cnt == 0) return find_range(off, k, i);
    int lo = 0, hi = tr.cnt - 1;  // largest j with off[l0 + j] <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tr.off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return tr.l0 + lo;
}

// local (state, label) ids -> union ids, with range checks per LTS
__global__ void k_batch_union(int k, const int64_t* __restrict__ state_off, const int64_t* __restrict__ trans_off,
                              const int32_t* __restrict__ num_act, const int32_t* __restrict__ src,
                              const int32_t* __restrict__ act, const int32_t* __restrict__ dst,
                              const int32_t* __restrict__ init, int64_t M, int64_t N, int32_t* usrc,
                              int32_t* uact, int32_t* udst, int32_t* uinit, int* status) {
    __shared__ TileRanges tr;
    int bad = 0;
    const int64_t tiles_m = (M + TILE - 1) / TILE, tiles_n = (N + TILE - 1) / TILE;
    for (int64_t t = blockIdx.x; t < tiles_m + tiles_n; t += gridDim.x) {
        const bool trans = t < tiles_m;
        const int64_t i0 = (trans ? t : t - tiles_m) * TILE;
        const int64_t i1 = min(i0 + TILE, trans ? M : N);
        tile_ranges(trans ? trans_off : state_off, k, i0, i1, tr);
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            if (trans) {
                const int li = range_of(trans_off, k, tr, i);
                const int64_t s0 = state_off[li];
                const int64_t ni = state_off[li + 1] - s0;
                const int32_t s = src[i], d = dst[i], a = act ? act[i] : 0;
                if ((int64_t)(unsigned)s >= ni || (int64_t)(unsigned)d >= ni ||
                    (unsigned)a >= (unsigned)num_act[li]) {
                    bad = 1;
                    usrc[i] = 0;
                    udst[i] = 0;
                    uact[i] = 0;
                } else {
                    usrc[i] = (int32_t)(s0 + s);
                    udst[i] = (int32_t)(s0 + d);
                    uact[i] = a;
                }
            } else {
                const int li = range_of(state_off, k, tr, i);
                const int64_t s0 = state_off[li];
                const int64_t ni = state_off[li + 1] - s0;
                const int32_t v = init ? init[i] : 0;
                if ((int64_t)(unsigned)v >= ni) {
                    bad = 1;
                    uinit[i] = (int32_t)s0;
                } else {
                    uinit[i] = (int32_t)(s0 + v);
                }
            }
        }
    }
    if (bad) atomicOr(status, ST_INVALID);
}

// union canonical ids -> ids local to each LTS (the first state of every LTS
// starts its first block, so subtracting its id renumbers from 0)
__global__ void k_batch_base(int k, const int64_t* __restrict__ state_off, const int32_t* __restrict__ out,
                             int32_t* base) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
        base[i] = state_off[i + 1] > state_off[i] ? out[state_off[i]] : 0;
}

// local ids and the block count of every LTS (largest local id + 1; one
// atomicMax per group of lanes of a warp that hold states of the same LTS)
__global__ void k_batch_local(int k, const int64_t* __restrict__ state_off, const int32_t* __restrict__ base,
                              int64_t N, int32_t* out, int32_t* nblocks) {
    __shared__ TileRanges tr;
    const unsigned lane = threadIdx.x & 31u;
    for (int64_t t = blockIdx.x; t * TILE < N; t += gridDim.x) {
        const int64_t i0 = t * TILE, i1 = min(i0 + TILE, N);
        tile_ranges(state_off, k, i0, i1, tr);
        // trip count rounded up to whole warps so that every lane reaches the match
        for (int64_t i = i0 + threadIdx.x; i - lane < i1; i += blockDim.x) {
            int li = -1 - (int)lane, v = 0;
            if (i < i1) {
                li = range_of(state_off, k, tr, i);
                v = out[i] - base[li];
                out[i] = v;
            }
            // lanes hold consecutive states, so the lanes of one LTS are a
            // contiguous run: a suffix max leaves the run's max at its lowest lane
            const unsigned peers = __match_any_sync(0xffffffffu, li);
            int mx = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_down_sync(0xffffffffu, mx, o);
                if (lane + o < 32u && ((peers >> (lane + o)) & 1u)) mx = max(mx, y);
            }
            if (li >= 0 && (peers & lanemask_lt()) == 0u) atomicMax(&nblocks[li], mx + 1);
        }
    }
}

int batch_plan_build(bisim_plan_s* p, int32_t k, const int64_t* state_off_h, const int64_t* trans_off_h,
                     const int32_t* num_act_h, const int32_t* src, const int32_t* act, const int32_t* dst,
                     const int32_t* init) {
    cudaStream_t st = p->st;
    const int64_t N = state_off_h[k], M = trans_off_h[k];
    p->batch_k = k;
    p->state_off_h.assign(state_off_h, state_off_h + k + 1);
    p->batch_act_h.assign(num_act_h, num_act_h + k);
    BISIM_TRY(p->state_off.alloc(8 * ((size_t)k + 1), st));
    BISIM_TRY(p->batch_act.alloc(4 * (size_t)k, st));
    BISIM_TRY(p->batch_order.alloc(4 * (size_t)k, st));
    BISIM_TRY(p->inst_rounds.alloc(8 * (size_t)k, st));
    BISIM_CUDA_TRY(cudaMemcpyAsync(p->state_off.p, state_off_h, 8 * ((size_t)k + 1), cudaMemcpyHostToDevice, st));
    BISIM_CUDA_TRY(cudaMemcpyAsync(p->batch_act.p, num_act_h, 4 * (size_t)k, cudaMemcpyHostToDevice, st));
    std::vector<int32_t> order((size_t)k);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        const int64_t wa = (state_off_h[a + 1] - state_off_h[a]) + (trans_off_h[a + 1] - trans_off_h[a]);
        const int64_t wb = (state_off_h[b + 1] - state_off_h[b]) + (trans_off_h[b + 1] - trans_off_h[b]);
        return wa > wb;
    });
    BISIM_CUDA_TRY(cudaMemcpyAsync(p->batch_order.p, order.data(), 4 * (size_t)k, cudaMemcpyHostToDevice, st));
    p->batch_order_h = order;
    DevMem toff, usrc, uact, udst, uinit;
    BISIM_TRY(toff.alloc(8 * ((size_t)k + 1), st));
    BISIM_CUDA_TRY(cudaMemcpyAsync(toff.p, trans_off_h, 8 * ((size_t)k + 1), cudaMemcpyHostToDevice, st));
    BISIM_TRY(usrc.alloc(4 * (size_t)M, st));
    BISIM_TRY(uact.alloc(4 * (size_t)M, st));
    BISIM_TRY(udst.alloc(4 * (size_t)M, st));
    BISIM_TRY(uinit.alloc(4 * (size_t)N, st));
    BISIM_TRY(p->ctrl.alloc(sizeof(bisim_ctrl), st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->ctrl.p, 0, sizeof(bisim_ctrl), st));
    k_batch_union<<<(unsigned)std::min<int64_t>((M + TILE - 1) / TILE + (N + TILE - 1) / TILE, 1 << 20), T, 0,
                    st>>>(
        k, p->state_off.as<int64_t>(), toff.as<int64_t>(), p->batch_act.as<int32_t>(), src, act, dst, init, M, N,
        usrc.as<int32_t>(), uact.as<int32_t>(), udst.as<int32_t>(), uinit.as<int32_t>(),
        &p->ctrl.as<bisim_ctrl>()->status);
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    BISIM_TRY(read_ctrl(p));
    if (p->ctrl_h->status & ST_INVALID) {
        set_last_error("a state, label or initial label is out of range for its LTS");
        return BISIM_EINVAL;
    }
    return plan_build(p, usrc.as<int32_t>(), uact.as<int32_t>(), udst.as<int32_t>(), uinit.as<int32_t>());
}

}  // namespace

extern "C" {

int bisim_batch_plan(int32_t k, const int64_t* state_off_h, const int64_t* trans_off_h, const int32_t* num_act_h,
                     const int32_t* src, const int32_t* act, const int32_t* dst, const int32_t* init_block,
                     const bisim_opts* opts, void* stream, bisim_plan_t* out) {
    if (!out) return BISIM_EINVAL;
    *out = nullptr;
    if (opts && (opts->threads < 0 || opts->threads > 1024 || (opts->threads & 31) || opts->wide_threads < 0 ||
                 opts->wide_threads > 1024 || (opts->wide_threads & 31))) {
        set_last_error("opts.threads / wide_threads must be multiples of 32 in [32, 1024] (or 0)");
        return BISIM_EINVAL;
    }
    if (opts && opts->engine == BISIM_ENGINE_PAIR) {
        set_last_error("bisim_batch_plan: the batch path runs frontier rounds; the pair engine is for single LTSs");
        return BISIM_ENOTSUP;
    }
    if (k < 1 || !state_off_h || !trans_off_h || !num_act_h) {
        set_last_error("bisim_batch_plan: need k >= 1 and the offset / label-count arrays");
        return BISIM_EINVAL;
    }
    int32_t A = 1;
    for (int32_t i = 0; i < k; i++) {
        if (state_off_h[i + 1] < state_off_h[i] || trans_off_h[i + 1] < trans_off_h[i] || num_act_h[i] < 1) {
            set_last_error("bisim_batch_plan: offsets must be non-decreasing and label counts >= 1");
            return BISIM_EINVAL;
        }
        A = std::max(A, num_act_h[i]);
    }
    if (state_off_h[0] != 0 || trans_off_h[0] != 0 || state_off_h[k] > 0x7fffffffll ||
        trans_off_h[k] > 0x7fffffffll || (trans_off_h[k] > 0 && (!src || !dst))) {
        set_last_error("bisim_batch_plan: offsets must start at 0 and the totals must be below 2^31");
        return BISIM_EINVAL;
    }
    bisim_plan_s* p = new (std::nothrow) bisim_plan_s();
    if (!p) return BISIM_ENOMEM;
    p->n = (int32_t)state_off_h[k];
    p->m = trans_off_h[k];
    p->A = A;
    p->st = (cudaStream_t)stream;
    if (opts) p->opts = *opts;
    int rc = device_setup(p);
    if (rc == BISIM_OK) {
        g_launches = 0;
        cudaEventRecord(p->ev0, p->st);
        rc = batch_plan_build(p, k, state_off_h, trans_off_h, num_act_h, src, act, dst, init_block);
        p->plan_launches = g_launches;
        float ms = 0;
        if (rc == BISIM_OK && cudaEventRecord(p->ev1, p->st) == cudaSuccess &&
            cudaEventSynchronize(p->ev1) == cudaSuccess && cudaEventElapsedTime(&ms, p->ev0, p->ev1) == cudaSuccess)
            p->t_plan_ms = ms;
    }
    if (rc) {
        cudaStreamSynchronize(p->st);
        delete p;
        return rc;
    }
    *out = p;
    return BISIM_OK;
}

int bisim_batch_refine(bisim_plan_t p, int32_t* out_block, bisim_stats* stats, bisim_batch_inst* inst_h) {
    if (!p || p->batch_k < 1 || (p->n > 0 && !out_block)) {
        set_last_error("bisim_batch_refine: needs a plan from bisim_batch_plan and an output array");
        return BISIM_EINVAL;
    }
    bisim_stats s;
    std::memset(&s, 0, sizeof(s));
    s.n = p->n;
    s.m = p->m;
    s.num_act = p->A;
    s.mark_length = p->L;
    s.pre_rounds = p->pre_rounds;
    s.initial_blocks = p->initial_blocks;
    s.t_plan_ms = p->t_plan_ms;
    s.t_pre_ms = p->t_pre_ms;
    const int32_t k = p->batch_k;
    cudaStream_t st = p->st;
    BISIM_CUDA_TRY(cudaEventRecord(p->ev0, st));
    g_launches = 0;
    std::vector<long long> rounds;
    int rc = BISIM_OK;
    if (p->n > 0) {
        rc = refine_frontier_batch(p, &s, rounds);
        if (rc == BISIM_OK) rc = write_output(p, out_block, &s.num_blocks);
    } else {
        rounds.assign((size_t)k, 1);
    }
    std::vector<int32_t> nb((size_t)k, 0);
    if (rc == BISIM_OK && p->n > 0 && !p->opts.raw_labels) {
        DevMem base, nbd;
        BISIM_TRY(base.alloc(4 * (size_t)k, st));
        BISIM_TRY(nbd.alloc(4 * (size_t)k, st));
        BISIM_CUDA_TRY(cudaMemsetAsync(nbd.p, 0, 4 * (size_t)k, st));
        k_batch_base<<<grid_for(k, T), T, 0, st>>>(k, p->state_off.as<int64_t>(), out_block, base.as<int32_t>());
        BISIM_LAUNCHED();
        k_batch_local<<<(unsigned)std::min<int64_t>(((int64_t)p->n + TILE - 1) / TILE, 1 << 20), T, 0, st>>>(
            k, p->state_off.as<int64_t>(), base.as<int32_t>(), p->n, out_block, nbd.as<int32_t>());
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        BISIM_CUDA_TRY(cudaMemcpyAsync(nb.data(), nbd.p, 4 * (size_t)k, cudaMemcpyDeviceToHost, st));
        BISIM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (rc == BISIM_OK) {
        float ms = 0;
        BISIM_CUDA_TRY(cudaEventRecord(p->ev1, st));
        BISIM_CUDA_TRY(cudaEventSynchronize(p->ev1));
        BISIM_CUDA_TRY(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        s.t_refine_ms = ms;
        if (inst_h)
            for (int32_t i = 0; i < k; i++) {
                inst_h[i].rounds = rounds[(size_t)i];
                inst_h[i].num_blocks = nb[(size_t)i];
            }
    }
    s.launches = p->plan_launches + g_launches;
    p->last = s;
    if (stats) *stats = s;
    return rc;
}

}  // extern "C"
