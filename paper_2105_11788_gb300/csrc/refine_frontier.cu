// Frontier refinement engine: the while-loop of Algorithm 3 (Algorithm 2 with
// rcpp_alg2) where a round touches only the splitter, the transitions into it
// and the blocks of the states that reach it.
//
// Layout: the states of every block b occupy the range [bbeg[b], bend[b]) of
// one of two member buffers (which[b] says which). A split writes all members
// of b to the other buffer over the same range, kept members first and split
// members last, so concurrent splits of different blocks never collide and no
// copy-back is needed.
//
// Round r (stamp = stamp0 + r), two grid barriers:
//   select  C := next label of the FIFO worklist; unstable_C := false
//   mark    for every member t of C and incoming transition s -a-> t:
//           mark[off(s) + order] := stamp, and block(s) is appended once
//           (touched stamp) to a list by size: warp / CTA / whole grid
//   split   every touched block compares each member's marks with its leader's;
//           members that differ move to a new block whose leader is elected
//           (warp and CTA teams: their smallest split state; grid teams:
//           compare-and-swap, the arbitrary write rule); the old label, the
//           new label and (Algorithm 3) C are pushed if they were stable.
// A block of one state cannot split and is never listed.
#include "plan.cuh"

using namespace bisim;

namespace {

constexpr int WARP_MAX = 64;  // blocks up to this size are split by one warp

struct FrontierArgs {
    int32_t n;
    const int32_t* __restrict__ off;
    const int32_t* __restrict__ in_ptr;
    const unsigned long long* __restrict__ in_edge;
    int32_t* block;
    uint32_t* mark;
    unsigned long long* nl64;
    uint32_t* unstable;
    int32_t* elems;  // [2n]
    uint8_t* which;
    int32_t* bbeg;
    int32_t* bend;
    unsigned long long* cnt;
    int32_t* done;
    uint32_t* touched;
    int32_t* tlist;  // [3n]: warp list, CTA list, grid list
    int32_t* queue;  // [n]
    bisim_ctrl* ctrl;
    GridBarrier gb;
    uint32_t stamp0;
    int64_t round_cap;
    int32_t cta_max;
    int alg2;
    int test_hook;
};

__device__ __forceinline__ unsigned long long elect_key(uint32_t stamp, int32_t s) {
    return ((unsigned long long)(0xffffffffu - stamp) << 32) | (uint32_t)s;
}
__device__ __forceinline__ bool key_is(unsigned long long v, uint32_t stamp) {
    return (uint32_t)(v >> 32) == 0xffffffffu - stamp;
}

__device__ __forceinline__ void push(const FrontierArgs& a, int32_t label) {
    unsigned long long pos = atomicAdd(&a.ctrl->q_tail, 1ull);
    a.queue[pos % (unsigned long long)a.n] = label;
}

// unstable_label := true; enqueue it if it was stable
__device__ __forceinline__ void set_unstable(const FrontierArgs& a, int32_t label) {
    if (atomicExch(&a.unstable[label], 1u) == 0u) push(a, label);
}

// Does state s have a mark vector different from the leader's? k = number of
// mark slots of the block's label set; lmask = the leader's marks (k <= 32).
__device__ __forceinline__ bool member_splits(const FrontierArgs& a, int32_t s, int32_t lo, int32_t k,
                                              unsigned lmask, uint32_t stamp) {
    const int32_t os = a.off[s];
    int32_t ks = a.off[s + 1] - os;
    if (ks != k) {
        atomicOr(&a.ctrl->status, ST_INTERNAL);
        ks = min(ks, k);
    }
    bool sp = false;
    if (k <= 32) {
        for (int32_t q = 0; q < ks; q++)
            sp |= (ldcg(&a.mark[os + q]) == stamp) != (bool)((lmask >> q) & 1u);
    } else {
        for (int32_t q = 0; q < ks; q++)
            sp |= (ldcg(&a.mark[os + q]) == stamp) != (ldcg(&a.mark[lo + q]) == stamp);
    }
    return sp;
}

// One warp splits block b (size <= WARP_MAX) entirely.
__device__ void warp_split(const FrontierArgs& a, int32_t b, uint32_t stamp, int32_t C, long long& states) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = lanemask_lt();
    const int w = ldcg(&a.which[b]);
    const int32_t b0 = ldcg(&a.bbeg[b]), e0 = ldcg(&a.bend[b]);
    const int32_t sz = e0 - b0;
    const int32_t* src = a.elems + (size_t)w * a.n;
    int32_t* dst = a.elems + (size_t)(1 - w) * a.n;
    const int32_t lo = a.off[b];
    const int32_t k = a.off[b + 1] - lo;
    unsigned lmask = 0;
    if (k <= 32) lmask = __ballot_sync(0xffffffffu, (int)lane < k && ldcg(&a.mark[lo + lane]) == stamp);
    const int32_t s0 = (int)lane < sz ? ldcg(&src[b0 + lane]) : -1;
    const int32_t s1 = (int)lane + 32 < sz ? ldcg(&src[b0 + 32 + lane]) : -1;
    const bool p0 = s0 >= 0 && member_splits(a, s0, lo, k, lmask, stamp);
    const bool p1 = s1 >= 0 && member_splits(a, s1, lo, k, lmask, stamp);
    const unsigned m0 = __ballot_sync(0xffffffffu, p0), m1 = __ballot_sync(0xffffffffu, p1);
    if (lane == 0) states += sz;
    if ((m0 | m1) == 0u) return;
    const unsigned v0 = __ballot_sync(0xffffffffu, s0 >= 0), v1 = __ballot_sync(0xffffffffu, s1 >= 0);
    const int32_t nsplit = __popc(m0) + __popc(m1);
    const int32_t nkeep = sz - nsplit;
    const int32_t leader = __reduce_min_sync(0xffffffffu, min(p0 ? s0 : NONE, p1 ? s1 : NONE));
    if (s0 >= 0) {
        const int32_t pos = p0 ? nkeep + __popc(m0 & lt) : __popc(~m0 & v0 & lt);
        dst[b0 + pos] = s0;
        if (p0) a.block[s0] = leader;
    }
    if (s1 >= 0) {
        const int32_t pos = p1 ? nkeep + __popc(m0) + __popc(m1 & lt)
                               : __popc(~m0 & v0) + __popc(~m1 & v1 & lt);
        dst[b0 + pos] = s1;
        if (p1) a.block[s1] = leader;
    }
    if (lane == 0) {
        a.which[b] = (uint8_t)(1 - w);
        a.bend[b] = b0 + nkeep;
        a.which[leader] = (uint8_t)(1 - w);
        a.bbeg[leader] = b0 + nkeep;
        a.bend[leader] = e0;
        set_unstable(a, b);
        set_unstable(a, leader);
        if (!a.alg2) set_unstable(a, C);
    }
}

struct CtaShared {
    int wkeep[32];
    int wsplit[32];
    int red[32];
    int leader;
    int kbase;
    int sbase;
    unsigned lmask;
};

// One CTA splits members [seg_lo, seg_hi) of block b. Several CTAs may work
// on disjoint segments of the same block: positions are reserved with one
// 64-bit atomicAdd per chunk (kept count low, split count high), the new
// leader is elected by compare-and-swap, and the CTA that completes the last
// member finalises the ranges and the worklist.
__device__ void cta_split_segment(const FrontierArgs& a, CtaShared& sh, int32_t b, int32_t seg_lo,
                                  int32_t seg_hi, uint32_t stamp, int32_t C, long long& states) {
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const unsigned nw = blockDim.x >> 5;
    const unsigned lt = lanemask_lt();
    const int w = ldcg(&a.which[b]);
    const int32_t b0 = ldcg(&a.bbeg[b]), e0 = ldcg(&a.bend[b]);
    const int32_t* src = a.elems + (size_t)w * a.n;
    int32_t* dst = a.elems + (size_t)(1 - w) * a.n;
    const int32_t lo = a.off[b];
    const int32_t k = a.off[b + 1] - lo;
    if (wid == 0) {
        unsigned lm = 0;
        if (k <= 32) lm = __ballot_sync(0xffffffffu, (int)lane < k && ldcg(&a.mark[lo + lane]) == stamp);
        if (lane == 0) {
            sh.lmask = lm;
            sh.leader = NONE;
        }
    }
    __syncthreads();
    const unsigned lmask = sh.lmask;
    for (int32_t base = seg_lo; base < seg_hi; base += blockDim.x) {
        const int32_t idx = base + threadIdx.x;
        const bool valid = idx < seg_hi;
        const int32_t s = valid ? ldcg(&src[idx]) : -1;
        const bool p = valid && member_splits(a, s, lo, k, lmask, stamp);
        const unsigned bs = __ballot_sync(0xffffffffu, p);
        const unsigned bk = __ballot_sync(0xffffffffu, valid && !p);
        if (lane == 0) {
            sh.wsplit[wid] = __popc(bs);
            sh.wkeep[wid] = __popc(bk);
        }
        int cand = __reduce_min_sync(0xffffffffu, p ? s : NONE);
        if (lane == 0) sh.red[wid] = cand;
        __syncthreads();
        if (wid == 0) {
            int ns = (int)lane < (int)nw ? sh.wsplit[lane] : 0;
            int nk = (int)lane < (int)nw ? sh.wkeep[lane] : 0;
            int c = (int)lane < (int)nw ? sh.red[lane] : NONE;
            // exclusive scans over warps
            int xs = ns, xk = nk;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int ys = __shfl_up_sync(0xffffffffu, xs, o);
                int yk = __shfl_up_sync(0xffffffffu, xk, o);
                if ((int)lane >= o) {
                    xs += ys;
                    xk += yk;
                }
            }
            const int tot_s = __shfl_sync(0xffffffffu, xs, 31);
            const int tot_k = __shfl_sync(0xffffffffu, xk, 31);
            c = __reduce_min_sync(0xffffffffu, c);
            if ((int)lane < (int)nw) {
                sh.wsplit[lane] = xs - ns;
                sh.wkeep[lane] = xk - nk;
            }
            if (lane == 0) {
                if (tot_s > 0 && sh.leader == NONE) {
                    // elect: first writer of this round wins
                    unsigned long long v = ldcg(&a.nl64[b]);
                    for (int it = 0; it < 4; it++) {
                        if (key_is(v, stamp)) {
                            sh.leader = (int32_t)(uint32_t)v;
                            break;
                        }
                        const unsigned long long want = elect_key(stamp, c);
                        const unsigned long long old = atomicCAS(&a.nl64[b], v, want);
                        if (old == v) {
                            sh.leader = c;
                            break;
                        }
                        v = old;
                    }
                    if (sh.leader == NONE) atomicOr(&a.ctrl->status, ST_INTERNAL);
                }
                const unsigned long long add = (unsigned long long)(uint32_t)tot_k |
                                               ((unsigned long long)(uint32_t)tot_s << 32);
                const unsigned long long old = atomicAdd(&a.cnt[b], add);
                sh.kbase = b0 + (int32_t)(uint32_t)old;
                sh.sbase = e0 - (int32_t)(uint32_t)(old >> 32) - tot_s;
            }
        }
        __syncthreads();
        if (valid) {
            int32_t pos;
            if (p) {
                pos = sh.sbase + sh.wsplit[wid] + __popc(bs & lt);
                if (sh.leader != NONE) a.block[s] = sh.leader;
            } else {
                pos = sh.kbase + sh.wkeep[wid] + __popc(bk & lt);
            }
            dst[pos] = s;
        }
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int32_t mine = seg_hi - seg_lo;
        states += mine;
        const int32_t d = atomicAdd(&a.done[b], mine) + mine;
        if (d == e0 - b0) {
            __threadfence();
            const unsigned long long c = atomicExch(&a.cnt[b], 0ull);
            const int32_t kept = (int32_t)(uint32_t)c;
            const int32_t spl = (int32_t)(uint32_t)(c >> 32);
            a.done[b] = 0;
            a.which[b] = (uint8_t)(1 - w);
            a.bend[b] = b0 + kept;
            if (kept + spl != e0 - b0) atomicOr(&a.ctrl->status, ST_INTERNAL);
            if (spl > 0) {
                const int32_t leader = (int32_t)(uint32_t)ldcg(&a.nl64[b]);
                a.which[leader] = (uint8_t)(1 - w);
                a.bbeg[leader] = b0 + kept;
                a.bend[leader] = e0;
                set_unstable(a, b);
                set_unstable(a, leader);
                if (!a.alg2) set_unstable(a, C);
            }
        }
    }
}

__global__ void __launch_bounds__(1024) k_frontier_main(FrontierArgs a) {
    __shared__ CtaShared sh;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int32_t n = a.n;
    unsigned long long tgt = 0;
    long long edges = 0, states = 0;
    if (a.test_hook == 1 && blockIdx.x == 0) return;  // testing: never arrive
    unsigned long long head = a.ctrl->q_head0;
    int64_t r = 0;
    const int32_t big_min = a.cta_max;
    for (;;) {
        r++;
        const uint32_t stamp = a.stamp0 + (uint32_t)r;
        const int par = (int)(r & 1);
        const unsigned long long tail = ldcg(&a.ctrl->q_tail);
        if (head >= tail) break;  // no unstable label: C = bottom
        if (r > a.round_cap) {
            if (gtid == 0) atomicOr(&a.ctrl->status, ST_ROUNDS);
            break;
        }
        const int32_t C = ldcg(&a.queue[head % (unsigned long long)n]);
        head++;
        if (gtid == 0) {
            a.unstable[C] = 0u;
            a.ctrl->n_touched[par ^ 1] = 0;
            a.ctrl->n_mid[par ^ 1] = 0;
            a.ctrl->n_big[par ^ 1] = 0;
        }
        // mark
        {
            const int w = ldcg(&a.which[C]);
            const int32_t b0 = ldcg(&a.bbeg[C]), e0 = ldcg(&a.bend[C]);
            const int32_t* mem = a.elems + (size_t)w * n;
            for (int64_t idx = b0 + gtid; idx < e0; idx += gsz) {
                const int32_t t = ldcg(&mem[idx]);
                const int32_t j0 = a.in_ptr[t], j1 = a.in_ptr[t + 1];
                edges += j1 - j0;
                for (int32_t j = j0; j < j1; j++) {
                    const unsigned long long e = a.in_edge[j];
                    const uint32_t slot = (uint32_t)e;
                    const int32_t s = (int32_t)(e >> 32);
                    a.mark[slot] = stamp;
                    const int32_t b = ldcg(&a.block[s]);
                    if (ldcg(&a.touched[b]) == stamp) continue;
                    if (atomicExch(&a.touched[b], stamp) == stamp) continue;
                    const int32_t sz = ldcg(&a.bend[b]) - ldcg(&a.bbeg[b]);
                    if (sz <= 1) continue;
                    if (sz <= WARP_MAX) {
                        a.tlist[atomicAdd(&a.ctrl->n_touched[par], 1)] = b;
                    } else if (sz <= big_min) {
                        a.tlist[n + atomicAdd(&a.ctrl->n_mid[par], 1)] = b;
                    } else {
                        a.tlist[2 * (size_t)n + atomicAdd(&a.ctrl->n_big[par], 1)] = b;
                    }
                }
            }
        }
        if (!grid_sync(a.gb, tgt)) return;
        // split
        {
            const int32_t ns = ldcg(&a.ctrl->n_touched[par]);
            const int32_t nm = ldcg(&a.ctrl->n_mid[par]);
            const int32_t nb = ldcg(&a.ctrl->n_big[par]);
            const int64_t gw = gtid >> 5, nwarps = gsz >> 5;
            for (int64_t i = gw; i < ns; i += nwarps) warp_split(a, ldcg(&a.tlist[i]), stamp, C, states);
            for (int32_t i = blockIdx.x; i < nm; i += gridDim.x) {
                const int32_t b = ldcg(&a.tlist[n + i]);
                const int32_t b0 = ldcg(&a.bbeg[b]), e0 = ldcg(&a.bend[b]);
                cta_split_segment(a, sh, b, b0, e0, stamp, C, states);
            }
            for (int32_t i = 0; i < nb; i++) {
                const int32_t b = ldcg(&a.tlist[2 * (size_t)n + i]);
                const int32_t b0 = ldcg(&a.bbeg[b]), e0 = ldcg(&a.bend[b]);
                const int32_t sz = e0 - b0;
                const int32_t chunk = (sz + (int32_t)gridDim.x - 1) / (int32_t)gridDim.x;
                const int32_t lo = b0 + (int32_t)blockIdx.x * chunk;
                const int32_t hi = min(e0, lo + chunk);
                if (lo < hi) cta_split_segment(a, sh, b, lo, hi, stamp, C, states);
            }
        }
        if (!grid_sync(a.gb, tgt)) return;
    }
    if (edges) atomicAdd((unsigned long long*)&a.ctrl->edges, (unsigned long long)edges);
    if (states) atomicAdd((unsigned long long*)&a.ctrl->states, (unsigned long long)states);
    if (gtid == 0) a.ctrl->rounds = r;
}

// ---------------------------------------------------------------- set-up

__global__ void k_front_init(const int32_t* __restrict__ block0, int32_t n, int32_t* block,
                             uint32_t* unstable, uint32_t* keys, uint32_t* vals, uint32_t* flags) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz) {
        const int32_t b = block0[i];
        block[i] = b;
        const bool leader = b == (int32_t)i;
        unstable[i] = leader;  // Algorithm 3, lines 1-3
        flags[i] = leader;
        keys[i] = (uint32_t)b;
        vals[i] = (uint32_t)i;
    }
}

// ranges of each label in the label-sorted member array; all members start
// in buffer 0
__global__ void k_front_ranges(const uint32_t* __restrict__ skeys, int32_t n, int32_t* bbeg,
                               int32_t* bend) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz) {
        const uint32_t b = skeys[i];
        if (i == 0 || skeys[i - 1] != b) bbeg[b] = (int32_t)i;
        if (i == n - 1 || skeys[i + 1] != b) bend[b] = (int32_t)i + 1;
    }
}

// initial worklist: every label in increasing order
__global__ void k_front_queue(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos,
                              int32_t n, int32_t* queue) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz)
        if (flags[i]) queue[pos[i]] = (int32_t)i;
}

int ensure_frontier(bisim_plan_s* p) {
    if (p->frontier_ready) return BISIM_OK;
    const size_t n = (size_t)p->n;
    cudaStream_t st = p->st;
    BISIM_TRY(p->elems.alloc(8 * n, st));
    BISIM_TRY(p->which.alloc(n, st));
    BISIM_TRY(p->bbeg.alloc(4 * n, st));
    BISIM_TRY(p->bend.alloc(4 * n, st));
    BISIM_TRY(p->cnt.alloc(8 * n, st));
    BISIM_TRY(p->done.alloc(4 * n, st));
    BISIM_TRY(p->touched.alloc(4 * n, st));
    BISIM_TRY(p->tlist.alloc(12 * n, st));
    BISIM_TRY(p->queue.alloc(4 * n, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->touched.p, 0, 4 * n, st));
    p->frontier_ready = true;
    return BISIM_OK;
}

}  // namespace

namespace bisim {

int refine_frontier(bisim_plan_s* p, bisim_stats* stats) {
    const int32_t n = p->n;
    cudaStream_t st = p->st;
    BISIM_TRY(ensure_frontier(p));
    const int64_t cap = p->opts.round_cap > 0 ? p->opts.round_cap : 3ll * n + p->A + 2;
    uint32_t base;
    BISIM_TRY(reserve_stamps(p, cap + 1, &base));
    bisim_ctrl* c = p->ctrl.as<bisim_ctrl>();
    BISIM_CUDA_TRY(cudaMemsetAsync(c, 0, sizeof(bisim_ctrl), st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->which.p, 0, (size_t)n, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->cnt.p, 0, 8 * (size_t)n, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->done.p, 0, 4 * (size_t)n, st));
    {
        DevMem keys, vals, keys2, flags;
        BISIM_TRY(keys.alloc(4 * (size_t)n, st));
        BISIM_TRY(vals.alloc(4 * (size_t)n, st));
        BISIM_TRY(keys2.alloc(4 * (size_t)n, st));
        BISIM_TRY(flags.alloc(4 * (size_t)n, st));
        const unsigned gn = grid_for(n, 256);
        k_front_init<<<gn, 256, 0, st>>>(p->block0.as<int32_t>(), n, p->block.as<int32_t>(),
                                         p->unstable.as<uint32_t>(), keys.as<uint32_t>(),
                                         vals.as<uint32_t>(), flags.as<uint32_t>());
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        // members grouped by label: sort (label, state); the sorted states are
        // buffer 0 of the member array
        uint32_t* e0 = p->elems.as<uint32_t>();
        bool alt = false;
        BISIM_TRY(radix_sort_pairs<uint32_t, uint32_t>(keys.as<uint32_t>(), vals.as<uint32_t>(),
                                                       keys2.as<uint32_t>(), e0, n,
                                                       ceil_log2_u64((uint64_t)n), st, &alt));
        uint32_t* skeys = alt ? keys2.as<uint32_t>() : keys.as<uint32_t>();
        if (!alt) BISIM_CUDA_TRY(cudaMemcpyAsync(e0, vals.p, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
        k_front_ranges<<<gn, 256, 0, st>>>(skeys, n, p->bbeg.as<int32_t>(), p->bend.as<int32_t>());
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        // worklist: all labels, increasing
        BISIM_TRY(scan_exclusive_u32(flags.as<uint32_t>(), keys.as<uint32_t>(), n,
                                     (uint32_t*)&c->q_tail, st));
        k_front_queue<<<gn, 256, 0, st>>>(flags.as<uint32_t>(), keys.as<uint32_t>(), n,
                                          p->queue.as<int32_t>());
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
    }
    FrontierArgs a;
    a.n = n;
    a.off = p->off.as<int32_t>();
    a.in_ptr = p->in_ptr.as<int32_t>();
    a.in_edge = p->in_edge.as<unsigned long long>();
    a.block = p->block.as<int32_t>();
    a.mark = p->mark.as<uint32_t>();
    a.nl64 = p->nl64.as<unsigned long long>();
    a.unstable = p->unstable.as<uint32_t>();
    a.elems = p->elems.as<int32_t>();
    a.which = p->which.as<uint8_t>();
    a.bbeg = p->bbeg.as<int32_t>();
    a.bend = p->bend.as<int32_t>();
    a.cnt = p->cnt.as<unsigned long long>();
    a.done = p->done.as<int32_t>();
    a.touched = p->touched.as<uint32_t>();
    a.tlist = p->tlist.as<int32_t>();
    a.queue = p->queue.as<int32_t>();
    a.ctrl = c;
    a.gb.counter = &c->barrier;
    a.gb.status = &c->status;
    a.gb.timeout_ns = (unsigned long long)(p->opts.timeout_ms > 0 ? p->opts.timeout_ms : 2000) * 1000000ull;
    a.stamp0 = base;
    a.round_cap = cap;
    a.alg2 = (p->opts.rcpp_alg2 && p->A == 1) ? 1 : 0;
    a.test_hook = p->opts.test_hook;
    const int threads = p->opts.threads > 0 ? p->opts.threads : 512;
    a.cta_max = 16 * threads;
    void* args[] = {&a};
    int grid = 0;
    BISIM_TRY(launch_persistent((const void*)k_frontier_main, args, threads, p, &grid));
    BISIM_TRY(read_ctrl(p));
    p->stamp = base + (uint32_t)std::min<long long>(p->ctrl_h->rounds + 1, cap + 1);
    if (stats) {
        BISIM_TRY(persistent_ms(p, &stats->t_main_ms));
        stats->rounds = p->ctrl_h->rounds;
        stats->edges_visited = p->ctrl_h->edges;
        stats->states_visited = p->ctrl_h->states;
        stats->engine = BISIM_ENGINE_FRONTIER;
        stats->grid_ctas = grid;
    }
    int code = status_to_code(p->ctrl_h->status);
    if (code) {
        set_last_error(p->ctrl_h->status & ST_TIMEOUT ? "grid barrier wait timed out"
                       : p->ctrl_h->status & ST_ROUNDS ? "round cap exceeded"
                                                       : "internal consistency check failed");
        return code;
    }
    return BISIM_OK;
}

}  // namespace bisim
