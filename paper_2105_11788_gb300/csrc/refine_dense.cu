// Dense refinement engine: the while-loop of Algorithm 3 (Algorithm 2 with
// rcpp_alg2) in one persistent cooperative kernel, four grid barriers per
// round, every concurrent write resolved by the priority rule:
//   select   C := smallest label with unstable_C (block-reduced atomicMin)
//   mark     for every state t with block_t = C and every incoming transition
//            s -a-> t: mark[off(s) + order] := round stamp
//   compare  split_s := some slot of s differs from the same slot of its
//            leader block_s; split states atomicMin (round, s) into
//            new_leader[block_s]
//   relabel  split states move to new_leader[block_s]; both labels and C
//            become unstable (C only for Algorithm 3)
// Marks are round stamps, so no reset pass is needed; new_leader words carry
// the round in their high half for the same reason. The loop ends in the
// iteration that finds no unstable label, which is counted, as in Table 1.
#include "plan.cuh"

using namespace bisim;

namespace {

struct DenseArgs {
    int32_t n;
    const int32_t* __restrict__ off;
    const int32_t* __restrict__ in_ptr;
    const unsigned long long* __restrict__ in_edge;
    int32_t* block;
    uint32_t* mark;
    unsigned long long* nl64;
    uint32_t* unstable;
    uint8_t* split;
    bisim_ctrl* ctrl;
    GridBarrier gb;
    uint32_t stamp0;
    int64_t round_cap;
    int alg2;
    int test_hook;
};

__device__ __forceinline__ unsigned long long elect_key(uint32_t stamp, int32_t s) {
    return ((unsigned long long)(0xffffffffu - stamp) << 32) | (uint32_t)s;
}

__global__ void k_dense_init(const int32_t* __restrict__ block0, int32_t n, int32_t* block,
                             uint32_t* unstable) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz) {
        int32_t b = block0[i];
        block[i] = b;
        unstable[i] = b == (int32_t)i;  // Algorithm 3, lines 1-3
    }
}

// the select, mark and relabel loops handle U states per thread per step and
// issue their loads before they use any of them, so a thread keeps several
// loads in flight; the compare step reads Q slots per lane per step
constexpr int U = 4;
constexpr int Q = 4;

template <int MAXT, int MINB>  // launch bounds: most threads per CTA, CTAs per SM to fit
__global__ void __launch_bounds__(MAXT, MINB) k_dense_main(DenseArgs a) {
    __shared__ int sh[32];
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int64_t lane = threadIdx.x & 31;
    const int32_t n = a.n;
    unsigned long long tgt = 0;
    long long edges = 0, states = 0;
    if (a.test_hook == 1 && blockIdx.x == 0) return;  // testing: never arrive
    int64_t r = 0;
    for (;;) {
        r++;
        const uint32_t stamp = a.stamp0 + (uint32_t)r;
        // select: smallest unstable label (this thread's states in increasing order)
        int loc = NONE;
        for (int64_t i0 = gtid; i0 < n && loc == NONE; i0 += U * gsz) {
            uint32_t v[U];
#pragma unroll
            for (int u = 0; u < U; u++) v[u] = i0 + u * gsz < n ? ldcg(&a.unstable[i0 + u * gsz]) : 0u;
#pragma unroll
            for (int u = 0; u < U; u++)
                if (v[u] && loc == NONE) loc = (int)(i0 + u * gsz);
        }
        const int bm = block_reduce_min(loc, sh);
        if (threadIdx.x == 0 && bm != NONE) atomicMin(&a.ctrl->sel[r & 1], bm);
        if (gtid == 0) a.ctrl->sel[(r + 1) & 1] = NONE;
        if (!grid_sync(a.gb, tgt)) return;
        const int C = ldcg(&a.ctrl->sel[r & 1]);
        if (C < 0 || C >= n) break;  // no unstable label: C = bottom
        if (r > a.round_cap) {
            if (gtid == 0) atomicOr(&a.ctrl->status, ST_ROUNDS);
            break;
        }
        // mark
        if (gtid == 0) a.unstable[C] = 0;
        for (int64_t t0 = gtid; t0 < n; t0 += U * gsz) {
            int32_t bt[U];
#pragma unroll
            for (int u = 0; u < U; u++) bt[u] = t0 + u * gsz < n ? ldcg(&a.block[t0 + u * gsz]) : -1;
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (bt[u] != C) continue;
                const int64_t t = t0 + u * gsz;
                const int32_t j1 = a.in_ptr[t + 1];
                for (int32_t j = a.in_ptr[t]; j < j1; j++) a.mark[(uint32_t)a.in_edge[j]] = stamp;
                edges += j1 - a.in_ptr[t];
            }
        }
        if (!grid_sync(a.gb, tgt)) return;
        // compare and elect: a warp takes 32 consecutive states, whose mark
        // slots form one contiguous range [base, end); lanes read that range
        // coalesced, compare each slot with the same slot of its state's leader
        // and set the state's bit in `diff` on a mismatch. The loop test uses
        // the warp's first state, so all lanes take every step together.
        for (int64_t w0 = gtid - lane; w0 < n; w0 += gsz) {
            const int64_t s = w0 + lane;
            const bool in = s < n;
            const int32_t b = in ? ldcg(&a.block[s]) : 0;
            const int32_t o = in ? a.off[s] : 0;
            const int32_t e = in ? a.off[s + 1] : 0;
            const int32_t ob = in ? a.off[b] : 0;
            if (in && a.off[b + 1] - ob != e - o)  // leader has a different label set: preprocessing broken
                atomicOr(&a.ctrl->status, ST_INTERNAL);
            const int nv = n - w0 < 32 ? (int)(n - w0) : 32;  // lanes holding a state
            const int32_t base = __shfl_sync(0xffffffffu, o, 0);
            const int32_t end = __shfl_sync(0xffffffffu, e, nv - 1);
            unsigned diff = 0;
            for (int32_t j0 = base; j0 < end; j0 += 32 * Q) {
                uint32_t x[Q], y[Q];
                int idx[Q];
#pragma unroll
                for (int u = 0; u < Q; u++) {
                    const int32_t jj = j0 + u * 32 + (int32_t)lane;
                    // owner of slot jj: the largest lane i < nv with o_i <= jj
                    int lo = 0;
#pragma unroll
                    for (int st = 16; st > 0; st >>= 1) {
                        const int cand = lo + st;
                        const int32_t oc = __shfl_sync(0xffffffffu, o, cand & 31);
                        if (cand < nv && oc <= jj) lo = cand;
                    }
                    idx[u] = lo;
                    const int32_t q = jj - __shfl_sync(0xffffffffu, o, lo);
                    const int32_t lj = __shfl_sync(0xffffffffu, ob, lo) + q;
                    const bool ok = jj < end;
                    x[u] = ok ? ldcg(&a.mark[jj]) : 0u;
                    y[u] = ok ? ldcg(&a.mark[lj]) : 0u;
                }
#pragma unroll
                for (int u = 0; u < Q; u++)
                    if (j0 + u * 32 + (int32_t)lane < end && (x[u] == stamp) != (y[u] == stamp)) diff |= 1u << idx[u];
            }
            diff = __reduce_or_sync(0xffffffffu, diff);
            const bool sp = in && ((diff >> lane) & 1u);
            if (in) {
                a.split[s] = sp;
                states++;
            }
            // lanes hold consecutive states: the lowest lane of a group of
            // splitting states with the same block holds the group's minimum;
            // it writes only if the election word can still drop
            const unsigned peers = __match_any_sync(0xffffffffu, sp ? b : -1);
            if (sp && (peers & lanemask_lt()) == 0u) {
                const unsigned long long key = elect_key(stamp, (int32_t)s);
                if (ldcg(&a.nl64[b]) > key) atomicMin(&a.nl64[b], key);
            }
        }
        if (!grid_sync(a.gb, tgt)) return;
        // relabel
        for (int64_t s0 = gtid; s0 < n; s0 += U * gsz) {
            uint8_t f[U];
            int32_t bb[U], v[U];
#pragma unroll
            for (int u = 0; u < U; u++) f[u] = s0 + u * gsz < n ? ldcg(&a.split[s0 + u * gsz]) : (uint8_t)0;
#pragma unroll
            for (int u = 0; u < U; u++) bb[u] = f[u] ? ldcg(&a.block[s0 + u * gsz]) : 0;
#pragma unroll
            for (int u = 0; u < U; u++) v[u] = f[u] ? (int32_t)(uint32_t)ldcg(&a.nl64[bb[u]]) : 0;
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (!f[u]) continue;
                a.block[s0 + u * gsz] = v[u];
                a.unstable[bb[u]] = 1;
                a.unstable[v[u]] = 1;
                if (!a.alg2) a.unstable[C] = 1;
            }
        }
        if (!grid_sync(a.gb, tgt)) return;
    }
    if (edges) atomicAdd((unsigned long long*)&a.ctrl->edges, (unsigned long long)edges);
    if (states) atomicAdd((unsigned long long*)&a.ctrl->states, (unsigned long long)states);
    if (gtid == 0) a.ctrl->rounds = r;
}

}  // namespace

namespace bisim {

int refine_dense(bisim_plan_s* p, bisim_stats* stats) {
    const int32_t n = p->n;
    cudaStream_t st = p->st;
    const int64_t cap = p->opts.round_cap > 0 ? p->opts.round_cap : 3ll * n + p->A + 2;
    uint32_t base;
    BISIM_TRY(reserve_stamps(p, cap + 1, &base));
    bisim_ctrl* c = p->ctrl.as<bisim_ctrl>();
    BISIM_CUDA_TRY(cudaMemsetAsync(c, 0, sizeof(bisim_ctrl), st));
    BISIM_CUDA_TRY(cudaMemsetAsync(c->sel, 0x7f, sizeof(c->sel), st));  // 0x7f7f7f7f > any label
    k_dense_init<<<grid_for(n, 256), 256, 0, st>>>(p->block0.as<int32_t>(), n, p->block.as<int32_t>(),
                                                   p->unstable.as<uint32_t>());
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    DenseArgs a;
    a.n = n;
    a.off = p->off.as<int32_t>();
    a.in_ptr = p->in_ptr.as<int32_t>();
    a.in_edge = p->in_edge.as<unsigned long long>();
    a.block = p->block.as<int32_t>();
    a.mark = p->mark.as<uint32_t>();
    a.nl64 = p->nl64.as<unsigned long long>();
    a.unstable = p->unstable.as<uint32_t>();
    a.split = p->split.as<uint8_t>();
    a.ctrl = c;
    a.gb.counter = &c->barrier;
    a.gb.status = &c->status;
    a.gb.timeout_ns = (unsigned long long)(p->opts.timeout_ms > 0 ? p->opts.timeout_ms : 2000) * 1000000ull;
    a.stamp0 = base;
    a.round_cap = cap;
    a.alg2 = (p->opts.rcpp_alg2 && p->A == 1) ? 1 : 0;
    a.test_hook = p->opts.test_hook;
    void* args[] = {&a};
    int threads = p->opts.threads > 0 ? p->opts.threads : 512;
    int grid = 0;
    // rounds over millions of states want many loads in flight (more CTAs per
    // SM); small LTSs want the cheaper barrier of one CTA per SM
    // large LTSs: 512-thread CTAs bounded to fit four per SM (full occupancy)
    const bool big = n >= (1 << 20) && threads <= 512;
    const void* fn = big ? (const void*)k_dense_main<512, 4> : (const void*)k_dense_main<1024, 1>;
    BISIM_TRY(launch_persistent(fn, args, threads, p, &grid, big ? 4 : 1));
    BISIM_TRY(read_ctrl(p));
    if (stats) BISIM_TRY(persistent_ms(p, &stats->t_main_ms));
    p->stamp = base + (uint32_t)std::min<long long>(p->ctrl_h->rounds + 1, cap + 1);
    if (stats) {
        stats->rounds = p->ctrl_h->rounds;
        stats->steps = p->ctrl_h->rounds;
        stats->edges_visited = p->ctrl_h->edges;
        stats->states_visited = p->ctrl_h->states;
        stats->engine = BISIM_ENGINE_DENSE;
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
