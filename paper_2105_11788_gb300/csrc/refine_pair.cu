// (C, a)-pair engine: Algorithm 2 applied with one action label at a time,
// in one persistent cooperative kernel, every concurrent write resolved by
// the priority rule. An iteration takes the splitter pair (C, a):
//   select   (when C has been used with every label that occurs)
//            C := smallest unstable label (block-reduced atomicMin);
//            unstable_C := false
//   mark     for every state t with block_t = C and every incoming
//            transition s -a-> t: pmark[s] := round stamp (one flag per
//            state, as in Algorithm 2)
//   compare  split_s := pmark[s] differs from pmark[block_s]; split states
//            atomicMin (round, s) into new_leader[block_s]
//   relabel  split states move to new_leader[block_s]; both labels become
//            unstable (the splitter is not set unstable again: Algorithm 2)
// Labels are taken in increasing order. No action-set preprocessing is
// needed: a block's first selection splits it by each label. With a single
// label this is Algorithm 2 iteration for iteration. Marks are round stamps
// and election words carry the round, so nothing is reset between rounds.
#include "plan.cuh"

using namespace bisim;

namespace {

struct PairArgs {
    int32_t n;
    int32_t n_labels;                  // labels that occur (0: no transitions)
    const int32_t* __restrict__ labels;  // [n_labels], increasing
    const int32_t* __restrict__ in_ptr;
    const unsigned long long* __restrict__ in_edge;  // (source << 32) | mark slot
    const int32_t* __restrict__ slot_act;            // label of each mark slot
    int32_t* block;
    uint32_t* pmark;
    unsigned long long* nl64;
    uint32_t* unstable;
    uint8_t* split;
    bisim_ctrl* ctrl;
    GridBarrier gb;
    uint32_t stamp0;
    int64_t round_cap;
    int test_hook;
};

__device__ __forceinline__ unsigned long long pair_key(uint32_t stamp, int32_t s) {
    return ((unsigned long long)(0xffffffffu - stamp) << 32) | (uint32_t)s;
}

__global__ void k_pair_init(const int32_t* __restrict__ block0, int32_t n, int32_t* block, uint32_t* unstable) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz) {
        const int32_t b = block0[i];
        block[i] = b;
        unstable[i] = b == (int32_t)i;  // every initial leader is unstable
    }
}

__global__ void __launch_bounds__(1024) k_pair_main(PairArgs a) {
    __shared__ int sh[32];
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int32_t n = a.n;
    unsigned long long tgt = 0;
    long long edges = 0, states = 0;
    if (a.test_hook == 1 && blockIdx.x == 0) return;  // testing: never arrive
    const int nl = max(a.n_labels, 1);
    int64_t r = 0, q = 0;  // iterations, selections
    int32_t C = -1;
    int li = 0;  // index of this iteration's label
    for (;;) {
        r++;
        const uint32_t stamp = a.stamp0 + (uint32_t)r;
        if (li == 0) {
            // select: smallest unstable label
            q++;
            int loc = NONE;
            for (int64_t i = gtid; i < n; i += gsz)
                if (ldcg(&a.unstable[i])) {
                    loc = (int)i;
                    break;
                }
            const int bm = block_reduce_min(loc, sh);
            if (threadIdx.x == 0 && bm != NONE) atomicMin(&a.ctrl->sel[q & 1], bm);
            if (gtid == 0) a.ctrl->sel[(q + 1) & 1] = NONE;
            if (!grid_sync(a.gb, tgt)) return;
            C = ldcg(&a.ctrl->sel[q & 1]);
            if (C < 0 || C >= n) break;  // no unstable label
        }
        if (r > a.round_cap) {
            if (gtid == 0) atomicOr(&a.ctrl->status, ST_ROUNDS);
            break;
        }
        if (li == 0 && gtid == 0) a.unstable[C] = 0u;
        const int32_t lab = a.n_labels > 0 ? a.labels[li] : -1;
        // mark
        for (int64_t t = gtid; t < n; t += gsz) {
            if (ldcg(&a.block[t]) != C) continue;
            const int32_t j1 = a.in_ptr[t + 1];
            for (int32_t j = a.in_ptr[t]; j < j1; j++) {
                const unsigned long long e = a.in_edge[j];
                if (a.slot_act[(uint32_t)e] == lab) a.pmark[(int32_t)(e >> 32)] = stamp;
            }
            edges += j1 - a.in_ptr[t];
        }
        if (!grid_sync(a.gb, tgt)) return;
        // compare and elect (trip count rounded up to whole warps so that
        // every lane reaches the match)
        const int64_t nlim = (n + 31) & ~(int64_t)31;
        for (int64_t s = gtid; s < nlim; s += gsz) {
            if (s >= n) {
                __match_any_sync(0xffffffffu, -1);
                continue;
            }
            const int32_t b = ldcg(&a.block[s]);
            const bool sp = (ldcg(&a.pmark[s]) == stamp) != (ldcg(&a.pmark[b]) == stamp);
            states++;
            a.split[s] = sp;
            // lanes hold consecutive states: the lowest lane of a group of
            // splitting states with the same block holds the group's minimum
            const unsigned peers = __match_any_sync(0xffffffffu, sp ? b : -1);
            if (sp && (peers & lanemask_lt()) == 0u) atomicMin(&a.nl64[b], pair_key(stamp, (int32_t)s));
        }
        if (!grid_sync(a.gb, tgt)) return;
        // relabel
        for (int64_t s = gtid; s < n; s += gsz) {
            if (!a.split[s]) continue;
            const int32_t b = a.block[s];
            const int32_t v = (int32_t)(uint32_t)ldcg(&a.nl64[b]);
            a.block[s] = v;
            a.unstable[b] = 1;
            a.unstable[v] = 1;
        }
        if (!grid_sync(a.gb, tgt)) return;
        li = li + 1 == nl ? 0 : li + 1;
    }
    if (edges) atomicAdd((unsigned long long*)&a.ctrl->edges, (unsigned long long)edges);
    if (states) atomicAdd((unsigned long long*)&a.ctrl->states, (unsigned long long)states);
    if (gtid == 0) a.ctrl->rounds = r;
}

}  // namespace

namespace bisim {

int refine_pair(bisim_plan_s* p, bisim_stats* stats) {
    const int32_t n = p->n;
    cudaStream_t st = p->st;
    const int64_t nl = std::max<int64_t>(p->n_labels, 1);
    // selections <= 2n (a label becomes unstable when created or split), so
    // iterations <= 2n * labels + 1
    const int64_t cap = p->opts.round_cap > 0 ? p->opts.round_cap : (2ll * n + 2) * nl + 2;
    uint32_t base;
    BISIM_TRY(reserve_stamps(p, cap + 1, &base));
    bisim_ctrl* c = p->ctrl.as<bisim_ctrl>();
    BISIM_CUDA_TRY(cudaMemsetAsync(c, 0, sizeof(bisim_ctrl), st));
    BISIM_CUDA_TRY(cudaMemsetAsync(c->sel, 0x7f, sizeof(c->sel), st));  // 0x7f7f7f7f > any label
    k_pair_init<<<grid_for(n, 256), 256, 0, st>>>(p->block0.as<int32_t>(), n, p->block.as<int32_t>(),
                                                  p->unstable.as<uint32_t>());
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    PairArgs a;
    a.n = n;
    a.n_labels = (int32_t)p->n_labels;
    a.labels = p->labels.as<int32_t>();
    a.in_ptr = p->in_ptr.as<int32_t>();
    a.in_edge = p->in_edge.as<unsigned long long>();
    BISIM_TRY(ensure_slot_arrays(p));
    a.slot_act = p->slot_act.as<int32_t>();
    a.block = p->block.as<int32_t>();
    a.pmark = p->lmark.as<uint32_t>();
    a.nl64 = p->nl64.as<unsigned long long>();
    a.unstable = p->unstable.as<uint32_t>();
    a.split = p->split.as<uint8_t>();
    a.ctrl = c;
    a.gb.counter = &c->barrier;
    a.gb.status = &c->status;
    a.gb.timeout_ns = (unsigned long long)(p->opts.timeout_ms > 0 ? p->opts.timeout_ms : 2000) * 1000000ull;
    a.stamp0 = base;
    a.round_cap = cap;
    a.test_hook = p->opts.test_hook;
    void* args[] = {&a};
    const int threads = p->opts.threads > 0 ? p->opts.threads : 512;
    int grid = 0;
    BISIM_TRY(launch_persistent((const void*)k_pair_main, args, threads, p, &grid));
    BISIM_TRY(read_ctrl(p));
    if (stats) BISIM_TRY(persistent_ms(p, &stats->t_main_ms));
    p->stamp = base + (uint32_t)std::min<long long>(p->ctrl_h->rounds + 1, cap + 1);
    if (stats) {
        stats->rounds = p->ctrl_h->rounds;
        stats->steps = p->ctrl_h->rounds;
        stats->edges_visited = p->ctrl_h->edges;
        stats->states_visited = p->ctrl_h->states;
        stats->engine = BISIM_ENGINE_PAIR;
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
