// Frontier refinement engine: the while-loop of Algorithm 3 (Algorithm 2 with
// rcpp_alg2) where a splitter iteration touches only the splitter C, the
// transitions into C, the states that reach C and - when a block's leader
// reaches C - the part of that block that moves out.
//
// Layout (refinable partition): the members of block b occupy
// elems[bbeg[b] .. bend[b]) and loc[s] is the position of state s. Splits
// rearrange a block's range in place by swapping members.
//
// A splitter iteration (stamp = stamp0 + round):
//   select  C := next label of the size-bucketed worklist; unstable_C := false
//   mark    one warp per member t of C, lanes over the transitions s -a-> t:
//           mark[off(s) + order] := stamp. The first time s is marked in the
//           round (smark stamp) it gets a rank r_s in its block b (atomicAdd)
//           and is written to mscr[bend[b] - 1 - r_s], so after the step the
//           marked members of b sit in the tail of b's range of mscr; the
//           first one appends b (with its range) to a list (warp list for
//           blocks of at most 64 states, CTA list otherwise). Blocks of one
//           state cannot split.
//   split   Algorithm 3's rule: s splits off iff its marks differ from the
//           leader's. If the leader is unmarked the split part is exactly the
//           marked members (k of them) and moves to the last k positions; if
//           the leader is marked, the kept part is the marked members whose
//           marks equal the leader's (kk of them) and moves to the first kk
//           positions, the rest is relabelled. The new label is the smallest
//           state of the split part; the old label, the new label and
//           (Algorithm 3) C are pushed if they were stable.
//
// A round carries out one iteration (mark, barrier, split, barrier), or
// several whose touched blocks do not overlap: claim, barrier, mark,
// barrier, split, barrier (see the section on rounds with several splitters
// below). Rounds run on the whole grid, on CTA 0 alone (light rounds of the
// hybrid schedule) or on the CTA that owns an LTS of a batch.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "plan.cuh"

namespace cg = cooperative_groups;

using namespace bisim;

// Phase timers of the hybrid kernel (diagnostic build only, -DBISIM_PHASE_TIMERS):
// thread 0 of CTA 0 adds the global-timer time of each phase of a round, and
// a few counts, to slots of a shared array that the kernel adds to
// g_phase_acc at exit. Slots: 0 selection, 1 publish, 2 claim, 3 barrier
// after claim, 4 mark, 5 barrier after mark, 6 split, 7 barrier after split,
// 8 one-splitter rounds (whole round), 9 multi-splitter rounds, 10
// one-splitter rounds, 11 rounds on CTA 0 alone, 12 splitters selected, 13
// their states, 14 touched blocks, 15 time between rounds.
#ifdef BISIM_PHASE_TIMERS
__device__ unsigned long long g_phase_acc[16];
// per-round trace of the hybrid kernel (rounds 1 .. BISIM_TRACE_MAX): splitters
// selected, worklist entries before the selection, touched blocks, winners,
// round time in ns, and 1 for a round on CTA 0 alone
constexpr int BISIM_TRACE_MAX = 1 << 16;
__device__ unsigned g_round_trace[BISIM_TRACE_MAX][6];
__device__ unsigned long long g_trace_wins;
__device__ __forceinline__ unsigned long long* phase_slots() {
    __shared__ unsigned long long s[20];  // [16] time of the last mark, [17] touched blocks of the round,
                                          // [18] wins before the round, [19] round start time
    return s;
}
#define TRACE_WIN() atomicAdd(&g_trace_wins, 1ull)
#define TRACE_TOUCHED(v)                                                      \
    do {                                                                      \
        if (blockIdx.x == 0 && threadIdx.x == 0) phase_slots()[17] = (v);     \
    } while (0)
#define TRACE_BEGIN(r, K, wl, head)                                           \
    do {                                                                      \
        if (blockIdx.x == 0 && threadIdx.x == 0 && (r) >= 1 && (r) <= BISIM_TRACE_MAX) { \
            unsigned long long av_ = 0;                                       \
            for (int b_ = 0; b_ < BISIM_BUCKETS; b_++)                        \
                av_ += *(volatile const unsigned long long*)&(wl).tail[b_] - (head)[b_]; \
            g_round_trace[(r) - 1][0] = (unsigned)(K);                        \
            g_round_trace[(r) - 1][1] = (unsigned)(av_ + (K));                \
            phase_slots()[17] = 0;                                            \
            phase_slots()[18] = *(volatile unsigned long long*)&g_trace_wins; \
            phase_slots()[19] = globaltimer_ns();                             \
        }                                                                     \
    } while (0)
#define TRACE_END(r, local)                                                   \
    do {                                                                      \
        if (blockIdx.x == 0 && threadIdx.x == 0 && (r) >= 1 && (r) <= BISIM_TRACE_MAX) { \
            g_round_trace[(r) - 1][2] = (unsigned)phase_slots()[17];          \
            g_round_trace[(r) - 1][3] =                                       \
                (unsigned)(*(volatile unsigned long long*)&g_trace_wins - phase_slots()[18]); \
            g_round_trace[(r) - 1][4] = (unsigned)(globaltimer_ns() - phase_slots()[19]); \
            g_round_trace[(r) - 1][5] = (local);                              \
        }                                                                     \
    } while (0)
#define PHASE_RESET()                                                         \
    do {                                                                      \
        if (threadIdx.x == 0) {                                               \
            for (int i_ = 0; i_ < 16; i_++) phase_slots()[i_] = 0;            \
            phase_slots()[16] = globaltimer_ns();                             \
        }                                                                     \
    } while (0)
#define PHASE(i)                                                              \
    do {                                                                      \
        if (blockIdx.x == 0 && threadIdx.x == 0) {                            \
            const unsigned long long t_ = globaltimer_ns();                   \
            phase_slots()[i] += t_ - phase_slots()[16];                       \
            phase_slots()[16] = t_;                                           \
        }                                                                     \
    } while (0)
#define PHASE_ADD(i, v)                                                       \
    do {                                                                      \
        if (blockIdx.x == 0 && threadIdx.x == 0) phase_slots()[i] += (v);     \
    } while (0)
#define PHASE_FLUSH()                                                         \
    do {                                                                      \
        if (blockIdx.x == 0 && threadIdx.x == 0)                              \
            for (int i_ = 0; i_ < 16; i_++) atomicAdd(&g_phase_acc[i_], phase_slots()[i_]); \
    } while (0)
#else
#define PHASE_RESET() do {} while (0)
#define PHASE(i) do {} while (0)
#define PHASE_ADD(i, v) do {} while (0)
#define PHASE_FLUSH() do {} while (0)
#define TRACE_WIN() do {} while (0)
#define TRACE_TOUCHED(v) do {} while (0)
#define TRACE_BEGIN(r, K, wl, head) do {} while (0)
#define TRACE_END(r, local) do {} while (0)
#endif

namespace {

constexpr int WARP_MAX = 64;  // blocks up to this size are split by one warp
constexpr int32_t MULTI = -2;  // splitter argument of a round with several splitters

struct FrontierArgs {
    int32_t n;
    const int32_t* __restrict__ off;
    const int32_t* __restrict__ in_ptr;
    const unsigned long long* __restrict__ in_edge;
    int32_t* block;
    uint32_t* mark;
    uint32_t* unstable;
    int32_t* elems;   // [n] members grouped by block
    int32_t* loc;     // [n] position of each state in elems
    int32_t* bbeg;    // [n] per label
    int32_t* bend;    // [n] per label
    int32_t* mcnt;    // [n] marked members per label in this round
    int32_t* mscr;    // [n] by position: marked members in the tail of their block's range
    int32_t* yscr;    // [n] by position: scratch for the swap pairing
    uint32_t* smark;  // [n] per state: stamp of the round that last marked it
    uint32_t* kmark;  // [n] per state: stamp of the round it was in a kept part
    int4* tlist;      // [2n]: warp list, CTA list of touched blocks (label, range begin, range end, 0)
    int32_t* queue;   // [n]
    unsigned long long* claim;  // [n] per label: (~stamp << 32) | index of the claiming splitter;
                                // peel rounds: the least key of all the round's claims
    unsigned long long* minx;   // [n] per label, peel rounds: the least key of the exclusive claims
    unsigned long long* smark64;  // [n] per state, peel rounds: the least key of the splitters
                                  // that mark it (the first to split it off)
    uint32_t* lostl;  // [n] per splitter label, peel rounds: the round in which it lost a claim
    int32_t* bspl;    // [n] per touched label: its splitter (multi-splitter rounds)
    bisim_ctrl* ctrl;
    GridBarrier gb;
    uint32_t stamp0;
    int64_t round_cap;
    int alg2;
    int test_hook;
};

// Loads of the round functions. Each one follows the barrier that orders it
// after the stores it must observe: __syncthreads within a CTA, and between
// CTAs the grid barrier (release arrive, acquire wait) or the release/acquire
// pair of a published command. By the memory model such a load sees those
// stores even when served from L1, so it takes the default caching. Waits on
// words that other CTAs change while this one spins (the heartbeat, the
// status word) read them with ld.global.cg instead.
template <typename T>
__device__ __forceinline__ T ld(const T* p) {
    return *p;
}

__device__ __forceinline__ int size_bucket(int32_t sz) { return 31 - __clz(max(sz, 1)); }

// The splitter worklist of one LTS: BISIM_BUCKETS FIFO rings of `cap`
// entries, bucket k at queue[k * stride + base ...]. `tail` holds the pushes
// per bucket; it lives in global memory for the grid engine (every CTA pops)
// and in shared memory for the CTA-per-instance engine.
// Pushes of one CTA collected in shared memory during a split step and
// appended to the rings at its end with one global atomic per ring
// (flush_pushes); a push that finds the buffer full goes to its ring at once.
constexpr int PUSH_BUF = 4096;
struct PushBuf {
    int n;  // pushes so far (may pass PUSH_BUF; the rest went to the rings)
    unsigned cnt[BISIM_BUCKETS];
    unsigned long long base[BISIM_BUCKETS];
    int32_t lab[PUSH_BUF];
    uint8_t bk[PUSH_BUF];
};

struct Worklist {
    unsigned long long* tail;
    int32_t* queue;
    size_t stride;
    int32_t base;
    int32_t cap;
    int nbk = BISIM_BUCKETS;  // rings in use: larger blocks share the last one
    PushBuf* buf = nullptr;   // this CTA's push buffer, if any
};

__device__ __forceinline__ void push_ring(const Worklist& wl, int32_t label, int bk) {
    if (wl.buf) {
        const int i = atomicAdd(&wl.buf->n, 1);
        if (i < PUSH_BUF) {
            wl.buf->lab[i] = label;
            wl.buf->bk[i] = (uint8_t)bk;
            return;
        }
    }
    const unsigned long long pos = atomicAdd(&wl.tail[bk], 1ull);
    wl.queue[(size_t)bk * wl.stride + wl.base + pos % (unsigned long long)wl.cap] = label;
}

// append a label whose block has `size` states to the FIFO ring of its size bucket
__device__ __forceinline__ void push_sized(const Worklist& wl, int32_t label, int32_t size) {
    push_ring(wl, label, min(size_bucket(size), wl.nbk - 1));
}

// Append a CTA's buffered pushes to the rings (the whole CTA calls, after a
// __syncthreads that follows the last push); the buffer is empty afterwards.
__device__ void flush_pushes(const Worklist& wl) {
    PushBuf* pb = wl.buf;
    const int n = min(pb->n, PUSH_BUF);
    if (threadIdx.x < BISIM_BUCKETS) pb->cnt[threadIdx.x] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&pb->cnt[pb->bk[i]], 1u);
    __syncthreads();
    if (threadIdx.x < BISIM_BUCKETS) {
        const unsigned c = pb->cnt[threadIdx.x];
        pb->base[threadIdx.x] = c ? atomicAdd(&wl.tail[threadIdx.x], (unsigned long long)c) : 0ull;
        pb->cnt[threadIdx.x] = 0u;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int bk = pb->bk[i];
        const unsigned long long pos = pb->base[bk] + atomicAdd(&pb->cnt[bk], 1u);
        wl.queue[(size_t)bk * wl.stride + wl.base + pos % (unsigned long long)wl.cap] = pb->lab[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) pb->n = 0;
    __syncthreads();
}

__device__ __forceinline__ void push(const FrontierArgs& a, const Worklist& wl, int32_t label) {
    push_sized(wl, label, ld(&a.bend[label]) - ld(&a.bbeg[label]));
}

// unstable_label := true; enqueue it if it was stable (size < 0: look it up)
__device__ __forceinline__ void set_unstable(const FrontierArgs& a, const Worklist& wl, int32_t label,
                                             int32_t size = -1) {
    if (atomicExch(&a.unstable[label], 1u) == 0u) {
        if (size < 0) size = ld(&a.bend[label]) - ld(&a.bbeg[label]);
        push_sized(wl, label, size);
    }
}

// finish_split by a whole warp: the (up to) three labels are pushed by three
// lanes at once; the kept part b has szb states and the split part szl. The
// caller's stores of the new ranges precede a __syncwarp.
__device__ __forceinline__ void finish_split_warp(const FrontierArgs& a, const Worklist& wl, int32_t b,
                                                  int32_t szb, int32_t leader, int32_t szl, int32_t C) {
    const unsigned lane = threadIdx.x & 31u;
    int32_t lab = lane == 0 ? b : lane == 1 ? leader : (lane == 2 && !a.alg2) ? C : -1;
    if (lab == MULTI) lab = ld(&a.bspl[b]);  // the splitter that touched b this round
    if (lab >= 0) set_unstable(a, wl, lab, lane == 0 ? szb : lane == 1 ? szl : -1);
}

// Does a member with mark slots [os, os + ks) have the same marks as the
// leader (slots [lo, lo + k); for k <= 32 their marks are the bits of
// lmask)? Loads go out eight at a time.
__device__ __forceinline__ bool same_marks_at(const FrontierArgs& a, int32_t os, int32_t ks, int32_t lo, int32_t k,
                                              unsigned lmask, uint32_t stamp) {
    if (ks != k) {  // members must share the leader's label set (preprocessing invariant)
        atomicOr(&a.ctrl->status, ST_INTERNAL);
        ks = min(ks, k);
    }
    bool diff = false;
    for (int32_t q0 = 0; q0 < ks; q0 += 8) {
        uint32_t v[8], w[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            v[u] = q0 + u < ks ? ld(&a.mark[os + q0 + u]) : 0u;
            w[u] = k > 32 && q0 + u < ks ? ld(&a.mark[lo + q0 + u]) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (q0 + u < ks)
                diff |= (v[u] == stamp) != (k <= 32 ? (bool)((lmask >> (q0 + u)) & 1u) : w[u] == stamp);
    }
    return !diff;
}

__device__ __forceinline__ bool same_marks(const FrontierArgs& a, int32_t s, int32_t lo, int32_t k,
                                           unsigned lmask, uint32_t stamp) {
    const int32_t os = a.off[s];
    return same_marks_at(a, os, a.off[s + 1] - os, lo, k, lmask, stamp);
}

// One warp splits block b (range [b0, e0), at most 64 members) from the
// members themselves. The loads are grouped by what they depend on: b and
// its range; then the members; then the members' marks.
__device__ void warp_split(const FrontierArgs& a, const Worklist& wl, int32_t b, int32_t b0, int32_t e0,
                           uint32_t stamp, int32_t C, long long& states) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = lanemask_lt();
    const int32_t sz = e0 - b0;
    const int32_t lo = a.off[b];
    const int32_t k = a.off[b + 1] - lo;
    const bool lead_marked = ld(&a.smark[b]) == stamp;
    const int32_t s0 = (int)lane < sz ? ld(&a.elems[b0 + lane]) : -1;
    const int32_t s1 = (int)lane + 32 < sz ? ld(&a.elems[b0 + 32 + lane]) : -1;
    if (lane == 0) a.mcnt[b] = 0;
    const bool mk0 = s0 >= 0 && ld(&a.smark[s0]) == stamp;
    const bool mk1 = s1 >= 0 && ld(&a.smark[s1]) == stamp;
    bool p0 = mk0, p1 = mk1;  // splits off (leader unmarked: exactly the marked members)
    if (lead_marked) {
        // slot ranges of the members, issued with the leader's marks
        const int32_t o0 = s0 >= 0 ? a.off[s0] : 0, q0 = s0 >= 0 ? a.off[s0 + 1] : 0;
        const int32_t o1 = s1 >= 0 ? a.off[s1] : 0, q1 = s1 >= 0 ? a.off[s1 + 1] : 0;
        unsigned lmask = 0;
        if (k <= 32) lmask = __ballot_sync(0xffffffffu, (int)lane < k && ld(&a.mark[lo + lane]) == stamp);
        p0 = s0 >= 0 && !(mk0 && same_marks_at(a, o0, q0 - o0, lo, k, lmask, stamp));
        p1 = s1 >= 0 && !(mk1 && same_marks_at(a, o1, q1 - o1, lo, k, lmask, stamp));
    }
    const unsigned m0 = __ballot_sync(0xffffffffu, p0), m1 = __ballot_sync(0xffffffffu, p1);
    if (lane == 0) states += sz;
    if ((m0 | m1) == 0u) return;
    const unsigned v0 = __ballot_sync(0xffffffffu, s0 >= 0), v1 = __ballot_sync(0xffffffffu, s1 >= 0);
    const int32_t nkeep = sz - __popc(m0) - __popc(m1);
    const int32_t leader = __reduce_min_sync(0xffffffffu, min(p0 ? s0 : NONE, p1 ? s1 : NONE));
    if (s0 >= 0) {
        const int32_t pos = b0 + (p0 ? nkeep + __popc(m0 & lt) : __popc(~m0 & v0 & lt));
        a.elems[pos] = s0;
        a.loc[s0] = pos;
        if (p0) a.block[s0] = leader;
    }
    if (s1 >= 0) {
        const int32_t pos = b0 + (p1 ? nkeep + __popc(m0) + __popc(m1 & lt)
                                     : __popc(~m0 & v0) + __popc(~m1 & v1 & lt));
        a.elems[pos] = s1;
        a.loc[s1] = pos;
        if (p1) a.block[s1] = leader;
    }
    if (lane == 0) {
        a.bend[b] = b0 + nkeep;
        a.bbeg[leader] = b0 + nkeep;
        a.bend[leader] = e0;
    }
    __syncwarp();
    finish_split_warp(a, wl, b, nkeep, leader, sz - nkeep, C);
}

struct CtaShared {
    int wcnt[32];
    int wmin[32];
    int total;
    int mn;
    unsigned lmask;
    int C;
    int bk;                 // select_splitter: size bucket of the popped label (-1: none)
    int bx[BISIM_BUCKETS];  // select_many: entries before each bucket
    int bn[BISIM_BUCKETS];  // select_many: entries taken from each bucket at most
    int hp[BISIM_BUCKETS];  // select_many: ring position of each bucket's head
    unsigned long long head[BISIM_BUCKETS];  // this CTA's copy of the worklist heads
    int k0;                 // select_peel: labels taken from size bucket 0
    int n1;                 // select_peel: listed labels whose block has one state
    unsigned long long h0;  // select_peel: ring-0 head before them
};

// Block-wide exclusive rank of predicate p and the block total (sh.total).
__device__ __forceinline__ int cta_rank(bool p, CtaShared& sh, int& total) {
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const unsigned nw = blockDim.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, p);
    if (lane == 0) sh.wcnt[wid] = __popc(bal);
    __syncthreads();
    if (wid == 0) {
        int c = (int)lane < (int)nw ? sh.wcnt[lane] : 0;
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        if ((int)lane < (int)nw) sh.wcnt[lane] = x - c;
        if (lane == 31) sh.total = x;
    }
    __syncthreads();
    const int r = sh.wcnt[wid] + __popc(bal & lanemask_lt());
    total = sh.total;
    __syncthreads();
    return r;
}

// Block-wide exclusive prefix sum of v and the block total.
__device__ __forceinline__ int cta_scan(int v, CtaShared& sh, int& total) {
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const unsigned nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    if (lane == 31) sh.wcnt[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int c = (int)lane < (int)nw ? sh.wcnt[lane] : 0;
        int y = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int z = __shfl_up_sync(0xffffffffu, y, o);
            if ((int)lane >= o) y += z;
        }
        if ((int)lane < (int)nw) sh.wcnt[lane] = y - c;
        if (lane == 31) sh.total = y;
    }
    __syncthreads();
    const int r = sh.wcnt[wid] + x - v;
    total = sh.total;
    __syncthreads();
    return r;
}

__device__ __forceinline__ int cta_min(int v, CtaShared& sh) {
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const unsigned nw = blockDim.x >> 5;
    v = __reduce_min_sync(0xffffffffu, v);
    if (lane == 0) sh.wmin[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int c = (int)lane < (int)nw ? sh.wmin[lane] : NONE;
        c = __reduce_min_sync(0xffffffffu, c);
        if (lane == 0) sh.mn = c;
    }
    __syncthreads();
    const int r = sh.mn;
    __syncthreads();
    return r;
}

// Move the set of states listed in mscr[t0 .. t0+cnt) (none of them already
// at a position in [r0, r0+cnt), except those whose loc says so) into the
// position range [r0, r0+cnt) by swapping with the states there that are not
// in the set. in_set(u) tells membership of the state u currently at a
// position of the range.
template <typename InSet>
__device__ void cta_gather_range(const FrontierArgs& a, CtaShared& sh, int32_t t0, int32_t cnt,
                                 int32_t r0, InSet in_set) {
    // outsiders of the set: X = members of the set outside [r0, r0+cnt),
    // compacted in place at mscr[t0 ..); Y = positions inside the range held
    // by non-members, compacted at yscr[t0 ..)
    int nx = 0;
    for (int32_t base = 0; base < cnt; base += blockDim.x) {
        const int32_t i = base + threadIdx.x;
        const int32_t s = i < cnt ? ld(&a.mscr[t0 + i]) : -1;
        const bool out = s >= 0 && (ld(&a.loc[s]) < r0 || ld(&a.loc[s]) >= r0 + cnt);
        int tot;
        const int rk = cta_rank(out, sh, tot);
        if (out) a.mscr[t0 + nx + rk] = s;  // stable in-place compaction (target <= source)
        nx += tot;
        __syncthreads();
    }
    int ny = 0;
    for (int32_t base = 0; base < cnt; base += blockDim.x) {
        const int32_t i = base + threadIdx.x;
        const int32_t q = r0 + i;
        const bool foreign = i < cnt && !in_set(ld(&a.elems[q]));
        int tot;
        const int rk = cta_rank(foreign, sh, tot);
        if (foreign) a.yscr[t0 + ny + rk] = q;
        ny += tot;
    }
    __syncthreads();
    if (nx != ny) {
        if (threadIdx.x == 0) atomicOr(&a.ctrl->status, ST_INTERNAL);
        return;
    }
    for (int32_t j = threadIdx.x; j < nx; j += blockDim.x) {
        const int32_t s = ld(&a.mscr[t0 + j]);
        const int32_t q = ld(&a.yscr[t0 + j]);
        const int32_t p = ld(&a.loc[s]);
        const int32_t u = ld(&a.elems[q]);
        a.elems[p] = u;
        a.loc[u] = p;
        a.elems[q] = s;
        a.loc[s] = q;
    }
    __syncthreads();
}

// One CTA splits block b (more than WARP_MAX members), touching only the
// marked members, plus the moved-out part when the leader is marked.
__device__ void cta_split(const FrontierArgs& a, const Worklist& wl, CtaShared& sh, int32_t b, uint32_t stamp,
                          int32_t C, long long& states) {
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const int32_t b0 = ld(&a.bbeg[b]), e0 = ld(&a.bend[b]);
    const int32_t km = ld(&a.mcnt[b]);
    const int32_t t0 = e0 - km;  // marked members are listed in mscr[t0 .. e0)
    const int32_t lo = a.off[b];
    const int32_t k = a.off[b + 1] - lo;
    const bool lead_marked = ld(&a.smark[b]) == stamp;
    __syncthreads();
    if (threadIdx.x == 0) a.mcnt[b] = 0;
    if (!lead_marked) {
        // split part = the km marked members; it moves to [t0, e0)
        int mn = NONE;
        for (int32_t i = threadIdx.x; i < km; i += blockDim.x) mn = min(mn, ld(&a.mscr[t0 + i]));
        const int32_t leader = cta_min(mn, sh);
        for (int32_t i = threadIdx.x; i < km; i += blockDim.x) a.block[ld(&a.mscr[t0 + i])] = leader;
        __syncthreads();
        cta_gather_range(a, sh, t0, km, t0, [&](int32_t u) { return ld(&a.smark[u]) == stamp; });
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) {
                states += km;
                a.bend[b] = t0;
                a.bbeg[leader] = t0;
                a.bend[leader] = e0;
            }
            __syncwarp();
            finish_split_warp(a, wl, b, t0 - b0, leader, e0 - t0, C);
        }
        __syncthreads();
        return;
    }
    // leader marked: kept part = marked members with the leader's marks
    if (wid == 0) {
        unsigned lm = 0;
        if (k <= 32) lm = __ballot_sync(0xffffffffu, (int)lane < k && ld(&a.mark[lo + lane]) == stamp);
        if (lane == 0) sh.lmask = lm;
    }
    __syncthreads();
    const unsigned lmask = sh.lmask;
    int kk = 0;
    for (int32_t base = 0; base < km; base += blockDim.x) {
        const int32_t i = base + threadIdx.x;
        const int32_t s = i < km ? ld(&a.mscr[t0 + i]) : -1;
        const bool keep = s >= 0 && same_marks(a, s, lo, k, lmask, stamp);
        int tot;
        const int rk = cta_rank(keep, sh, tot);
        if (keep) {
            a.kmark[s] = stamp;
            a.mscr[t0 + kk + rk] = s;  // kept members compacted in place
        }
        kk += tot;
        __syncthreads();
    }
    const int32_t sz = e0 - b0;
    if (threadIdx.x == 0) states += km;
    if (kk == sz) return;  // every member kept: no split
    cta_gather_range(a, sh, t0, kk, b0, [&](int32_t u) { return ld(&a.kmark[u]) == stamp; });
    // split part = [b0 + kk, e0)
    int mn = NONE;
    for (int32_t q = b0 + kk + threadIdx.x; q < e0; q += blockDim.x) mn = min(mn, ld(&a.elems[q]));
    const int32_t leader = cta_min(mn, sh);
    for (int32_t q = b0 + kk + threadIdx.x; q < e0; q += blockDim.x) a.block[ld(&a.elems[q])] = leader;
    __syncthreads();
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) {
            states += sz - kk;
            a.bend[b] = b0 + kk;
            a.bbeg[leader] = b0 + kk;
            a.bend[leader] = e0;
        }
        __syncwarp();
        finish_split_warp(a, wl, b, kk, leader, e0 - b0 - kk, C);
    }
    __syncthreads();
}

// Warp version of the gather: lanes l < cnt hold the members s_l of a set
// (cnt <= 32) that must end up at positions [r0, r0 + cnt). Members outside
// the range swap with the non-members inside it, paired by rank.
template <typename InSet>
__device__ __forceinline__ void warp_gather(const FrontierArgs& a, int32_t s, int32_t cnt, int32_t r0,
                                            InSet in_set) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = lanemask_lt();
    const bool mine = (int)lane < cnt;
    const int32_t p = mine ? ld(&a.loc[s]) : -1;
    const bool x = mine && (p < r0 || p >= r0 + cnt);
    const int32_t q = r0 + (int32_t)lane;
    const bool y = mine && !in_set(ld(&a.elems[q]));
    const unsigned xm = __ballot_sync(0xffffffffu, x), ym = __ballot_sync(0xffffffffu, y);
    if (__popc(xm) != __popc(ym)) {
        if (lane == 0) atomicOr(&a.ctrl->status, ST_INTERNAL);
        return;
    }
    int src = (int)lane;
    if (x) {
        unsigned mm = ym;
        for (int j = __popc(xm & lt); j > 0; j--) mm &= mm - 1u;  // drop the j lowest set bits
        src = __ffs(mm) - 1;
    }
    const int32_t qq = __shfl_sync(0xffffffffu, q, src);
    if (x) {
        const int32_t u = ld(&a.elems[qq]);
        a.elems[p] = u;
        a.loc[u] = p;
        a.elems[qq] = s;
        a.loc[s] = qq;
    }
    __syncwarp();
}

// One warp splits block b (more than WARP_MAX members) that has at most 32
// marked members this round.
__device__ void warp_split_sparse(const FrontierArgs& a, const Worklist& wl, int32_t b, int32_t b0, int32_t e0,
                                  int32_t km, uint32_t stamp, int32_t C, long long& states) {
    const unsigned lane = threadIdx.x & 31u;
    const int32_t t0 = e0 - km;  // marked members listed in mscr[t0 .. e0)
    const int32_t lo = a.off[b];
    const int32_t k = a.off[b + 1] - lo;
    const bool lead_marked = ld(&a.smark[b]) == stamp;
    const int32_t s = (int)lane < km ? ld(&a.mscr[t0 + lane]) : -1;
    __syncwarp();
    if (lane == 0) a.mcnt[b] = 0;
    if (!lead_marked) {
        // split part = the marked members; they move to [t0, e0)
        const int32_t leader = __reduce_min_sync(0xffffffffu, s >= 0 ? s : NONE);
        if (s >= 0) a.block[s] = leader;
        warp_gather(a, s, km, t0, [&](int32_t u) { return ld(&a.smark[u]) == stamp; });
        if (lane == 0) {
            states += km;
            a.bend[b] = t0;
            a.bbeg[leader] = t0;
            a.bend[leader] = e0;
        }
        __syncwarp();
        finish_split_warp(a, wl, b, t0 - b0, leader, e0 - t0, C);
        return;
    }
    // leader marked: kept part = marked members with the leader's marks
    unsigned lmask = 0;
    if (k <= 32) lmask = __ballot_sync(0xffffffffu, (int)lane < k && ld(&a.mark[lo + lane]) == stamp);
    const bool keep = s >= 0 && same_marks(a, s, lo, k, lmask, stamp);
    const unsigned km_mask = __ballot_sync(0xffffffffu, keep);
    const int32_t kk = __popc(km_mask);
    // compact the kept members into lanes 0..kk-1
    int src = (int)lane;
    {
        unsigned mm = km_mask;
        for (int j = (int)lane; j > 0 && mm; j--) mm &= mm - 1u;
        src = mm ? __ffs(mm) - 1 : 0;
    }
    const int32_t ks = __shfl_sync(0xffffffffu, s, src);
    if ((int)lane < kk) a.kmark[ks] = stamp;
    __syncwarp();
    warp_gather(a, (int)lane < kk ? ks : -1, kk, b0, [&](int32_t u) { return ld(&a.kmark[u]) == stamp; });
    // split part = [b0 + kk, e0): every other member
    int mn = NONE;
    for (int32_t q = b0 + kk + (int32_t)lane; q < e0; q += 32) mn = min(mn, ld(&a.elems[q]));
    const int32_t leader = __reduce_min_sync(0xffffffffu, mn);
    for (int32_t q = b0 + kk + (int32_t)lane; q < e0; q += 32) a.block[ld(&a.elems[q])] = leader;
    __syncwarp();
    if (lane == 0) {
        states += e0 - b0;
        a.bend[b] = b0 + kk;
        a.bbeg[leader] = b0 + kk;
        a.bend[leader] = e0;
    }
    __syncwarp();
    finish_split_warp(a, wl, b, kk, leader, e0 - b0 - kk, C);
}

// ------------------------------------------------ splits of peel rounds
//
// In a peel round a block may be touched by several winning splitters, each
// of which marked exactly one member of it and not its leader (the round's
// rule, see peel_round). Carried out one after the other in increasing label
// order, each such iteration finds the leader unmarked, so its split part is
// exactly its marked member: the first splitter to mark a member splits it
// off into a block of its own, a later one that marks the same member finds
// it alone and splits nothing. So every marked member ends in a block of one
// state, the block keeps its label and the unmarked members, and the
// splitters that split something are, per member, the least label among its
// markers - the low word of smark64. Pushes as Algorithm 3: the block's
// label, every new label, and (not with Algorithm 2) those splitters.

// set_unstable for every lane with `active` (every lane of the warp calls
// it); each size bucket's ring slots are taken with one atomicAdd per warp
__device__ __forceinline__ void set_unstable_warp(const FrontierArgs& a, const Worklist& wl, int32_t label,
                                                  int32_t size, bool active) {
    const unsigned lane = threadIdx.x & 31u;
    bool need = active && atomicExch(&a.unstable[label], 1u) == 0u;
    int bk = 32 + (int)lane;  // a group of its own when nothing is pushed
    if (need) {
        if (size < 0) size = ld(&a.bend[label]) - ld(&a.bbeg[label]);
        bk = min(size_bucket(size), wl.nbk - 1);
    }
    if (wl.buf) {
        if (need) push_ring(wl, label, bk);
        return;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, bk);
    const int first = __ffs(peers) - 1;
    unsigned long long pos = 0;
    if (need && (int)lane == first) pos = atomicAdd(&wl.tail[bk], (unsigned long long)__popc(peers));
    pos = __shfl_sync(0xffffffffu, pos, first) + __popc(peers & lanemask_lt());
    if (need) wl.queue[(size_t)bk * wl.stride + wl.base + pos % (unsigned long long)wl.cap] = label;
}

__device__ __forceinline__ bool peeled(const FrontierArgs& a, int32_t s, uint32_t stamp, unsigned long long* key) {
    const unsigned long long k = ld(&a.smark64[s]);
    *key = k;
    return (uint32_t)(k >> 32) == ~stamp;
}

// A peeled member s at position q: a block of its own labelled s; its own
// label and the splitter that split it off become unstable.
__device__ __forceinline__ void peel_member(const FrontierArgs& a, int32_t s, int32_t q) {
    a.block[s] = s;
    a.bbeg[s] = q;
    a.bend[s] = q + 1;
}

__device__ __forceinline__ void peel_pushes(const FrontierArgs& a, const Worklist& wl, int32_t s,
                                            unsigned long long key, bool active) {
    set_unstable_warp(a, wl, s, 1, active);
    set_unstable_warp(a, wl, (int32_t)(uint32_t)key, -1, active && !a.alg2);
}

// One warp peels block b (range [b0, e0), at most 64 members) from the members.
__device__ void warp_peel(const FrontierArgs& a, const Worklist& wl, int32_t b, int32_t b0, int32_t e0,
                          uint32_t stamp, long long& states) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = lanemask_lt();
    const int32_t sz = e0 - b0;
    const int32_t s0 = (int)lane < sz ? ld(&a.elems[b0 + lane]) : -1;
    const int32_t s1 = (int)lane + 32 < sz ? ld(&a.elems[b0 + 32 + lane]) : -1;
    if (lane == 0) a.mcnt[b] = 0;
    unsigned long long k0 = 0, k1 = 0;
    const bool p0 = s0 >= 0 && peeled(a, s0, stamp, &k0);
    const bool p1 = s1 >= 0 && peeled(a, s1, stamp, &k1);
    const unsigned m0 = __ballot_sync(0xffffffffu, p0), m1 = __ballot_sync(0xffffffffu, p1);
    if (lane == 0) states += sz;
    const unsigned v0 = __ballot_sync(0xffffffffu, s0 >= 0), v1 = __ballot_sync(0xffffffffu, s1 >= 0);
    const int32_t nkeep = sz - __popc(m0) - __popc(m1);
    if (nkeep < 1 || (m0 | m1) == 0u) {  // the leader is never marked here, and a listed block has a mark
        if (lane == 0) atomicOr(&a.ctrl->status, ST_INTERNAL);
        return;
    }
    if (s0 >= 0) {
        const int32_t pos = b0 + (p0 ? nkeep + __popc(m0 & lt) : __popc(~m0 & v0 & lt));
        a.elems[pos] = s0;
        a.loc[s0] = pos;
        if (p0) peel_member(a, s0, pos);
    }
    if (s1 >= 0) {
        const int32_t pos = b0 + (p1 ? nkeep + __popc(m0) + __popc(m1 & lt)
                                     : __popc(~m0 & v0) + __popc(~m1 & v1 & lt));
        a.elems[pos] = s1;
        a.loc[s1] = pos;
        if (p1) peel_member(a, s1, pos);
    }
    if (lane == 0) a.bend[b] = b0 + nkeep;
    __syncwarp();
    set_unstable_warp(a, wl, b, nkeep, lane == 0);
    peel_pushes(a, wl, s0, k0, p0);
    peel_pushes(a, wl, s1, k1, p1);
}

// One warp peels block b (more than WARP_MAX members) with km <= 32 marked
// members, listed in mscr[e0 - km, e0).
__device__ void warp_peel_sparse(const FrontierArgs& a, const Worklist& wl, int32_t b, int32_t b0, int32_t e0,
                                 int32_t km, uint32_t stamp, long long& states) {
    const unsigned lane = threadIdx.x & 31u;
    const int32_t t0 = e0 - km;
    const int32_t s = (int)lane < km ? ld(&a.mscr[t0 + lane]) : -1;
    __syncwarp();
    if (lane == 0) a.mcnt[b] = 0;
    const unsigned long long k = s >= 0 ? ld(&a.smark64[s]) : 0ull;
    const unsigned hi = ~stamp;
    warp_gather(a, s, km, t0, [&](int32_t u) { return (uint32_t)(ld(&a.smark64[u]) >> 32) == hi; });
    if (s >= 0) peel_member(a, s, ld(&a.loc[s]));
    if (lane == 0) {
        states += km;
        a.bend[b] = t0;
    }
    __syncwarp();
    set_unstable_warp(a, wl, b, t0 - b0, lane == 0);
    peel_pushes(a, wl, s, k, s >= 0);
}

// One CTA peels block b with more than 32 marked members.
__device__ void cta_peel(const FrontierArgs& a, const Worklist& wl, CtaShared& sh, int32_t b, uint32_t stamp,
                         long long& states) {
    const int32_t b0 = ld(&a.bbeg[b]), e0 = ld(&a.bend[b]);
    const int32_t km = ld(&a.mcnt[b]);
    const int32_t t0 = e0 - km;
    const unsigned hi = ~stamp;
    __syncthreads();
    if (threadIdx.x == 0) a.mcnt[b] = 0;
    cta_gather_range(a, sh, t0, km, t0, [&](int32_t u) { return (uint32_t)(ld(&a.smark64[u]) >> 32) == hi; });
    for (int32_t base = 0; base < km; base += blockDim.x) {
        const int32_t i = base + (int32_t)threadIdx.x;
        const bool act = i < km;
        const int32_t s = act ? ld(&a.elems[t0 + i]) : -1;
        const unsigned long long k = act ? ld(&a.smark64[s]) : 0ull;
        if (act) peel_member(a, s, t0 + i);
        peel_pushes(a, wl, s, k, act);
    }
    if (threadIdx.x == 0) {
        states += km;
        a.bend[b] = t0;
    }
    __syncthreads();
    if (threadIdx.x < 32) set_unstable_warp(a, wl, b, t0 - b0, threadIdx.x == 0);
    __syncthreads();
}

// Split step of a round for the touched blocks listed by the mark step:
// blocks of at most WARP_MAX states one per warp; larger blocks one per warp
// when at most 32 members are marked, otherwise one per CTA. CTA `cta` of
// `ncta` takes its share; `defer` is a CTA-local list of at least
// blockDim/32 entries.
__device__ void split_step(const FrontierArgs& a, const Worklist& wl, CtaShared& sh, int* defer, int* ndefer,
                           uint32_t stamp, int32_t C, int ns, const int4* small_list, int nm,
                           const int4* mid_list, int cta, int ncta,
                           long long& states) {
    const int wid = (int)(threadIdx.x >> 5);
    const int nw = (int)(blockDim.x >> 5);
    // entry i of either list goes to CTA i % ncta, so the first ncta entries
    // land on different CTAs; inside a CTA, warp-list entries take the first
    // warps and CTA-list entries the last, and the first pass over the CTA
    // list runs alongside the warp list
    auto mid_entry = [&](int i) {
        const int4 t = ld(&mid_list[i]);
        const int32_t km = ld(&a.mcnt[t.x]);
        if (km <= 32) {
            if (t.w)
                warp_peel_sparse(a, wl, t.x, t.y, t.z, km, stamp, states);
            else
                warp_split_sparse(a, wl, t.x, t.y, t.z, km, stamp, C, states);
        } else if ((threadIdx.x & 31) == 0) {
            defer[atomicAdd(ndefer, 1)] = t.w ? ~t.x : t.x;  // a peeled block is listed as ~label
        }
    };
    if (threadIdx.x == 0) *ndefer = 0;
    __syncthreads();
    for (int base = 0; base < max(nm, 1); base += ncta * nw) {
        const int i = base + (nw - 1 - wid) * ncta + cta;
        if (i < nm) mid_entry(i);
        if (base == 0)
            for (int64_t q = cta + (int64_t)wid * ncta; q < ns; q += (int64_t)ncta * nw) {
                const int4 t = ld(&small_list[q]);
                if (t.w)
                    warp_peel(a, wl, t.x, t.y, t.z, stamp, states);
                else
                    warp_split(a, wl, t.x, t.y, t.z, stamp, C, states);
            }
        __syncthreads();
        const int nd = *ndefer;
        for (int jd = 0; jd < nd; jd++) {
            const int d = defer[jd];
            if (d < 0)
                cta_peel(a, wl, sh, ~d, stamp, states);
            else
                cta_split(a, wl, sh, d, stamp, C, states);
        }
        __syncthreads();
        if (threadIdx.x == 0) *ndefer = 0;
        __syncthreads();
    }
}

// Mark step of one round (Algorithm 3, mark lines) for splitter C, done by the
// warps gw, gw + nwarps, ... (the whole grid or one CTA): one warp per member
// of C, lanes over its incoming transitions. The first mark of a source s in
// the round ranks it among the marked members of its block; the first marked
// member of a block appends the block to the warp list or the CTA list.
// Marks of one member t of a splitter, by one warp (lanes over t's incoming
// transitions). Cw >= 0 is recorded as the splitter of each newly touched
// block (rounds with several splitters).
// The part of a mark step after the first mark of a source s in its block b
// (range [bb, be)): rank s among the block's marked members and list b when
// it is the first. Blocks of one state cannot split and are skipped.
// mode (the list entry's fourth field): 0 = the block is split by one splitter
// (Algorithm 3's rule); 1 = peel rounds: every marked member is split off on
// its own (each was marked by splitters that mark no other member of the
// block and not its leader).
__device__ __forceinline__ void rank_marked(const FrontierArgs& a, int32_t s, int32_t b, int32_t bb, int32_t be,
                                            int32_t Cw, int* n_small, int* n_mid, int4* small_list,
                                            int4* mid_list, int mode = 0) {
    if (be - bb <= 1) return;
    const int32_t rk = atomicAdd(&a.mcnt[b], 1);
    a.mscr[be - 1 - rk] = s;
    if (rk == 0) {
        if (Cw >= 0) a.bspl[b] = Cw;
        // the lanes here that list a block into the same list take their
        // entries with one atomic (the list lengths are one word each for the
        // whole grid)
        const bool small = be - bb <= WARP_MAX;
        const cg::coalesced_group g = cg::coalesced_threads();
        const cg::coalesced_group part = cg::labeled_partition(g, small ? 1 : 0);
        int base = 0;
        if (part.thread_rank() == 0) base = atomicAdd(small ? n_small : n_mid, (int)part.size());
        base = part.shfl(base, 0) + (int)part.thread_rank();
        (small ? small_list : mid_list)[base] = make_int4(b, bb, be, mode);
    }
}

__device__ __forceinline__ void mark_member(const FrontierArgs& a, int32_t t, uint32_t stamp, int32_t Cw,
                                            int* n_small, int* n_mid, int4* small_list, int4* mid_list,
                                            long long& edges) {
    const int lane = threadIdx.x & 31;
    const int32_t j0 = a.in_ptr[t], j1 = a.in_ptr[t + 1];
    if (lane == 0) edges += j1 - j0;
    for (int32_t j = j0 + lane; j < j1; j += 32) {
        const unsigned long long e = a.in_edge[j];
        const int32_t s = (int32_t)(e >> 32);
        a.mark[(uint32_t)e] = stamp;
        const int32_t b = ld(&a.block[s]);  // issued before the atomic: both depend on s only
        if (atomicExch(&a.smark[s], stamp) == stamp) continue;
        rank_marked(a, s, b, ld(&a.bbeg[b]), ld(&a.bend[b]), Cw, n_small, n_mid, small_list, mid_list);
    }
}

__device__ __forceinline__ void mark_step(const FrontierArgs& a, int32_t C, uint32_t stamp, int64_t gw,
                                          int64_t nwarps, int* n_small, int* n_mid, int4* small_list,
                                          int4* mid_list, long long& edges) {
    const int32_t b0 = ld(&a.bbeg[C]), e0 = ld(&a.bend[C]);
    for (int64_t idx = b0 + gw; idx < e0; idx += nwarps)
        mark_member(a, ld(&a.elems[idx]), stamp, -1, n_small, n_mid, small_list, mid_list, edges);
}

// ------------------------------------------- rounds with several splitters
//
// A round may take K splitters C_0 .. C_{K-1} at once. The splitter rounds
// of Algorithm 3 for C_i and C_j touch disjoint data, and so may run
// concurrently with the effect of running them one after the other, when
// neither C_j nor any block holding a predecessor of C_j is C_i or a block
// holding a predecessor of C_i. (Blocks of one state are exempt: they are
// read, never split.) Before marking, every splitter claims its block and
// the blocks of its predecessors with atomicMin on a per-label word
// (~stamp << 32 | j); a splitter that meets a claim of a smaller index, or
// whose claim is displaced by one, has lost and goes back to the worklist.
// Splitter 0 never loses, so every round carries out at least one splitter
// iteration. The winners then mark with one shared stamp (their marked
// slots are disjoint) and split exactly as in a one-splitter round.

// loads that read shared memory, or global memory past L1, through a generic pointer
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) { return *(volatile const uint32_t*)p; }
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *(volatile const int*)p; }

// entries of a multi-splitter selection per thread at most
constexpr int SEL_E = 8;

// Pops up to kmax labels (lowest size bucket first, FIFO inside a bucket;
// at most SEL_E per thread of the CTA) while their blocks hold at most
// `budget` states together; the first is always taken. selC[0..K) gets the
// labels, selP[0..K] the exclusive prefix of their block sizes. Returns K to
// every thread (0: the worklist is empty). The labels are read with
// consecutive threads on consecutive ring entries; the sizes of bucket-0
// entries are known without a load (blocks only shrink and are never empty,
// so a label pushed with one state still has one).
__device__ int select_many(const FrontierArgs& a, const Worklist& wl, unsigned long long* head, CtaShared& sh,
                           int32_t* selC, int32_t* selP, int kmax, int32_t budget) {
    const unsigned lane = threadIdx.x & 31u;
    kmax = min(kmax, SEL_E * (int)blockDim.x);
    if (threadIdx.x < 32) {
        const unsigned long long h = head[lane];
        const unsigned long long t = *(volatile const unsigned long long*)&wl.tail[lane];
        const int av = (int)min(t - h, (unsigned long long)kmax);
        int x = av;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        sh.bx[lane] = x - av;
        sh.bn[lane] = av;
        sh.hp[lane] = (int)(h % (unsigned long long)wl.cap);
        if (lane == 31) sh.total = min(x, kmax);
    }
    __syncthreads();
    const int k0 = sh.total;
    {
        // all of this thread's ring loads are issued before the first store
        int32_t lv[SEL_E];
        int bk = 0;
#pragma unroll
        for (int e = 0; e < SEL_E; e++) {
            const int j = e * (int)blockDim.x + (int)threadIdx.x;
            lv[e] = -1;
            if (j < k0) {
                while (j >= sh.bx[bk] + sh.bn[bk]) bk++;
                int pos = sh.hp[bk] + (j - sh.bx[bk]);  // < 2 cap: the bucket holds at most cap entries
                if (pos >= wl.cap) pos -= wl.cap;
                lv[e] = ld(&wl.queue[(size_t)bk * wl.stride + wl.base + pos]);
            }
        }
#pragma unroll
        for (int e = 0; e < SEL_E; e++) {
            const int j = e * (int)blockDim.x + (int)threadIdx.x;
            if (j < k0) selC[j] = lv[e];
        }
    }
    __syncthreads();
    const int n0 = sh.bn[0];  // entries [0, n0) come from bucket 0
    if (n0 >= k0) {
        // every entry is a block of one state: prefix j, the budget caps the count
        const int K = k0 > 0 ? min(k0, max(budget, 1)) : 0;
        for (int j = threadIdx.x; j <= K; j += blockDim.x) selP[j] = j;
        if (threadIdx.x == 0) head[0] += (unsigned long long)K;
        __syncthreads();
        return K;
    }
    const int E = (k0 + (int)blockDim.x - 1) / (int)blockDim.x;
    const int j0 = (int)threadIdx.x * E;
    int32_t cs[SEL_E];
    int sz[SEL_E];
#pragma unroll
    for (int e = 0; e < SEL_E; e++) {
        const int j = j0 + e;
        cs[e] = e < E && j < k0 ? selC[j] : -1;
    }
    int mine = 0;
#pragma unroll
    for (int e = 0; e < SEL_E; e++) {
        sz[e] = cs[e] < 0 ? 0 : j0 + e < n0 ? 1 : ld(&a.bend[cs[e]]) - ld(&a.bbeg[cs[e]]);
        mine += sz[e];
    }
    int tot;
    int ex = cta_scan(mine, sh, tot);
    // sizes are positive, so the taken entries are a prefix
    int taken = 0;
#pragma unroll
    for (int e = 0; e < SEL_E; e++) {
        const int j = j0 + e;
        if (cs[e] >= 0 && (j == 0 || ex + sz[e] <= budget)) {
            selP[j] = ex;
            selP[j + 1] = ex + sz[e];  // the next entry's prefix (same value if it is taken)
            taken++;
        }
        ex += sz[e];
    }
    int K;
    cta_scan(taken, sh, K);
    if (threadIdx.x < 32) head[lane] += (unsigned long long)max(0, min(sh.bn[lane], K - sh.bx[lane]));
    __syncthreads();
    return K;
}

// index j of the splitter whose member range holds item i (selP[0] = 0)
__device__ __forceinline__ int find_sel(const int32_t* selP, int K, int32_t i) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (selP[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void claim_label(const FrontierArgs& a, int32_t b, unsigned long long key,
                                            uint32_t* lost, uint32_t stamp) {
    const unsigned long long old = atomicMin(&a.claim[b], key);
    if ((old >> 32) == (key >> 32)) {
        const uint32_t jo = (uint32_t)old, j = (uint32_t)key;
        if (jo < j)
            lost[j] = stamp;
        else if (jo > j)
            lost[jo] = stamp;
    }
}

// Claim phase: splitter j claims its own block and every block of more than
// one state that holds a predecessor of one of its members. Items (members
// of the K splitters, in order) go to warps gw, gw + nwarps, ...
__device__ void claim_step(const FrontierArgs& a, const int32_t* selC, const int32_t* selP, int K, uint32_t* lost,
                           uint32_t stamp, int64_t gw, int64_t nwarps) {
    const int lane = threadIdx.x & 31;
    const int32_t tot = selP[K];
    const unsigned long long hi = (unsigned long long)(~stamp) << 32;
    for (int64_t i = gw; i < tot; i += nwarps) {
        const int j = find_sel(selP, K, (int32_t)i);
        const int32_t C = selC[j];
        const unsigned long long key = hi | (unsigned)j;
        if (i == selP[j] && lane == 0 && ld(&a.bend[C]) - ld(&a.bbeg[C]) > 1) claim_label(a, C, key, lost, stamp);
        const int32_t t = ld(&a.elems[ld(&a.bbeg[C]) + (int32_t)i - selP[j]]);
        const int32_t j0 = a.in_ptr[t], j1 = a.in_ptr[t + 1];
        for (int32_t q = j0 + lane; q < j1; q += 32) {
            const int32_t s = (int32_t)(a.in_edge[q] >> 32);
            const int32_t b = ld(&a.block[s]);
            if (ld(&a.bend[b]) - ld(&a.bbeg[b]) > 1) claim_label(a, b, key, lost, stamp);
        }
    }
}

// Mark phase of a round with several splitters: a splitter that lost a claim
// goes back to the worklist (its unstable flag is still set); a winner
// clears its unstable flag (Algorithm 3, line 23) and marks as mark_step.
__device__ void mark_many(const FrontierArgs& a, const Worklist& wl, const int32_t* selC, const int32_t* selP,
                          int K, const uint32_t* lost, uint32_t stamp, int64_t gw, int64_t nwarps, int* n_small,
                          int* n_mid, int4* small_list, int4* mid_list, long long& edges,
                          long long& commits) {
    const int lane = threadIdx.x & 31;
    const int32_t tot = selP[K];
    for (int64_t i = gw; i < tot; i += nwarps) {
        const int j = find_sel(selP, K, (int32_t)i);
        const int32_t C = selC[j];
        const bool lose = ld_volatile_u32(&lost[j]) == stamp;
        if (i == selP[j] && lane == 0) {
            if (lose) {
                push(a, wl, C);
            } else {
                a.unstable[C] = 0u;
                commits++;
                TRACE_WIN();
            }
        }
        if (lose) continue;
        const int32_t t = ld(&a.elems[ld(&a.bbeg[C]) + (int32_t)i - selP[j]]);
        mark_member(a, t, stamp, C, n_small, n_mid, small_list, mid_list, edges);
    }
}

// Pop the next splitter (lowest non-empty size bucket) with warp 0 of the CTA;
// returns it to every thread, or -1 when the worklist is empty.
__device__ __forceinline__ int32_t select_splitter(const Worklist& wl, unsigned long long* head, CtaShared& sh) {
    const unsigned lane = threadIdx.x & 31u;
    if (threadIdx.x < 32) {
        const unsigned long long h = head[lane];
        // the tails are global (grid engine) or shared (batch engine): a
        // volatile generic load serves both without using a stale L1 line
        const bool ne = h < *(volatile const unsigned long long*)&wl.tail[lane];
        const unsigned bal = __ballot_sync(0xffffffffu, ne);
        if (bal == 0u) {
            if (lane == 0) {
                sh.C = -1;
                sh.bk = -1;
            }
        } else if ((int)lane == __ffs(bal) - 1) {
            sh.C = ld(&wl.queue[(size_t)lane * wl.stride + wl.base + h % (unsigned long long)wl.cap]);
            sh.bk = (int)lane;
            head[lane] = h + 1;
        }
    }
    __syncthreads();
    const int32_t C = sh.C;
    __syncthreads();
    return C;
}

__global__ void __launch_bounds__(1024) k_frontier_main(FrontierArgs a) {
    __shared__ CtaShared sh;
    __shared__ int s_defer[32];
    __shared__ int s_ndefer;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int32_t n = a.n;
    const int64_t gw = gtid >> 5, nwarps = gsz >> 5;
    unsigned long long tgt = 0;
    long long edges = 0, states = 0;
    if (a.test_hook == 1 && blockIdx.x == 0) return;  // testing: never arrive
    if (threadIdx.x < BISIM_BUCKETS) sh.head[threadIdx.x] = 0;
    const Worklist wl{a.ctrl->bq_tail, a.queue, (size_t)n, 0, n};
    int64_t r = 0;
    for (;;) {
        r++;
        const uint32_t stamp = a.stamp0 + (uint32_t)r;
        const int par = (int)(r & 1);
        // every CTA pops the same label
        const int32_t C = select_splitter(wl, sh.head, sh);
        if (C < 0) break;  // no unstable label: C = bottom
        if (r > a.round_cap) {
            if (gtid == 0) atomicOr(&a.ctrl->status, ST_ROUNDS);
            break;
        }
        if (gtid == 0) {
            a.unstable[C] = 0u;
            a.ctrl->n_touched[par ^ 1] = 0;
            a.ctrl->n_mid[par ^ 1] = 0;
        }
        mark_step(a, C, stamp, gw, nwarps, &a.ctrl->n_touched[par], &a.ctrl->n_mid[par], a.tlist,
                  a.tlist + n, edges);
        if (!grid_sync(a.gb, tgt)) return;
        split_step(a, wl, sh, s_defer, &s_ndefer, stamp, C, ldcg(&a.ctrl->n_touched[par]), a.tlist,
                   ldcg(&a.ctrl->n_mid[par]), a.tlist + n, (int)blockIdx.x, (int)gridDim.x, states);
        if (!grid_sync(a.gb, tgt)) return;
    }
    if (edges) atomicAdd((unsigned long long*)&a.ctrl->edges, (unsigned long long)edges);
    if (states) atomicAdd((unsigned long long*)&a.ctrl->states, (unsigned long long)states);
    if (gtid == 0) {
        a.ctrl->rounds = r;
        a.ctrl->commits = r - 1;  // one splitter per round
    }
}

__device__ __forceinline__ unsigned long long ld_acquire_u64_g(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Hybrid schedule for one LTS. CTA 0 selects every splitter. A light round
// (at most 32 members whose incoming transitions number at most light_edges)
// is done by CTA 0 alone with CTA barriers; a heavy round is published
// (cmd_C, cmd_stamp, then cmd_seq with release order) and done by the whole
// grid with two grid barriers, exactly as k_frontier_main. The other CTAs
// wait for commands; their wait is bounded by timeout_ns without progress,
// where progress is a new command or a new heartbeat from CTA 0.
// One item per warp (a round's splitters hold at most as many states as
// there are warps): the claim pass keeps what it loaded in registers for the
// mark pass - the member t, its incoming-transition range and, one per
// lane, the first 32 transitions with their source's block and its range
// (nothing changes them between the two passes).
struct ItemCarry {
    int32_t j;  // splitter index, -1: this warp has no item
    int32_t C;
    int32_t j0, j1;
    unsigned long long e;  // this lane's transition j0 + lane, when < j1
    int32_t b, bb, be;     // its source's block and block range
};

__device__ __forceinline__ void claim_item(const FrontierArgs& a, const int32_t* selC, const int32_t* selP, int K,
                                           uint32_t* lost, uint32_t stamp, int64_t i, ItemCarry& ic) {
    const int lane = threadIdx.x & 31;
    ic.j = -1;
    if (i >= selP[K]) return;
    const int j = find_sel(selP, K, (int32_t)i);
    const int32_t C = selC[j];
    ic.j = j;
    ic.C = C;
    const unsigned long long key = ((unsigned long long)(~stamp) << 32) | (unsigned)j;
    int32_t t = C;  // a block of one state holds its label only
    if (selP[j + 1] - selP[j] > 1) {
        const int32_t cb = ld(&a.bbeg[C]);
        if (i == selP[j] && lane == 0) claim_label(a, C, key, lost, stamp);
        t = ld(&a.elems[cb + (int32_t)i - selP[j]]);
    }
    ic.j0 = a.in_ptr[t];
    ic.j1 = a.in_ptr[t + 1];
    const bool has = ic.j0 + lane < ic.j1;
    if (has) {
        ic.e = a.in_edge[ic.j0 + lane];
        ic.b = ld(&a.block[(int32_t)(ic.e >> 32)]);
        ic.bb = ld(&a.bbeg[ic.b]);
        ic.be = ld(&a.bend[ic.b]);
    }
    // one claim per distinct block of the warp (sources often share a block)
    const bool cl = has && ic.be - ic.bb > 1;
    const unsigned peers = __match_any_sync(0xffffffffu, cl ? ic.b : -1 - lane);  // every lane gets here
    if (cl && (peers & lanemask_lt()) == 0u) claim_label(a, ic.b, key, lost, stamp);
    for (int32_t q = ic.j0 + 32 + lane; q < ic.j1; q += 32) {
        const int32_t b = ld(&a.block[(int32_t)(a.in_edge[q] >> 32)]);
        if (ld(&a.bend[b]) - ld(&a.bbeg[b]) > 1) claim_label(a, b, key, lost, stamp);
    }
}

__device__ __forceinline__ void mark_item(const FrontierArgs& a, const Worklist& wl, const int32_t* selP,
                                          const uint32_t* lost, uint32_t stamp, int64_t i, const ItemCarry& ic,
                                          int* n_small, int* n_mid, int4* small_list, int4* mid_list,
                                          long long& edges, long long& commits) {
    const int lane = threadIdx.x & 31;
    if (ic.j < 0) return;
    const bool lose = ld_volatile_u32(&lost[ic.j]) == stamp;
    if (i == selP[ic.j] && lane == 0) {
        if (lose) {
            push(a, wl, ic.C);
        } else {
            a.unstable[ic.C] = 0u;
            commits++;
            TRACE_WIN();
        }
    }
    if (lose) return;
    if (lane == 0) edges += ic.j1 - ic.j0;
    if (ic.j0 + lane < ic.j1) {
        const int32_t s = (int32_t)(ic.e >> 32);
        a.mark[(uint32_t)ic.e] = stamp;
        if (atomicExch(&a.smark[s], stamp) != stamp)
            rank_marked(a, s, ic.b, ic.bb, ic.be, ic.C, n_small, n_mid, small_list, mid_list);
    }
    for (int32_t q = ic.j0 + 32 + lane; q < ic.j1; q += 32) {
        const unsigned long long e = a.in_edge[q];
        const int32_t s = (int32_t)(e >> 32);
        a.mark[(uint32_t)e] = stamp;
        const int32_t b = ld(&a.block[s]);
        if (atomicExch(&a.smark[s], stamp) == stamp) continue;
        rank_marked(a, s, b, ld(&a.bbeg[b]), ld(&a.bend[b]), ic.C, n_small, n_mid, small_list, mid_list);
    }
}

struct HybridArgs {
    int light_edges;   // a one-splitter round with at most 32 members and this many
                       // incoming transitions runs on CTA 0 alone
    int kmax;          // most splitters per round (1: one per round); the dynamic shared
                       // memory holds kmax labels and kmax + 1 prefix entries
    int budget;        // states of a round's splitters at most (grid rounds)
    int local_budget;  // rounds with several splitters and at most this many states (<= 32)
                       // run on CTA 0
    int32_t* g_selC;   // [BISIM_KMAX_GRID] published splitters
    int32_t* g_selP;   // [BISIM_KMAX_GRID + 1] their size prefix
    uint32_t* g_lost;  // [BISIM_KMAX_GRID] round in which each lost a claim
    int peel;          // 1: grid rounds with several splitters are peel rounds
    int cap0;          // peel rounds: most splitters of one state per round
};

// The three phases of a round with several splitters, by the warps gw,
// gw + nwarps, ... of the grid (sync = grid barrier) or of one CTA.
template <typename Sync>
__device__ __forceinline__ bool multi_round(const FrontierArgs& a, const Worklist& wl, CtaShared& sh, int* defer,
                                            int* ndefer, const int32_t* selC, const int32_t* selP, int K,
                                            uint32_t* lost, uint32_t stamp, int64_t gw, int64_t nwarps, int* n_small,
                                            int* n_mid, int4* small_list, int4* mid_list, int cta, int ncta,
                                            long long& edges, long long& states, long long& commits, Sync sync) {
    if (selP[K] <= nwarps) {
        ItemCarry ic;
        claim_item(a, selC, selP, K, lost, stamp, gw, ic);
        PHASE(2);
        if (!sync()) return false;
        PHASE(3);
        mark_item(a, wl, selP, lost, stamp, gw, ic, n_small, n_mid, small_list, mid_list, edges, commits);
    } else {
        claim_step(a, selC, selP, K, lost, stamp, gw, nwarps);
        PHASE(2);
        if (!sync()) return false;
        PHASE(3);
        mark_many(a, wl, selC, selP, K, lost, stamp, gw, nwarps, n_small, n_mid, small_list, mid_list, edges,
                  commits);
    }
    PHASE(4);
    if (!sync()) return false;
    PHASE(5);
    const int ns = ld_volatile_i32(n_small), nm = ld_volatile_i32(n_mid);
    PHASE_ADD(14, (unsigned long long)(ns + nm));
    TRACE_TOUCHED((unsigned long long)(ns + nm));
    split_step(a, wl, sh, defer, ndefer, stamp, MULTI, ns, small_list, nm, mid_list, cta, ncta, states);
    PHASE(6);
    const bool ok = sync();
    PHASE(7);
    return ok;
}

// ------------------------------------------------------------- peel rounds
//
// Grid rounds with several splitters, generalising the claim rule above so
// that a block may be split by several splitters of the same round. Keys
// order the round's splitters by label: key = (~stamp << 32) | (C << 1) | x.
// A splitter touches a block b (of more than one state) that holds a
// predecessor of one of its members; the touch is a "peel" (x = 0) when the
// splitter has one state, all its incoming transitions are walked by one
// warp, and among them exactly one member of b and not b's leader is a
// source; every other touch, and a splitter's claim on its own block when it
// has several states, is exclusive (x = 1). Every touch lowers claim[b] to
// its key, exclusive ones also minx[b]. The least touch of b decides:
//   exclusive (minx[b] == claim[b]): that splitter alone splits b, with
//     Algorithm 3's rule, and every other toucher of b loses;
//   peel (otherwise): every exclusive toucher of b loses, the peeling ones
//     do not, and b is split as described before warp_peel.
// A splitter that loses anywhere goes back to the worklist and marks nothing
// (exclusive losers are known from the claims themselves: an exclusive touch
// that meets or is displaced by a lesser key records the loss in lostl; a
// peeling splitter checks its blocks' words after the barrier). The least
// splitter of the round never loses, so every round carries out at least one
// iteration. The winners' iterations touch disjoint data except on peeled
// blocks, where running them one after the other in label order gives the
// same split; so a round again has the effect of a sequence of Algorithm 3
// iterations. The splitters of one state come by position from the ring of
// size bucket 0, so a round may take tens of thousands of them.

#ifndef BISIM_PEEL_CHUNKS
#define BISIM_PEEL_CHUNKS 4
#endif
constexpr int PEEL_CHUNKS = BISIM_PEEL_CHUNKS;  // chunks of 32 transitions a warp loads at once
constexpr int PEEL_MIN_SINGLES = 256;    // a peel round needs this many labels in size bucket 0
constexpr int PEEL_QUIET = 32;           // a peel round is quiet below one touched block per 32 splitters
constexpr int PEEL_SWEEP_GROWTH = 4;     // after a quiet round the next takes this many times the labels
constexpr int PEEL_SWEEP_MAX = 1 << 24;  // labels one sweep round takes at most

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    return *(volatile const unsigned long long*)p;
}

__device__ __forceinline__ unsigned long long peel_key(uint32_t stamp, int32_t C, bool x) {
    return ((unsigned long long)(~stamp) << 32) | ((unsigned long long)(uint32_t)C << 1) | (x ? 1ull : 0ull);
}

__device__ __forceinline__ void claim_peel(const FrontierArgs& a, int32_t b, unsigned long long key, bool x,
                                           uint32_t stamp) {
    const unsigned long long old = atomicMin(&a.claim[b], key);
    if (x) atomicMin(&a.minx[b], key);
    if ((old >> 32) == (key >> 32)) {
        if (old < key) {
            if (x) a.lostl[(uint32_t)key >> 1] = stamp;
        } else if (old > key && (old & 1ull)) {
            a.lostl[(uint32_t)old >> 1] = stamp;
        }
    }
}

// Selection of a peel round by every CTA: K0 labels of size bucket 0 (blocks
// of one state; blocks only shrink and are never empty) from the head of its
// ring, at most cap0 (sh.k0, and the ring-0 head before them in sh.h0), and
// up to kmax1 labels of the higher buckets (lowest first, FIFO inside a
// bucket) while their blocks hold at most budget1 states together, listed in
// selC with the exclusive prefix of their sizes in selP. Returns the number
// of the higher-bucket labels to every thread.
constexpr int PEEL_SEL_E = 16;  // listed labels per thread of a peel selection at most

__device__ int select_peel(const FrontierArgs& a, const Worklist& wl, unsigned long long* head, CtaShared& sh,
                           int32_t* selC, int32_t* selP, int kmax1, int32_t budget1, int cap0, bool sweep) {
    const unsigned lane = threadIdx.x & 31u;
    if (sweep) {
        // sweep round: up to cap0 labels by position from the rings, lowest
        // bucket first, nothing listed; ring b's run starts at ring position
        // hp[b], holds bn[b] labels and is items [bx[b], bx[b] + bn[b])
        if (threadIdx.x < 32) {
            const unsigned long long h = head[lane];
            const unsigned long long t = *(volatile const unsigned long long*)&wl.tail[lane];
            const long long av = (long long)(t - h);
            long long x = av;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, x, o);
                if ((int)lane >= o) x += y;
            }
            const long long ex = x - av;
            const int take = (int)max(0ll, min(av, (long long)cap0 - ex));
            sh.bx[lane] = (int)min(ex, (long long)cap0);
            sh.bn[lane] = take;
            sh.hp[lane] = (int)(h % (unsigned long long)wl.cap);
            head[lane] = h + (unsigned long long)take;
            if (lane == 31) sh.k0 = (int)min(x, (long long)cap0);
            if (lane == 0) sh.h0 = h;
        }
        if (threadIdx.x == 0) selP[0] = 0;
        __syncthreads();
        return 0;
    }
    kmax1 = min(kmax1, PEEL_SEL_E * (int)blockDim.x);
    if (threadIdx.x < 32) {
        const unsigned long long h = head[lane];
        const unsigned long long t = *(volatile const unsigned long long*)&wl.tail[lane];
        const int av = lane == 0 ? 0 : (int)min(t - h, (unsigned long long)kmax1);
        int x = av;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        sh.bx[lane] = x - av;
        sh.bn[lane] = av;
        sh.hp[lane] = (int)(h % (unsigned long long)wl.cap);
        if (lane == 0) {
            sh.k0 = (int)min(t - h, (unsigned long long)max(cap0, 0));
            sh.h0 = h;
        }
        if (lane == 31) sh.total = min(x, kmax1);
    }
    __syncthreads();
    const int k1 = sh.total;
    const int K0 = sh.k0;
    {
        int32_t lv[PEEL_SEL_E];
        int bk = 1;
#pragma unroll
        for (int e = 0; e < PEEL_SEL_E; e++) {
            const int j = e * (int)blockDim.x + (int)threadIdx.x;
            lv[e] = -1;
            if (j < k1) {
                while (j >= sh.bx[bk] + sh.bn[bk]) bk++;
                int pos = sh.hp[bk] + (j - sh.bx[bk]);
                if (pos >= wl.cap) pos -= wl.cap;
                lv[e] = ld(&wl.queue[(size_t)bk * wl.stride + wl.base + pos]);
            }
        }
#pragma unroll
        for (int e = 0; e < PEEL_SEL_E; e++) {
            const int j = e * (int)blockDim.x + (int)threadIdx.x;
            if (j < k1) selC[j] = lv[e];
        }
    }
    if (threadIdx.x == 0) selP[0] = 0;
    __syncthreads();
    const int E = (k1 + (int)blockDim.x - 1) / (int)blockDim.x;
    const int j0 = (int)threadIdx.x * E;
    int32_t cs[PEEL_SEL_E];
    int sz[PEEL_SEL_E];
    int mine = 0, mine_w = 0;  // states, and states of blocks of several states
#pragma unroll
    for (int e = 0; e < PEEL_SEL_E; e++) {
        const int j = j0 + e;
        cs[e] = e < E && j < k1 ? selC[j] : -1;
        sz[e] = cs[e] < 0 ? 0 : ld(&a.bend[cs[e]]) - ld(&a.bbeg[cs[e]]);
        mine += sz[e];
        mine_w += sz[e] > 1 ? sz[e] : 0;
    }
    int tot;
    int ex = cta_scan(mine, sh, tot);
    // the budget counts the splitters of several states only (a label pushed
    // with a larger block whose block now has one state costs as little as a
    // label of bucket 0); the costs are non-negative, so the taken entries
    // are again a prefix
    int exw = cta_scan(mine_w, sh, tot);
    int taken = 0;
#pragma unroll
    for (int e = 0; e < PEEL_SEL_E; e++) {
        const int j = j0 + e;
        const int w = sz[e] > 1 ? sz[e] : 0;
        // the first is taken when nothing else is, so a round is never empty
        if (cs[e] >= 0 && ((j == 0 && K0 == 0) || exw + w <= budget1)) {
            selP[j] = ex;
            selP[j + 1] = ex + sz[e];
            taken++;
        }
        ex += sz[e];
        exw += w;
    }
    int K1;
    cta_scan(taken, sh, K1);
    // listed labels whose block now has one state (they may peel)
    int ones = 0;
#pragma unroll
    for (int e = 0; e < PEEL_SEL_E; e++) ones += (cs[e] >= 0 && j0 + e < K1 && sz[e] == 1) ? 1 : 0;
    int n1;
    cta_scan(ones, sh, n1);
    if (threadIdx.x == 0) sh.n1 = n1;
    if (threadIdx.x < 32) {
        if (lane == 0)
            head[0] += (unsigned long long)K0;
        else
            head[lane] += (unsigned long long)max(0, min(sh.bn[lane], K1 - sh.bx[lane]));
    }
    __syncthreads();
    return K1;
}

// One item of a peel round: a member t of splitter C with its incoming range.
struct PeelItem {
    int32_t C, t, d0, deg;
    bool first;   // the first member of its splitter
    bool single;  // the splitter has one state
    bool defer;   // sweep rounds: a label whose block has several states, pushed back untouched
};

__device__ __forceinline__ PeelItem peel_item(const FrontierArgs& a, const Worklist& wl, unsigned long long h0,
                                              const CtaShared* sw, int K0, const int32_t* selC,
                                              const int32_t* selP, int K1, int64_t item) {
    PeelItem it;
    it.defer = false;
    if (item < K0) {
        int bk = 0;
        unsigned long long pos;
        if (sw) {
            // sweep round: entry (item - bx[bk]) of ring bk's taken run
            const int i = (int)item;
            while (i >= sw->bx[bk] + sw->bn[bk]) bk++;
            pos = (unsigned long long)sw->hp[bk] + (unsigned long long)(i - sw->bx[bk]);
            if (pos >= (unsigned long long)wl.cap) pos -= (unsigned long long)wl.cap;
        } else {
            pos = (h0 + (unsigned long long)item) % (unsigned long long)wl.cap;
        }
        it.C = ld(&wl.queue[(size_t)bk * wl.stride + wl.base + pos]);
        it.t = it.C;  // the label of a block of one state is that state
        it.first = true;
        it.single = true;
        if (bk > 0 && ld(&a.bend[it.C]) - ld(&a.bbeg[it.C]) != 1) {
            it.defer = true;
            it.d0 = 0;
            it.deg = 0;
            return it;
        }
    } else {
        const int32_t i = (int32_t)(item - K0);
        const int j = find_sel(selP, K1, i);
        it.C = selC[j];
        it.first = i == selP[j];
        it.single = selP[j + 1] - selP[j] == 1;
        it.t = it.single ? it.C : ld(&a.elems[ld(&a.bbeg[it.C]) + i - selP[j]]);
    }
    it.d0 = a.in_ptr[it.t];
    it.deg = a.in_ptr[it.t + 1] - it.d0;
    return it;
}

// The loads of one packed chunk lane: its transition, source, source block
// and the block's range.
struct PeelEdge {
    unsigned long long e;
    int32_t b, bb, be;
};

// The claim (pass 0) and mark (pass 1) work of a warp on the items
// [g0, g1) of the round (at most 32; lane l holds item g0 + l). Items with
// at most 32 incoming transitions are packed whole into chunks of 32 lanes
// (so one ballot sees all of an item's transitions); larger ones are walked
// by the whole warp afterwards and touch exclusively.
template <int PASS>
__device__ void peel_items(const FrontierArgs& a, const Worklist& wl, unsigned long long h0, const CtaShared* sw,
                           int K0, const int32_t* selC, const int32_t* selP, int K1, int64_t g0, int64_t g1,
                           uint32_t stamp, int* n_small, int* n_mid, int4* small_list, int4* mid_list,
                           int* n_defer, long long& edges, long long& commits) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned FULL = 0xffffffffu;
    const int ng = (int)(g1 - g0);
    PeelItem it;
    it.C = -1;
    it.deg = 0;
    it.single = true;
    it.first = false;
    it.defer = false;
    it.t = 0;
    it.d0 = 0;
    if ((int)lane < ng) it = peel_item(a, wl, h0, sw, K0, selC, selP, K1, g0 + lane);
    // pass 1: an item of one state that pass 0 carried out already (it touched
    // no block of several states) is done
    bool done = false;
    if (PASS == 1 && (int)lane < ng && it.single && !it.defer && ld(&a.unstable[it.C]) == 0u) {
        done = true;
        it.deg = 0;
    }
    // pass 1: exclusive losses recorded by the claims
    bool lost_x = false;
    if (PASS == 1 && (int)lane < ng) lost_x = ld_volatile_u32(&a.lostl[it.C]) == stamp;
    const bool packable = (int)lane < ng && it.deg > 0 && it.deg <= 32;
    // greedy packing: chunk and first lane of every packable item
    int my_chunk = -1, my_start = 0, nchunks = 0;
    {
        int cur = 0, chunk = 0;
        const int dp = packable ? it.deg : 0;
        for (int i = 0; i < ng; i++) {
            const int d = __shfl_sync(FULL, dp, i);
            if (d == 0) continue;
            if (cur + d > 32) {
                chunk++;
                cur = 0;
            }
            if ((int)lane == i) {
                my_chunk = chunk;
                my_start = cur;
            }
            cur += d;
        }
        nchunks = cur > 0 ? chunk + 1 : chunk;
    }
    // pass 1: the item's loss as seen from its peel touches (filled per chunk);
    // pass 0: whether one of its transitions comes from a block of several states
    bool lost_p = false, touched = false;
    for (int c0 = 0; c0 < nchunks; c0 += PEEL_CHUNKS) {
        PeelEdge ed[PEEL_CHUNKS];
        int src_lane[PEEL_CHUNKS];
        bool val[PEEL_CHUNKS];
#pragma unroll
        for (int u = 0; u < PEEL_CHUNKS; u++) {
            const int c = c0 + u;
            const unsigned mc = __ballot_sync(FULL, my_chunk == c);
            const unsigned starts = __reduce_or_sync(FULL, my_chunk == c ? (1u << my_start) : 0u);
            // the r-th item of the chunk owns this lane
            const int r = __popc(starts & (0xffffffffu >> (31 - lane))) - 1;
            const int il = (mc != 0u && r >= 0) ? (int)__fns(mc, 0, r + 1) : 0;
            const int st = __shfl_sync(FULL, my_start, il);
            const int dg = __shfl_sync(FULL, it.deg, il);
            const int d0 = __shfl_sync(FULL, it.d0, il);
            val[u] = c < nchunks && mc != 0u && r >= 0 && (int)lane < st + dg;
            src_lane[u] = il;
            ed[u].e = val[u] ? a.in_edge[d0 + (int)lane - st] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < PEEL_CHUNKS; u++) ed[u].b = val[u] ? ld(&a.block[(int32_t)(ed[u].e >> 32)]) : 0;
#pragma unroll
        for (int u = 0; u < PEEL_CHUNKS; u++) {
            ed[u].bb = val[u] ? ld(&a.bbeg[ed[u].b]) : 0;
            ed[u].be = val[u] ? ld(&a.bend[ed[u].b]) : 0;
        }
#pragma unroll
        for (int u = 0; u < PEEL_CHUNKS; u++) {
            if (c0 + u >= nchunks) break;  // warp-uniform
            const int il = src_lane[u];
            const int32_t s = (int32_t)(ed[u].e >> 32);
            const int32_t b = ed[u].b;
            const bool ns = val[u] && ed[u].be - ed[u].bb > 1;
            const int32_t C = __shfl_sync(FULL, it.C, il);
            const bool single = __shfl_sync(FULL, it.single, il);
            // lanes of this item that reach block b, and those among them from source s
            const unsigned long long vb = ns ? ((unsigned long long)il << 32) | (uint32_t)b : ~0ull - lane;
            const unsigned mb = __match_any_sync(FULL, vb);
            const unsigned long long vbs = ns ? ((unsigned long long)(uint32_t)b << 32) | (uint32_t)s : ~0ull - lane;
            const unsigned mbs = __match_any_sync(FULL, vbs) & mb;
            const bool lead = (__ballot_sync(FULL, ns && s == b) & mb) != 0u;
            const bool x = !single || mbs != mb || lead;
            if (PASS == 0) {
                if (ns && (mb & lanemask_lt()) == 0u) claim_peel(a, b, peel_key(stamp, C, x), x, stamp);
                const unsigned nsm = __ballot_sync(FULL, ns);
                if (my_chunk == c0 + u) {
                    const unsigned mine = (it.deg >= 32 ? 0xffffffffu : ((1u << it.deg) - 1u)) << my_start;
                    touched = (nsm & mine) != 0u;
                }
            } else {
                // a peel touch of a block whose least touch is exclusive: this splitter loses
                const bool lp = ns && !x && ld_volatile_u64(&a.minx[b]) == ld_volatile_u64(&a.claim[b]);
                const unsigned lpm = __ballot_sync(FULL, lp);
                const int st = __shfl_sync(FULL, my_start, il);
                const int dg = __shfl_sync(FULL, it.deg, il);
                const unsigned range = (dg >= 32 ? 0xffffffffu : ((1u << dg) - 1u)) << st;
                const bool lose = __shfl_sync(FULL, lost_x, il) || (lpm & range) != 0u;
                if (my_chunk == c0 + u) {
                    const unsigned mine = (it.deg >= 32 ? 0xffffffffu : ((1u << it.deg) - 1u)) << my_start;
                    lost_p = lost_x || (lpm & mine) != 0u;
                }
                if (ns && !lose) {
                    if (x) {
                        a.mark[(uint32_t)ed[u].e] = stamp;
                        if (atomicExch(&a.smark[s], stamp) != stamp)
                            rank_marked(a, s, b, ed[u].bb, ed[u].be, C, n_small, n_mid, small_list, mid_list, 0);
                    } else {
                        const unsigned long long pk = ((unsigned long long)(~stamp) << 32) | (uint32_t)C;
                        const unsigned long long old = atomicMin(&a.smark64[s], pk);
                        if ((old >> 32) != (pk >> 32))
                            rank_marked(a, s, b, ed[u].bb, ed[u].be, C, n_small, n_mid, small_list, mid_list, 1);
                    }
                }
            }
        }
    }
    // items with more than 32 incoming transitions: the whole warp walks each;
    // all their touches are exclusive (no unit check across chunks)
    unsigned big = __ballot_sync(FULL, (int)lane < ng && it.deg > 32);
    while (big) {
        const int il = __ffs(big) - 1;
        big &= big - 1u;
        const int32_t C = __shfl_sync(FULL, it.C, il);
        const int32_t d0 = __shfl_sync(FULL, it.d0, il);
        const int32_t dg = __shfl_sync(FULL, it.deg, il);
        const bool lose = PASS == 1 && __shfl_sync(FULL, lost_x, il);
        bool tb = false;
        for (int32_t q0 = 0; q0 < dg; q0 += 32) {
            const bool v = q0 + (int32_t)lane < dg;
            const unsigned long long e = v ? a.in_edge[d0 + q0 + (int32_t)lane] : 0ull;
            const int32_t s = (int32_t)(e >> 32);
            const int32_t b = v ? ld(&a.block[s]) : 0;
            const int32_t bb = v ? ld(&a.bbeg[b]) : 0, be = v ? ld(&a.bend[b]) : 0;
            const bool ns = v && be - bb > 1;
            tb |= __any_sync(FULL, ns);
            if (PASS == 0) {
                const unsigned mb = __match_any_sync(FULL, ns ? b : -1 - (int)lane);
                if (ns && (mb & lanemask_lt()) == 0u) claim_peel(a, b, peel_key(stamp, C, true), true, stamp);
            } else if (ns && !lose) {
                a.mark[(uint32_t)e] = stamp;
                if (atomicExch(&a.smark[s], stamp) != stamp)
                    rank_marked(a, s, b, bb, be, C, n_small, n_mid, small_list, mid_list, 0);
            }
        }
        if ((int)lane == il) {
            lost_p = lost_x;
            touched = tb;
        }
    }
    if (PASS == 0 && n_defer) {
        const unsigned dm = __ballot_sync(FULL, (int)lane < ng && it.defer);
        if (dm != 0u && lane == 0) atomicAdd(n_defer, __popc(dm));
    }
    if ((int)lane < ng && !done) {
        if (PASS == 0) {
            // a splitter of several states claims its own block
            if (it.first && !it.single) claim_peel(a, it.C, peel_key(stamp, it.C, true), true, stamp);
            if (it.single && !touched && !it.defer) {
                // nothing to claim, nothing to mark: this iteration is carried out now
                a.unstable[it.C] = 0u;
                commits++;
                edges += it.deg;
                TRACE_WIN();
            }
        } else {
            const bool lose = lost_x || lost_p || it.defer;
            if (it.first) {
                if (lose) {
                    push(a, wl, it.C);
                } else {
                    a.unstable[it.C] = 0u;
                    commits++;
                    TRACE_WIN();
                }
            }
            if (!lose) edges += it.deg;
        }
    }
}

// What a warp's claim pass keeps for its mark pass when its share of the
// round is one group of at most 32 items in at most PEEL_CARRY_CHUNKS chunks
// of 32 transitions with no item of more than 32 transitions: per lane its
// item (registers), and per chunk the lane's transition, its source's block
// and flags (the lane of the transition's item, whether the block has several
// states, whether the touch is exclusive) in the warp's slice of shared
// memory, each lane reading back only what it wrote.
constexpr int PEEL_CARRY_CHUNKS = 8;
constexpr int PEEL_CARRY_BYTES = PEEL_CARRY_CHUNKS * 32 * 16;  // per warp

struct PeelCarry {
    int32_t C, deg;
    bool first, pending;  // pending: the item is decided in the mark pass
    bool defer;           // pushed back untouched (sweep rounds)
    int my_chunk, my_start, nchunks;
    unsigned long long* e;  // [chunk * 32 + lane]
    int32_t* b;
    int* fl;                // item lane | 32 (block of several states) | 64 (exclusive touch)
};

__device__ __forceinline__ void peel_carry_at(PeelCarry& cy, unsigned char* warp_slice) {
    cy.e = reinterpret_cast<unsigned long long*>(warp_slice);
    cy.b = reinterpret_cast<int32_t*>(warp_slice + PEEL_CARRY_CHUNKS * 32 * 8);
    cy.fl = reinterpret_cast<int*>(warp_slice + PEEL_CARRY_CHUNKS * 32 * 12);
}

// Claim pass of a warp's items [g0, g1) (g1 - g0 <= 32). Returns true (to
// every lane) when everything the mark pass needs is in `cy`; then the items
// of one state that touched no block of several states are carried out here
// already (they claim nothing, so they cannot lose, and they mark nothing).
// Otherwise the claims are made by peel_items<0> and the mark pass must
// recompute.
__device__ bool peel_claim(const FrontierArgs& a, const Worklist& wl, unsigned long long h0, const CtaShared* sw,
                           int K0, const int32_t* selC, const int32_t* selP, int K1, int64_t g0, int64_t g1,
                           uint32_t stamp, PeelCarry& cy, int* n_defer, long long& edges, long long& commits) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned FULL = 0xffffffffu;
    const int ng = (int)(g1 - g0);
    PeelItem it;
    it.C = -1;
    it.deg = 0;
    it.single = true;
    it.first = false;
    it.defer = false;
    it.t = 0;
    it.d0 = 0;
    if ((int)lane < ng) it = peel_item(a, wl, h0, sw, K0, selC, selP, K1, g0 + lane);
    const bool packable = (int)lane < ng && it.deg > 0 && it.deg <= 32;
    int cur = 0, chunk = 0;
    cy.my_chunk = -1;
    cy.my_start = 0;
    {
        const int dp = packable ? it.deg : 0;
        for (int i = 0; i < ng; i++) {
            const int d = __shfl_sync(FULL, dp, i);
            if (d == 0) continue;
            if (cur + d > 32) {
                chunk++;
                cur = 0;
            }
            if ((int)lane == i) {
                cy.my_chunk = chunk;
                cy.my_start = cur;
            }
            cur += d;
        }
    }
    const int nchunks = cur > 0 ? chunk + 1 : chunk;  // the same on every lane
    const bool fits =
        nchunks <= PEEL_CARRY_CHUNKS && __ballot_sync(FULL, (int)lane < ng && it.deg > 32) == 0u;
    if (!fits) {
        peel_items<0>(a, wl, h0, sw, K0, selC, selP, K1, g0, g1, stamp, nullptr, nullptr, nullptr, nullptr, n_defer,
                      edges, commits);
        return false;
    }
    if (n_defer) {
        const unsigned dm = __ballot_sync(FULL, (int)lane < ng && it.defer);
        if (dm != 0u && lane == 0) atomicAdd(n_defer, __popc(dm));
    }
    cy.C = it.C;
    cy.deg = it.deg;
    cy.first = it.first;
    cy.defer = it.defer;
    cy.nchunks = nchunks;
    bool touched = false;  // item lane: one of its transitions comes from a block of several states
    for (int u0 = 0; u0 < nchunks; u0 += PEEL_CHUNKS) {
        bool val[PEEL_CHUNKS];
        int ils[PEEL_CHUNKS], bb[PEEL_CHUNKS], be[PEEL_CHUNKS];
        unsigned long long e[PEEL_CHUNKS];
        int32_t b[PEEL_CHUNKS];
#pragma unroll
        for (int k = 0; k < PEEL_CHUNKS; k++) {
            const int u = u0 + k;
            const unsigned mc = __ballot_sync(FULL, cy.my_chunk == u);
            const unsigned starts = __reduce_or_sync(FULL, cy.my_chunk == u ? (1u << cy.my_start) : 0u);
            const int r = __popc(starts & (0xffffffffu >> (31 - lane))) - 1;
            const int il = (mc != 0u && r >= 0) ? (int)__fns(mc, 0, r + 1) : 0;
            const int st = __shfl_sync(FULL, cy.my_start, il);
            const int dg = __shfl_sync(FULL, it.deg, il);
            const int d0 = __shfl_sync(FULL, it.d0, il);
            val[k] = u < nchunks && mc != 0u && r >= 0 && (int)lane < st + dg;
            ils[k] = il;
            e[k] = val[k] ? a.in_edge[d0 + (int)lane - st] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < PEEL_CHUNKS; k++) b[k] = val[k] ? ld(&a.block[(int32_t)(e[k] >> 32)]) : 0;
#pragma unroll
        for (int k = 0; k < PEEL_CHUNKS; k++) {
            bb[k] = val[k] ? ld(&a.bbeg[b[k]]) : 0;
            be[k] = val[k] ? ld(&a.bend[b[k]]) : 0;
        }
#pragma unroll
        for (int k = 0; k < PEEL_CHUNKS; k++) {
            const int u = u0 + k;
            const int il = ils[k];
            const int32_t s = (int32_t)(e[k] >> 32);
            const bool ns = val[k] && be[k] - bb[k] > 1;
            const int32_t C = __shfl_sync(FULL, it.C, il);
            const bool single = __shfl_sync(FULL, it.single, il);
            const unsigned long long vb = ns ? ((unsigned long long)il << 32) | (uint32_t)b[k] : ~0ull - lane;
            const unsigned mb = __match_any_sync(FULL, vb);
            const unsigned long long vbs = ns ? ((unsigned long long)(uint32_t)b[k] << 32) | (uint32_t)s : ~0ull - lane;
            const unsigned mbs = __match_any_sync(FULL, vbs) & mb;
            const bool lead = (__ballot_sync(FULL, ns && s == b[k]) & mb) != 0u;
            const bool x = !single || mbs != mb || lead;
            if (u < nchunks) {
                cy.e[u * 32 + lane] = e[k];
                cy.b[u * 32 + lane] = b[k];
                cy.fl[u * 32 + lane] = il | (ns ? 32 : 0) | (x ? 64 : 0);
            }
            if (ns && (mb & lanemask_lt()) == 0u) claim_peel(a, b[k], peel_key(stamp, C, x), x, stamp);
            const unsigned nsm = __ballot_sync(FULL, ns);
            if (cy.my_chunk == u) {
                const unsigned mine = (it.deg >= 32 ? 0xffffffffu : ((1u << it.deg) - 1u)) << cy.my_start;
                touched = (nsm & mine) != 0u;
            }
        }
    }
    cy.pending = false;
    if ((int)lane < ng) {
        if (it.first && !it.single) claim_peel(a, it.C, peel_key(stamp, it.C, true), true, stamp);
        if (it.single && !touched && !it.defer) {
            // nothing to claim, nothing to mark: this iteration is carried out now
            a.unstable[it.C] = 0u;
            commits++;
            edges += it.deg;
            TRACE_WIN();
        } else {
            cy.pending = true;
        }
    }
    return true;
}

// Mark pass from what the claim pass kept (the block ranges are read again
// for the few transitions from blocks of several states).
__device__ void peel_mark_carried(const FrontierArgs& a, const Worklist& wl, uint32_t stamp, const PeelCarry& cy,
                                  int* n_small, int* n_mid, int4* small_list, int4* mid_list, long long& edges,
                                  long long& commits) {
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    if (__ballot_sync(FULL, cy.pending) == 0u) return;
    const bool lost_x = cy.pending && ld_volatile_u32(&a.lostl[cy.C]) == stamp;
    bool lost_p = false;
    for (int u0 = 0; u0 < cy.nchunks; u0 += PEEL_CHUNKS) {
        int fl[PEEL_CHUNKS];
        int32_t b[PEEL_CHUNKS];
        bool ns[PEEL_CHUNKS], lp[PEEL_CHUNKS];
#pragma unroll
        for (int k = 0; k < PEEL_CHUNKS; k++) {
            const int u = u0 + k;
            fl[k] = u < cy.nchunks ? cy.fl[u * 32 + lane] : 0;
            b[k] = u < cy.nchunks ? cy.b[u * 32 + lane] : 0;
        }
#pragma unroll
        for (int k = 0; k < PEEL_CHUNKS; k++) {
            const bool pend = __shfl_sync(FULL, cy.pending, fl[k] & 31);
            ns[k] = u0 + k < cy.nchunks && pend && (fl[k] & 32);
            lp[k] = ns[k] && !(fl[k] & 64) && ld_volatile_u64(&a.minx[b[k]]) == ld_volatile_u64(&a.claim[b[k]]);
        }
#pragma unroll
        for (int k = 0; k < PEEL_CHUNKS; k++) {
            const int u = u0 + k;
            const int il = fl[k] & 31;
            const bool x = fl[k] & 64;
            const unsigned lpm = __ballot_sync(FULL, lp[k]);
            const int st = __shfl_sync(FULL, cy.my_start, il);
            const int dg = __shfl_sync(FULL, cy.deg, il);
            const int32_t C = __shfl_sync(FULL, cy.C, il);
            const unsigned range = (dg >= 32 ? 0xffffffffu : ((1u << dg) - 1u)) << st;
            const bool lose = __shfl_sync(FULL, lost_x, il) || (lpm & range) != 0u;
            if (cy.my_chunk == u) {
                const unsigned mine = (cy.deg >= 32 ? 0xffffffffu : ((1u << cy.deg) - 1u)) << cy.my_start;
                lost_p = (lpm & mine) != 0u;
            }
            if (ns[k] && !lose) {
                const unsigned long long e = cy.e[u * 32 + lane];
                const int32_t s = (int32_t)(e >> 32);
                const int32_t bb = ld(&a.bbeg[b[k]]), be = ld(&a.bend[b[k]]);
                if (x) {
                    a.mark[(uint32_t)e] = stamp;
                    if (atomicExch(&a.smark[s], stamp) != stamp)
                        rank_marked(a, s, b[k], bb, be, C, n_small, n_mid, small_list, mid_list, 0);
                } else {
                    const unsigned long long pk = ((unsigned long long)(~stamp) << 32) | (uint32_t)C;
                    const unsigned long long old = atomicMin(&a.smark64[s], pk);
                    if ((old >> 32) != (pk >> 32))
                        rank_marked(a, s, b[k], bb, be, C, n_small, n_mid, small_list, mid_list, 1);
                }
            }
        }
    }
    if (cy.pending) {
        const bool lose = lost_x || lost_p || cy.defer;
        if (cy.first) {
            if (lose) {
                push(a, wl, cy.C);
            } else {
                a.unstable[cy.C] = 0u;
                commits++;
                TRACE_WIN();
            }
        }
        if (!lose) edges += cy.deg;
    }
}

// A peel round on the whole grid: claim pass, barrier, mark pass, barrier,
// split step, barrier. The items (members of the round's splitters: K0 of
// one state from the ring of bucket 0 - in a sweep round, `sweep`, the runs
// select_peel took from every ring, whose labels of blocks of several states
// are pushed back untouched and counted in n_defer - then the members of the
// K1 listed ones) are cut into one contiguous share per warp.
template <typename Sync>
__device__ __forceinline__ bool peel_round(const FrontierArgs& a, const Worklist& wl, CtaShared& sh, int* defer,
                                           int* ndefer, const int32_t* selC, const int32_t* selP, int K1, int K0,
                                           unsigned long long h0, uint32_t stamp, int64_t gw, int64_t nwarps,
                                           int* n_small, int* n_mid, int4* small_list, int4* mid_list, int cta,
                                           int ncta, long long& edges, long long& states, long long& commits,
                                           unsigned char* carry, PushBuf* pbuf, bool sweep, int* n_defer,
                                           int& touched, Sync sync) {
    const CtaShared* sw = sweep ? &sh : nullptr;
    const int64_t I = (int64_t)K0 + selP[K1];
    const int64_t per = (I + nwarps - 1) / nwarps;
    const int64_t i0 = gw * per, i1 = min(I, i0 + per);
    if (per <= 32) {
        // one group per warp: what the claim pass loaded is kept for the mark pass
        PeelCarry cy;
        peel_carry_at(cy, carry);
        const bool carried =
            i0 < i1 && peel_claim(a, wl, h0, sw, K0, selC, selP, K1, i0, i1, stamp, cy, n_defer, edges, commits);
        PHASE(2);
        if (!sync()) return false;
        PHASE(3);
        if (carried)
            peel_mark_carried(a, wl, stamp, cy, n_small, n_mid, small_list, mid_list, edges, commits);
        else if (i0 < i1)
            peel_items<1>(a, wl, h0, sw, K0, selC, selP, K1, i0, i1, stamp, n_small, n_mid, small_list, mid_list,
                          nullptr, edges, commits);
    } else {
        for (int64_t g = i0; g < i1; g += 32)
            peel_items<0>(a, wl, h0, sw, K0, selC, selP, K1, g, min(i1, g + 32), stamp, n_small, n_mid,
                          small_list, mid_list, n_defer, edges, commits);
        PHASE(2);
        if (!sync()) return false;
        PHASE(3);
        for (int64_t g = i0; g < i1; g += 32)
            peel_items<1>(a, wl, h0, sw, K0, selC, selP, K1, g, min(i1, g + 32), stamp, n_small, n_mid,
                          small_list, mid_list, nullptr, edges, commits);
    }
    PHASE(4);
    if (!sync()) return false;
    PHASE(5);
    const int ns = ld_volatile_i32(n_small), nm = ld_volatile_i32(n_mid);
    // final after the barrier: the same on every thread of the grid
    touched = ns + nm + (n_defer ? ld_volatile_i32(n_defer) : 0);
    PHASE_ADD(14, (unsigned long long)(ns + nm));
    TRACE_TOUCHED((unsigned long long)(ns + nm));
    // the split step's pushes (peeled members, their splitters, the blocks)
    // gather in shared memory and reach the rings once per CTA
    Worklist wlb = wl;
    wlb.buf = pbuf;
    split_step(a, wlb, sh, defer, ndefer, stamp, MULTI, ns, small_list, nm, mid_list, cta, ncta, states);
    if (pbuf) flush_pushes(wlb);
    PHASE(6);
    const bool ok = sync();
    PHASE(7);
    return ok;
}

// Hybrid schedule for one LTS. A round of one light splitter (at most 32
// members whose incoming transitions number at most light_edges), or of
// several splitters with at most local_budget states together, is done by
// CTA 0 alone with CTA barriers; every other round is done by the whole grid
// with grid barriers. After a grid round every CTA selects the next round's
// splitters itself: the selection reads only what the barrier made visible
// (worklist tails and entries, block ranges) and each CTA's copy of the
// worklist heads, so all CTAs choose the same round. When that round is a
// CTA-0 round the other CTAs park; CTA 0 then publishes the next grid round
// (cmd_C, cmd_K, cmd_stamp, the splitter list and its worklist heads, then
// cmd_seq with release order), which brings them back in step. A parked
// CTA's wait is bounded by timeout_ns without progress, where progress is a
// new command or a new heartbeat from CTA 0. The touched-block counters of
// grid rounds alternate by round parity; CTA 0 clears the next round's pair.
// Dynamic shared memory of the hybrid kernel: the selection (kmax + 32
// labels and kmax + 33 offsets), then, with peel rounds, PEEL_CARRY_BYTES per
// warp and the CTA's push buffer.
__host__ __device__ inline size_t peel_carry_offset(int kmax) {
    return (sizeof(int32_t) * (2 * ((size_t)kmax + 32) + 1) + 7) / 8 * 8;
}

template <int MAXT>  // most threads per CTA (sets the register budget)
__global__ void __launch_bounds__(MAXT, 1) k_frontier_hybrid(FrontierArgs a, HybridArgs h) {
    __shared__ CtaShared sh;
    __shared__ int s_defer[32];
    __shared__ int s_ndefer;
    __shared__ int s_ns, s_nm, s_heavy, s_cmd, s_K, s_K0, s_av0, s_avall;
    __shared__ bool s_peel;
    __shared__ unsigned long long s_h0;
    __shared__ unsigned s_stamp;
    __shared__ uint32_t s_lost[32];  // rounds on CTA 0 alone take at most 32 splitters
    extern __shared__ int32_t s_dyn[];
    const int kmax = max(h.kmax, 1);
    // kmax labels plus 32 for the singletons a CTA-0 round of a peel selection appends
    int32_t* s_selC = s_dyn;
    int32_t* s_selP = s_dyn + kmax + 32;
    // peel rounds: each warp's claim-pass carry, after the selection (8-byte aligned)
    unsigned char* s_carry = reinterpret_cast<unsigned char*>(s_dyn) + peel_carry_offset(kmax);
    PushBuf* s_pbuf = h.peel ? reinterpret_cast<PushBuf*>(s_carry + (size_t)(blockDim.x >> 5) * PEEL_CARRY_BYTES)
                             : nullptr;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int32_t n = a.n;
    const int64_t wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t gw = gtid >> 5, nwarps = gsz >> 5;
    const bool lead = blockIdx.x == 0;
    bisim_ctrl* c = a.ctrl;
    unsigned long long tgt = 0;
    long long edges = 0, states = 0, commits = 0;
    if (a.test_hook == 1 && lead) return;  // testing: never publish, never arrive
    const Worklist wl{c->bq_tail, a.queue, (size_t)n, 0, n};
    auto gsync = [&]() { return grid_sync(a.gb, tgt); };
    // one-state splitters a peel round takes from ring 0: cap0, or, after a
    // quiet round (fewer than one touched block per PEEL_QUIET splitters),
    // PEEL_SWEEP_GROWTH times the last cap (at most PEEL_SWEEP_MAX): most of
    // them then touch no block of several states and are carried out in the
    // claim pass, so a round sweeps many of them. Every CTA updates it from
    // the same counts, so all select alike.
    int peel_cap = h.cap0;
    int peel_touched = 0;
    auto next_peel_cap = [&](int K) {
        peel_cap = (long long)peel_touched * PEEL_QUIET < (long long)K
                       ? (int)min((long long)peel_cap * PEEL_SWEEP_GROWTH, (long long)PEEL_SWEEP_MAX)
                       : h.cap0;
    };
    auto csync = [&]() {
        __syncthreads();
        return true;
    };
    // a grid round: K > 1 splitters in selC / selP (peel rounds: K listed ones
    // and K0 of one state from ring 0 after h0), or the single splitter C
    auto grid_round = [&](int K, int K0, unsigned long long h0, int32_t C, uint32_t stamp, int par,
                          bool peel_now, bool sweep) -> bool {
        int* ns = &c->n_touched[par];
        int* nm = &c->n_mid[par];
        if (peel_now && K + K0 > 1)
            return peel_round(a, wl, sh, s_defer, &s_ndefer, s_selC, s_selP, K, K0, h0, stamp, gw, nwarps, ns, nm,
                              a.tlist, a.tlist + n, (int)blockIdx.x, (int)gridDim.x, edges, states, commits,
                              s_carry + wid * PEEL_CARRY_BYTES, s_pbuf, sweep, &c->n_defer[par], peel_touched,
                              gsync);
        if (K > 1)
            return multi_round(a, wl, sh, s_defer, &s_ndefer, s_selC, s_selP, K, h.g_lost, stamp, gw, nwarps, ns, nm,
                               a.tlist, a.tlist + n, (int)blockIdx.x, (int)gridDim.x, edges, states, commits, gsync);
        mark_step(a, C, stamp, gw, nwarps, ns, nm, a.tlist, a.tlist + n, edges);
        if (!gsync()) return false;
        split_step(a, wl, sh, s_defer, &s_ndefer, stamp, C, ld_volatile_i32(ns), a.tlist, ld_volatile_i32(nm),
                   a.tlist + n, (int)blockIdx.x, (int)gridDim.x, states);
        return gsync();
    };
    // zero, or where a one-CTA start handed the refinement over (a field that
    // CTA 0's commands never overwrite, so a late-starting CTA reads it too)
    if (threadIdx.x < BISIM_BUCKETS) sh.head[threadIdx.x] = ldcg(&c->start_heads[threadIdx.x]);
    if (threadIdx.x < 32) s_lost[threadIdx.x] = 0u;
    if (s_pbuf && threadIdx.x == 0) s_pbuf->n = 0;
    PHASE_RESET();
    __syncthreads();
    bool in_step = true;  // the other CTAs follow the selection (CTA 0: they are not parked)
    unsigned long long seen = 0;
    int64_t r = 0;
    for (;;) {
        if (!lead && !in_step) {
            // parked: wait for CTA 0's next grid round
            if (threadIdx.x == 0) {
                int ab = 0;
                unsigned long long t0 = 0, hb = ~0ull, v;
                unsigned spins = 0;
                while ((v = ld_acquire_u64_g(&c->cmd_seq)) == seen) {
                    __nanosleep(64);
                    if ((++spins & 31u) == 0) {
                        const unsigned long long now = globaltimer_ns();
                        const unsigned long long hbv = ldcg(&c->heartbeat);
                        if (hbv != hb) {
                            hb = hbv;
                            t0 = now;
                        } else if (now - t0 > a.gb.timeout_ns) {
                            atomicOr(&c->status, ST_TIMEOUT);
                            ab = 1;
                            break;
                        }
                        if (ldcg(&c->status) & ST_ABORT_MASK) {
                            ab = 1;
                            break;
                        }
                    }
                }
                seen = v;
                s_cmd = ab ? -1 : ldcg(&c->cmd_C);
                s_stamp = ldcg(&c->cmd_stamp);
                s_K = ldcg(&c->cmd_K);
                s_K0 = ldcg(&c->cmd_K0);
                s_h0 = ldcg(&c->cmd_h0);
                s_peel = ldcg(&c->cmd_peel) != 0;
            }
            __syncthreads();
            const int32_t C = s_cmd;
            const uint32_t stamp = s_stamp;
            const int K = s_K;
            const int K0c = s_K0;
            const unsigned long long h0c = s_h0;
            if (C == -1) break;
            if (threadIdx.x < BISIM_BUCKETS) sh.head[threadIdx.x] = ldcg(&c->cmd_heads[threadIdx.x]);
            if (C == MULTI)
                for (int i = threadIdx.x; i <= K; i += blockDim.x) {
                    if (i < K) s_selC[i] = ldcg(&h.g_selC[i]);
                    s_selP[i] = ldcg(&h.g_selP[i]);
                }
            __syncthreads();
            r = (int64_t)(stamp - a.stamp0);
            if (!grid_round(C == MULTI ? K : 1, C == MULTI ? K0c : 0, h0c, C, stamp, (int)(r & 1), s_peel, false))
                return;
            if (s_peel && C == MULTI) next_peel_cap(K + K0c);  // as CTA 0 does after this round
            in_step = true;
            continue;
        }
        PHASE(15);
        r++;
        const uint32_t stamp = a.stamp0 + (uint32_t)r;
        const int par = (int)(r & 1);
        int K;       // splitters of the round
        bool peel_now = false;  // a peel round (else a multi_round with these listed splitters)
        int K1 = 0;  // of those, listed in s_selC / s_selP (the rest: ring 0 after h0, peel rounds)
        int K0 = 0;
        unsigned long long h0 = 0;
        int32_t C;
        // Peel rounds pay when splitters of one state are many (each warp then
        // walks several small items); with fewer than PEEL_MIN_SINGLES labels
        // in size bucket 0 the round is selected and run as in multi_round
        // (one splitter per touched block). Every CTA reads the same tail
        // after the barrier, so all decide alike.
        bool peel_sel = false;
        // a sweep round needs every CTA to select it (none parked)
        const bool sweep_ok = peel_cap > h.cap0 && (!lead || in_step);
        bool sweep_now = false;
        if (kmax > 1 && h.peel) {
            if (threadIdx.x == 0) {
                s_av0 = (int)min(*(volatile const unsigned long long*)&wl.tail[0] - sh.head[0],
                                 (unsigned long long)PEEL_MIN_SINGLES);
                unsigned long long av = 0;
                if (sweep_ok)
                    for (int b = 0; b < BISIM_BUCKETS; b++)
                        av += *(volatile const unsigned long long*)&wl.tail[b] - sh.head[b];
                s_avall = (int)min(av, (unsigned long long)PEEL_MIN_SINGLES);
            }
            __syncthreads();
            sweep_now = sweep_ok && s_avall >= PEEL_MIN_SINGLES;
            peel_sel = sweep_now || s_av0 >= PEEL_MIN_SINGLES;
            __syncthreads();
        }
        if (peel_sel) {
            K1 = select_peel(a, wl, sh.head, sh, s_selC, s_selP, kmax, h.budget, peel_cap, sweep_now);
            K0 = sh.k0;
            h0 = sh.h0;
            peel_now = true;
            K = K0 + K1;
            C = K0 > 0 ? ld(&wl.queue[wl.base + h0 % (unsigned long long)wl.cap]) : K1 > 0 ? s_selC[0] : -1;
        } else if (kmax > 1) {
            K = select_many(a, wl, sh.head, sh, s_selC, s_selP, kmax, h.budget);
            K1 = K;
            C = K > 0 ? s_selC[0] : -1;
        } else {
            C = select_splitter(wl, sh.head, sh);
            K = C >= 0 ? 1 : 0;
            K1 = K;
        }
        PHASE(0);
        PHASE_ADD(K > 1 ? 9 : 10, K > 0 ? 1ull : 0ull);
        if (K > 0 && r > a.round_cap) {
            if (lead && threadIdx.x == 0) atomicOr(&c->status, ST_ROUNDS);
            K = 0;
        }
        if (K == 0) {
            if (lead && threadIdx.x == 0) {
                if (!in_step) {
                    c->cmd_C = -1;
                    __threadfence();
                    atomicAdd(&c->cmd_seq, 1ull);
                }
                c->rounds = r;
            }
            break;
        }
        // CTA 0 alone, or the grid?
        bool local;
        if (K > 1) {
            local = !sweep_now && K0 + s_selP[K1] <= h.local_budget;
            if (local && K0 > 0) {
                // the splitters of one state join the list (at most local_budget <= 32 of them)
                for (int i = threadIdx.x; i < K0; i += blockDim.x) {
                    s_selC[K1 + i] = ld(&wl.queue[wl.base + (h0 + (unsigned long long)i) % (unsigned long long)wl.cap]);
                    s_selP[K1 + i + 1] = s_selP[K1] + i + 1;
                }
                __syncthreads();
                K1 = K;
                K0 = 0;
            }
        } else {
            if (threadIdx.x < 32) {
                const int32_t b0 = ld(&a.bbeg[C]), e0 = ld(&a.bend[C]);
                int heavy = 1;
                if (e0 - b0 <= 32) {
                    int deg = 0;
                    if ((int)threadIdx.x < e0 - b0) {
                        const int32_t t = ld(&a.elems[b0 + threadIdx.x]);
                        deg = a.in_ptr[t + 1] - a.in_ptr[t];
                    }
                    heavy = __reduce_add_sync(0xffffffffu, deg) > h.light_edges;
                }
                if (threadIdx.x == 0) s_heavy = heavy;
            }
            __syncthreads();
            local = !s_heavy;
        }
        if (lead && threadIdx.x == 0) {
            c->n_touched[par ^ 1] = 0;  // the next grid round's counters
            c->n_mid[par ^ 1] = 0;
            c->n_defer[par ^ 1] = 0;
            if (K == 1) {
                a.unstable[C] = 0u;
                commits++;
                TRACE_WIN();
            }
        }
        TRACE_BEGIN(r, K, wl, sh.head);
        if (local) {
            if (!lead) {
                in_step = false;  // park until CTA 0 publishes a grid round
                continue;
            }
            if (threadIdx.x == 0) {
                s_ns = 0;
                s_nm = 0;
            }
            PHASE_ADD(11, 1ull);
            __syncthreads();
            if (K > 1) {
                multi_round(a, wl, sh, s_defer, &s_ndefer, s_selC, s_selP, K, s_lost, stamp, wid, nw, &s_ns, &s_nm,
                            a.tlist, a.tlist + n, 0, 1, edges, states, commits, csync);
            } else {
                mark_step(a, C, stamp, wid, nw, &s_ns, &s_nm, a.tlist, a.tlist + n, edges);
                __syncthreads();
                split_step(a, wl, sh, s_defer, &s_ndefer, stamp, C, s_ns, a.tlist, s_nm, a.tlist + n, 0, 1, states);
                __syncthreads();
            }
            if (threadIdx.x == 0) *(volatile unsigned long long*)&c->heartbeat = (unsigned long long)r;
            TRACE_END(r, 1u);
            in_step = false;
            continue;
        }
        if (lead && !in_step) {
            // wake the parked CTAs with this round and the heads after its selection
            if (K > 1)
                for (int i = threadIdx.x; i <= K1; i += blockDim.x) {
                    if (i < K1) h.g_selC[i] = s_selC[i];
                    h.g_selP[i] = s_selP[i];
                }
            if (threadIdx.x < BISIM_BUCKETS) c->cmd_heads[threadIdx.x] = sh.head[threadIdx.x];
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                c->cmd_C = K > 1 ? MULTI : C;
                c->cmd_K = K > 1 ? K1 : K;
                c->cmd_K0 = K > 1 ? K0 : 0;
                c->cmd_h0 = h0;
                c->cmd_peel = peel_now ? 1 : 0;
                c->cmd_stamp = stamp;
                __threadfence();
                atomicAdd(&c->cmd_seq, 1ull);
            }
        }
        in_step = true;
        PHASE(1);
        if (K > 1) {
            PHASE_ADD(12, (unsigned long long)K);
            PHASE_ADD(13, (unsigned long long)(K0 + s_selP[K1]));
        }
        if (!grid_round(K > 1 ? K1 : 1, K > 1 ? K0 : 0, h0, C, stamp, par, peel_now, sweep_now)) return;
        if (peel_now && K > 1) next_peel_cap(K);
        if (K == 1) PHASE(8);
        TRACE_END(r, 0u);
    }
    PHASE_FLUSH();
    if (edges) atomicAdd((unsigned long long*)&c->edges, (unsigned long long)edges);
    if (states) atomicAdd((unsigned long long*)&c->states, (unsigned long long)states);
    if (commits) atomicAdd((unsigned long long*)&c->commits, (unsigned long long)commits);
}

// Many LTSs in one launch, one CTA per LTS at a time: the same rounds, with
// __syncthreads in place of the grid barrier and the worklist cursors in
// shared memory. LTS i owns states, labels and member positions
// [state_off[i], state_off[i+1]) of the batch arrays; CTAs take LTSs from a
// counter in `order` (largest first). Nothing waits on another CTA, so the
// launch is an ordinary one and may overlap other work. With state_off,
// order and num_act null the batch is the plan's single LTS (states 0..n-1,
// round cap a.round_cap), refined by one CTA.
struct BatchArgs {
    int32_t k;
    const int64_t* __restrict__ state_off;  // [k+1]
    const int32_t* __restrict__ order;      // [k] LTS indices, largest first
    const int32_t* __restrict__ num_act;    // [k]
    int* next;                              // LTS counter
    long long* inst_rounds;                 // [k] out: splitter iterations + 1
    int32_t* block0;
    int kmax;                               // most splitters per round (1: one per round)
    int budget_per_warp;                    // states of a round's splitters per warp at most
    int multi_min_states;                   // smaller LTSs take one splitter per round
    // single LTS only: hand the refinement to the grid before a round whose
    // splitters hold more than handoff_states states (0 = never), or after
    // handoff_busy rounds in a row with at least kmax / 2 winners, or
    // handoff_busy rounds in a row of more than handoff_round_ns each
    // (handoff_busy 0 = neither)
    int handoff_states;
    int handoff_busy;
    unsigned long long handoff_round_ns;
};

__global__ void __launch_bounds__(1024) k_frontier_batch(FrontierArgs a, BatchArgs bt) {
    __shared__ CtaShared sh;
    __shared__ int s_defer[32];
    __shared__ int s_ndefer;
    __shared__ unsigned long long s_tail[BISIM_BUCKETS];
    __shared__ int s_ns, s_nm, s_inst;
    __shared__ int32_t s_selC[BISIM_KMAX_CTA];
    __shared__ int32_t s_selP[BISIM_KMAX_CTA + 1];
    __shared__ uint32_t s_lost[BISIM_KMAX_CTA];
    __shared__ unsigned long long s_commits;
    __shared__ int s_slow;  // rounds in a row longer than handoff_round_ns
    const int64_t gw = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int kmax = min(max(bt.kmax, 1), BISIM_KMAX_CTA);
    const int32_t budget = bt.budget_per_warp * (int32_t)nwarps;
    long long edges = 0, states = 0, steps = 0;
    for (;;) {
        if (threadIdx.x == 0) s_inst = atomicAdd(bt.next, 1);
        __syncthreads();
        const int inst = s_inst;
        __syncthreads();
        if (inst >= bt.k) break;
        const int32_t li = bt.order ? bt.order[inst] : 0;
        const int32_t s0 = bt.state_off ? (int32_t)bt.state_off[li] : 0;
        const int32_t ni = bt.state_off ? (int32_t)(bt.state_off[li + 1] - s0) : a.n;
        if (threadIdx.x < BISIM_BUCKETS) {
            // a single LTS finds its worklist filled by the whole grid (k_front_queue)
            s_tail[threadIdx.x] = bt.order ? 0ull : ldcg(&a.ctrl->bq_tail[threadIdx.x]);
            sh.head[threadIdx.x] = 0;
        }
        // the round stamps restart with every LTS: forget this CTA's last losses
        for (int i = threadIdx.x; i < BISIM_KMAX_CTA; i += blockDim.x) s_lost[i] = 0u;
        if (threadIdx.x == 0) {
            s_commits = 0;
            s_slow = 0;
        }
        __syncthreads();
        const Worklist wl{s_tail, a.queue, (size_t)a.n, s0, max(ni, 1)};
        // Algorithm 3, lines 1-3: every label of this LTS is unstable
        if (bt.order)
            for (int32_t l = s0 + threadIdx.x; l < s0 + ni; l += blockDim.x)
                if (bt.block0[l] == l) push(a, wl, l);
        __syncthreads();
        const int64_t cap = bt.num_act ? min((long long)a.round_cap, 3ll * ni + bt.num_act[li] + 2) : a.round_cap;
        const int kmax_i = ni >= bt.multi_min_states ? kmax : 1;
        int64_t r = 0;
        long long commits = 0;
        // A round of several splitters costs about as much as two rounds of
        // one (claim phase, one more barrier). After a round with at most two
        // winners (the others touch the same blocks, as in Fan_out_n, or only
        // two splitters were ready, as in a chain) the next `skip` rounds take
        // one splitter; each further such round doubles the stretch (to 64),
        // a round with three or more winners ends it.
        int skip = 0, backoff = 0, busy = 0;
        bool handoff = false;
        for (;;) {
            r++;
            const uint32_t stamp = a.stamp0 + (uint32_t)r;
            const unsigned long long head0 = threadIdx.x < BISIM_BUCKETS ? sh.head[threadIdx.x] : 0ull;
            const unsigned long long t0 = threadIdx.x == 0 && bt.handoff_busy > 0 ? globaltimer_ns() : 0ull;
            int K;
            int32_t C;
            const bool many = kmax_i > 1 && skip == 0;
            if (skip > 0) skip--;
            if (many) {
                K = select_many(a, wl, sh.head, sh, s_selC, s_selP, kmax_i, budget);
                C = K > 0 ? s_selC[0] : -1;
            } else {
                C = select_splitter(wl, sh.head, sh);
                K = C >= 0 ? 1 : 0;
            }
            if (K == 0) break;
            if (bt.handoff_states > 0 || bt.handoff_busy > 0) {
                int32_t rs = many ? s_selP[K] : 0;
                // a popped label of size bucket k had at least 2^k states when it was
                // pushed; it may have shrunk since, so only then is its size looked up
                if (!many && bt.handoff_states > 0 && (1ll << sh.bk) > bt.handoff_states) {
                    if (threadIdx.x == 0) s_ns = ld(&a.bend[C]) - ld(&a.bbeg[C]);
                    __syncthreads();
                    rs = s_ns;
                    __syncthreads();
                }
                if ((bt.handoff_states > 0 && rs > bt.handoff_states) ||
                    (bt.handoff_busy > 0 && (busy >= bt.handoff_busy || s_slow >= bt.handoff_busy))) {
                    // leave this round's labels in the worklist for the grid
                    if (threadIdx.x < BISIM_BUCKETS) {
                        a.ctrl->start_heads[threadIdx.x] = head0;
                        a.ctrl->bq_tail[threadIdx.x] = s_tail[threadIdx.x];
                    }
                    if (threadIdx.x == 0) a.ctrl->handoff = 1;
                    handoff = true;
                    break;
                }
            }
            if (r > cap) {
                if (threadIdx.x == 0) atomicOr(&a.ctrl->status, ST_ROUNDS);
                break;
            }
            if (threadIdx.x == 0) {
                if (K == 1) {
                    a.unstable[C] = 0u;
                    commits++;
                }
                s_ns = 0;
                s_nm = 0;
            }
            __syncthreads();
            if (K == 1) {
                mark_step(a, C, stamp, gw, nwarps, &s_ns, &s_nm, a.tlist + s0, a.tlist + a.n + s0, edges);
                __syncthreads();
                split_step(a, wl, sh, s_defer, &s_ndefer, stamp, C, s_ns, a.tlist + s0, s_nm, a.tlist + a.n + s0,
                           0, 1, states);
            } else {
                multi_round(a, wl, sh, s_defer, &s_ndefer, s_selC, s_selP, K, s_lost, stamp, gw, nwarps, &s_ns, &s_nm,
                            a.tlist + s0, a.tlist + a.n + s0, 0, 1, edges, states, commits, [] {
                                __syncthreads();
                                return true;
                            });
                // winners of this round: every warp counts the same losers
                int nlost = 0;
                for (int j0 = 0; j0 < K; j0 += 32) {
                    const int j = j0 + (int)(threadIdx.x & 31);
                    nlost += __popc(__ballot_sync(0xffffffffu, j < K && s_lost[j] == stamp));
                }
                if (K - nlost <= 2) {
                    backoff = min(max(2 * backoff, 2), 64);
                    skip = backoff;
                } else {
                    backoff = 0;
                }
                busy = 2 * (K - nlost) >= kmax_i ? busy + 1 : 0;
            }
            if (threadIdx.x == 0 && bt.handoff_busy > 0)
                s_slow = globaltimer_ns() - t0 > bt.handoff_round_ns ? s_slow + 1 : 0;
            __syncthreads();
        }
        if (commits) atomicAdd(&s_commits, (unsigned long long)commits);
        __syncthreads();
        if (threadIdx.x == 0) bt.inst_rounds[li] = (long long)s_commits + 1;
        steps += handoff ? r - 1 : r;  // the round that found the hand-off did not run
        __syncthreads();
    }
    if (edges) atomicAdd((unsigned long long*)&a.ctrl->edges, (unsigned long long)edges);
    if (states) atomicAdd((unsigned long long*)&a.ctrl->states, (unsigned long long)states);
    if (threadIdx.x == 0 && steps) atomicAdd((unsigned long long*)&a.ctrl->rounds, (unsigned long long)steps);
}

// ------------------------------------------------------------ small LTSs
//
// An LTS small enough to live in one CTA's shared memory is reduced by one
// kernel launch: validation happened in bisim_plan; this kernel computes the
// mark-slot layout from label sets (the reading of Algorithm 4 in plan.cu),
// the incoming-transition CSR, the initial leaders (Algorithm 2, lines 1-6,
// priority rule), the partition after the action-set preprocessing
// (Algorithm 5's result: one block per (initial block, label set), led by
// its smallest state), the refinable partition and worklist, the rounds of
// the frontier engine (the same round functions, on shared-memory arrays
// through generic pointers, with CTA barriers), and the canonical ids. Every
// block's label is its smallest state throughout (a split keeps the label
// with the part that holds it; the new label is the smallest state of the
// other part), so the canonical id of a block is the number of labels below
// it.
constexpr int SMALL_THREADS = 1024;         // most threads of the CTA
constexpr int SMALL_THREADS_DEFAULT = 512;
constexpr int SMALL_RINGS = 4;   // worklist rings: blocks of 1, 2-3, 4-7 and more states
constexpr int SMALL_KMAX = 32;   // splitters per round at most

struct SmallLayout {
    size_t tlist, in_edge, claim, mark, mask, off, in_ptr, block, elems, loc, bbeg, bend, mcnt, mscr, yscr, smark,
        kmark, unstable, bspl, queue, total;
};

__host__ __device__ inline size_t small_take(size_t& o, size_t bytes, size_t align) {
    o = (o + align - 1) / align * align;
    const size_t r = o;
    o += bytes;
    return r;
}

__host__ __device__ inline SmallLayout small_layout(int32_t n, int64_t m) {
    SmallLayout L;
    size_t o = 0;
    const size_t N = (size_t)n, M = (size_t)(m > 0 ? m : 1);
    L.tlist = small_take(o, 32 * N, 16);  // int4 [2n]; the grouping's hash table while planning
    L.in_edge = small_take(o, 8 * M, 8);
    L.claim = small_take(o, 8 * N, 8);
    L.mark = small_take(o, 4 * M, 4);  // mark_length <= m
    L.mask = small_take(o, 4 * N, 4);
    L.off = small_take(o, 4 * (N + 1), 4);
    L.in_ptr = small_take(o, 4 * (N + 1), 4);
    L.block = small_take(o, 4 * N, 4);
    L.elems = small_take(o, 4 * N, 4);
    L.loc = small_take(o, 4 * N, 4);
    L.bbeg = small_take(o, 4 * N, 4);
    L.bend = small_take(o, 4 * N, 4);
    L.mcnt = small_take(o, 4 * N, 4);
    L.mscr = small_take(o, 4 * N, 4);
    L.yscr = small_take(o, 4 * N, 4);
    L.smark = small_take(o, 4 * N, 4);
    L.kmark = small_take(o, 4 * N, 4);
    L.unstable = small_take(o, 4 * N, 4);
    L.bspl = small_take(o, 4 * N, 4);
    L.queue = small_take(o, 4 * SMALL_RINGS * N, 4);
    L.total = o;
    return L;
}

struct SmallArgs {
    int32_t n;
    int64_t m;
    const int32_t* src;
    const int32_t* act;   // null: every label 0
    const int32_t* dst;
    const int32_t* init;  // null: one initial block
    int32_t* out;         // canonical ids
    long long* res;       // [8]: iterations + 1, rounds, labels present, blocks after preprocessing,
                          //      blocks, mark_length, transitions walked, states compared
    bisim_ctrl* ctrl;     // status word
    int64_t round_cap;
    int alg2;
    int kmax;
    int32_t budget;
};

// exclusive prefix sum of arr[0 .. cnt) in place; returns the total
__device__ int32_t cta_scan_array(int32_t* arr, int32_t cnt, CtaShared& sh) {
    int32_t carry = 0;
    for (int32_t base = 0; base < cnt; base += blockDim.x) {
        const int32_t i = base + (int32_t)threadIdx.x;
        const int32_t v = i < cnt ? arr[i] : 0;
        int tot;
        const int ex = cta_scan(v, sh, tot);
        if (i < cnt) arr[i] = carry + ex;
        carry += tot;
    }
    return carry;
}

__device__ __forceinline__ uint32_t mix64(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return (uint32_t)x;
}

__global__ void __launch_bounds__(SMALL_THREADS, 1) k_small(SmallArgs g) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ CtaShared sh;
    __shared__ int s_defer[32];
    __shared__ int s_ndefer;
    __shared__ unsigned long long s_tail[BISIM_BUCKETS];
    __shared__ int s_ns, s_nm;
    __shared__ int32_t s_selC[SMALL_KMAX];
    __shared__ int32_t s_selP[SMALL_KMAX + 1];
    __shared__ uint32_t s_lost[SMALL_KMAX];
    __shared__ unsigned s_orm;  // labels present (bits)
    __shared__ int s_lead;
    const int32_t n = g.n;
    const int64_t m = g.m;
    const int tid = threadIdx.x, T = blockDim.x;
    const SmallLayout Lo = small_layout(n, m);
    int4* tlist = reinterpret_cast<int4*>(smem + Lo.tlist);
    unsigned long long* in_edge = reinterpret_cast<unsigned long long*>(smem + Lo.in_edge);
    unsigned long long* claim = reinterpret_cast<unsigned long long*>(smem + Lo.claim);
    uint32_t* mark = reinterpret_cast<uint32_t*>(smem + Lo.mark);
    uint32_t* mask = reinterpret_cast<uint32_t*>(smem + Lo.mask);
    int32_t* off = reinterpret_cast<int32_t*>(smem + Lo.off);
    int32_t* in_ptr = reinterpret_cast<int32_t*>(smem + Lo.in_ptr);
    int32_t* block = reinterpret_cast<int32_t*>(smem + Lo.block);
    int32_t* elems = reinterpret_cast<int32_t*>(smem + Lo.elems);
    int32_t* loc = reinterpret_cast<int32_t*>(smem + Lo.loc);
    int32_t* bbeg = reinterpret_cast<int32_t*>(smem + Lo.bbeg);
    int32_t* bend = reinterpret_cast<int32_t*>(smem + Lo.bend);
    int32_t* mcnt = reinterpret_cast<int32_t*>(smem + Lo.mcnt);
    int32_t* mscr = reinterpret_cast<int32_t*>(smem + Lo.mscr);
    int32_t* yscr = reinterpret_cast<int32_t*>(smem + Lo.yscr);
    uint32_t* smark = reinterpret_cast<uint32_t*>(smem + Lo.smark);
    uint32_t* kmark = reinterpret_cast<uint32_t*>(smem + Lo.kmark);
    uint32_t* unstable = reinterpret_cast<uint32_t*>(smem + Lo.unstable);
    int32_t* bspl = reinterpret_cast<int32_t*>(smem + Lo.bspl);
    int32_t* queue = reinterpret_cast<int32_t*>(smem + Lo.queue);

    // label sets and in-degrees
    for (int32_t i = tid; i < n; i += T) {
        mask[i] = 0u;
        in_ptr[i] = 0;
    }
    if (tid == 0) {
        in_ptr[n] = 0;
        off[n] = 0;
        s_orm = 0u;
        s_lead = 0;
    }
    if (tid < BISIM_BUCKETS) {
        s_tail[tid] = 0ull;
        sh.head[tid] = 0ull;
    }
    if (tid < SMALL_KMAX) s_lost[tid] = 0u;  // older than every round stamp
    __syncthreads();
    for (int64_t i = tid; i < m; i += T) {
        const int32_t s = g.src[i], a = g.act ? g.act[i] : 0, d = g.dst[i];
        atomicOr(&mask[s], 1u << a);
        atomicAdd(&in_ptr[d], 1);
    }
    __syncthreads();
    unsigned orm = 0u;
    for (int32_t i = tid; i < n; i += T) {
        off[i] = __popc(mask[i]);
        orm |= mask[i];
    }
    orm = __reduce_or_sync(0xffffffffu, orm);
    if ((tid & 31) == 0 && orm) atomicOr(&s_orm, orm);
    __syncthreads();
    // off = exclusive sum of nr_marks (off[n] = L), in_ptr likewise over in-degrees
    const int32_t L = cta_scan_array(off, n + 1, sh);
    cta_scan_array(in_ptr, n + 1, sh);
    // incoming-transition CSR, entries (source << 32) | slot; mcnt counts per target
    for (int32_t i = tid; i < n; i += T) mcnt[i] = 0;
    for (int32_t i = tid; i < L; i += T) mark[i] = 0u;
    __syncthreads();
    for (int64_t i = tid; i < m; i += T) {
        const int32_t s = g.src[i], a = g.act ? g.act[i] : 0, d = g.dst[i];
        const uint32_t slot = (uint32_t)off[s] + __popc(mask[s] & ((1u << a) - 1u));
        in_edge[in_ptr[d] + atomicAdd(&mcnt[d], 1)] = ((unsigned long long)(uint32_t)s << 32) | slot;
    }
    // initial leaders: the smallest member of every initial block
    for (int32_t i = tid; i < n; i += T) yscr[i] = NONE;
    __syncthreads();
    if (g.init)
        for (int32_t i = tid; i < n; i += T) atomicMin(&yscr[g.init[i]], i);
    __syncthreads();
    for (int32_t i = tid; i < n; i += T) block[i] = g.init ? yscr[g.init[i]] : 0;
    // action-set preprocessing: one block per (initial block, label set), led
    // by its smallest state, found through a hash table of 2n entries in the
    // (not yet used) touched-list area
    const int32_t cap = 2 * n;
    unsigned long long* hkey = reinterpret_cast<unsigned long long*>(tlist);
    int32_t* hval = reinterpret_cast<int32_t*>(hkey + cap);
    for (int32_t h = tid; h < cap; h += T) {
        hkey[h] = ~0ull;
        hval[h] = NONE;
    }
    __syncthreads();
    for (int32_t i = tid; i < n; i += T) {
        const unsigned long long key = ((unsigned long long)(uint32_t)block[i] << 32) | mask[i];
        int32_t h = (int32_t)(mix64(key) % (uint32_t)cap);
        for (;;) {
            const unsigned long long old = atomicCAS(&hkey[h], ~0ull, key);
            if (old == ~0ull || old == key) {
                atomicMin(&hval[h], i);
                break;
            }
            h = h + 1 == cap ? 0 : h + 1;
        }
    }
    __syncthreads();
    for (int32_t i = tid; i < n; i += T) {
        const unsigned long long key = ((unsigned long long)(uint32_t)block[i] << 32) | mask[i];
        int32_t h = (int32_t)(mix64(key) % (uint32_t)cap);
        while (hkey[h] != key) h = h + 1 == cap ? 0 : h + 1;
        yscr[i] = hval[h];
    }
    __syncthreads();
    // refinable partition: members grouped by label (counting sort), ranges, worklist
    for (int32_t i = tid; i < n; i += T) {
        block[i] = yscr[i];
        mcnt[i] = 0;
    }
    __syncthreads();
    for (int32_t i = tid; i < n; i += T) atomicAdd(&mcnt[block[i]], 1);
    __syncthreads();
    for (int32_t i = tid; i < n; i += T) bbeg[i] = mcnt[i];
    __syncthreads();
    cta_scan_array(bbeg, n, sh);
    for (int32_t i = tid; i < n; i += T) {
        bend[i] = bbeg[i] + mcnt[i];
        yscr[i] = 0;
    }
    __syncthreads();
    for (int32_t i = tid; i < n; i += T) {
        const int32_t pos = bbeg[block[i]] + atomicAdd(&yscr[block[i]], 1);
        elems[pos] = i;
        loc[i] = pos;
    }
    for (int32_t i = tid; i < n; i += T) {
        smark[i] = 0u;
        kmark[i] = 0u;
        bspl[i] = 0;
        claim[i] = ~0ull;
        unstable[i] = block[i] == i ? 1u : 0u;
    }
    __syncthreads();
    for (int32_t i = tid; i < n; i += T) mcnt[i] = 0;
    FrontierArgs a;
    a.n = n;
    a.off = off;
    a.in_ptr = in_ptr;
    a.in_edge = in_edge;
    a.block = block;
    a.mark = mark;
    a.unstable = unstable;
    a.elems = elems;
    a.loc = loc;
    a.bbeg = bbeg;
    a.bend = bend;
    a.mcnt = mcnt;
    a.mscr = mscr;
    a.yscr = yscr;
    a.smark = smark;
    a.kmark = kmark;
    a.tlist = tlist;
    a.queue = queue;
    a.claim = claim;
    a.minx = nullptr;
    a.smark64 = nullptr;
    a.lostl = nullptr;
    a.bspl = bspl;
    a.ctrl = g.ctrl;
    a.gb.counter = nullptr;
    a.gb.status = &g.ctrl->status;
    a.gb.timeout_ns = 0;
    a.stamp0 = 0;
    a.round_cap = g.round_cap;
    a.alg2 = g.alg2;
    a.test_hook = 0;
    Worklist wl{s_tail, queue, (size_t)n, 0, n};
    wl.nbk = SMALL_RINGS;
    __syncthreads();
    // Algorithm 3, lines 1-3: every label is unstable
    int leaders = 0;
    for (int32_t i = tid; i < n; i += T)
        if (block[i] == i) {
            push_sized(wl, i, bend[i] - bbeg[i]);
            leaders++;
        }
    leaders = __reduce_add_sync(0xffffffffu, leaders);
    if ((tid & 31) == 0 && leaders) atomicAdd(&s_lead, leaders);
    __syncthreads();
    // rounds, as the one-CTA rounds of the batch kernel: after a round of
    // several splitters with at most two winners, single splitters for a
    // stretch of rounds that doubles (2 ... 64) while such rounds repeat
    const int64_t gw = tid >> 5, nwarps = T >> 5;
    long long edges = 0, states = 0, commits = 0;
    int64_t r = 0;
    int skip = 0, backoff = 0;
    for (;;) {
        r++;
        const uint32_t stamp = (uint32_t)r;
        int K;
        int32_t C;
        const bool many = g.kmax > 1 && skip == 0;
        if (skip > 0) skip--;
        if (many) {
            K = select_many(a, wl, sh.head, sh, s_selC, s_selP, g.kmax, g.budget);
            C = K > 0 ? s_selC[0] : -1;
        } else {
            C = select_splitter(wl, sh.head, sh);
            K = C >= 0 ? 1 : 0;
        }
        if (K == 0) break;
        if (r > g.round_cap) {
            if (tid == 0) atomicOr(&g.ctrl->status, ST_ROUNDS);
            break;
        }
        if (tid == 0) {
            if (K == 1) {
                unstable[C] = 0u;
                commits++;
            }
            s_ns = 0;
            s_nm = 0;
        }
        __syncthreads();
        if (K == 1) {
            mark_step(a, C, stamp, gw, nwarps, &s_ns, &s_nm, tlist, tlist + n, edges);
            __syncthreads();
            split_step(a, wl, sh, s_defer, &s_ndefer, stamp, C, s_ns, tlist, s_nm, tlist + n, 0, 1, states);
        } else {
            multi_round(a, wl, sh, s_defer, &s_ndefer, s_selC, s_selP, K, s_lost, stamp, gw, nwarps, &s_ns, &s_nm,
                        tlist, tlist + n, 0, 1, edges, states, commits, [] {
                            __syncthreads();
                            return true;
                        });
            int nlost = 0;  // every warp counts the same losers
            for (int j0 = 0; j0 < K; j0 += 32) {
                const int j = j0 + (tid & 31);
                nlost += __popc(__ballot_sync(0xffffffffu, j < K && s_lost[j] == stamp));
            }
            if (K - nlost <= 2) {
                backoff = min(max(2 * backoff, 2), 64);
                skip = backoff;
            } else {
                backoff = 0;
            }
        }
        __syncthreads();
    }
    // canonical ids: a block's label is its smallest state, so its id is the
    // number of labels below it
    for (int32_t i = tid; i < n; i += T) mcnt[i] = block[i] == i ? 1 : 0;
    __syncthreads();
    const int32_t nb = cta_scan_array(mcnt, n, sh);
    for (int32_t i = tid; i < n; i += T) g.out[i] = mcnt[block[i]];
    // counts of each thread (commits by the threads that carried splitters out)
    if (edges) atomicAdd((unsigned long long*)&g.res[6], (unsigned long long)edges);
    if (states) atomicAdd((unsigned long long*)&g.res[7], (unsigned long long)states);
    if (commits) atomicAdd((unsigned long long*)&g.res[0], (unsigned long long)commits);
    if (tid == 0) {
        atomicAdd((unsigned long long*)&g.res[0], 1ull);  // the final empty iteration
        g.res[1] = r;
        g.res[2] = __popc(s_orm);
        g.res[3] = s_lead;
        g.res[4] = nb;
        g.res[5] = L;
    }
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

// ranges of each label in the label-sorted member array, and loc
__global__ void k_front_ranges(const uint32_t* __restrict__ skeys, const int32_t* __restrict__ elems,
                               int32_t n, int32_t* bbeg, int32_t* bend, int32_t* loc) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz) {
        const uint32_t b = skeys[i];
        if (i == 0 || skeys[i - 1] != b) bbeg[b] = (int32_t)i;
        if (i == n - 1 || skeys[i + 1] != b) bend[b] = (int32_t)i + 1;
        loc[elems[i]] = (int32_t)i;
    }
}

// initial worklist: every label, in the bucket of its block size (one
// atomicAdd per bucket and warp; the lanes of a bucket take consecutive slots)
__global__ void k_front_queue(const uint32_t* __restrict__ flags, const int32_t* __restrict__ bbeg,
                              const int32_t* __restrict__ bend, int32_t n, bisim_ctrl* ctrl,
                              int32_t* queue) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int lane = (int)(threadIdx.x & 31);
    // trip count rounded up to whole warps so that every lane reaches the match
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i - lane < n; i += gsz) {
        const bool has = i < n && flags[i];
        const int bk = has ? size_bucket(bend[i] - bbeg[i]) : 32 + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, bk);
        const int first = __ffs(peers) - 1;
        unsigned long long base = 0;
        if (has && lane == first) base = atomicAdd(&ctrl->bq_tail[bk], (unsigned long long)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, first);
        if (has) queue[(size_t)bk * n + base + __popc(peers & lanemask_lt())] = (int32_t)i;
    }
}

int ensure_frontier(bisim_plan_s* p) {
    if (p->frontier_ready) return BISIM_OK;
    const size_t n = (size_t)p->n;
    cudaStream_t st = p->st;
    BISIM_TRY(p->elems.alloc(4 * n, st));
    BISIM_TRY(p->loc.alloc(4 * n, st));
    BISIM_TRY(p->bbeg.alloc(4 * n, st));
    BISIM_TRY(p->bend.alloc(4 * n, st));
    BISIM_TRY(p->mcnt.alloc(4 * n, st));
    BISIM_TRY(p->mscr.alloc(4 * n, st));
    BISIM_TRY(p->yscr.alloc(4 * n, st));
    BISIM_TRY(p->smark.alloc(4 * n, st));
    BISIM_TRY(p->kmark.alloc(4 * n, st));
    BISIM_TRY(p->tlist.alloc(32 * n, st));
    BISIM_TRY(p->queue.alloc(4 * n * BISIM_BUCKETS, st));
    BISIM_TRY(p->claim.alloc(8 * n, st));
    BISIM_TRY(p->bspl.alloc(4 * n, st));
    BISIM_TRY(p->msel.alloc(4 * (3 * (size_t)BISIM_KMAX_GRID + 1), st));
    BISIM_TRY(p->minx.alloc(8 * n, st));
    BISIM_TRY(p->smark64.alloc(8 * n, st));
    BISIM_TRY(p->lostl.alloc(4 * n, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->claim.p, 0xff, 8 * n, st));  // older than every round
    BISIM_CUDA_TRY(cudaMemsetAsync(p->minx.p, 0xff, 8 * n, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->smark64.p, 0xff, 8 * n, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->lostl.p, 0, 4 * n, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->smark.p, 0, 4 * n, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->kmark.p, 0, 4 * n, st));
    p->frontier_ready = true;
    return BISIM_OK;
}

// Grouped member array, ranges, loc, labels and unstable flags from block0;
// with fill_queue, also the global worklist (grid engine).
int frontier_setup(bisim_plan_s* p, bool fill_queue) {
    const int32_t n = p->n;
    cudaStream_t st = p->st;
    BISIM_TRY(ensure_frontier(p));
    bisim_ctrl* c = p->ctrl.as<bisim_ctrl>();
    BISIM_CUDA_TRY(cudaMemsetAsync(c, 0, sizeof(bisim_ctrl), st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->mcnt.p, 0, 4 * (size_t)n, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->msel.p, 0, p->msel.bytes, st));
    DevMem keys, vals, keys2, flags;
    BISIM_TRY(keys.alloc(4 * (size_t)n, st));
    BISIM_TRY(vals.alloc(4 * (size_t)n, st));
    BISIM_TRY(keys2.alloc(4 * (size_t)n, st));
    BISIM_TRY(flags.alloc(4 * (size_t)n, st));
    const unsigned gn = grid_for(n, 256);
    k_front_init<<<gn, 256, 0, st>>>(p->block0.as<int32_t>(), n, p->block.as<int32_t>(),
                                     p->unstable.as<uint32_t>(), keys.as<uint32_t>(), vals.as<uint32_t>(),
                                     flags.as<uint32_t>());
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    // members grouped by label: sort (label, state)
    uint32_t* el = p->elems.as<uint32_t>();
    bool alt = false;
    BISIM_TRY(radix_sort_pairs<uint32_t, uint32_t>(keys.as<uint32_t>(), vals.as<uint32_t>(), keys2.as<uint32_t>(),
                                                   el, n, ceil_log2_u64((uint64_t)n), st, &alt));
    uint32_t* skeys = alt ? keys2.as<uint32_t>() : keys.as<uint32_t>();
    if (!alt) BISIM_CUDA_TRY(cudaMemcpyAsync(el, vals.p, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    k_front_ranges<<<gn, 256, 0, st>>>(skeys, p->elems.as<int32_t>(), n, p->bbeg.as<int32_t>(),
                                       p->bend.as<int32_t>(), p->loc.as<int32_t>());
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    if (fill_queue) {
        k_front_queue<<<gn, 256, 0, st>>>(flags.as<uint32_t>(), p->bbeg.as<int32_t>(), p->bend.as<int32_t>(), n,
                                          c, p->queue.as<int32_t>());
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
    }
    return BISIM_OK;
}

FrontierArgs make_args(bisim_plan_s* p, uint32_t base, int64_t cap) {
    FrontierArgs a;
    bisim_ctrl* c = p->ctrl.as<bisim_ctrl>();
    a.n = p->n;
    a.off = p->off.as<int32_t>();
    a.in_ptr = p->in_ptr.as<int32_t>();
    a.in_edge = p->in_edge.as<unsigned long long>();
    a.block = p->block.as<int32_t>();
    a.mark = p->mark.as<uint32_t>();
    a.unstable = p->unstable.as<uint32_t>();
    a.elems = p->elems.as<int32_t>();
    a.loc = p->loc.as<int32_t>();
    a.bbeg = p->bbeg.as<int32_t>();
    a.bend = p->bend.as<int32_t>();
    a.mcnt = p->mcnt.as<int32_t>();
    a.mscr = p->mscr.as<int32_t>();
    a.yscr = p->yscr.as<int32_t>();
    a.smark = p->smark.as<uint32_t>();
    a.kmark = p->kmark.as<uint32_t>();
    a.tlist = p->tlist.as<int4>();
    a.queue = p->queue.as<int32_t>();
    a.claim = p->claim.as<unsigned long long>();
    a.minx = p->minx.as<unsigned long long>();
    a.smark64 = p->smark64.as<unsigned long long>();
    a.lostl = p->lostl.as<uint32_t>();
    a.bspl = p->bspl.as<int32_t>();
    a.ctrl = c;
    a.gb.counter = &c->barrier;
    a.gb.status = &c->status;
    a.gb.timeout_ns = (unsigned long long)(p->opts.timeout_ms > 0 ? p->opts.timeout_ms : 2000) * 1000000ull;
    a.stamp0 = base;
    a.round_cap = cap;
    a.alg2 = (p->opts.rcpp_alg2 && p->A == 1) ? 1 : 0;
    a.test_hook = p->opts.test_hook;
    return a;
}

int report(bisim_plan_s* p) {
    int code = status_to_code(p->ctrl_h->status);
    if (code)
        set_last_error(p->ctrl_h->status & ST_TIMEOUT ? "grid barrier wait timed out"
                       : p->ctrl_h->status & ST_ROUNDS ? "round cap exceeded"
                                                       : "internal consistency check failed");
    return code;
}

// One LTS on one CTA: the batch kernel with the plan's LTS as its only
// instance, every round between CTA barriers. With a hand-off rule it stops
// before a round that the whole grid would do faster and leaves the worklist
// (tails, and the heads before that round) in ctrl for the hybrid kernel.
int refine_frontier_local(bisim_plan_s* p, int64_t cap, uint32_t base, int handoff_states, int handoff_busy,
                          double* ms) {
    cudaStream_t st = p->st;
    FrontierArgs a = make_args(p, base, cap);
    bisim_ctrl* c = p->ctrl.as<bisim_ctrl>();
    BatchArgs bt;
    bt.k = 1;
    bt.state_off = nullptr;
    bt.order = nullptr;
    bt.num_act = nullptr;
    bt.next = &c->next_inst;
    bt.inst_rounds = &c->local_rounds;
    bt.block0 = p->block0.as<int32_t>();
    bt.kmax = p->opts.splitters > 0 ? std::min(p->opts.splitters, BISIM_KMAX_CTA) : 32;
    bt.budget_per_warp = p->opts.split_budget > 0 ? std::min(p->opts.split_budget, 1 << 20) : 4;
    bt.multi_min_states = 0;
    bt.handoff_states = handoff_states;
    bt.handoff_busy = handoff_busy;
    bt.handoff_round_ns = BISIM_HANDOFF_ROUND_NS;
    const int threads = p->opts.threads > 0 ? p->opts.threads : 1024;
    BISIM_CUDA_TRY(cudaEventRecord(p->evk0, st));
    k_frontier_batch<<<1, threads, 0, st>>>(a, bt);
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    BISIM_CUDA_TRY(cudaEventRecord(p->evk1, st));
    BISIM_TRY(read_ctrl(p));
    return persistent_ms(p, ms);
}

}  // namespace

namespace bisim {

int refine_frontier(bisim_plan_s* p, bisim_stats* stats) {
    const int32_t n = p->n;
    const int64_t cap = p->opts.round_cap > 0 ? p->opts.round_cap : 3ll * n + p->A + 2;
    uint32_t base;
    BISIM_TRY(reserve_stamps(p, cap + 1, &base));
    // A sparse LTS (m <= 4n) starts on one CTA, whose rounds cost a few
    // CTA barriers instead of grid barriers, and moves to the grid before a
    // round of a large splitter or once many splitters win every round.
    const int32_t lo = p->opts.local_states;
    const bool start_local = p->opts.light_edges >= 0 && (lo > 0 || (lo == 0 && p->m <= 4ll * n));
    int64_t done = 0;            // rounds carried out on one CTA
    long long done_commits = 0;  // splitter iterations among them
    double local_ms = 0;
    BISIM_TRY(frontier_setup(p, true));
    if (start_local) {
        BISIM_TRY(refine_frontier_local(p, cap, base, lo > 0 ? lo : BISIM_HANDOFF_STATES,
                                        lo > 0 ? 0 : BISIM_HANDOFF_BUSY, &local_ms));
        BISIM_TRY(report(p));
        if (!p->ctrl_h->handoff) {
            p->stamp = base + (uint32_t)std::min<long long>(p->ctrl_h->rounds + 1, cap + 1);
            if (stats) {
                stats->t_main_ms = local_ms;
                stats->rounds = p->ctrl_h->local_rounds;
                stats->steps = p->ctrl_h->rounds;
                stats->local_steps = p->ctrl_h->rounds;
                stats->edges_visited = p->ctrl_h->edges;
                stats->states_visited = p->ctrl_h->states;
                stats->engine = BISIM_ENGINE_FRONTIER;
                stats->grid_ctas = 1;
            }
            return BISIM_OK;
        }
        done = p->ctrl_h->rounds;
        done_commits = p->ctrl_h->local_rounds - 1;
    }
    FrontierArgs a = make_args(p, base + (uint32_t)done, cap - done);
    const int threads = p->opts.threads > 0 ? p->opts.threads : 512;
    const int light = p->opts.light_edges == 0 ? 256 : p->opts.light_edges;
    int grid = 0;
    if (light < 0) {  // every round on the whole grid, one splitter per round
        void* args[] = {&a};
        BISIM_TRY(launch_persistent((const void*)k_frontier_main, args, threads, p, &grid));
    } else {
        HybridArgs h;
        h.light_edges = light;
        h.kmax = p->opts.splitters > 0 ? std::min(p->opts.splitters, BISIM_KMAX_GRID) : BISIM_KMAX_GRID;
        h.kmax = std::min(h.kmax, (p->opts.peel >= 0 ? PEEL_SEL_E : SEL_E) * threads);
        h.local_budget = std::min(threads / 32, 32);
        h.g_selC = p->msel.as<int32_t>();
        h.g_selP = h.g_selC + BISIM_KMAX_GRID;
        h.g_lost = reinterpret_cast<uint32_t*>(h.g_selP + BISIM_KMAX_GRID + 1);
        h.budget = 0;  // set from the grid size below
        void* args[] = {&a, &h};
        const void* fn = threads <= 512 ? (const void*)k_frontier_hybrid<512> : (const void*)k_frontier_hybrid<1024>;
        int occ = 0;
        BISIM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0));
        // (an estimate for the budget only; launch_persistent sizes the grid)
        int per_sm = p->opts.ctas_per_sm > 0 ? std::min(p->opts.ctas_per_sm, std::max(occ, 1)) : 1;
        int g = p->sm_count * per_sm;
        if (p->opts.max_ctas > 0) g = std::min(g, p->opts.max_ctas);
        const int per_warp = p->opts.split_budget > 0 ? p->opts.split_budget : 1;
        h.budget = (int)std::min<int64_t>((int64_t)per_warp * g * (threads / 32), 1 << 30);
        h.peel = p->opts.peel >= 0 && h.kmax > 1 ? 1 : 0;
        const int peel_items = p->opts.peel_items > 0 ? std::min(p->opts.peel_items, 1 << 12) : 96;
        int64_t cap0 = (int64_t)peel_items * g * (threads / 32);
        if (p->opts.splitters > 0) cap0 = std::min<int64_t>(cap0, p->opts.splitters);
        h.cap0 = (int)std::min<int64_t>(cap0, 1 << 30);
        const size_t dyn = h.peel ? peel_carry_offset(h.kmax) + (size_t)(threads / 32) * PEEL_CARRY_BYTES +
                                        sizeof(PushBuf)
                                  : sizeof(int32_t) * (2 * ((size_t)h.kmax + 32) + 1);
        BISIM_TRY(launch_persistent(fn, args, threads, p, &grid, 1, dyn));
    }
    BISIM_TRY(read_ctrl(p));
    p->stamp = base + (uint32_t)std::min<long long>(done + p->ctrl_h->rounds + 1, cap + 1);
    if (stats) {
        BISIM_TRY(persistent_ms(p, &stats->t_main_ms));
        stats->t_main_ms += local_ms;
        stats->rounds = done_commits + p->ctrl_h->commits + 1;
        stats->steps = done + p->ctrl_h->rounds;
        stats->local_steps = done;
        stats->edges_visited = p->ctrl_h->edges;
        stats->states_visited = p->ctrl_h->states;
        stats->engine = BISIM_ENGINE_FRONTIER;
        stats->grid_ctas = grid;
    }
    return report(p);
}

int refine_frontier_batch(bisim_plan_s* p, bisim_stats* stats, std::vector<long long>& rounds) {
    const int32_t k = p->batch_k;
    cudaStream_t st = p->st;
    int64_t cap = 0;
    for (int32_t i = 0; i < k; i++)
        cap = std::max<int64_t>(cap, 3ll * (p->state_off_h[i + 1] - p->state_off_h[i]) + p->batch_act_h[i] + 2);
    uint32_t base;
    BISIM_TRY(reserve_stamps(p, cap + 1, &base));
    BISIM_TRY(frontier_setup(p, false));
    FrontierArgs a = make_args(p, base, cap);
    BatchArgs bt;
    bt.k = k;
    bt.state_off = p->state_off.as<int64_t>();
    bt.order = p->batch_order.as<int32_t>();
    bt.num_act = p->batch_act.as<int32_t>();
    bt.next = &p->ctrl.as<bisim_ctrl>()->next_inst;
    bt.inst_rounds = p->inst_rounds.as<long long>();
    bt.block0 = p->block0.as<int32_t>();
    bt.kmax = p->opts.splitters > 0 ? std::min(p->opts.splitters, BISIM_KMAX_CTA) : 1;
    bt.budget_per_warp = p->opts.split_budget > 0 ? std::min(p->opts.split_budget, 1 << 20) : 8;
    bt.multi_min_states = std::max(p->opts.multi_min_states, 0);
    bt.handoff_states = 0;
    bt.handoff_busy = 0;
    bt.handoff_round_ns = 0;
    const int threads = p->opts.threads > 0 ? p->opts.threads : 256;
    // optional split schedule: the LTSs with at least wide_min_states states
    // (a prefix of the largest-first order) run in a second launch of wide
    // CTAs on an auxiliary stream, concurrently with the narrow launch
    int32_t kw = 0;
    if (p->opts.wide_threads > 0 && p->opts.wide_min_states > 0)
        while (kw < k) {
            const int32_t li = p->batch_order_h[(size_t)kw];
            if (p->state_off_h[li + 1] - p->state_off_h[li] < p->opts.wide_min_states) break;
            kw++;
        }
    auto grid_of = [&](int thr, int cnt, int* g) -> int {
        int occ = 0;
        BISIM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_frontier_batch, thr, 0));
        int per_sm = p->opts.ctas_per_sm > 0 ? std::min(p->opts.ctas_per_sm, occ) : occ;
        int gg = std::max(1, std::min(cnt, p->sm_count * std::max(per_sm, 1)));
        if (p->opts.max_ctas > 0) gg = std::min(gg, p->opts.max_ctas);
        *g = gg;
        return BISIM_OK;
    };
    int grid = 0, gridw = 0;
    BISIM_CUDA_TRY(cudaEventRecord(p->evk0, st));
    if (kw > 0) {
        if (!p->aux_stream) BISIM_CUDA_TRY(cudaStreamCreateWithFlags(&p->aux_stream, cudaStreamNonBlocking));
        if (!p->aux_event) BISIM_CUDA_TRY(cudaEventCreateWithFlags(&p->aux_event, cudaEventDisableTiming));
        BISIM_CUDA_TRY(cudaStreamWaitEvent(p->aux_stream, p->evk0, 0));
        BISIM_TRY(grid_of(p->opts.wide_threads, kw, &gridw));
        BatchArgs bw = bt;
        bw.k = kw;
        bw.next = &p->ctrl.as<bisim_ctrl>()->next_inst_wide;
        k_frontier_batch<<<gridw, p->opts.wide_threads, 0, p->aux_stream>>>(a, bw);
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        BISIM_CUDA_TRY(cudaEventRecord(p->aux_event, p->aux_stream));
    }
    if (kw < k) {
        BISIM_TRY(grid_of(threads, k - kw, &grid));
        BatchArgs bn = bt;
        bn.k = k - kw;
        bn.order = bt.order + kw;
        k_frontier_batch<<<grid, threads, 0, st>>>(a, bn);
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
    }
    if (kw > 0) BISIM_CUDA_TRY(cudaStreamWaitEvent(st, p->aux_event, 0));
    BISIM_CUDA_TRY(cudaEventRecord(p->evk1, st));
    grid += gridw;
    rounds.assign((size_t)k, 0);
    if (k) BISIM_CUDA_TRY(cudaMemcpyAsync(rounds.data(), p->inst_rounds.p, 8 * (size_t)k, cudaMemcpyDeviceToHost, st));
    BISIM_TRY(read_ctrl(p));
    long long rmax = 0, rsum = 0;
    for (long long r : rounds) {
        rmax = std::max(rmax, r);
        rsum += r;
    }
    p->stamp = base + (uint32_t)std::min<long long>(rmax + 1, cap + 1);
    if (stats) {
        BISIM_TRY(persistent_ms(p, &stats->t_main_ms));
        stats->rounds = rsum;
        stats->steps = p->ctrl_h->rounds;
        stats->edges_visited = p->ctrl_h->edges;
        stats->states_visited = p->ctrl_h->states;
        stats->engine = BISIM_ENGINE_FRONTIER;
        stats->grid_ctas = grid;
    }
    return report(p);
}

// Dynamic shared memory k_small may take on `dev`: the opt-in maximum per
// CTA less the kernel's static shared arrays. The kernel's limit is raised
// to that once per device; 0 if either query fails.
static size_t small_smem_room(int dev) {
    constexpr int MAXDEV = 64;
    static std::mutex mu;
    static size_t room[MAXDEV];
    static bool known[MAXDEV];
    if (dev < 0 || dev >= MAXDEV) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!known[dev]) {
        int optin = 0;
        cudaFuncAttributes fa{};
        size_t r = 0;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, k_small) == cudaSuccess && (size_t)optin > fa.sharedSizeBytes) {
            r = (size_t)optin - fa.sharedSizeBytes;
            if (cudaFuncSetAttribute(k_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r) != cudaSuccess)
                r = 0;
        }
        (void)cudaGetLastError();
        room[dev] = r;
        known[dev] = true;
    }
    return room[dev];
}

// Does this plan's LTS take the one-CTA shared-memory path?
bool small_fits(const bisim_plan_s* p) {
    const bisim_opts& o = p->opts;
    if (o.small < 0 || p->n < 1 || p->A > 32) return false;
    if (o.engine != BISIM_ENGINE_AUTO && o.engine != BISIM_ENGINE_FRONTIER) return false;
    if (o.raw_labels || o.local_states != 0 || o.light_edges != 0 || o.preprocess == 1 || o.test_hook) return false;
    const size_t room = small_smem_room(p->dev);
    return small_layout(p->n, p->m).total <= room;
}

int small_refine(bisim_plan_s* p, int32_t* out_block, bisim_stats* stats) {
    cudaStream_t st = p->st;
    const SmallLayout Lo = small_layout(p->n, p->m);
    SmallArgs g;
    g.n = p->n;
    g.m = p->m;
    const int32_t* base = p->small_in.as<int32_t>();
    g.src = base;
    g.act = p->small_has_act ? base + p->m : nullptr;
    g.dst = base + 2 * p->m;
    g.init = p->small_has_init ? base + 3 * p->m : nullptr;
    g.out = out_block;
    g.res = p->small_res.as<long long>();
    g.ctrl = p->ctrl.as<bisim_ctrl>();
    g.round_cap = p->opts.round_cap > 0 ? p->opts.round_cap : 3ll * p->n + p->A + 2;
    g.alg2 = (p->opts.rcpp_alg2 && p->A == 1) ? 1 : 0;
    g.kmax = p->opts.splitters > 0 ? std::min(p->opts.splitters, SMALL_KMAX) : SMALL_KMAX;
    const int budget_per_warp = p->opts.split_budget > 0 ? std::min(p->opts.split_budget, 1 << 20) : 4;
    const int threads = p->opts.threads > 0 ? p->opts.threads : SMALL_THREADS_DEFAULT;
    g.budget = budget_per_warp * (threads / 32);
    BISIM_CUDA_TRY(cudaMemsetAsync(p->small_res.p, 0, 8 * 8, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(&g.ctrl->status, 0, sizeof(int), st));
    BISIM_CUDA_TRY(cudaEventRecord(p->evk0, st));
    k_small<<<1, threads, Lo.total, st>>>(g);
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    BISIM_CUDA_TRY(cudaEventRecord(p->evk1, st));
    long long res[8];
    BISIM_CUDA_TRY(cudaMemcpyAsync(res, p->small_res.p, sizeof(res), cudaMemcpyDeviceToHost, st));
    BISIM_TRY(read_ctrl(p));
    BISIM_TRY(report(p));
    if (stats) {
        BISIM_TRY(persistent_ms(p, &stats->t_main_ms));
        stats->rounds = res[0];
        stats->steps = res[1];
        stats->local_steps = res[1];
        stats->pre_rounds = res[2];
        stats->initial_blocks = res[3];
        stats->num_blocks = res[4];
        stats->mark_length = res[5];
        stats->edges_visited = res[6];
        stats->states_visited = res[7];
        stats->engine = BISIM_ENGINE_SMALL;
        stats->grid_ctas = 1;
    }
    p->L = res[5];
    p->pre_rounds = res[2];
    p->initial_blocks = res[3];
    return BISIM_OK;
}

}  // namespace bisim

extern "C" {

int bisim_phase_times(uint64_t* out16) {
#ifdef BISIM_PHASE_TIMERS
    if (!out16) return BISIM_EINVAL;
    BISIM_CUDA_TRY(cudaDeviceSynchronize());
    BISIM_CUDA_TRY(cudaMemcpyFromSymbol(out16, g_phase_acc, sizeof(g_phase_acc)));
    return BISIM_OK;
#else
    (void)out16;
    set_last_error("built without BISIM_PHASE_TIMERS");
    return BISIM_ENOTSUP;
#endif
}

int bisim_phase_trace(uint32_t* out, int32_t max_rounds) {
#ifdef BISIM_PHASE_TIMERS
    if (!out || max_rounds < 0) return BISIM_EINVAL;
    BISIM_CUDA_TRY(cudaDeviceSynchronize());
    const size_t nr = (size_t)std::min(max_rounds, BISIM_TRACE_MAX);
    BISIM_CUDA_TRY(cudaMemcpyFromSymbol(out, g_round_trace, nr * 6 * sizeof(unsigned)));
    return BISIM_OK;
#else
    (void)out;
    (void)max_rounds;
    set_last_error("built without BISIM_PHASE_TIMERS");
    return BISIM_ENOTSUP;
#endif
}

int bisim_phase_reset(void) {
#ifdef BISIM_PHASE_TIMERS
    unsigned long long z[16] = {0};
    BISIM_CUDA_TRY(cudaDeviceSynchronize());
    BISIM_CUDA_TRY(cudaMemcpyToSymbol(g_phase_acc, z, sizeof(z)));
    void* tr = nullptr;
    BISIM_CUDA_TRY(cudaGetSymbolAddress(&tr, g_round_trace));
    BISIM_CUDA_TRY(cudaMemset(tr, 0, sizeof(g_round_trace)));
    return BISIM_OK;
#else
    set_last_error("built without BISIM_PHASE_TIMERS");
    return BISIM_ENOTSUP;
#endif
}

}  // extern "C"
