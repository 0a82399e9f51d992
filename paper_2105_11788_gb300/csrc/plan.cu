// Plan construction (everything before the main while-loop):
//  - range validation of the input arrays;
//  - sort of the transitions by (source, label) and the mark-slot layout of
//    Section 4.1.1: a new (source, label) pair starts where Algorithm 4 would
//    see a source change or an action switch, so the running count of pair
//    starts gives slot = off(source) + order for every transition, nr_marks
//    is the number of pairs of a state and off their exclusive prefix sum;
//  - the incoming-transition CSR by target, every entry carrying (source,
//    slot), built by target bins (or, for very many states and on the sort
//    route, with a counting sort);
//  - initial leaders (Algorithm 2, lines 1-6, priority rule: the smallest
//    member of each initial block);
//  - action-set preprocessing (Algorithm 5): for every label that occurs, in
//    increasing order, mark the sources of that label's transitions and split
//    every block into marked / unmarked parts, the part not containing the
//    leader getting its smallest member as new leader.
// Plus the canonical output step shared by both engines.
#include <algorithm>
#include <mutex>
#include <vector>

#include "plan.cuh"

using namespace bisim;

namespace {

constexpr int T = 256;

// The transition arrays are read as int4 (four transitions per load) when
// all of them start on a 16-byte boundary; `vec` says so (checked on the
// host), and the last m % 4 transitions, or all of them otherwise, are read
// one by one.
__device__ __forceinline__ int4 ld4(const int32_t* p, int64_t q) { return reinterpret_cast<const int4*>(p)[q]; }

__device__ __forceinline__ int check_transition(int32_t s, int32_t a, int32_t d, int32_t n, int32_t A,
                                                uint32_t* used) {
    if ((unsigned)s >= (unsigned)n || (unsigned)d >= (unsigned)n || (unsigned)a >= (unsigned)A) return 1;
    if (used[a] == 0) used[a] = 1;  // benign same-value store
    return 0;
}

__global__ void k_validate(const int32_t* __restrict__ src, const int32_t* __restrict__ act,
                           const int32_t* __restrict__ dst, const int32_t* __restrict__ init,
                           int32_t n, int64_t m, int32_t A, int* status, uint32_t* used, int vec) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int bad = 0;
    const int64_t m4 = vec ? m / 4 : 0;
    for (int64_t q = gtid; q < m4; q += gsz) {
        const int4 s = ld4(src, q), d = ld4(dst, q);
        const int4 a = act ? ld4(act, q) : make_int4(0, 0, 0, 0);
        bad |= check_transition(s.x, a.x, d.x, n, A, used) | check_transition(s.y, a.y, d.y, n, A, used) |
               check_transition(s.z, a.z, d.z, n, A, used) | check_transition(s.w, a.w, d.w, n, A, used);
    }
    for (int64_t i = 4 * m4 + gtid; i < m; i += gsz)
        bad |= check_transition(src[i], act ? act[i] : 0, dst[i], n, A, used);
    if (init)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz)
            if ((unsigned)init[i] >= (unsigned)n) bad = 1;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_INVALID);
}

template <typename K>
__global__ void k_make_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ act,
                            const int32_t* __restrict__ dst, int64_t m, int32_t A, K* keys,
                            uint32_t* vals, int vec) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m4 = vec ? m / 4 : 0;  // keys and vals are fresh allocations: 16-byte aligned
    for (int64_t q = gtid; q < m4; q += gsz) {
        const int4 s = ld4(src, q), d = ld4(dst, q);
        const int4 a = act ? ld4(act, q) : make_int4(0, 0, 0, 0);
        keys[4 * q + 0] = (K)s.x * (K)A + (K)a.x;
        keys[4 * q + 1] = (K)s.y * (K)A + (K)a.y;
        keys[4 * q + 2] = (K)s.z * (K)A + (K)a.z;
        keys[4 * q + 3] = (K)s.w * (K)A + (K)a.w;
        reinterpret_cast<uint4*>(vals)[q] = make_uint4((uint32_t)d.x, (uint32_t)d.y, (uint32_t)d.z, (uint32_t)d.w);
    }
    for (int64_t i = 4 * m4 + gtid; i < m; i += gsz) {
        keys[i] = (K)src[i] * (K)A + (K)(act ? act[i] : 0);
        vals[i] = (uint32_t)dst[i];
    }
}

// flag[i] = 1 where a new (source, label) pair starts in sorted order
template <typename K>
__global__ void k_pair_flags(const K* __restrict__ keys, int64_t m, uint32_t* flags) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gsz)
        flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// slot of every sorted transition, the owner and label of every slot, the
// in-CSR key (target) and payload (source << 32 | slot), and the in-degree.
template <typename K>
__global__ void k_slots(const K* __restrict__ keys, const uint32_t* __restrict__ dst_sorted,
                        const uint32_t* __restrict__ excl, int64_t m, int32_t A,
                        int32_t* slot_src, int32_t* slot_act, uint32_t* tkey, uint64_t* tval,
                        uint32_t* nr_cnt, uint32_t* indeg) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gsz) {
        const K k = keys[i];
        const bool first = (i == 0 || k != keys[i - 1]);
        const uint32_t slot = first ? excl[i] : excl[i] - 1u;
        const int32_t s = (int32_t)(k / (K)A);
        if (first) {
            slot_src[slot] = s;
            slot_act[slot] = (int32_t)(k % (K)A);
            atomicAdd(&nr_cnt[s], 1u);
        }
        const uint32_t d = dst_sorted[i];
        tkey[i] = d;
        tval[i] = ((uint64_t)(uint32_t)s << 32) | slot;
        atomicAdd(&indeg[d], 1u);
    }
}

__global__ void k_csr_scatter(const uint32_t* __restrict__ tkey, const uint64_t* __restrict__ tval, int64_t m,
                              uint32_t* cursor, uint64_t* in_edge) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gsz)
        in_edge[atomicAdd(&cursor[tkey[i]], 1u)] = tval[i];
}

// Mark-slot layout from label sets (|Act| <= 32 * MASK_WORDS_MAX). One pass
// over the transitions validates them and, for valid ones, ORs the label
// into its source's label-set bitmask and counts the target's in-degree.
// Then for a state s with label set M(s): nr_marks(s) = |M(s)|, off = the
// exclusive prefix sum of nr_marks, and the slot of a transition s -a-> t is
// off(s) + |{b in M(s) : b < a}| - the rank of (s, a) among the distinct
// (source, label) pairs in (source, label) order, which is exactly what
// Algorithm 4's sort, action_switch and segmented scans compute.
constexpr int MASK_WORDS_MAX = 4;
// The incoming-transition CSR is built by bins of 2^bin_bits targets, at most
// CSR_MAX_BINS of them (see k_csr_bin).
constexpr int CSR_MAX_BINS = 4096;

// In-degrees, counted either per target (a global atomic per transition,
// indeg != null) or per bin of 2^bin_bits targets in the CTA's shared
// histogram, added to bin_cnt at the end (the CSR passes then derive the
// per-target offsets bin by bin).
struct InCount {
    uint32_t* indeg;
    uint32_t* hist;  // shared, or null
    int bin_bits;
    __device__ __forceinline__ void add(int32_t d) const {
        if (hist)
            atomicAdd(&hist[(uint32_t)d >> bin_bits], 1u);
        else
            atomicAdd(&indeg[d], 1u);
    }
};

__device__ __forceinline__ void count_transition(int32_t s, int32_t a, int32_t d, int mask_words, uint32_t* amask,
                                                 const InCount& ic) {
    atomicOr(&amask[(size_t)s * mask_words + (a >> 5)], 1u << (a & 31));
    ic.add(d);
}

__global__ void k_validate_count(const int32_t* __restrict__ src, const int32_t* __restrict__ act,
                                 const int32_t* __restrict__ dst, const int32_t* __restrict__ init, int32_t n,
                                 int64_t m, int32_t A, int* status, uint32_t* used, int vec, int mask_words,
                                 uint32_t* amask, uint32_t* indeg, int bin_bits, int nbins, uint32_t* bin_cnt) {
    __shared__ uint32_t hist[CSR_MAX_BINS];
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const InCount ic{indeg, bin_cnt ? hist : nullptr, bin_bits};
    if (bin_cnt) {
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0u;
        __syncthreads();
    }
    int bad = 0;
    const int64_t m4 = vec ? m / 4 : 0;
    for (int64_t q = gtid; q < m4; q += gsz) {
        const int4 s = ld4(src, q), d = ld4(dst, q);
        const int4 a = act ? ld4(act, q) : make_int4(0, 0, 0, 0);
        const int b0 = check_transition(s.x, a.x, d.x, n, A, used), b1 = check_transition(s.y, a.y, d.y, n, A, used);
        const int b2 = check_transition(s.z, a.z, d.z, n, A, used), b3 = check_transition(s.w, a.w, d.w, n, A, used);
        bad |= b0 | b1 | b2 | b3;
        if (!(b0 | b1 | b2 | b3)) {
            // consecutive transitions with the same label-set word (one source,
            // when the input is grouped by source) set their bits with one atomic
            const int sv[4] = {s.x, s.y, s.z, s.w}, av[4] = {a.x, a.y, a.z, a.w}, dv[4] = {d.x, d.y, d.z, d.w};
            size_t wprev = (size_t)sv[0] * mask_words + (av[0] >> 5);
            uint32_t bits = 1u << (av[0] & 31);
#pragma unroll
            for (int k = 1; k < 4; k++) {
                const size_t w = (size_t)sv[k] * mask_words + (av[k] >> 5);
                if (w != wprev) {
                    atomicOr(&amask[wprev], bits);
                    wprev = w;
                    bits = 0u;
                }
                bits |= 1u << (av[k] & 31);
            }
            atomicOr(&amask[wprev], bits);
#pragma unroll
            for (int k = 0; k < 4; k++) ic.add(dv[k]);
        } else {
            if (!b0) count_transition(s.x, a.x, d.x, mask_words, amask, ic);
            if (!b1) count_transition(s.y, a.y, d.y, mask_words, amask, ic);
            if (!b2) count_transition(s.z, a.z, d.z, mask_words, amask, ic);
            if (!b3) count_transition(s.w, a.w, d.w, mask_words, amask, ic);
        }
    }
    for (int64_t i = 4 * m4 + gtid; i < m; i += gsz) {
        const int32_t s = src[i], a = act ? act[i] : 0, d = dst[i];
        const int b = check_transition(s, a, d, n, A, used);
        if (!b) count_transition(s, a, d, mask_words, amask, ic);
        bad |= b;
    }
    if (init)
        for (int64_t i = gtid; i < n; i += gsz)
            if ((unsigned)init[i] >= (unsigned)n) bad = 1;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_INVALID);
    if (bin_cnt) {
        __syncthreads();
        for (int b = threadIdx.x; b < nbins; b += blockDim.x)
            if (hist[b]) atomicAdd(&bin_cnt[b], hist[b]);
    }
}

// nr_marks of every state (into off, scanned afterwards)
__global__ void k_mask_count(const uint32_t* __restrict__ amask, int32_t n, int mask_words, uint32_t* nr) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gsz) {
        uint32_t c = 0;
        for (int w = 0; w < mask_words; w++) c += __popc(amask[(size_t)s * mask_words + w]);
        nr[s] = c;
    }
}

// owner and label of every mark slot
__global__ void k_mask_slots(const uint32_t* __restrict__ amask, const uint32_t* __restrict__ off, int32_t n,
                             int mask_words, int32_t* slot_src, int32_t* slot_act) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gsz) {
        uint32_t k = off[s];
        for (int w = 0; w < mask_words; w++) {
            uint32_t bits = amask[(size_t)s * mask_words + w];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                slot_src[k] = (int32_t)s;
                slot_act[k] = 32 * w + b;
                k++;
            }
        }
    }
}

// incoming-transition CSR by target with (source << 32 | slot) entries
__device__ __forceinline__ void csr_put(int32_t s, int32_t a, int32_t d, const uint32_t* __restrict__ amask,
                                        const uint32_t* __restrict__ off, int mask_words, uint32_t* cursor,
                                        unsigned long long* in_edge) {
    uint32_t order = 0;
    const uint32_t* ms = amask + (size_t)s * mask_words;
    for (int w = 0; w < (a >> 5); w++) order += __popc(ms[w]);
    order += __popc(ms[a >> 5] & ((1u << (a & 31)) - 1u));
    const uint32_t slot = off[s] + order;
    in_edge[atomicAdd(&cursor[d], 1u)] = ((unsigned long long)(uint32_t)s << 32) | slot;  // (large n only)
}

__global__ void k_mask_csr(const int32_t* __restrict__ src, const int32_t* __restrict__ act,
                           const int32_t* __restrict__ dst, int64_t m, const uint32_t* __restrict__ amask,
                           const uint32_t* __restrict__ off, int mask_words, int vec, uint32_t* cursor,
                           unsigned long long* in_edge) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m4 = vec ? m / 4 : 0;
    for (int64_t q = gtid; q < m4; q += gsz) {
        const int4 s = ld4(src, q), d = ld4(dst, q);
        const int4 a = act ? ld4(act, q) : make_int4(0, 0, 0, 0);
        csr_put(s.x, a.x, d.x, amask, off, mask_words, cursor, in_edge);
        csr_put(s.y, a.y, d.y, amask, off, mask_words, cursor, in_edge);
        csr_put(s.z, a.z, d.z, amask, off, mask_words, cursor, in_edge);
        csr_put(s.w, a.w, d.w, amask, off, mask_words, cursor, in_edge);
    }
    for (int64_t i = 4 * m4 + gtid; i < m; i += gsz)
        csr_put(src[i], act ? act[i] : 0, dst[i], amask, off, mask_words, cursor, in_edge);
}

// The incoming-transition CSR in two passes, without a returning global
// atomic per transition. Targets are cut into bins of 2^bin_bits states; the
// validation pass counted the transitions of every bin, so a bin's entries
// occupy a known range of in_edge (the exclusive scan of those counts).
//   pass A: a CTA takes a tile of transitions, ranks them per bin with
//     shared-memory atomics, reserves each bin's share of the tile with one
//     global atomic per (CTA, bin), sorts the tile's (target, source << 32 |
//     slot) records by bin in shared memory and writes each bin's records as
//     one run into the bin's range of two scratch arrays;
//   pass B: one CTA per bin counts the bin's records per target, writes
//     in_ptr for its targets from the scan of the counts, and places every
//     record at in_ptr[t] + (rank among t's records).
#ifndef BISIM_CSR_A_THREADS
#define BISIM_CSR_A_THREADS 1024
#endif
#ifndef BISIM_CSR_A_ITEMS
#define BISIM_CSR_A_ITEMS 8
#endif
constexpr int CSR_A_THREADS = BISIM_CSR_A_THREADS;
constexpr int CSR_A_ITEMS = BISIM_CSR_A_ITEMS;   // transitions per thread of pass A
constexpr int CSR_A_TILE = CSR_A_THREADS * CSR_A_ITEMS;
constexpr int CSR_B_THREADS = 1024;

__device__ __forceinline__ uint32_t slot_of(int32_t s, int32_t a, const uint32_t* __restrict__ amask,
                                            const uint32_t* __restrict__ off, int mask_words) {
    uint32_t order = 0;
    const uint32_t* ms = amask + (size_t)s * mask_words;
    for (int w = 0; w < (a >> 5); w++) order += __popc(ms[w]);
    order += __popc(ms[a >> 5] & ((1u << (a & 31)) - 1u));
    return off[s] + order;
}

// With at most 32 labels a state's first slot and label set fit one word
// (off << 32 | label set): one gather per transition instead of two.
__global__ void k_pack_sinfo(const uint32_t* __restrict__ off, const uint32_t* __restrict__ amask, int32_t n,
                             unsigned long long* sinfo) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gsz)
        sinfo[s] = ((unsigned long long)off[s] << 32) | amask[s];
}

__global__ void __launch_bounds__(CSR_A_THREADS, 1) k_csr_bin(const int32_t* __restrict__ src,
                                                           const int32_t* __restrict__ act,
                                                           const int32_t* __restrict__ dst, int64_t m,
                                                           const uint32_t* __restrict__ amask,
                                                           const uint32_t* __restrict__ off, int mask_words,
                                                           const unsigned long long* __restrict__ sinfo,
                                                           int bin_bits, int nbins, uint32_t* bin_cursor,
                                                           uint32_t* rec_t, unsigned long long* rec_v) {
    // dynamic shared memory: per bin the tile's count, then its first
    // position in the tile (exclusive scan) and its reserved global position;
    // the tile's records sorted by bin
    extern __shared__ __align__(16) unsigned char csr_smem[];
    unsigned long long* vs = reinterpret_cast<unsigned long long*>(csr_smem);  // [CSR_A_TILE]
    uint32_t* ts = reinterpret_cast<uint32_t*>(vs + CSR_A_TILE);              // [CSR_A_TILE]
    uint32_t* cnt = ts + CSR_A_TILE;                                           // [nbins]
    uint32_t* toff = cnt + CSR_MAX_BINS;                                       // [nbins]
    uint32_t* base = toff + CSR_MAX_BINS;                                      // [nbins]
    __shared__ uint32_t wsum[CSR_A_THREADS / 32];
    const int64_t tile0 = (int64_t)blockIdx.x * CSR_A_TILE;
    const int tn = (int)min((int64_t)CSR_A_TILE, m - tile0);
    for (int b = threadIdx.x; b < nbins; b += CSR_A_THREADS) cnt[b] = 0;
    __syncthreads();
    int32_t t[CSR_A_ITEMS];
    uint32_t rk[CSR_A_ITEMS];
#pragma unroll
    for (int j = 0; j < CSR_A_ITEMS; j++) {
        const int k = j * CSR_A_THREADS + (int)threadIdx.x;
        t[j] = k < tn ? dst[tile0 + k] : -1;
    }
#pragma unroll
    for (int j = 0; j < CSR_A_ITEMS; j++)
        if (t[j] >= 0) rk[j] = atomicAdd(&cnt[t[j] >> bin_bits], 1u);
    __syncthreads();
    // exclusive scan of the counts over the bins (CSR_MAX_BINS / CSR_A_THREADS per thread)
    {
        constexpr int E = CSR_MAX_BINS / CSR_A_THREADS;
        const int b0 = (int)threadIdx.x * E;
        uint32_t c[E], sum = 0;
#pragma unroll
        for (int e = 0; e < E; e++) {
            c[e] = b0 + e < nbins ? cnt[b0 + e] : 0u;
            sum += c[e];
        }
        const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t v = lane < CSR_A_THREADS / 32 ? wsum[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= (unsigned)o) v += y;
            }
            if (lane < CSR_A_THREADS / 32) wsum[lane] = v;
        }
        __syncthreads();
        uint32_t ex = x - sum + (w > 0 ? wsum[w - 1] : 0u);
#pragma unroll
        for (int e = 0; e < E; e++) {
            if (b0 + e < nbins) {
                toff[b0 + e] = ex;
                base[b0 + e] = c[e] ? atomicAdd(&bin_cursor[b0 + e], c[e]) : 0u;
            }
            ex += c[e];
        }
    }
    __syncthreads();
    // the tile's sources and labels again (just read, so close) and its
    // records, placed by bin in shared memory
#pragma unroll
    for (int j = 0; j < CSR_A_ITEMS; j++)
        if (t[j] >= 0) {
            const int64_t i = tile0 + (int64_t)j * CSR_A_THREADS + threadIdx.x;
            const int32_t s = src[i], a = act ? act[i] : 0;
            uint32_t slot;
            if (sinfo) {
                const unsigned long long si = sinfo[s];
                slot = (uint32_t)(si >> 32) + __popc((uint32_t)si & ((1u << (a & 31)) - 1u));
            } else {
                slot = slot_of(s, a, amask, off, mask_words);
            }
            const uint32_t q = toff[t[j] >> bin_bits] + rk[j];
            ts[q] = (uint32_t)t[j];
            vs[q] = ((unsigned long long)(uint32_t)s << 32) | slot;
        }
    __syncthreads();
    // consecutive records of a bin go to consecutive global positions
    for (int q = threadIdx.x; q < tn; q += CSR_A_THREADS) {
        const uint32_t tt = ts[q];
        const int b = (int)(tt >> bin_bits);
        const uint32_t g = base[b] + (uint32_t)q - toff[b];
        rec_t[g] = tt;
        rec_v[g] = vs[q];
    }
}

// dynamic shared memory of k_csr_bin
constexpr size_t CSR_A_SMEM = (size_t)CSR_A_TILE * 12 + (size_t)CSR_MAX_BINS * 12;

// Pass B: bin b's records are rec_t / rec_v[bin_end[b - 1], bin_end[b])
// (bin_end: the bin cursors after pass A). The CTA counts them per target,
// writes in_ptr for the bin's targets (and in_ptr[n] = m in the last bin)
// from the exclusive scan of the counts, and places every record by target
// with shared-memory cursors.
__global__ void __launch_bounds__(CSR_B_THREADS) k_csr_place(const uint32_t* __restrict__ bin_end, int32_t n,
                                                             int64_t m, int bin_bits,
                                                             const uint32_t* __restrict__ rec_t,
                                                             const unsigned long long* __restrict__ rec_v,
                                                             uint32_t* in_ptr, unsigned long long* in_edge) {
    extern __shared__ uint32_t tcnt[];  // 2^bin_bits counters
    __shared__ uint32_t wsum[CSR_B_THREADS / 32];
    const int b = (int)blockIdx.x;
    const int64_t lo = (int64_t)b << bin_bits;
    const int nt = (int)(min((int64_t)n, lo + ((int64_t)1 << bin_bits)) - lo);
    for (int i = threadIdx.x; i < nt; i += CSR_B_THREADS) tcnt[i] = 0;
    __syncthreads();
    const uint32_t r0 = b ? bin_end[b - 1] : 0u, r1 = bin_end[b];
    for (uint32_t i = r0 + threadIdx.x; i < r1; i += CSR_B_THREADS) atomicAdd(&tcnt[rec_t[i] - (uint32_t)lo], 1u);
    __syncthreads();
    // exclusive scan of tcnt[0, nt): each thread a run of E counters
    const int E = (nt + CSR_B_THREADS - 1) / CSR_B_THREADS;
    const int i0 = (int)threadIdx.x * E, i1 = min(nt, i0 + E);
    uint32_t sum = 0;
    for (int i = i0; i < i1; i++) sum += tcnt[i];
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t v = lane < CSR_B_THREADS / 32 ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= (unsigned)o) v += y;
        }
        if (lane < CSR_B_THREADS / 32) wsum[lane] = v;
    }
    __syncthreads();
    uint32_t ex = x - sum + (w > 0 ? wsum[w - 1] : 0u);
    for (int i = i0; i < i1; i++) {
        const uint32_t c = tcnt[i];
        tcnt[i] = ex;
        in_ptr[lo + i] = r0 + ex;
        ex += c;
    }
    if (lo + nt == (int64_t)n && threadIdx.x == 0) in_ptr[n] = (uint32_t)m;
    __syncthreads();
    for (uint32_t i = r0 + threadIdx.x; i < r1; i += CSR_B_THREADS) {
        const uint32_t tt = rec_t[i];
        const uint32_t r = atomicAdd(&tcnt[tt - (uint32_t)lo], 1u);
        in_edge[r0 + r] = rec_v[i];
    }
}

// label set of every state as a bitmask of mask_words 32-bit words
__global__ void k_label_masks(const int32_t* __restrict__ slot_src, const int32_t* __restrict__ slot_act,
                              int64_t L, int mask_words, uint32_t* amask) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gsz) {
        const int32_t a = slot_act[k];
        atomicOr(&amask[(size_t)slot_src[k] * mask_words + (a >> 5)], 1u << (a & 31));
    }
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz) p[i] = v;
}

__global__ void k_init_min(const int32_t* __restrict__ init, int32_t n, int32_t* nl) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    // uniform trip count per warp (n rounded up), so every lane reaches the match
    const int64_t lim = (n + 31) & ~(int64_t)31;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < lim; i += gsz) {
        const int32_t v = i < n ? init[i] : -1;
        // consecutive lanes hold consecutive states: one atomic per label per warp
        const unsigned peers = __match_any_sync(0xffffffffu, v);
        if (v >= 0 && (peers & lanemask_lt()) == 0u) atomicMin(&nl[v], (int32_t)i);
    }
}

__global__ void k_init_relabel(const int32_t* __restrict__ init, int32_t n,
                               const int32_t* __restrict__ nl, int32_t* block) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz)
        block[i] = nl[init[i]];
}

__device__ __forceinline__ unsigned long long elect_key(uint32_t stamp, int32_t s) {
    // newer stamps compare smaller, so atomicMin keeps this round's smallest state
    return ((unsigned long long)(0xffffffffu - stamp) << 32) | (uint32_t)s;
}

struct LabelArgs {
    int32_t n;
    int64_t L;
    int32_t n_labels;
    const int32_t* labels;
    const int32_t* slot_src;
    const int32_t* slot_act;
    int32_t* block;
    uint32_t* lmark;
    unsigned long long* nl64;
    uint8_t* split;
    const uint32_t* amask;  // label sets as bitmasks (NULL: mark by scanning the slots)
    int mask_words;
    uint32_t stamp0;
    GridBarrier gb;
};

// Algorithm 5: one round per label that occurs. The mark of state s in the
// round of label a is "s has an a-transition": read from the state's label
// bitmask when there is one (two grid barriers per round), else written by
// one thread per mark slot (three).
__global__ void __launch_bounds__(512, 4) k_label_rounds(LabelArgs a) {  // launched with 512 threads
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    unsigned long long tgt = 0;
    for (int li = 0; li < a.n_labels; li++) {
        const int32_t lab = a.labels[li];
        const uint32_t stamp = a.stamp0 + (uint32_t)li + 1u;
        if (!a.amask) {
            for (int64_t k = gtid; k < a.L; k += gsz)
                if (a.slot_act[k] == lab) a.lmark[a.slot_src[k]] = stamp;
            if (!grid_sync(a.gb, tgt)) return;
        }
        const int w = lab >> 5;
        const uint32_t bit = 1u << (lab & 31);
        // four states per thread per step, so their independent loads overlap;
        // the loop test uses the warp's first state, so all lanes iterate
        // together and reach the match below
        const int64_t lane = threadIdx.x & 31;
        for (int64_t s0 = gtid; s0 - lane < a.n; s0 += 4 * gsz) {
            int32_t b[4];
            bool ms[4], mb[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int64_t s = s0 + u * gsz;
                b[u] = s < a.n ? a.block[s] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int64_t s = s0 + u * gsz;
                if (s >= a.n) {
                    ms[u] = mb[u] = false;
                } else if (a.amask) {
                    ms[u] = (a.amask[(size_t)s * a.mask_words + w] & bit) != 0u;
                    mb[u] = (a.amask[(size_t)b[u] * a.mask_words + w] & bit) != 0u;
                } else {
                    ms[u] = ldcg(&a.lmark[s]) == stamp;
                    mb[u] = ldcg(&a.lmark[b[u]]) == stamp;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int64_t s = s0 + u * gsz;
                const bool sp = s < a.n && ms[u] != mb[u];
                if (s < a.n) a.split[s] = sp;
                // lanes hold consecutive states: the lowest lane of each group of
                // splitting states with the same block holds the group's minimum
                const unsigned peers = __match_any_sync(0xffffffffu, sp ? b[u] : -1);
                if (sp && (peers & lanemask_lt()) == 0u) {
                    // early rounds split a few huge blocks: skip the atomic when
                    // the election word already holds a smaller key
                    // (a cached, possibly stale read is enough: election words
                    // only drop within a round, and older rounds' keys are larger)
                    const unsigned long long key = elect_key(stamp, (int32_t)s);
                    if (a.nl64[b[u]] > key) atomicMin(&a.nl64[b[u]], key);
                }
            }
        }
        if (!grid_sync(a.gb, tgt)) return;
        // relabel: each level of loads (flags, blocks, election words) of the
        // thread's four states is issued together
        for (int64_t s0 = gtid; s0 < a.n; s0 += 4 * gsz) {
            uint8_t f[4];
            int32_t bb[4];
            uint32_t v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) f[u] = s0 + u * gsz < a.n ? ldcg(&a.split[s0 + u * gsz]) : (uint8_t)0;
#pragma unroll
            for (int u = 0; u < 4; u++) bb[u] = f[u] ? a.block[s0 + u * gsz] : 0;
            // after the barrier's acquire, cached loads of the election words see
            // their final values; they keep the few words of big blocks in L1
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = f[u] ? (uint32_t)a.nl64[bb[u]] : 0u;
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (f[u]) a.block[s0 + u * gsz] = (int32_t)v[u];
        }
        if (!grid_sync(a.gb, tgt)) return;
    }
}

__global__ void k_count_leaders(const int32_t* __restrict__ block, int32_t n,
                                unsigned long long* count) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    unsigned c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz)
        c += block[i] == (int32_t)i;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

// canonical output
__global__ void k_first_min(const int32_t* __restrict__ block, int32_t n, int32_t* first) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz)
        atomicMin(&first[block[i]], (int32_t)i);
}
__global__ void k_is_first(const int32_t* __restrict__ block, const int32_t* __restrict__ first,
                           int32_t n, uint32_t* flag) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz)
        flag[i] = first[block[i]] == (int32_t)i;
}
__global__ void k_gather_ids(const int32_t* __restrict__ block, const int32_t* __restrict__ first,
                             const uint32_t* __restrict__ rank, int32_t n, int32_t* out) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz)
        out[i] = (int32_t)rank[first[block[i]]];
}

// key of state vals[i] for the sort pass over label-set word w (w < mask_words)
// or over the block after the initial election (w == mask_words)
__global__ void k_group_keys(const uint32_t* __restrict__ vals, const uint32_t* __restrict__ amask,
                             const int32_t* __restrict__ block, int mask_words, int w, int32_t n,
                             uint32_t* keys) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz) {
        const uint32_t s = vals[i];
        keys[i] = w < mask_words ? amask[(size_t)s * mask_words + w] : (uint32_t)block[s];
    }
}

// 1 where sorted position i starts a new (block, label set) group
__global__ void k_group_starts(const uint32_t* __restrict__ vals, const uint32_t* __restrict__ amask,
                               const int32_t* __restrict__ block, int mask_words, int32_t n,
                               uint32_t* start) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz) {
        bool st = i == 0;
        if (!st) {
            const uint32_t s = vals[i], t = vals[i - 1];
            st = block[s] != block[t];
            for (int w = 0; w < mask_words && !st; w++)
                st = amask[(size_t)s * mask_words + w] != amask[(size_t)t * mask_words + w];
        }
        start[i] = st;
    }
}

// leader of each group = its first sorted state (the smallest, the sorts being
// stable over states in increasing order). excl = exclusive scan of start, so
// the group of position i is excl[i] + start[i] - 1.
__global__ void k_group_first(const uint32_t* __restrict__ vals, const uint32_t* __restrict__ start,
                              const uint32_t* __restrict__ excl, int32_t n, int32_t* first) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz)
        if (start[i]) first[excl[i]] = (int32_t)vals[i];
}

__global__ void k_group_assign(const uint32_t* __restrict__ vals, const uint32_t* __restrict__ start,
                               const uint32_t* __restrict__ excl, const int32_t* __restrict__ first,
                               int32_t n, int32_t* block) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz)
        block[vals[i]] = first[excl[i] + start[i] - 1u];
}

__global__ void k_iota(uint32_t* v, int32_t n) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz) v[i] = (uint32_t)i;
}

}  // namespace

namespace bisim {

// Literal preprocessing rounds (Algorithm 5, one per label) are kept for the
// dense engine, whose leader labels are checked against the lock-step
// program, and on request; otherwise the rounds' result is computed directly.
bool preprocess_fused(const bisim_plan_s* p) {
    if (p->opts.preprocess == 1) return false;
    if (p->opts.preprocess == 2) return true;
    return p->opts.engine != BISIM_ENGINE_DENSE;
}

// block <- one block per (block, label set), led by its smallest state: the
// partition every sequence of Algorithm 5's label rounds ends in. Stable LSD
// radix sorts of the states by each label-set word and then by the block,
// group boundaries, and a scan numbering the groups.
int group_by_label_set(bisim_plan_s* p, const uint32_t* amask, int mask_words) {
    const int32_t n = p->n;
    cudaStream_t st = p->st;
    const unsigned gn = grid_for(n, T);
    DevMem keys, keys2, vals, vals2, flags;
    BISIM_TRY(keys.alloc(4 * (size_t)n, st));
    BISIM_TRY(keys2.alloc(4 * (size_t)n, st));
    BISIM_TRY(vals.alloc(4 * (size_t)n, st));
    BISIM_TRY(vals2.alloc(4 * (size_t)n, st));
    BISIM_TRY(flags.alloc(4 * (size_t)n, st));
    k_iota<<<gn, T, 0, st>>>(vals.as<uint32_t>(), n);
    BISIM_LAUNCHED();
    int32_t* block = p->block.as<int32_t>();
    for (int w = 0; w <= mask_words; w++) {
        k_group_keys<<<gn, T, 0, st>>>(vals.as<uint32_t>(), amask, block, mask_words, w, n, keys.as<uint32_t>());
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        bool alt = false;
        const int bits = w < mask_words ? 32 : ceil_log2_u64((uint64_t)n);
        BISIM_TRY(radix_sort_pairs<uint32_t, uint32_t>(keys.as<uint32_t>(), vals.as<uint32_t>(),
                                                       keys2.as<uint32_t>(), vals2.as<uint32_t>(), n, bits, st,
                                                       &alt));
        if (alt) {
            std::swap(vals.p, vals2.p);
            std::swap(keys.p, keys2.p);
        }
    }
    k_group_starts<<<gn, T, 0, st>>>(vals.as<uint32_t>(), amask, block, mask_words, n, flags.as<uint32_t>());
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    // keys <- number of group starts before each sorted position
    BISIM_TRY(scan_exclusive_u32(flags.as<uint32_t>(), keys.as<uint32_t>(), n, nullptr, st));
    k_group_first<<<gn, T, 0, st>>>(vals.as<uint32_t>(), flags.as<uint32_t>(), keys.as<uint32_t>(), n,
                                    (int32_t*)keys2.p);
    BISIM_LAUNCHED();
    k_group_assign<<<gn, T, 0, st>>>(vals.as<uint32_t>(), flags.as<uint32_t>(), keys.as<uint32_t>(),
                                     (const int32_t*)keys2.p, n, block);
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    return BISIM_OK;
}

}  // namespace bisim

namespace {

// Pinned control mirrors and timing events outlive their plans: creating
// them (a page-locked host allocation and four events) costs more than a
// whole small reduction, so released sets wait here, per device, for the
// next plan.
struct HostRes {
    int dev;
    bisim_ctrl* ctrl_h;
    cudaEvent_t ev[4];
};
constexpr size_t HOST_RES_KEEP = 64;
std::mutex g_res_mu;
std::vector<HostRes> g_res;

}  // namespace

namespace bisim {

int device_setup(bisim_plan_s* p) {
    int dev = 0;
    BISIM_CUDA_TRY(cudaGetDevice(&dev));
    BISIM_CUDA_TRY(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev));
    BISIM_TRY(retain_pool_memory());
    p->dev = dev;
    {
        std::lock_guard<std::mutex> lk(g_res_mu);
        for (size_t i = g_res.size(); i-- > 0;) {
            if (g_res[i].dev != dev) continue;
            const HostRes r = g_res[i];
            g_res.erase(g_res.begin() + (std::ptrdiff_t)i);
            p->ctrl_h = r.ctrl_h;
            p->ev0 = r.ev[0];
            p->ev1 = r.ev[1];
            p->evk0 = r.ev[2];
            p->evk1 = r.ev[3];
            return BISIM_OK;
        }
    }
    BISIM_CUDA_TRY(cudaMallocHost(&p->ctrl_h, sizeof(bisim_ctrl)));
    BISIM_CUDA_TRY(cudaEventCreate(&p->ev0));
    BISIM_CUDA_TRY(cudaEventCreate(&p->ev1));
    BISIM_CUDA_TRY(cudaEventCreate(&p->evk0));
    BISIM_CUDA_TRY(cudaEventCreate(&p->evk1));
    return BISIM_OK;
}

}  // namespace bisim

bisim_plan_s::~bisim_plan_s() {
    // the destroy call synchronised the stream: nothing in flight uses these
    bool kept = false;
    if (ctrl_h && ev0 && ev1 && evk0 && evk1) {
        std::lock_guard<std::mutex> lk(g_res_mu);
        if (g_res.size() < HOST_RES_KEEP) {
            g_res.push_back(HostRes{dev, ctrl_h, {ev0, ev1, evk0, evk1}});
            kept = true;
        }
    }
    if (!kept) {
        if (ctrl_h) cudaFreeHost(ctrl_h);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (evk0) cudaEventDestroy(evk0);
        if (evk1) cudaEventDestroy(evk1);
    }
    if (aux_event) cudaEventDestroy(aux_event);
    if (aux_stream) {
        cudaStreamSynchronize(aux_stream);
        cudaStreamDestroy(aux_stream);
    }
}

namespace bisim {

int read_ctrl(bisim_plan_s* p) {
    BISIM_CUDA_TRY(cudaMemcpyAsync(p->ctrl_h, p->ctrl.p, sizeof(bisim_ctrl), cudaMemcpyDeviceToHost,
                                   p->st));
    BISIM_CUDA_TRY(cudaStreamSynchronize(p->st));
    return BISIM_OK;
}

int reserve_stamps(bisim_plan_s* p, int64_t rounds, uint32_t* base) {
    if ((uint64_t)p->stamp + (uint64_t)rounds + 2 >= 0xffffffffull) {
        if (p->L) BISIM_CUDA_TRY(cudaMemsetAsync(p->mark.p, 0, sizeof(uint32_t) * p->L, p->st));
        if (p->n) {
            BISIM_CUDA_TRY(cudaMemsetAsync(p->lmark.p, 0, sizeof(uint32_t) * p->n, p->st));
            BISIM_CUDA_TRY(cudaMemsetAsync(p->nl64.p, 0xff, sizeof(uint64_t) * p->n, p->st));
            if (p->frontier_ready) {
                BISIM_CUDA_TRY(cudaMemsetAsync(p->smark.p, 0, sizeof(uint32_t) * p->n, p->st));
                BISIM_CUDA_TRY(cudaMemsetAsync(p->kmark.p, 0, sizeof(uint32_t) * p->n, p->st));
                BISIM_CUDA_TRY(cudaMemsetAsync(p->claim.p, 0xff, sizeof(uint64_t) * p->n, p->st));
                BISIM_CUDA_TRY(cudaMemsetAsync(p->minx.p, 0xff, sizeof(uint64_t) * p->n, p->st));
                BISIM_CUDA_TRY(cudaMemsetAsync(p->smark64.p, 0xff, sizeof(uint64_t) * p->n, p->st));
                BISIM_CUDA_TRY(cudaMemsetAsync(p->lostl.p, 0, sizeof(uint32_t) * p->n, p->st));
            }
        }
        p->stamp = 0;
    }
    *base = p->stamp;
    return BISIM_OK;
}

int launch_persistent(const void* fn, void** args, int threads, bisim_plan_s* p, int* grid_out,
                      int per_sm_default, size_t dyn_smem) {
    int occ = 0;
    if (dyn_smem > 48 * 1024)
        BISIM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem));
    BISIM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, dyn_smem));
    if (occ < 1) {
        set_last_error("persistent kernel does not fit on an SM");
        return BISIM_ECUDA;
    }
    int per_sm = p->opts.ctas_per_sm > 0 ? p->opts.ctas_per_sm : per_sm_default;
    per_sm = std::min(per_sm, occ);
    int grid = p->sm_count * per_sm;
    if (p->opts.max_ctas > 0) grid = std::min(grid, p->opts.max_ctas);
    *grid_out = grid;
    BISIM_CUDA_TRY(cudaEventRecord(p->evk0, p->st));
    BISIM_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(threads), args, dyn_smem, p->st));
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaEventRecord(p->evk1, p->st));
    return BISIM_OK;
}

int persistent_ms(bisim_plan_s* p, double* ms) {
    float f = 0;
    BISIM_CUDA_TRY(cudaEventSynchronize(p->evk1));
    BISIM_CUDA_TRY(cudaEventElapsedTime(&f, p->evk0, p->evk1));
    *ms = f;
    return BISIM_OK;
}

// a2 + a3 by Algorithm 4's route: sort the transitions by (source, label),
// flag where a new (source, label) pair starts, scan the flags; the slots,
// nr_marks and off follow, then the incoming-transition CSR by target
// (counting sort; the order inside one target's list is whatever the atomics
// give: marking is idempotent, so it never matters).
static int slots_by_sort(bisim_plan_s* p, const int32_t* src, const int32_t* act, const int32_t* dst, int vec) {
    const int32_t n = p->n;
    const int64_t m = p->m;
    const int32_t A = p->A;
    cudaStream_t st = p->st;
    const uint64_t keyspace = (uint64_t)n * (uint64_t)A;

    const bool wide = keyspace > 0xffffffffull;
    const int kbits = ceil_log2_u64(keyspace);
    const size_t ksz = wide ? 8 : 4;
    DevMem keys, keys_alt, vals, vals_alt;
    BISIM_TRY(keys.alloc(ksz * (size_t)m, st));
    BISIM_TRY(keys_alt.alloc(ksz * (size_t)m, st));
    BISIM_TRY(vals.alloc(4 * (size_t)m, st));
    BISIM_TRY(vals_alt.alloc(4 * (size_t)m, st));
    const unsigned gm = grid_for(m, T);
    bool alt = false;
    if (wide) {
        k_make_keys<uint64_t><<<gm, T, 0, st>>>(src, act, dst, m, A, keys.as<uint64_t>(),
                                                vals.as<uint32_t>(), vec);
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        BISIM_TRY(radix_sort_pairs<uint64_t, uint32_t>(keys.as<uint64_t>(), vals.as<uint32_t>(),
                                                       keys_alt.as<uint64_t>(),
                                                       vals_alt.as<uint32_t>(), m, kbits, st, &alt));
    } else {
        k_make_keys<uint32_t><<<gm, T, 0, st>>>(src, act, dst, m, A, keys.as<uint32_t>(),
                                                vals.as<uint32_t>(), vec);
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        BISIM_TRY(radix_sort_pairs<uint32_t, uint32_t>(keys.as<uint32_t>(), vals.as<uint32_t>(),
                                                       keys_alt.as<uint32_t>(),
                                                       vals_alt.as<uint32_t>(), m, kbits, st, &alt));
    }
    void* skeys = alt ? keys_alt.p : keys.p;
    uint32_t* sdst = alt ? vals_alt.as<uint32_t>() : vals.as<uint32_t>();

    DevMem flags, Ldev;
    BISIM_TRY(flags.alloc(4 * (size_t)m, st));
    BISIM_TRY(Ldev.alloc(4, st));
    if (wide)
        k_pair_flags<uint64_t><<<gm, T, 0, st>>>((const uint64_t*)skeys, m, flags.as<uint32_t>());
    else
        k_pair_flags<uint32_t><<<gm, T, 0, st>>>((const uint32_t*)skeys, m, flags.as<uint32_t>());
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    BISIM_TRY(scan_exclusive_u32(flags.as<uint32_t>(), flags.as<uint32_t>(), m, Ldev.as<uint32_t>(), st));
    uint32_t L_h = 0;
    BISIM_CUDA_TRY(cudaMemcpyAsync(&L_h, Ldev.p, 4, cudaMemcpyDeviceToHost, st));
    BISIM_CUDA_TRY(cudaStreamSynchronize(st));
    p->L = m ? (int64_t)L_h : 0;
    const int64_t L = p->L;

    BISIM_TRY(p->slot_src.alloc(4 * (size_t)L, st));
    BISIM_TRY(p->slot_act.alloc(4 * (size_t)L, st));
    BISIM_TRY(p->off.alloc(4 * ((size_t)n + 1), st));
    BISIM_TRY(p->in_ptr.alloc(4 * ((size_t)n + 1), st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->off.p, 0, 4 * ((size_t)n + 1), st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->in_ptr.p, 0, 4 * ((size_t)n + 1), st));
    DevMem tkey, tval;
    BISIM_TRY(tkey.alloc(4 * (size_t)m, st));
    BISIM_TRY(tval.alloc(8 * (size_t)m, st));
    if (wide)
        k_slots<uint64_t><<<gm, T, 0, st>>>((const uint64_t*)skeys, sdst, flags.as<uint32_t>(), m, A,
                                            p->slot_src.as<int32_t>(), p->slot_act.as<int32_t>(),
                                            tkey.as<uint32_t>(), tval.as<uint64_t>(),
                                            p->off.as<uint32_t>(), p->in_ptr.as<uint32_t>());
    else
        k_slots<uint32_t><<<gm, T, 0, st>>>((const uint32_t*)skeys, sdst, flags.as<uint32_t>(), m, A,
                                            p->slot_src.as<int32_t>(), p->slot_act.as<int32_t>(),
                                            tkey.as<uint32_t>(), tval.as<uint64_t>(),
                                            p->off.as<uint32_t>(), p->in_ptr.as<uint32_t>());
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    keys.release(); keys_alt.release(); vals.release(); vals_alt.release(); flags.release();
    // off = exclusive sum of nr_marks (off[n] = L); in_ptr likewise over in-degrees
    BISIM_TRY(scan_exclusive_u32(p->off.as<uint32_t>(), p->off.as<uint32_t>(), (int64_t)n + 1,
                                 nullptr, st));
    BISIM_TRY(scan_exclusive_u32(p->in_ptr.as<uint32_t>(), p->in_ptr.as<uint32_t>(), (int64_t)n + 1,
                                 nullptr, st));

    // a3: incoming transitions grouped by target
    {
        DevMem cursor;
        BISIM_TRY(cursor.alloc(4 * ((size_t)n + 1), st));
        BISIM_CUDA_TRY(cudaMemcpyAsync(cursor.p, p->in_ptr.p, 4 * ((size_t)n + 1), cudaMemcpyDeviceToDevice, st));
        BISIM_TRY(p->in_edge.alloc(8 * (size_t)m, st));
        k_csr_scatter<<<gm, T, 0, st>>>(tkey.as<uint32_t>(), tval.as<uint64_t>(), m, cursor.as<uint32_t>(),
                                        p->in_edge.as<uint64_t>());
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
    }
    tkey.release();
    tval.release();

    return BISIM_OK;
}

// a2 + a3 from the label sets recorded by k_validate_count (see there).
// Bins of the incoming-transition CSR: 2^bin_bits targets each, at most
// CSR_MAX_BINS of them, whose counters fit in shared memory (2^15 targets:
// 128 KB); 0 when n needs more (the CSR then takes one atomic per transition).
static int csr_bin_bits(int32_t n) {
    int bin_bits = 11;
    while (((int64_t)n + ((int64_t)1 << bin_bits) - 1) >> bin_bits > CSR_MAX_BINS) bin_bits++;
    return bin_bits <= 15 ? bin_bits : 0;
}

// a2 + a3 from the label sets recorded by k_validate_count (see there). With
// bin_cnt the validation counted transitions per target bin (bin_bits) and
// the CSR passes write in_ptr; otherwise it counted in-degrees into in_ptr.
static int slots_from_masks(bisim_plan_s* p, const int32_t* src, const int32_t* act, const int32_t* dst,
                            const uint32_t* amask, int mask_words, int vec, const uint32_t* bin_cnt,
                            int bin_bits) {
    const int32_t n = p->n;
    const int64_t m = p->m;
    cudaStream_t st = p->st;
    const unsigned gn = grid_for(n, T);
    uint32_t* off = p->off.as<uint32_t>();
    if (n) {
        k_mask_count<<<gn, T, 0, st>>>(amask, n, mask_words, off);
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
    }
    // off = exclusive sum of nr_marks (off[n] = L); in_ptr likewise over in-degrees
    BISIM_TRY(scan_exclusive_u32(off, off, (int64_t)n + 1, nullptr, st));
    if (!bin_cnt)
        BISIM_TRY(scan_exclusive_u32(p->in_ptr.as<uint32_t>(), p->in_ptr.as<uint32_t>(), (int64_t)n + 1, nullptr,
                                     st));
    uint32_t L_h = 0;
    BISIM_CUDA_TRY(cudaMemcpyAsync(&L_h, off + n, 4, cudaMemcpyDeviceToHost, st));
    BISIM_CUDA_TRY(cudaStreamSynchronize(st));
    p->L = (int64_t)L_h;
    BISIM_TRY(p->in_edge.alloc(8 * (size_t)m, st));
    if (!m) return BISIM_OK;
    if (bin_cnt) {
        const int nbins = (int)(((int64_t)n + ((int64_t)1 << bin_bits) - 1) >> bin_bits);
        DevMem bin_cursor, rec_t, rec_v, sinfo;
        if (mask_words == 1) {
            BISIM_TRY(sinfo.alloc(8 * (size_t)n, st));
            k_pack_sinfo<<<gn, T, 0, st>>>(off, amask, n, sinfo.as<unsigned long long>());
            BISIM_LAUNCHED();
        }
        BISIM_TRY(bin_cursor.alloc(4 * (size_t)nbins, st));
        BISIM_TRY(rec_t.alloc(4 * (size_t)m, st));
        BISIM_TRY(rec_v.alloc(8 * (size_t)m, st));
        // the bins' first records: exclusive scan of the per-bin counts
        BISIM_TRY(scan_exclusive_u32(bin_cnt, bin_cursor.as<uint32_t>(), nbins, nullptr, st));
        const int64_t tile = CSR_A_TILE;
        BISIM_CUDA_TRY(cudaFuncSetAttribute(k_csr_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CSR_A_SMEM));
        k_csr_bin<<<(unsigned)((m + tile - 1) / tile), CSR_A_THREADS, CSR_A_SMEM, st>>>(
            src, act, dst, m, amask, off, mask_words, sinfo.p ? sinfo.as<unsigned long long>() : nullptr, bin_bits,
            nbins, bin_cursor.as<uint32_t>(), rec_t.as<uint32_t>(), rec_v.as<unsigned long long>());
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        // bin_cursor now holds each bin's end
        const size_t smem = sizeof(uint32_t) << bin_bits;
        BISIM_CUDA_TRY(cudaFuncSetAttribute(k_csr_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_csr_place<<<nbins, CSR_B_THREADS, smem, st>>>(bin_cursor.as<uint32_t>(), n, m, bin_bits,
                                                        rec_t.as<uint32_t>(), rec_v.as<unsigned long long>(),
                                                        p->in_ptr.as<uint32_t>(), p->in_edge.as<unsigned long long>());
        BISIM_LAUNCHED();
        BISIM_CUDA_TRY(cudaGetLastError());
        return BISIM_OK;
    }
    // very many states: one returning atomic per transition on a cursor per target
    DevMem cursor;
    BISIM_TRY(cursor.alloc(4 * ((size_t)n + 1), st));
    BISIM_CUDA_TRY(cudaMemcpyAsync(cursor.p, p->in_ptr.p, 4 * ((size_t)n + 1), cudaMemcpyDeviceToDevice, st));
    k_mask_csr<<<grid_for(m, T), T, 0, st>>>(src, act, dst, m, amask, off, mask_words, vec,
                                             cursor.as<uint32_t>(), p->in_edge.as<unsigned long long>());
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    return BISIM_OK;
}

int ensure_slot_arrays(bisim_plan_s* p) {
    if (p->slot_src.p || !p->amask.p || p->L == 0) return BISIM_OK;
    cudaStream_t st = p->st;
    BISIM_TRY(p->slot_src.alloc(4 * (size_t)p->L, st));
    BISIM_TRY(p->slot_act.alloc(4 * (size_t)p->L, st));
    k_mask_slots<<<grid_for(p->n, T), T, 0, st>>>(p->amask.as<uint32_t>(), p->off.as<uint32_t>(), p->n,
                                                  p->mask_words, p->slot_src.as<int32_t>(),
                                                  p->slot_act.as<int32_t>());
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    return BISIM_OK;
}

int plan_build(bisim_plan_s* p, const int32_t* src, const int32_t* act, const int32_t* dst,
               const int32_t* init) {
    const int32_t n = p->n;
    const int64_t m = p->m;
    const int32_t A = p->A;
    cudaStream_t st = p->st;

    BISIM_TRY(p->ctrl.alloc(sizeof(bisim_ctrl), st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->ctrl.p, 0, sizeof(bisim_ctrl), st));
    int* status = &p->ctrl.as<bisim_ctrl>()->status;

    // a1: validation and the set of labels that occur (with label sets of at
    // most MASK_WORDS_MAX words, the same pass records every state's label
    // set and every state's in-degree)
    DevMem used;
    BISIM_TRY(used.alloc(sizeof(uint32_t) * (size_t)A, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(used.p, 0, sizeof(uint32_t) * (size_t)A, st));
    const int vec = (((uintptr_t)src | (uintptr_t)dst | (uintptr_t)act) & 15u) == 0 ? 1 : 0;
    const int mask_words = (A + 31) / 32;
    const bool by_masks = mask_words <= MASK_WORDS_MAX && p->opts.slots == 0;
    DevMem amask_local, bin_cnt;
    DevMem& amask = by_masks ? p->amask : amask_local;
    const int bin_bits = by_masks && m > 0 ? csr_bin_bits(n) : 0;
    const int nbins = bin_bits ? (int)(((int64_t)n + ((int64_t)1 << bin_bits) - 1) >> bin_bits) : 0;
    if (by_masks) {
        p->mask_words = mask_words;
        if (bin_bits) {
            BISIM_TRY(bin_cnt.alloc(4 * (size_t)nbins, st));
            BISIM_CUDA_TRY(cudaMemsetAsync(bin_cnt.p, 0, 4 * (size_t)nbins, st));
        }
        BISIM_TRY(amask.alloc(4 * (size_t)mask_words * n, st));
        BISIM_TRY(p->off.alloc(4 * ((size_t)n + 1), st));
        BISIM_TRY(p->in_ptr.alloc(4 * ((size_t)n + 1), st));
        BISIM_CUDA_TRY(cudaMemsetAsync(amask.p, 0, 4 * (size_t)mask_words * n, st));
        BISIM_CUDA_TRY(cudaMemsetAsync(p->off.p, 0, 4 * ((size_t)n + 1), st));
        BISIM_CUDA_TRY(cudaMemsetAsync(p->in_ptr.p, 0, 4 * ((size_t)n + 1), st));
        k_validate_count<<<grid_for(std::max<int64_t>(m, n), T), T, 0, st>>>(
            src, act, dst, init, n, m, A, status, used.as<uint32_t>(), vec, mask_words, amask.as<uint32_t>(),
            p->in_ptr.as<uint32_t>(), bin_bits, nbins, bin_bits ? bin_cnt.as<uint32_t>() : nullptr);
    } else {
        k_validate<<<grid_for(std::max<int64_t>(m, n), T), T, 0, st>>>(src, act, dst, init, n, m, A,
                                                                       status, used.as<uint32_t>(), vec);
    }
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    std::vector<uint32_t> used_h((size_t)A);
    BISIM_CUDA_TRY(cudaMemcpyAsync(used_h.data(), used.p, sizeof(uint32_t) * (size_t)A,
                                   cudaMemcpyDeviceToHost, st));
    BISIM_TRY(read_ctrl(p));
    if (p->ctrl_h->status & ST_INVALID) {
        set_last_error("an input array entry is out of range");
        return BISIM_EINVAL;
    }
    std::vector<int32_t> labels_h;
    for (int32_t a = 0; a < A; a++)
        if (used_h[a]) labels_h.push_back(a);
    p->n_labels = (int64_t)labels_h.size();
    // the pair engine splits by one label per round and needs no preprocessing
    p->pre_rounds = p->opts.engine == BISIM_ENGINE_PAIR ? 0 : p->n_labels;

    if (by_masks) {
        BISIM_TRY(slots_from_masks(p, src, act, dst, amask.as<uint32_t>(), mask_words, vec,
                                   bin_bits ? bin_cnt.as<uint32_t>() : nullptr, bin_bits));
    } else {
        BISIM_TRY(slots_by_sort(p, src, act, dst, vec));
    }
    const int64_t L = p->L;

    if (!labels_h.empty()) {
        BISIM_TRY(p->labels.alloc(4 * labels_h.size(), st));
        BISIM_CUDA_TRY(cudaMemcpyAsync(p->labels.p, labels_h.data(), 4 * labels_h.size(),
                                       cudaMemcpyHostToDevice, st));
    }

    // refinement state
    BISIM_TRY(p->block.alloc(4 * (size_t)n, st));
    BISIM_TRY(p->block0.alloc(4 * (size_t)n, st));
    BISIM_TRY(p->mark.alloc(4 * (size_t)L, st));
    BISIM_TRY(p->lmark.alloc(4 * (size_t)n, st));
    BISIM_TRY(p->nl64.alloc(8 * (size_t)n, st));
    BISIM_TRY(p->unstable.alloc(4 * (size_t)n, st));
    BISIM_TRY(p->split.alloc((size_t)n, st));
    if (L) BISIM_CUDA_TRY(cudaMemsetAsync(p->mark.p, 0, 4 * (size_t)L, st));
    if (n) {
        BISIM_CUDA_TRY(cudaMemsetAsync(p->lmark.p, 0, 4 * (size_t)n, st));
        BISIM_CUDA_TRY(cudaMemsetAsync(p->nl64.p, 0xff, 8 * (size_t)n, st));
    }
    p->stamp = 0;

    // a4: initial leaders
    const unsigned gn = grid_for(n, T);
    if (n) {
        if (init) {
            int32_t* nl = p->block0.as<int32_t>();  // scratch for the election
            k_fill_i32<<<gn, T, 0, st>>>(nl, n, NONE);
            BISIM_LAUNCHED();
            k_init_min<<<gn, T, 0, st>>>(init, n, nl);
            BISIM_LAUNCHED();
            k_init_relabel<<<gn, T, 0, st>>>(init, n, nl, p->block.as<int32_t>());
            BISIM_LAUNCHED();
        } else {
            BISIM_CUDA_TRY(cudaMemsetAsync(p->block.p, 0, 4 * (size_t)n, st));
        }
        BISIM_CUDA_TRY(cudaGetLastError());
    }

    // a5: action-set preprocessing
    if (n && p->pre_rounds > 0) {
        uint32_t base;
        BISIM_TRY(reserve_stamps(p, p->pre_rounds, &base));
        BISIM_CUDA_TRY(cudaMemsetAsync(&p->ctrl.as<bisim_ctrl>()->barrier, 0, 8, st));
        LabelArgs a;
        a.n = n;
        a.L = L;
        a.n_labels = (int32_t)p->pre_rounds;
        a.labels = p->labels.as<int32_t>();
        a.block = p->block.as<int32_t>();
        a.lmark = p->lmark.as<uint32_t>();
        a.nl64 = p->nl64.as<unsigned long long>();
        a.split = p->split.as<uint8_t>();
        a.stamp0 = base;
        a.amask = nullptr;
        a.mask_words = (A + 31) / 32;
        if (by_masks) {
            a.amask = amask.as<uint32_t>();  // recorded by the validation pass
        } else if (a.mask_words <= MASK_WORDS_MAX) {  // up to 128 labels: 16 B or less per state
            BISIM_TRY(amask.alloc(4 * (size_t)a.mask_words * n, st));
            BISIM_CUDA_TRY(cudaMemsetAsync(amask.p, 0, 4 * (size_t)a.mask_words * n, st));
            k_label_masks<<<grid_for(L, T), T, 0, st>>>(p->slot_src.as<int32_t>(), p->slot_act.as<int32_t>(), L,
                                                        a.mask_words, amask.as<uint32_t>());
            BISIM_LAUNCHED();
            BISIM_CUDA_TRY(cudaGetLastError());
            a.amask = amask.as<uint32_t>();
        }
        const bool fused = a.amask && preprocess_fused(p);
        if (!fused) BISIM_TRY(ensure_slot_arrays(p));  // the literal label rounds walk the slots
        a.slot_src = p->slot_src.as<int32_t>();
        a.slot_act = p->slot_act.as<int32_t>();
        if (fused) {
            // the partition after every label round: one block per (initial
            // block, label set), led by its smallest state
            BISIM_CUDA_TRY(cudaEventRecord(p->evk0, st));
            BISIM_TRY(group_by_label_set(p, a.amask, a.mask_words));
            BISIM_CUDA_TRY(cudaEventRecord(p->evk1, st));
            BISIM_TRY(persistent_ms(p, &p->t_pre_ms));
        } else {
            a.gb.counter = &p->ctrl.as<bisim_ctrl>()->barrier;
            a.gb.status = status;
            a.gb.timeout_ns = (unsigned long long)(p->opts.timeout_ms > 0 ? p->opts.timeout_ms : 2000) * 1000000ull;
            void* args[] = {&a};
            int grid = 0;
            BISIM_TRY(launch_persistent((const void*)k_label_rounds, args, 512, p, &grid, 4));
            BISIM_TRY(persistent_ms(p, &p->t_pre_ms));
        }
        p->stamp = base + (uint32_t)p->pre_rounds;
    }
    if (n) BISIM_CUDA_TRY(cudaMemcpyAsync(p->block0.p, p->block.p, 4 * (size_t)n,
                                          cudaMemcpyDeviceToDevice, st));
    // |pi_0'|
    {
        unsigned long long* cnt = &p->ctrl.as<bisim_ctrl>()->count;
        BISIM_CUDA_TRY(cudaMemsetAsync(cnt, 0, 8, st));
        if (n) {
            k_count_leaders<<<gn, T, 0, st>>>(p->block0.as<int32_t>(), n, cnt);
            BISIM_LAUNCHED();
        }
        BISIM_CUDA_TRY(cudaGetLastError());
        BISIM_TRY(read_ctrl(p));
        p->initial_blocks = (int64_t)p->ctrl_h->count;
        int code = status_to_code(p->ctrl_h->status);
        if (code) {
            set_last_error("preprocessing rounds failed");
            return code;
        }
    }
    return BISIM_OK;
}

// The plan of a small LTS (one CTA in shared memory, see small_refine):
// validation as in plan_build, and a copy of the inputs, which bisim_refine
// reduces in one kernel launch.
int small_plan(bisim_plan_s* p, const int32_t* src, const int32_t* act, const int32_t* dst, const int32_t* init) {
    const int32_t n = p->n;
    const int64_t m = p->m;
    const int32_t A = p->A;
    cudaStream_t st = p->st;
    BISIM_TRY(p->ctrl.alloc(sizeof(bisim_ctrl), st));
    BISIM_CUDA_TRY(cudaMemsetAsync(p->ctrl.p, 0, sizeof(bisim_ctrl), st));
    DevMem used;
    BISIM_TRY(used.alloc(sizeof(uint32_t) * (size_t)A, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(used.p, 0, sizeof(uint32_t) * (size_t)A, st));
    const int vec = (((uintptr_t)src | (uintptr_t)dst | (uintptr_t)act) & 15u) == 0 ? 1 : 0;
    k_validate<<<grid_for(std::max<int64_t>(m, n), T), T, 0, st>>>(src, act, dst, init, n, m, A,
                                                                   &p->ctrl.as<bisim_ctrl>()->status,
                                                                   used.as<uint32_t>(), vec);
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    BISIM_TRY(p->small_in.alloc(4 * (3 * (size_t)m + (size_t)n), st));
    BISIM_TRY(p->small_res.alloc(8 * 8, st));
    int32_t* base = p->small_in.as<int32_t>();
    if (m) {
        BISIM_CUDA_TRY(cudaMemcpyAsync(base, src, 4 * (size_t)m, cudaMemcpyDeviceToDevice, st));
        if (act) BISIM_CUDA_TRY(cudaMemcpyAsync(base + m, act, 4 * (size_t)m, cudaMemcpyDeviceToDevice, st));
        BISIM_CUDA_TRY(cudaMemcpyAsync(base + 2 * m, dst, 4 * (size_t)m, cudaMemcpyDeviceToDevice, st));
    }
    if (init) BISIM_CUDA_TRY(cudaMemcpyAsync(base + 3 * m, init, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    p->small_has_act = act != nullptr;
    p->small_has_init = init != nullptr;
    BISIM_TRY(read_ctrl(p));
    if (p->ctrl_h->status & ST_INVALID) {
        set_last_error("an input array entry is out of range");
        return BISIM_EINVAL;
    }
    p->small = true;
    return BISIM_OK;
}

int write_output(bisim_plan_s* p, int32_t* out, int64_t* num_blocks) {
    const int32_t n = p->n;
    cudaStream_t st = p->st;
    if (n == 0) {
        *num_blocks = 0;
        return BISIM_OK;
    }
    const int32_t* block = p->block.as<int32_t>();
    const unsigned gn = grid_for(n, T);
    DevMem first, flag, tot;
    BISIM_TRY(first.alloc(4 * (size_t)n, st));
    BISIM_TRY(flag.alloc(4 * (size_t)n, st));
    BISIM_TRY(tot.alloc(4, st));
    k_fill_i32<<<gn, T, 0, st>>>(first.as<int32_t>(), n, NONE);
    BISIM_LAUNCHED();
    k_first_min<<<gn, T, 0, st>>>(block, n, first.as<int32_t>());
    BISIM_LAUNCHED();
    k_is_first<<<gn, T, 0, st>>>(block, first.as<int32_t>(), n, flag.as<uint32_t>());
    BISIM_LAUNCHED();
    BISIM_CUDA_TRY(cudaGetLastError());
    BISIM_TRY(scan_exclusive_u32(flag.as<uint32_t>(), flag.as<uint32_t>(), n, tot.as<uint32_t>(), st));
    if (p->opts.raw_labels)
        BISIM_CUDA_TRY(cudaMemcpyAsync(out, block, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    else {
        k_gather_ids<<<gn, T, 0, st>>>(block, first.as<int32_t>(), flag.as<uint32_t>(), n, out);
        BISIM_LAUNCHED();
    }
    BISIM_CUDA_TRY(cudaGetLastError());
    uint32_t nb = 0;
    BISIM_CUDA_TRY(cudaMemcpyAsync(&nb, tot.p, 4, cudaMemcpyDeviceToHost, st));
    BISIM_CUDA_TRY(cudaStreamSynchronize(st));
    *num_blocks = nb;
    return BISIM_OK;
}

}  // namespace bisim
