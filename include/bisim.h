/*
 * bisim.h - C ABI of the GB300 (sm_103a) strong-bisimulation library.
 *
 * The library computes the coarsest partition of the states of a labelled
 * transition system (LTS) that refines an initial partition and is a
 * bisimulation: the Bisimulation Coarsest Refinement Problem (BCRP) and, for
 * one action label, the Relational Coarsest Partition Problem (RCPP), as
 * stated in Section 2.2 of Martens, Groote, van den Haak, Hijma and Wijs,
 * "A linear parallel algorithm to compute bisimulation and relational
 * coarsest partitions" (arXiv:2105.11788). The method is the CRCW-PRAM
 * refinement of Sections 3 and 4 (Algorithms 2, 3, 4 and 5): every round
 * elects one splitter block, marks the (state, action) pairs that reach it,
 * and splits every block into the states whose marks equal the block
 * leader's and those whose marks differ, the latter led by a freshly elected
 * leader; rounds repeat until no block is unstable.
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers unless the name ends in _h (host).
 *    The caller owns them; the library never frees them.
 *  - Inputs are read only during the call that receives them.
 *  - All work is ordered on the CUDA stream given to bisim_plan (NULL = the
 *    legacy default stream). Calls synchronise that stream before returning
 *    because they report device-side errors.
 *  - Return value: BISIM_OK (0) or a negative BISIM_E* code. No exception
 *    crosses the ABI and the library never traps or aborts the device; after
 *    any error the plan (if one was returned) may still be destroyed.
 *  - Not thread-safe per plan: one host thread at a time per plan.
 */
#ifndef BISIM_H
#define BISIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BISIM_OK 0
#define BISIM_EINVAL (-1)   /* bad scalar argument or out-of-range array entry */
#define BISIM_ENOMEM (-2)   /* device memory allocation failed */
#define BISIM_ECUDA (-3)    /* a CUDA runtime call failed (see bisim_last_error) */
#define BISIM_EROUNDS (-4)  /* round cap exceeded (Theorem 3 bound; indicates a bug) */
#define BISIM_ETIMEOUT (-5) /* a grid-wide barrier wait exceeded its time limit */
#define BISIM_ENOTSUP (-6)  /* requested engine/option not supported for this input */

/* Refinement engines. */
#define BISIM_ENGINE_AUTO 0
/* Dense rounds as printed in Algorithms 3 and 5: every round scans all
 * states and mark slots; splitter = smallest unstable label and new leader =
 * smallest splitting state (the priority write rule of Section 2.1), so the
 * round count and the leader labels equal the lock-step PRAM program. */
#define BISIM_ENGINE_DENSE 1
/* Frontier rounds: states kept grouped by block; a round touches only the
 * splitter's members, their incoming transitions and the blocks of the
 * marked states. Splitters come from a FIFO worklist and new leaders are
 * elected by compare-and-swap (the arbitrary write rule). Same partition;
 * round count may differ and may vary between runs. */
#define BISIM_ENGINE_FRONTIER 2
/* (C, a)-pair rounds: Algorithm 2 applied with one action label at a time,
 * one mark flag per state, every write under the priority rule (splitter =
 * smallest unstable label, labels in increasing order, new leader =
 * smallest splitting state). Needs no action-set preprocessing (pre_rounds
 * is 0) and up to |Act| times as many rounds; a second, independent engine
 * for cross-checks. Single LTSs only (bisim_batch_plan rejects it). */
#define BISIM_ENGINE_PAIR 3
/* Reported in bisim_stats.engine only (not an option): a small LTS reduced by
 * one CTA in shared memory with the frontier engine's rounds (opts.small). */
#define BISIM_ENGINE_SMALL 4

typedef struct bisim_opts {
    int32_t engine;      /* BISIM_ENGINE_* (0 = auto) */
    int32_t rcpp_alg2;   /* 1: with |Act| = 1, follow Algorithm 2 (the splitter is
                            not set unstable again after a split); 0: Algorithm 3 */
    int32_t raw_labels;  /* 1: bisim_refine writes leader labels instead of
                            canonical ids (testing the election rule) */
    int32_t threads;     /* threads per CTA for the persistent kernels (0 = 512; the
                            one-CTA start of the frontier engine: 0 = 1024; a batch:
                            0 = 256) */
    int32_t ctas_per_sm; /* CTAs per SM for the persistent kernels (0 = 1) */
    int32_t test_hook;   /* testing only: 1 = CTA 0 of the refinement kernel
                            leaves before its first barrier, so the other CTAs'
                            barrier waits run out and BISIM_ETIMEOUT is returned */
    int64_t round_cap;   /* 0 = 3n + |Act| + 2 (Theorem 3 plus slack) */
    int64_t timeout_ms;  /* limit on one grid-barrier wait (0 = 2000 ms) */
    int32_t max_ctas;    /* cap on the CTAs of the persistent launches (0 = no cap;
                            fewer CTAs make the grid barrier cheaper) */
    int32_t light_edges; /* frontier engine: a round whose splitter has at most 32
                            members and at most this many incoming transitions runs
                            on one CTA without grid barriers (0 = 256; negative =
                            every round on the whole grid) */
    int32_t preprocess;  /* action-set preprocessing (Algorithm 5): 0 = auto (literal
                            rounds for the dense engine, else direct grouping);
                            1 = one round per label; 2 = direct grouping by
                            (initial block, label set) when |Act| <= 128. Same
                            partition; leader labels may differ */
    int32_t wide_threads;    /* batch: threads per CTA of a second, concurrent launch
                                that takes the largest LTSs (0 = single launch) */
    int32_t wide_min_states; /* batch: LTSs with at least this many states go to the
                                wide launch */
    int32_t splitters;       /* frontier engine: most splitters per round (0 = 8192 for
                                one LTS on the grid, at most 8 per thread of a CTA;
                                0 = 32 on the one-CTA start and 1 for a batch, at most
                                128 per CTA; 1 = one splitter per round, as in
                                Algorithm 3).
                                Splitters whose touched blocks overlap are deferred to
                                a later round */
    int32_t split_budget;    /* frontier engine, rounds with several splitters: at most
                                this many splitter states per warp (0 = 1 on the grid,
                                4 on the one-CTA start, 8 per CTA of a batch) */
    int32_t multi_min_states; /* batch: only LTSs with at least this many states take
                                 several splitters per round (0 = every LTS) */
    int32_t local_states;     /* frontier engine, one LTS: start on a single CTA with CTA
                                 barriers (the batch schedule on one LTS; threads 0 =
                                 1024, splitters 0 = 32, split_budget 0 = 4) and hand
                                 the rest to the hybrid schedule before a round whose
                                 splitters hold more than this many states.
                                 0 = sparse LTSs only (m <= 4n), 16384 states, and also
                                 hand off after 3 rounds in a row in which at least
                                 half of the splitters won or that took more than
                                 25 us each; negative = never (hybrid or grid
                                 schedule from the start) */
    int32_t peel;             /* frontier engine, grid rounds with several splitters:
                                 0 = several splitters may split one block in the same
                                 round when each of them marks exactly one member of
                                 it and not its leader (the members are split off one
                                 by one, as the iterations would do one after the
                                 other); -1 = every touched block is taken by one
                                 splitter per round */
    int32_t peel_items;       /* frontier engine, grid rounds with several splitters:
                                 at most this many splitters of one state per warp of
                                 the grid (0 = 96) */
    int32_t small;            /* engine auto or frontier with the default schedule: an
                                 LTS with |Act| <= 32 whose arrays fit in one CTA's
                                 shared memory (about 12 B per transition and 116 B
                                 per state, at most 227 KB: e.g. 1,000 states and
                                 9,000 transitions) is reduced by one kernel launch
                                 on one CTA (bisim_plan validates and keeps a copy
                                 of the inputs). 0 = when it fits, -1 = never */
    int32_t slots;            /* mark-slot layout (Section 4.1.1): 0 = from every state's
                                 label set when |Act| <= 128 (the validation pass
                                 records the label sets; no sort), else by sorting
                                 the transitions by (source, label); 1 = always by
                                 the sort. Same arrays */
} bisim_opts;

typedef struct bisim_stats {
    int64_t n, m, num_act;
    int64_t mark_length;    /* L: number of distinct (source, label) pairs */
    int64_t pre_rounds;     /* action-set preprocessing rounds (labels that occur) */
    int64_t initial_blocks; /* blocks after preprocessing (|pi_0'|) */
    int64_t rounds;         /* main-loop iterations incl. the final empty one */
    int64_t num_blocks;     /* blocks of the result */
    int64_t edges_visited;  /* incoming transitions walked by mark steps */
    int64_t states_visited; /* states whose marks were compared */
    double t_plan_ms;       /* device time of bisim_plan (sort, CSR, preprocessing) */
    double t_refine_ms;     /* device time of the last bisim_refine */
    double t_pre_ms;        /* device time of the preprocessing-round kernel */
    double t_main_ms;       /* device time of the main-loop kernel of the last refine */
    int64_t launches;       /* kernels launched by bisim_plan + the last bisim_refine */
    int32_t engine;         /* engine that ran */
    int32_t grid_ctas;      /* CTAs of the persistent launch */
    int64_t steps;          /* barrier-separated rounds incl. the final empty one; equals
                               rounds when every round takes one splitter */
    int64_t local_steps;    /* frontier engine, one LTS: of those, the rounds run on one CTA
                               before the grid took over (= steps when it never did) */
} bisim_stats;

typedef struct bisim_plan_s* bisim_plan_t;

/*
 * bisim_plan - validate an LTS and build everything the rounds need.
 *
 * Steps (all on the device): range checks of every array entry; the sort of
 * the transitions by (source, label) with the action_switch / order /
 * nr_marks / off arrays of Section 4.1.1 (Algorithm 4 and its scans; off is
 * the exclusive prefix sum of nr_marks, slot(s,a) = off(s) + order); the
 * incoming-transition index by target (CSR, each entry carrying its source
 * and mark slot); the initial leaders of Algorithm 2, lines 1-6 (the smallest
 * member of each initial block); and the action-set preprocessing of
 * Algorithm 5, one round per label that occurs, in increasing label order.
 *
 * n          number of states, 0 <= n < 2^31
 * m          number of transitions, 0 <= m < 2^31
 * num_act    number of action labels, >= 1
 * src, dst   int32 [m], values in [0, n)
 * act        int32 [m], values in [0, num_act); NULL means every label is 0
 * init_block int32 [n], values in [0, n) (the I_i of Section 3.2.2; states
 *            with equal values form one initial block); NULL = one block
 * opts       NULL = defaults
 * stream     cudaStream_t as void*, NULL = legacy default stream
 * out        receives the plan; the plan owns its device workspace until
 *            bisim_plan_destroy (about 40 bytes per transition and 80 bytes
 *            per state)
 * Errors: BISIM_EINVAL for bad scalars or any out-of-range entry (found on
 * the device), BISIM_ENOMEM, BISIM_ECUDA. On error *out is NULL.
 */
int bisim_plan(int32_t n, int64_t m, int32_t num_act, const int32_t* src, const int32_t* act,
               const int32_t* dst, const int32_t* init_block, const bisim_opts* opts,
               void* stream, bisim_plan_t* out);

/*
 * bisim_refine - run the refinement rounds (the while-loop of Algorithm 3,
 * or Algorithm 2 with rcpp_alg2) from the preprocessed partition and write
 * the result. May be called again on the same plan; every call starts from
 * the partition left by bisim_plan.
 *
 * out_block  int32 [n] device: block id per state, canonical (blocks
 *            numbered 0.. in order of their smallest state), or the leader
 *            label of the state's block if opts.raw_labels was set.
 * stats      NULL or receives counters and device times.
 * Errors: BISIM_EROUNDS, BISIM_ETIMEOUT, BISIM_ECUDA, BISIM_EINVAL (NULL plan).
 */
int bisim_refine(bisim_plan_t plan, int32_t* out_block, bisim_stats* stats);

/* Release the plan's device memory (stream-ordered). NULL is ignored. */
void bisim_plan_destroy(bisim_plan_t plan);

/*
 * bisim_plan_arrays - copy a plan's mark-slot layout and incoming-transition
 * index to host memory (for checking them against Section 4.1.1; not needed
 * to reduce an LTS). With the transitions sorted by (source, label), off is
 * the exclusive prefix sum of nr_marks (off[n] = mark_length, Algorithm 4's
 * off read as start offsets), and the slot of a transition s -a-> t is
 * off(s) + order, order = the number of labels of s smaller than a.
 * off_h       int32 [n + 1] or NULL
 * slot_src_h  int32 [mark_length] or NULL: the state owning each slot (plans
 *             that took the slots from label sets fill these on this call)
 * slot_act_h  int32 [mark_length] or NULL: its label
 * in_ptr_h    int32 [n + 1] or NULL: incoming transitions of t are entries
 *             in_ptr[t] .. in_ptr[t+1]-1 of in_edge
 * in_edge_h   int64 [m] or NULL: (source << 32) | slot per incoming
 *             transition (the order inside one target's range is arbitrary)
 * mark_length NULL or receives mark_length
 * Synchronises the plan's stream. Errors: BISIM_EINVAL (plan NULL), BISIM_ECUDA.
 */
int bisim_plan_arrays(bisim_plan_t plan, int32_t* off_h, int32_t* slot_src_h, int32_t* slot_act_h,
                      int32_t* in_ptr_h, int64_t* in_edge_h, int64_t* mark_length);

/*
 * bisim_reduce_host - one whole reduction from HOST buffers: copies the
 * arrays to the device (on three streams of the library at once, ordered
 * before the plan on `stream`), plans, refines, copies the canonical block
 * ids back into out_block_h, synchronises `stream` and releases everything.
 * Same arguments and errors as bisim_plan + bisim_refine; all pointers
 * ending in _h are host memory (pinned memory gives faster copies) and must
 * stay valid until the call returns; act_h and init_h may be NULL.
 */
int bisim_reduce_host(int32_t n, int64_t m, int32_t num_act, const int32_t* src_h,
                      const int32_t* act_h, const int32_t* dst_h, const int32_t* init_h,
                      int32_t* out_block_h, const bisim_opts* opts, void* stream,
                      bisim_stats* stats);

/* Per-LTS results of bisim_batch_refine. */
typedef struct bisim_batch_inst {
    int64_t rounds;     /* main-loop iterations of this LTS, incl. the final empty one */
    int64_t num_blocks; /* blocks of its result */
} bisim_batch_inst;

/*
 * bisim_batch_plan - plan k LTSs at once (not in the paper: a throughput
 * mode). The LTSs are packed into one union whose state ranges are disjoint;
 * the union's initial partition separates the LTSs, so its coarsest stable
 * refinement is the union of theirs, and one sort, one CSR and one set of
 * preprocessing rounds (Algorithm 5, one per label occurring anywhere) serve
 * the batch.
 *
 * k            number of LTSs, >= 1
 * state_off_h  host int64 [k+1]: LTS i has states [state_off_h[i], state_off_h[i+1])
 *              of the concatenated state arrays; state_off_h[0] = 0, total < 2^31
 * trans_off_h  host int64 [k+1]: LTS i has transitions [trans_off_h[i], trans_off_h[i+1])
 * num_act_h    host int32 [k]: label count of each LTS (>= 1)
 * src, dst     device int32 [total m]: LOCAL state numbers in [0, n_i)
 * act          device int32 [total m]: local labels in [0, num_act_h[i]), or NULL (all 0)
 * init_block   device int32 [total n]: local initial labels in [0, n_i), or NULL
 * Same ownership, stream and error rules as bisim_plan.
 */
int bisim_batch_plan(int32_t k, const int64_t* state_off_h, const int64_t* trans_off_h,
                     const int32_t* num_act_h, const int32_t* src, const int32_t* act,
                     const int32_t* dst, const int32_t* init_block, const bisim_opts* opts,
                     void* stream, bisim_plan_t* out);

/*
 * bisim_batch_refine - refine every LTS of a batch plan in one launch: each
 * CTA takes one LTS at a time (largest first) and runs the frontier rounds
 * for it with CTA-local barriers and a CTA-local worklist, so different LTSs
 * proceed concurrently on different SMs. The launch is not cooperative and
 * can overlap other work on the device.
 *
 * out_block  device int32 [total n]: canonical ids local to each LTS (blocks
 *            of LTS i numbered 0.. by their smallest state), or union leader
 *            labels with opts.raw_labels
 * stats      NULL or aggregate counters (rounds = sum over the LTSs)
 * inst_h     NULL or host array of k per-LTS results
 * Errors as bisim_refine; BISIM_EINVAL if the plan is not a batch plan.
 */
int bisim_batch_refine(bisim_plan_t plan, int32_t* out_block, bisim_stats* stats,
                       bisim_batch_inst* inst_h);

/*
 * bisim_barrier_cost - diagnostic: time `iters` back-to-back grid-wide
 * barriers (the synchronisation the persistent kernels use between the steps
 * of a round; §5 of the paper needs four such points per iteration, the
 * frontier engine two) in one cooperative launch of `ctas` CTAs of `threads`
 * threads, and return the average device time per barrier in nanoseconds.
 * Errors: BISIM_EINVAL (bad argument or more CTAs than can be co-resident),
 * BISIM_ECUDA, BISIM_ETIMEOUT.
 */
int bisim_barrier_cost(int32_t ctas, int32_t threads, int32_t iters, void* stream,
                       double* ns_per_barrier);

/*
 * bisim_phase_times / bisim_phase_reset - diagnostic: per-phase device time of
 * the frontier engine's hybrid rounds, accumulated over launches since the
 * last reset by thread 0 of CTA 0 with the global timer. Only a library built
 * with -DBISIM_PHASE_TIMERS records them; the default build returns
 * BISIM_ENOTSUP (the paper has no counterpart; this is a profiling aid).
 * out16: host array of 16 uint64 entries, nanoseconds unless noted:
 *   0 selection, 1 publish to parked CTAs, 2 claim pass, 3 barrier after it,
 *   4 mark pass, 5 barrier after it, 6 split pass, 7 barrier after it,
 *   8 one-splitter grid rounds (whole round), 9 multi-splitter rounds (count),
 *   10 one-splitter rounds (count), 11 rounds run by CTA 0 alone (count),
 *   12 splitters selected by grid rounds (count), 13 their states (count),
 *   14 touched blocks (count), 15 time between rounds.
 * Both synchronise the device. Errors: BISIM_EINVAL (out16 NULL), BISIM_ECUDA,
 * BISIM_ENOTSUP.
 */
int bisim_phase_times(uint64_t* out16);
int bisim_phase_reset(void);

/*
 * bisim_phase_trace - diagnostic, same build and purpose as bisim_phase_times:
 * a per-round record of the hybrid rounds of the last launches (rounds
 * 1 .. 65536, later rounds are not recorded; cleared by bisim_phase_reset).
 * out: host array of 6 * max_rounds uint32, per round: splitters selected,
 * worklist entries before the selection, touched blocks, splitter iterations
 * carried out, round time in ns (CTA 0's view), 1 if the round ran on CTA 0
 * alone. Synchronises the device. Errors: BISIM_EINVAL (out NULL or
 * max_rounds < 0), BISIM_ECUDA, BISIM_ENOTSUP (default build).
 */
int bisim_phase_trace(uint32_t* out, int32_t max_rounds);

/*
 * Device memory of the library (the paper has no counterpart; this is for
 * admission control by a serving loop). Plans allocate stream-ordered from the
 * current device's default memory pool, whose release threshold the library
 * raises so that memory a destroyed plan frees is kept for the next plan
 * instead of being returned at every synchronisation. So the pool can hold
 * more than the plans alive use:
 *
 * bisim_pool_usage      used: bytes of the pool in use by live allocations;
 *                       used_high: the most in use since the last
 *                       bisim_pool_reset_high; reserved: bytes the pool holds
 *                       from the device, in use or not. Any pointer may be NULL.
 * bisim_pool_reset_high restarts the high-water mark at the current use.
 * bisim_pool_trim       synchronises the device, then returns the pool's unused
 *                       memory to the device until at most keep_bytes of
 *                       unused memory stay reserved.
 * These act on the default pool of the current device, which other users of
 * that pool (cudaMallocAsync with the default pool) share.
 * Errors: BISIM_ECUDA.
 */
int bisim_pool_usage(uint64_t* used, uint64_t* used_high, uint64_t* reserved);
int bisim_pool_reset_high(void);
int bisim_pool_trim(uint64_t keep_bytes);

/* Largest n accepted by bisim_canonical_ids_noalloc. */
#define BISIM_NOALLOC_MAX_N (1 << 20)

/*
 * bisim_canonical_ids_noalloc - renumber block labels canonically without
 * allocating any memory. The paper has no counterpart: this is a service for
 * callers that cannot allocate device memory, e.g. because a framework's
 * caching allocator owns the whole device budget, or because a cudaMalloc /
 * cudaFree in a latency-critical loop would synchronise the device.
 *
 * Same result as the output step of bisim_refine: given any labelling of
 * states (labels[i] in [0, n), equal labels = same block), out_ids[i] is the
 * block's rank when blocks are ordered by their smallest state.
 *
 * labels       int32 [n] device, values in [0, n) (caller-owned, read only)
 * n            0 <= n <= BISIM_NOALLOC_MAX_N (1,048,576); larger n returns
 *              BISIM_EINVAL without touching anything
 * out_ids      int32 [n] device (caller-owned), written
 * num_blocks_h NULL or host int32 receiving the number of blocks
 * stream       cudaStream_t as void*, NULL = legacy default stream; the call
 *              synchronises it before returning
 *
 * Scratch: a fixed file-scope device array of about 8 MB (two int32 arrays of
 * BISIM_NOALLOC_MAX_N plus counters), held on every GPU that loads the
 * library until the process exits. The call makes no cudaMalloc, cudaFree or
 * other allocating call. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture. Every call on a device shares the
 * one array and resets the parts that must start at zero; calls that overlap
 * on the GPU (other streams, other host threads) race on it and must be
 * serialised by the caller.
 * Errors (return code only; bisim_last_error is not updated): BISIM_EINVAL
 * (n out of range, NULL pointer, or a label outside [0, n)), BISIM_ETIMEOUT,
 * BISIM_ECUDA, BISIM_ENOTSUP (device ordinal >= 64).
 */
int bisim_canonical_ids_noalloc(const int32_t* labels, int32_t n, int32_t* out_ids,
                                int32_t* num_blocks_h, void* stream);

/* Static description of an error code. */
const char* bisim_strerror(int code);

/* Detail of the last error raised on the calling host thread ("" if none). */
const char* bisim_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t bisim_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BISIM_H */
