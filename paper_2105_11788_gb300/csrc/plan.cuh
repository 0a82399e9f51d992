// Internal plan object shared by the plan builder, the refinement engines
// and the C ABI.
#pragma once

#include <vector>

#include "common.cuh"
#include "prim.cuh"

// Device control block: barrier counter, status word, splitter election
// slots, worklist cursors and counters. Zeroed (then initialised) before
// every persistent launch.
struct bisim_ctrl {
    unsigned long long barrier;  // grid barrier counter (monotonic)
    int status;                  // ST_* bits
    int sel[2];                  // priority splitter election, double-buffered by round parity
    int pad0;
    long long rounds;            // main-loop iterations incl. the final empty one
    long long edges;             // incoming transitions walked by mark steps
    long long states;            // states whose marks were compared
    unsigned long long count;    // scratch counter for host queries
    int n_touched[2];            // frontier: warp-list length by round parity
    int n_mid[2];                // frontier: CTA-list length by round parity
    unsigned long long bq_tail[32];  // frontier worklist: pushes per size bucket
    int next_inst;                   // batch engine: next LTS to take (narrow launch)
    int next_inst_wide;              // batch engine: next LTS of the wide launch
    // hybrid engine: CTA 0 publishes heavy rounds to the parked CTAs
    unsigned long long cmd_seq;      // number of commands published
    unsigned long long heartbeat;    // rounds CTA 0 has finished (progress for the parked CTAs' limit)
    int cmd_C;                       // splitter of the published heavy round, -1 = stop, -2 = several
    unsigned cmd_stamp;              // its round stamp
    int cmd_K;                       // number of splitters of a published multi-splitter round
    int pad3;
    long long commits;               // splitter iterations carried out (multi-splitter schedules)
    unsigned long long cmd_heads[32];  // worklist heads after the published round's selection
    long long local_rounds;            // one LTS on one CTA: splitter iterations + 1
    int handoff;                       // one LTS on one CTA: 1 = the grid takes over
    int pad4;
    unsigned long long start_heads[32];  // worklist heads at the hand-off to the grid
    // hybrid engine, a published round with several splitters: its splitters of
    // one state, taken by position from the ring of size bucket 0
    int cmd_K0;                          // how many
    int cmd_peel;                        // 1: the published round is a peel round
    unsigned long long cmd_h0;           // ring-0 head before them
    int n_defer[2];                      // hybrid sweep rounds: labels pushed back untouched, by round parity
};

// Most splitters one multi-splitter round takes: grid rounds of the hybrid
// schedule, and CTA rounds of the batch schedule.
constexpr int BISIM_KMAX_GRID = 8192;
constexpr int BISIM_KMAX_CTA = 128;
// A sparse single LTS starting on one CTA moves to the grid before a round
// whose splitters hold more than BISIM_HANDOFF_STATES states, or after
// BISIM_HANDOFF_BUSY rounds in a row in which half the splitters won, or
// that took longer than BISIM_HANDOFF_ROUND_NS each (about a grid round)
constexpr int BISIM_HANDOFF_STATES = 16384;
constexpr int BISIM_HANDOFF_BUSY = 3;
constexpr unsigned long long BISIM_HANDOFF_ROUND_NS = 25000;

// Frontier worklist: one FIFO ring of n entries per size bucket
// floor(log2(block size)); the splitter is taken from the lowest non-empty
// bucket, so small blocks are split on first (any unstable block is a valid
// splitter under the arbitrary write rule).
constexpr int BISIM_BUCKETS = 32;

struct bisim_plan_s {
    int32_t n = 0;
    int64_t m = 0;
    int32_t A = 1;
    int64_t L = 0;
    cudaStream_t st = nullptr;
    bisim_opts opts{};
    int sm_count = 0;
    int dev = 0;

    // read-only after planning
    bisim::DevMem off;       // int32 [n+1]: first mark slot of each state; off[n] = L
    bisim::DevMem in_ptr;    // int32 [n+1]: CSR of incoming transitions by target
    bisim::DevMem in_edge;   // uint64 [m]: (source << 32) | mark slot of the transition
    bisim::DevMem slot_src;  // int32 [L]: state owning each mark slot
    bisim::DevMem slot_act;  // int32 [L]: label of each mark slot
    // label set of every state (mask_words 32-bit words) when the slots came
    // from label sets; slot_src / slot_act are then filled on first use
    bisim::DevMem amask;
    int mask_words = 0;
    bisim::DevMem labels;    // int32 [n_labels]: labels that occur, increasing
    bisim::DevMem block0;    // int32 [n]: leader labels after preprocessing

    // refinement state
    bisim::DevMem block;     // int32 [n]: current leader label per state
    bisim::DevMem mark;      // uint32 [L]: round stamp of the last mark of each slot
    bisim::DevMem lmark;     // uint32 [n]: round stamp of the last label mark per state
    bisim::DevMem nl64;      // uint64 [n]: new-leader election word per label
    bisim::DevMem unstable;  // uint32 [n]: unstable flag per label
    bisim::DevMem split;     // uint8 [n]
    bisim::DevMem ctrl;      // bisim_ctrl
    bisim_ctrl* ctrl_h = nullptr;  // pinned mirror

    // frontier engine state (allocated on first use)
    bool frontier_ready = false;
    bisim::DevMem elems;     // int32 [n]: states grouped by block
    bisim::DevMem loc;       // int32 [n]: position of each state in elems
    bisim::DevMem bbeg;      // int32 [n]: member range [bbeg, bend) of each label
    bisim::DevMem bend;      // int32 [n]
    bisim::DevMem mcnt;      // int32 [n]: marked members per label in the current round
    bisim::DevMem mscr;      // int32 [n]: by position, marked members of each touched block
    bisim::DevMem yscr;      // int32 [n]: by position, swap-pairing scratch
    bisim::DevMem smark;     // uint32 [n]: round stamp of the last mark of each state
    bisim::DevMem kmark;     // uint32 [n]: round stamp of membership in a kept part
    bisim::DevMem tlist;     // int32 [2n]: touched-label lists (warp, CTA)
    bisim::DevMem queue;     // int32 [BISIM_BUCKETS * n]: FIFO rings of unstable labels
    bisim::DevMem claim;     // uint64 [n]: per label, (~stamp << 32 | splitter index) of the round's claim
    bisim::DevMem bspl;      // int32 [n]: per touched label, the splitter that touched it
    bisim::DevMem msel;      // int32 [2 * KMAX_GRID + 1] + uint32 [KMAX_GRID]: published splitters,
                             // their size prefix, and the round in which each lost a claim
    bisim::DevMem minx;      // uint64 [n]: per label, the least key of this round's exclusive claims
    bisim::DevMem smark64;   // uint64 [n]: per state, the least key of the splitters that peel it
    bisim::DevMem lostl;     // uint32 [n]: per splitter label, the round in which it lost a claim

    // batch plans: k LTSs over disjoint state ranges of one union LTS
    int32_t batch_k = 0;
    std::vector<int64_t> state_off_h;   // [k+1]
    std::vector<int32_t> batch_act_h;   // [k] label count of each LTS
    bisim::DevMem state_off;            // int64 [k+1]
    bisim::DevMem batch_act;            // int32 [k]
    bisim::DevMem batch_order;          // int32 [k]: LTS indices, largest first
    bisim::DevMem inst_rounds;          // int64 [k]
    std::vector<int32_t> batch_order_h; // [k]
    cudaStream_t aux_stream = nullptr;  // second stream of the split batch schedule
    cudaEvent_t aux_event = nullptr;

    // small LTSs (one CTA, shared memory): the inputs kept by the plan
    // (src, act, dst, init back to back), and the kernel's results
    bool small = false;
    bool small_has_act = false, small_has_init = false;
    bisim::DevMem small_in;
    bisim::DevMem small_res;            // int64 [8]

    uint32_t stamp = 0;      // last round stamp used (marks are never cleared)
    int64_t pre_rounds = 0;  // action-set preprocessing rounds run (0 for the pair engine)
    int64_t n_labels = 0;    // labels that occur
    int64_t initial_blocks = 0;
    double t_plan_ms = 0;
    double t_pre_ms = 0;
    long long plan_launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;    // whole call
    cudaEvent_t evk0 = nullptr, evk1 = nullptr;  // around the persistent kernel
    bisim_stats last{};

    ~bisim_plan_s();
};

namespace bisim {

int plan_build(bisim_plan_s* p, const int32_t* src, const int32_t* act, const int32_t* dst,
               const int32_t* init);
int refine_dense(bisim_plan_s* p, bisim_stats* st);
int refine_frontier(bisim_plan_s* p, bisim_stats* st);
int refine_pair(bisim_plan_s* p, bisim_stats* st);
// CTA-per-LTS frontier rounds over a batch plan; rounds[i] = iterations of LTS i
int refine_frontier_batch(bisim_plan_s* p, bisim_stats* st, std::vector<long long>& rounds);
int write_output(bisim_plan_s* p, int32_t* out_block, int64_t* num_blocks);
// small LTSs: one CTA holds the whole reduction in shared memory
bool small_fits(const bisim_plan_s* p);
int small_plan(bisim_plan_s* p, const int32_t* src, const int32_t* act, const int32_t* dst, const int32_t* init);
int small_refine(bisim_plan_s* p, int32_t* out_block, bisim_stats* st);
bool preprocess_fused(const bisim_plan_s* p);
int group_by_label_set(bisim_plan_s* p, const uint32_t* amask, int mask_words);

// Reserve `rounds` fresh stamps (resetting stamped arrays if the 32-bit
// stamp space would wrap); returns the first stamp minus one.
int reserve_stamps(bisim_plan_s* p, int64_t rounds, uint32_t* base);

// Cooperative launch on one SM-multiple grid, bracketed by evk0 / evk1.
int launch_persistent(const void* fn, void** args, int threads, bisim_plan_s* p, int* grid_out,
                      int per_sm_default = 1, size_t dyn_smem = 0);
// Device time between evk0 and evk1 of the last persistent launch.
int persistent_ms(bisim_plan_s* p, double* ms);
int read_ctrl(bisim_plan_s* p);
// Device, SM count, pool settings, the pinned control mirror and the timing
// events of a new plan (the last three reused from destroyed plans).
int device_setup(bisim_plan_s* p);
// Fill slot_src / slot_act from the label sets if the plan has not yet.
int ensure_slot_arrays(bisim_plan_s* p);

}  // namespace bisim
