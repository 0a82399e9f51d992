// C ABI entry points (include/bisim.h): argument checks, plan lifetime,
// engine selection, device timing and error reporting.
#include <array>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "plan.cuh"

namespace bisim {

static thread_local std::string g_last_error;
thread_local long long g_launches = 0;

void set_last_error(const std::string& s) { g_last_error = s; }

}  // namespace bisim

using namespace bisim;

static int choose_engine(const bisim_plan_s* p) {
    int e = p->opts.engine;
    if (e == BISIM_ENGINE_DENSE || e == BISIM_ENGINE_FRONTIER || e == BISIM_ENGINE_PAIR) return e;
    return BISIM_ENGINE_FRONTIER;
}

static void fill_static_stats(const bisim_plan_s* p, bisim_stats* s) {
    s->n = p->n;
    s->m = p->m;
    s->num_act = p->A;
    s->mark_length = p->L;
    s->pre_rounds = p->pre_rounds;
    s->initial_blocks = p->initial_blocks;
    s->t_plan_ms = p->t_plan_ms;
    s->t_pre_ms = p->t_pre_ms;
}

namespace {

// Streams for the input copies of bisim_reduce_host, three per device,
// created on first use and kept for the process.
std::mutex g_copy_mu;
std::vector<std::pair<int, std::array<cudaStream_t, 3>>> g_copy_streams;

int copy_streams(cudaStream_t* cs) {
    int dev = 0;
    BISIM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_copy_mu);
    for (auto& e : g_copy_streams)
        if (e.first == dev) {
            for (int k = 0; k < 3; k++) cs[k] = e.second[k];
            return BISIM_OK;
        }
    std::array<cudaStream_t, 3> a{};
    for (int k = 0; k < 3; k++) BISIM_CUDA_TRY(cudaStreamCreateWithFlags(&a[k], cudaStreamNonBlocking));
    g_copy_streams.emplace_back(dev, a);
    for (int k = 0; k < 3; k++) cs[k] = a[k];
    return BISIM_OK;
}

// Events of one call (destroyed with it; a destroyed event that a stream
// still waits on is released once the wait completes).
struct EventSet {
    cudaEvent_t e[4] = {};
    int n = 0;
    int create(int k) {
        for (; n < k; n++) BISIM_CUDA_TRY(cudaEventCreateWithFlags(&e[n], cudaEventDisableTiming));
        return BISIM_OK;
    }
    ~EventSet() {
        for (int i = 0; i < n; i++) cudaEventDestroy(e[i]);
    }
};

}  // namespace

extern "C" {

const char* bisim_strerror(int code) {
    switch (code) {
        case BISIM_OK: return "ok";
        case BISIM_EINVAL: return "invalid argument or out-of-range array entry";
        case BISIM_ENOMEM: return "out of device memory";
        case BISIM_ECUDA: return "CUDA runtime error";
        case BISIM_EROUNDS: return "round cap exceeded";
        case BISIM_ETIMEOUT: return "grid barrier wait timed out";
        case BISIM_ENOTSUP: return "not supported";
        default: return "unknown error";
    }
}

const char* bisim_last_error(void) { return g_last_error.c_str(); }

int32_t bisim_version(void) { return 100; }

int bisim_plan(int32_t n, int64_t m, int32_t num_act, const int32_t* src, const int32_t* act,
               const int32_t* dst, const int32_t* init_block, const bisim_opts* opts, void* stream,
               bisim_plan_t* out) {
    if (!out) {
        set_last_error("out is NULL");
        return BISIM_EINVAL;
    }
    *out = nullptr;
    if (n < 0 || m < 0 || m > 0x7fffffffll || num_act < 1 || (m > 0 && (!src || !dst))) {
        set_last_error("bad scalar argument (need 0 <= n, 0 <= m < 2^31, num_act >= 1, src/dst)");
        return BISIM_EINVAL;
    }
    if (n == 0 && m > 0) {
        set_last_error("transitions given for an LTS without states");
        return BISIM_EINVAL;
    }
    if (opts && (opts->threads < 0 || opts->threads > 1024 || (opts->threads & 31))) {
        set_last_error("opts.threads must be a multiple of 32 in [32, 1024] (or 0)");
        return BISIM_EINVAL;
    }
    if (opts && (opts->engine < BISIM_ENGINE_AUTO || opts->engine > BISIM_ENGINE_PAIR)) {
        set_last_error("opts.engine must be one of BISIM_ENGINE_*");
        return BISIM_EINVAL;
    }
    bisim_plan_s* p = new (std::nothrow) bisim_plan_s();
    if (!p) return BISIM_ENOMEM;
    p->n = n;
    p->m = m;
    p->A = num_act;
    p->st = (cudaStream_t)stream;
    if (opts) p->opts = *opts;
    int rc = BISIM_OK;
    do {
        rc = device_setup(p);
        if (rc) break;
        cudaError_t e = cudaEventRecord(p->ev0, p->st);
        if (e != cudaSuccess) {
            set_last_error(std::string("cudaEventRecord: ") + cudaGetErrorString(e));
            rc = BISIM_ECUDA;
            break;
        }
        g_launches = 0;
        rc = small_fits(p) ? small_plan(p, src, act, dst, init_block) : plan_build(p, src, act, dst, init_block);
        p->plan_launches = g_launches;
        if (rc) break;
        float ms = 0;
        e = cudaEventRecord(p->ev1, p->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(p->ev1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p->ev0, p->ev1);
        if (e != cudaSuccess) {
            set_last_error(std::string("plan timing: ") + cudaGetErrorString(e));
            rc = BISIM_ECUDA;
            break;
        }
        p->t_plan_ms = ms;
    } while (0);
    if (rc) {
        cudaStreamSynchronize(p->st);
        delete p;
        return rc;
    }
    *out = p;
    return BISIM_OK;
}

int bisim_refine(bisim_plan_t p, int32_t* out_block, bisim_stats* stats) {
    if (!p || (p->n > 0 && !out_block)) {
        set_last_error("plan or out_block is NULL");
        return BISIM_EINVAL;
    }
    bisim_stats s;
    std::memset(&s, 0, sizeof(s));
    fill_static_stats(p, &s);
    if (p->n == 0) {
        if (stats) *stats = s;
        return BISIM_OK;
    }
    BISIM_CUDA_TRY(cudaEventRecord(p->ev0, p->st));
    g_launches = 0;
    int rc;
    if (p->small) {
        rc = small_refine(p, out_block, &s);
    } else {
        const int engine = choose_engine(p);
        rc = engine == BISIM_ENGINE_DENSE  ? refine_dense(p, &s)
             : engine == BISIM_ENGINE_PAIR ? refine_pair(p, &s)
                                           : refine_frontier(p, &s);
        if (rc == BISIM_OK) rc = write_output(p, out_block, &s.num_blocks);
    }
    s.launches = p->plan_launches + g_launches;
    if (rc == BISIM_OK) {
        float ms = 0;
        BISIM_CUDA_TRY(cudaEventRecord(p->ev1, p->st));
        BISIM_CUDA_TRY(cudaEventSynchronize(p->ev1));
        BISIM_CUDA_TRY(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        s.t_refine_ms = ms;
    }
    p->last = s;
    if (stats) *stats = s;
    return rc;
}

void bisim_plan_destroy(bisim_plan_t p) {
    if (!p) return;
    cudaStreamSynchronize(p->st);
    delete p;
}

int bisim_plan_arrays(bisim_plan_t p, int32_t* off_h, int32_t* slot_src_h, int32_t* slot_act_h, int32_t* in_ptr_h,
                      int64_t* in_edge_h, int64_t* mark_length) {
    if (!p) {
        set_last_error("bad argument");
        return BISIM_EINVAL;
    }
    if (slot_src_h || slot_act_h) BISIM_TRY(ensure_slot_arrays(p));
    const size_t n1 = (size_t)p->n + 1, L = (size_t)p->L, m = (size_t)p->m;
    if (mark_length) *mark_length = p->L;
    if (off_h && p->off.p) BISIM_CUDA_TRY(cudaMemcpyAsync(off_h, p->off.p, 4 * n1, cudaMemcpyDeviceToHost, p->st));
    if (in_ptr_h && p->in_ptr.p)
        BISIM_CUDA_TRY(cudaMemcpyAsync(in_ptr_h, p->in_ptr.p, 4 * n1, cudaMemcpyDeviceToHost, p->st));
    if (slot_src_h && L)
        BISIM_CUDA_TRY(cudaMemcpyAsync(slot_src_h, p->slot_src.p, 4 * L, cudaMemcpyDeviceToHost, p->st));
    if (slot_act_h && L)
        BISIM_CUDA_TRY(cudaMemcpyAsync(slot_act_h, p->slot_act.p, 4 * L, cudaMemcpyDeviceToHost, p->st));
    if (in_edge_h && m)
        BISIM_CUDA_TRY(cudaMemcpyAsync(in_edge_h, p->in_edge.p, 8 * m, cudaMemcpyDeviceToHost, p->st));
    BISIM_CUDA_TRY(cudaStreamSynchronize(p->st));
    return BISIM_OK;
}

int bisim_reduce_host(int32_t n, int64_t m, int32_t num_act, const int32_t* src_h,
                      const int32_t* act_h, const int32_t* dst_h, const int32_t* init_h,
                      int32_t* out_block_h, const bisim_opts* opts, void* stream,
                      bisim_stats* stats) {
    if (n < 0 || m < 0 || m > 0x7fffffffll || (m > 0 && (!src_h || !dst_h)) ||
        (n > 0 && !out_block_h)) {
        set_last_error("bad argument");
        return BISIM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    DevMem dsrc, dact, ddst, dinit, dout;
    BISIM_TRY(dsrc.alloc(4 * (size_t)m, st));
    BISIM_TRY(ddst.alloc(4 * (size_t)m, st));
    BISIM_TRY(dout.alloc(4 * (size_t)n, st));
    if (act_h) BISIM_TRY(dact.alloc(4 * (size_t)m, st));
    if (init_h) BISIM_TRY(dinit.alloc(4 * (size_t)n, st));
    // the input arrays travel on separate streams at once (one copy each),
    // after the allocations and before the plan
    {
        cudaStream_t cs[3];
        BISIM_TRY(copy_streams(cs));
        struct Copy {
            void* d;
            const void* h;
            size_t bytes;
        } copies[4] = {{dsrc.p, src_h, 4 * (size_t)m},
                       {ddst.p, dst_h, 4 * (size_t)m},
                       {act_h ? dact.p : nullptr, act_h, act_h ? 4 * (size_t)m : 0},
                       {init_h ? dinit.p : nullptr, init_h, init_h ? 4 * (size_t)n : 0}};
        EventSet ev;
        BISIM_TRY(ev.create(4));
        BISIM_CUDA_TRY(cudaEventRecord(ev.e[0], st));
        for (int k = 0; k < 3; k++) BISIM_CUDA_TRY(cudaStreamWaitEvent(cs[k], ev.e[0], 0));
        for (int k = 0; k < 4; k++)
            if (copies[k].bytes)
                BISIM_CUDA_TRY(cudaMemcpyAsync(copies[k].d, copies[k].h, copies[k].bytes, cudaMemcpyHostToDevice,
                                               cs[k % 3]));
        for (int k = 0; k < 3; k++) {
            BISIM_CUDA_TRY(cudaEventRecord(ev.e[1 + k], cs[k]));
            BISIM_CUDA_TRY(cudaStreamWaitEvent(st, ev.e[1 + k], 0));
        }
    }
    bisim_plan_t plan = nullptr;
    int rc = bisim_plan(n, m, num_act, dsrc.as<int32_t>(), act_h ? dact.as<int32_t>() : nullptr,
                        ddst.as<int32_t>(), init_h ? dinit.as<int32_t>() : nullptr, opts, stream, &plan);
    if (rc) return rc;
    rc = bisim_refine(plan, dout.as<int32_t>(), stats);
    bisim_plan_destroy(plan);
    if (rc) return rc;
    if (n) BISIM_CUDA_TRY(cudaMemcpyAsync(out_block_h, dout.p, 4 * (size_t)n, cudaMemcpyDeviceToHost, st));
    BISIM_CUDA_TRY(cudaStreamSynchronize(st));
    return BISIM_OK;
}

}  // extern "C"
