// Diagnostics: cost of the grid-wide barrier the persistent kernels use.
#include "prim.cuh"

namespace {

using namespace bisim;

__global__ void k_barrier_loop(GridBarrier gb, int iters) {
    unsigned long long tgt = 0;
    for (int i = 0; i < iters; i++)
        if (!grid_sync(gb, tgt)) return;
}

}  // namespace

extern "C" int bisim_barrier_cost(int32_t ctas, int32_t threads, int32_t iters, void* stream,
                                  double* ns_per_barrier) {
    if (ctas < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 || !ns_per_barrier) {
        set_last_error("bisim_barrier_cost: bad argument");
        return BISIM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0, occ = 0;
    BISIM_CUDA_TRY(cudaGetDevice(&dev));
    BISIM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BISIM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_barrier_loop, threads, 0));
    if (ctas > sms * occ) {
        set_last_error("bisim_barrier_cost: more CTAs than can be co-resident");
        return BISIM_EINVAL;
    }
    DevMem words;
    BISIM_TRY(words.alloc(16, st));
    BISIM_CUDA_TRY(cudaMemsetAsync(words.p, 0, 16, st));
    GridBarrier gb;
    gb.counter = words.as<unsigned long long>();
    gb.status = (int*)(words.as<char>() + 8);
    gb.timeout_ns = 2000000000ull;
    cudaEvent_t e0, e1;
    BISIM_CUDA_TRY(cudaEventCreate(&e0));
    BISIM_CUDA_TRY(cudaEventCreate(&e1));
    void* args[] = {&gb, &iters};
    int rc = BISIM_OK;
    cudaError_t e = cudaEventRecord(e0, st);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void*)k_barrier_loop, dim3(ctas), dim3(threads), args, 0, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, gb.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_last_error(std::string("bisim_barrier_cost: ") + cudaGetErrorString(e));
        rc = BISIM_ECUDA;
    } else if (status) {
        rc = status_to_code(status);
    } else {
        *ns_per_barrier = (double)ms * 1e6 / iters;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
