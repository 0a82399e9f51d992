// Frontier refinement engine (placeholder until the kernel lands).
#include "plan.cuh"

namespace bisim {

int refine_frontier(bisim_plan_s* p, bisim_stats* st) {
    (void)p;
    (void)st;
    set_last_error("frontier engine not built");
    return BISIM_ENOTSUP;
}

}  // namespace bisim
