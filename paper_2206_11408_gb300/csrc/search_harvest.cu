// Search kernel instances for the harvest mode (see search_impl.cuh).
#include "search_impl.cuh"

namespace fg {
cudaError_t launch_mode_harvest(const DevIndex& ix, const SearchArgs& a, const SearchPlan& p,
                                cudaStream_t s) {
    return launch_mode<MODE_HARVEST>(ix, a, p, s);
}
cudaError_t occupancy_mode_harvest(const SearchPlan& p, int* blocks) {
    return occupancy_mode<MODE_HARVEST>(p, blocks);
}
}  // namespace fg
