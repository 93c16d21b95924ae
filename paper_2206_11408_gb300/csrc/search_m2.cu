// Search kernel instances for mode 2 (see search_impl.cuh).
#include "search_impl.cuh"

namespace fg {
cudaError_t launch_mode2(const DevIndex& ix, const SearchArgs& a, const SearchPlan& p,
                          cudaStream_t s) {
    return launch_mode<2>(ix, a, p, s);
}
cudaError_t occupancy_mode2(const SearchPlan& p, int* blocks) { return occupancy_mode<2>(p, blocks); }
}  // namespace fg
