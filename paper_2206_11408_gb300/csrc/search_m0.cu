// Search kernel instances for mode 0 (see search_impl.cuh).
#include "search_impl.cuh"

namespace fg {
cudaError_t launch_mode0(const DevIndex& ix, const SearchArgs& a, const SearchPlan& p,
                          cudaStream_t s) {
    return launch_mode<0>(ix, a, p, s);
}
cudaError_t occupancy_mode0(const SearchPlan& p, int* blocks) { return occupancy_mode<0>(p, blocks); }
}  // namespace fg
