// Search kernel instances for mode 1 (see search_impl.cuh).
#include "search_impl.cuh"

namespace fg {
cudaError_t launch_mode1(const DevIndex& ix, const SearchArgs& a, const SearchPlan& p,
                          cudaStream_t s) {
    return launch_mode<1>(ix, a, p, s);
}
cudaError_t occupancy_mode1(const SearchPlan& p, int* blocks) { return occupancy_mode<1>(p, blocks); }
}  // namespace fg
