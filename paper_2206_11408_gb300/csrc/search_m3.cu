// Search kernel instances for mode 3 (see search_impl.cuh).
#include "search_impl.cuh"

namespace fg {
cudaError_t launch_mode3(const DevIndex& ix, const SearchArgs& a, const SearchPlan& p,
                          cudaStream_t s) {
    return launch_mode<3>(ix, a, p, s);
}
cudaError_t occupancy_mode3(const SearchPlan& p, int* blocks) { return occupancy_mode<3>(p, blocks); }
}  // namespace fg
