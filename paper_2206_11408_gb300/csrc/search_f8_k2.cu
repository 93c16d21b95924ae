// Search kernel instances of mode FINGER_F8 (FP32 rows, FP8 codes) for code
// tables of 2 k steps (see search_impl.cuh).
#include "search_impl.cuh"

namespace fg {
cudaError_t launch_f8_k2(const DevIndex& ix, const SearchArgs& a, const SearchPlan& p,
                         cudaStream_t s) {
    return launch_mode<MODE_F8_K2>(ix, a, p, s);
}
cudaError_t occupancy_f8_k2(const SearchPlan& p, int* blocks) {
    return occupancy_mode<MODE_F8_K2>(p, blocks);
}
}  // namespace fg
