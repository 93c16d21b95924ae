// Search kernel instances of mode FINGER_F8 (FP32 rows, FP8 codes) for code
// tables of 4 k steps (see search_impl.cuh).
#include "search_impl.cuh"

namespace fg {
cudaError_t launch_f8_k4(const DevIndex& ix, const SearchArgs& a, const SearchPlan& p,
                         cudaStream_t s) {
    return launch_mode<MODE_F8_K4>(ix, a, p, s);
}
cudaError_t occupancy_f8_k4(const SearchPlan& p, int* blocks) {
    return occupancy_mode<MODE_F8_K4>(p, blocks);
}
}  // namespace fg
