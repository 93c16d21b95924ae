// Learned skip predictor (placeholder upload path; training kernels follow).
#include <vector>

#include "internal.cuh"

finger_status finger_load_mlp_internal(finger_index* ix, const float* w, int64_t count, float eps) {
    (void)ix;
    (void)w;
    (void)count;
    (void)eps;
    return FINGER_ERR_UNSUPPORTED;
}
