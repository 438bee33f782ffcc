// FP32 storage and arithmetic.
#include "lbm_launchers.cuh"

namespace lbm {
LBM_INSTANTIATE(float)
}  // namespace lbm
