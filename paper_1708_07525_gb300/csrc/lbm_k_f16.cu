// BF16 and FP16 storage with FP32 arithmetic.
#include "lbm_launchers.cuh"

namespace lbm {
LBM_INSTANTIATE(__nv_bfloat16)
LBM_INSTANTIATE(__half)
}  // namespace lbm
