// Batched kernels, BF16 and FP16 storage with FP32 arithmetic.
#include "lbm_kb_launchers.cuh"

namespace lbm {
LBM_BATCH_INSTANTIATE(__nv_bfloat16)
LBM_BATCH_INSTANTIATE(__half)
}  // namespace lbm
