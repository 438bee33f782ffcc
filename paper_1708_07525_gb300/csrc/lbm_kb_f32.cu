// Batched kernels, FP32 storage.
#include "lbm_kb_launchers.cuh"

namespace lbm {
LBM_BATCH_INSTANTIATE(float)
}  // namespace lbm
