// Launch interface of the batched kernels (lbm_batch_kernels.cuh), explicitly
// instantiated in lbm_kb_*.cu for S = float, __nv_bfloat16, __half.
#pragma once
#include "lbm_launch.h"

namespace lbm {

template <typename R> struct BatchInst;

// One step of the cavities owning tiles [tile_begin, tile_end) (one CTA per tile);
// one_node: every tile has exactly BATCH_THREADS nodes (loop-free kernel); nee: some
// cavity of the batch has wall nodes (Sec. 3.3), so the kernel with the rebuild runs.
template <typename S>
cudaError_t launch_batch_step(const BatchInst<float>* table, const int* owner, int tile_begin,
                              int tile_end, int parity, bool aa, bool one_node, bool nee,
                              cudaStream_t st);
template <typename S>
cudaError_t launch_batch_residual(const BatchInst<float>* table, const int* owner,
                                  const int* ntiles, int total_tiles, int n_inst, int parity,
                                  bool aa, int grid, double* partial, double* out, cudaStream_t st);
template <typename S>
cudaError_t launch_batch_nush(const BatchInst<float>* table, const WallSpec* walls, int n_inst,
                              int parity, bool aa, double* out, cudaStream_t st);
// Resident blocks per SM of the batched step kernel.
template <typename S>
int batch_step_blocks_per_sm(bool aa);

}  // namespace lbm
