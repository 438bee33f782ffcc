// Definitions of the batched-kernel launchers (instantiated per precision).
#pragma once
#include "lbm_batch.h"
#include "lbm_batch_kernels.cuh"

namespace lbm {

// One-node tile steps go out as programmatic dependent launches: the next step's CTAs are
// placed, and read their descriptors, while the current step's last wave drains (also
// inside a captured graph, where the attribute becomes a programmatic edge).  GB300, 512
// mixed cavities, FP32: 39.6 -> 40.2 GLUPS two-buffer, 34.6 -> 34.9 in place; a 32^2
// cavity stepped alone 8.3 -> 5.3 us per step.
template <typename... P, typename... A>
cudaError_t launch_tiles(void (*kernel)(P...), int grid, cudaStream_t st, A... args) {
    return launch_pdl(kernel, dim3((unsigned)grid), dim3(BATCH_THREADS), st, args...);
}

template <typename S>
cudaError_t launch_batch_step(const BatchInst<float>* table, const int* owner, int tile_begin,
                              int tile_end, int parity, bool aa, bool one_node, bool nee,
                              cudaStream_t st) {
    const int grid = tile_end - tile_begin;
    if (grid <= 0) return cudaSuccess;
    if (one_node) {
        if (aa) return launch_tiles(batch_step1_kernel<S, true>, grid, st, table, owner, tile_begin, parity);
        if (nee) return launch_tiles(batch_step1_kernel<S, false, true>, grid, st, table, owner, tile_begin, parity);
        return launch_tiles(batch_step1_kernel<S, false>, grid, st, table, owner, tile_begin, parity);
    }
    if (aa)
        batch_step_kernel<S, true><<<grid, BATCH_THREADS, 0, st>>>(table, owner, tile_begin, tile_end, parity);
    else if (nee)
        batch_step_kernel<S, false, true><<<grid, BATCH_THREADS, 0, st>>>(table, owner, tile_begin, tile_end, parity);
    else
        batch_step_kernel<S, false><<<grid, BATCH_THREADS, 0, st>>>(table, owner, tile_begin, tile_end, parity);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_batch_residual(const BatchInst<float>* table, const int* owner,
                                  const int* ntiles, int total_tiles, int n_inst, int parity,
                                  bool aa, int grid, double* partial, double* out, cudaStream_t st) {
    if (total_tiles <= 0 || n_inst <= 0) return cudaSuccess;
    if (aa)
        batch_residual_kernel<S, true><<<grid, BATCH_THREADS, 0, st>>>(table, owner, total_tiles,
                                                                       parity, partial);
    else
        batch_residual_kernel<S, false><<<grid, BATCH_THREADS, 0, st>>>(table, owner, total_tiles,
                                                                        parity, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_residual_fold_kernel<float><<<n_inst, BATCH_THREADS, 0, st>>>(table, ntiles, partial, out);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_batch_nush(const BatchInst<float>* table, const WallSpec* walls, int n_inst,
                              int parity, bool aa, double* out, cudaStream_t st) {
    if (n_inst <= 0) return cudaSuccess;
    if (aa)
        batch_nush_kernel<S, true><<<n_inst, BATCH_THREADS, 0, st>>>(table, walls, parity, out);
    else
        batch_nush_kernel<S, false><<<n_inst, BATCH_THREADS, 0, st>>>(table, walls, parity, out);
    return cudaGetLastError();
}

template <typename S>
int batch_step_blocks_per_sm(bool aa) {
    int n = 0;
    if (aa)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<S, true>, BATCH_THREADS, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<S, false>, BATCH_THREADS, 0);
    return n > 0 ? n : 1;
}

#define LBM_BATCH_INSTANTIATE(S)                                                                  \
    template cudaError_t launch_batch_step<S>(const BatchInst<float>*, const int*, int, int, int,  \
                                              bool, bool, bool, cudaStream_t);                     \
    template cudaError_t launch_batch_residual<S>(const BatchInst<float>*, const int*, const int*, \
                                                  int, int, int, bool, int, double*, double*,      \
                                                  cudaStream_t);                                   \
    template cudaError_t launch_batch_nush<S>(const BatchInst<float>*, const WallSpec*, int, int,  \
                                              bool, double*, cudaStream_t);                        \
    template int batch_step_blocks_per_sm<S>(bool);

}  // namespace lbm
