// FP64 storage and arithmetic; also the precision-independent residual fold.
#include "lbm_launchers.cuh"

namespace lbm {

__global__ void __launch_bounds__(RES_THREADS)
residual_final_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
    __shared__ double red[RES_THREADS / 32][9];
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] = fmax(v[q], partial[(size_t)b * 9 + q]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const double r = warp_max(v[q]);
        if (lane == 0) red[warp][q] = r;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, red[w][threadIdx.x]);
        out[threadIdx.x] = s;
    }
}

LBM_INSTANTIATE(double)

}  // namespace lbm
