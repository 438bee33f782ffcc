// Kernels that advance many cavities of different sizes and parameters in one
// launch.  The work is cut into tiles (tile_w x tile_h nodes of one cavity);
// a grid of resident CTAs (a multiple of the SM count) walks the global tile
// list, each CTA taking every gridDim.x-th tile.  Per cavity the tile shape is
// chosen by the autotuner (lbm_batch.cu).  The per-node work is exactly the
// single-cavity step (gather_pull / collide / put of lbm_kernels.cuh), so a
// cavity gives bit-identical results alone or in a batch.
#pragma once
#include "lbm_kernels.cuh"

namespace lbm {

// One cavity of a batch, as the kernels see it (device memory, 16-byte aligned).
template <typename R>
struct alignas(16) BatchInst {
    void* buf[2];          // two-buffer layout: both; in-place layout: buf[0]
    void* hist;            // 4 history planes in R
    R* snap;               // residual snapshot [4][ny][nx] (u_x, u_y, T - T0, C - C0) or NULL
    Geom G;
    Coef<R> c;
    int tile_w_log2;       // tile width = 1 << tile_w_log2 (32 .. 256)
    int tile_h;            // tile height (rows)
    int tiles_x;           // tiles along x
    int tile_begin;        // index of the cavity's first tile in the global list
    int phase;             // the cavity's level parity = (batch step parity + phase) & 1
    int active;            // 0: skipped (free slot)
};

constexpr int BATCH_THREADS = 128;

// Copies the descriptor of cavity k into shared memory (all threads take part).
template <typename R>
__device__ __forceinline__ void load_inst(const BatchInst<R>* __restrict__ table, int k,
                                          BatchInst<R>& s) {
    static_assert(sizeof(BatchInst<R>) % 4 == 0, "descriptor size");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(table + k);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&s);
    for (int w = threadIdx.x; w < (int)(sizeof(BatchInst<R>) / 4); w += blockDim.x) dst[w] = src[w];
}

// One time step of every active cavity.  tile_owner[t] = cavity of global tile t.
// Launched with one CTA per tile (the loop then runs once).
// NEE = true: the batch holds cavities with wall nodes (Sec. 3.3); their nodes gather
// through the rebuild (two-buffer layout only).
template <typename S, bool AA, bool NEE = false>
__global__ void __launch_bounds__(BATCH_THREADS, 4)
batch_step_kernel(const BatchInst<typename Real<S>::type>* __restrict__ table,
                  const int* __restrict__ tile_owner, int tile_begin, int tile_end, int parity) {
    using R = typename Real<S>::type;
    __shared__ BatchInst<R> I;
    for (int tile = tile_begin + blockIdx.x; tile < tile_end; tile += gridDim.x) {
        const int k = tile_owner[tile];
        __syncthreads();                      // previous tile done with I
        load_inst(table, k, I);
        __syncthreads();
        if (!I.active) continue;
        const int local = tile - I.tile_begin;
        const int ty = local / I.tiles_x, tx = local - ty * I.tiles_x;
        const int tw = 1 << I.tile_w_log2;
        const int x0 = tx << I.tile_w_log2, y0 = ty * I.tile_h;
        const int odd = (parity + I.phase) & 1;
        const Geom G = I.G;
        for (int n = threadIdx.x; n < tw * I.tile_h; n += BATCH_THREADS) {
            const int i = x0 + (n & (tw - 1)), j = y0 + (n >> I.tile_w_log2);
            if (i >= G.nx || j >= G.ny) continue;
            R f[9], g[5], h[5], hv[4];
            const size_t self = (size_t)j * G.pitch + i;
            R* hist = (R*)I.hist;
            if (!AA) {
                const S* src = (const S*)I.buf[odd];
                S* dst = (S*)I.buf[odd ^ 1];
                if (NEE && I.c.nee)
                    gather_nee(src, G, i, j, I.c, f, g, h);
                else
                    gather_pull<false, true, false>(src, G, i, j, I.c, f, g, h);
                load_hist(hist, G, self, hv);
                uint32_t seed = Store<S>::kLow ? node_seed(self, f[0], g[0]) : 0u;
                collide(I.c, f, g, h, hv);
                store_ab(dst, G, self, I.c, f, g, h, seed);
            } else {
                S* buf = (S*)I.buf[0];
                if (odd)
                    gather_pull<true, true, false>(buf, G, i, j, I.c, f, g, h);
                else
                    gather_local<true>(buf, G, i, j, f, g, h);
                load_hist(hist, G, self, hv);
                uint32_t seed = Store<S>::kLow ? node_seed(self, f[0], g[0]) : 0u;
                collide(I.c, f, g, h, hv);
                if (odd)
                    store_aa_odd<false>(buf, G, i, j, self, I.c, f, g, h, seed);
                else
                    store_aa_even(buf, G, self, I.c, f, g, h, seed);
            }
            store_hist(hist, G, self, hv);
        }
    }
}

// The same step for tiles of exactly BATCH_THREADS nodes: one node per thread,
// one tile per CTA and no loop, so nothing loop-invariant is hoisted into
// registers (the descriptor stays in shared memory and occupancy stays high).
// The two-buffer variant is held to 64 registers (8 CTAs per SM instead of 7; 12
// bytes of spills with the flow and scalar collisions as two calls).  The in-place
// one holds both parities' code (cavities in one launch may be at different
// parities) and was compiled to 146 registers (3 CTAs per SM) when left alone;
// held to 5 CTAs per SM it fits 96 (24 bytes of spills).
template <typename S, bool AA, bool NEE = false>
__global__ void __launch_bounds__(BATCH_THREADS, NEE ? 1 : (AA ? 5 : 8))
batch_step1_kernel(const BatchInst<typename Real<S>::type>* __restrict__ table,
                   const int* __restrict__ tile_owner, int tile_begin, int parity) {
    using R = typename Real<S>::type;
    __shared__ BatchInst<R> I;
    pdl_trigger();                            // launched by launch_pdl() (launch_batch_step)
    const int tile = tile_begin + blockIdx.x;
    load_inst(table, tile_owner[tile], I);    // only host copies write the table and owners
    __syncthreads();
    pdl_wait();                               // the previous step's writes are visible
    if (!I.active) return;
    const int local = tile - I.tile_begin;
    const int ty = local / I.tiles_x, tx = local - ty * I.tiles_x;
    const int n = threadIdx.x;
    const int i = (tx << I.tile_w_log2) + (n & ((1 << I.tile_w_log2) - 1));
    const int j = ty * I.tile_h + (n >> I.tile_w_log2);
    const Geom G = I.G;
    if (i >= G.nx || j >= G.ny) return;
    const int odd = (parity + I.phase) & 1;
    R f[9], g[5], h[5], hv[4];
    const size_t self = (size_t)j * G.pitch + i;
    R* hist = (R*)I.hist;
    if (!AA) {
        const S* src = (const S*)I.buf[odd];
        S* dst = (S*)I.buf[odd ^ 1];
        if (NEE && I.c.nee)
            gather_nee(src, G, i, j, I.c, f, g, h);
        else
            gather_pull<false, true, false>(src, G, i, j, I.c, f, g, h);
        load_hist(hist, G, self, hv);
        uint32_t seed = Store<S>::kLow ? node_seed(self, f[0], g[0]) : 0u;
        collide(I.c, f, g, h, hv);
        store_ab(dst, G, self, I.c, f, g, h, seed);
    } else {
        S* buf = (S*)I.buf[0];
        if (odd)
            gather_pull<true, true, false>(buf, G, i, j, I.c, f, g, h);
        else
            gather_local<true>(buf, G, i, j, f, g, h);
        load_hist(hist, G, self, hv);
        uint32_t seed = Store<S>::kLow ? node_seed(self, f[0], g[0]) : 0u;
        collide(I.c, f, g, h, hv);
        if (odd)
            store_aa_odd<false>(buf, G, i, j, self, I.c, f, g, h, seed);
        else
            store_aa_even(buf, G, self, I.c, f, g, h, seed);
    }
    store_hist(hist, G, self, hv);
}

// Gather mode of cavity I at batch step parity `parity`.
template <typename R>
__device__ __forceinline__ int batch_mode(const BatchInst<R>& I, int parity, bool aa) {
    const int odd = (parity + I.phase) & 1;
    if (!aa) return I.c.nee ? GATHER_NEE_AB : GATHER_PULL_AB;
    return odd ? GATHER_PULL_AA : GATHER_LOCAL;
}
template <typename R>
__device__ __forceinline__ const void* batch_cur(const BatchInst<R>& I, int parity, bool aa) {
    return aa ? I.buf[0] : I.buf[(parity + I.phase) & 1];
}

// Residual pass 1 over tiles: partial[tile][9] as in residual_kernel.
template <typename S, bool AA>
__global__ void __launch_bounds__(BATCH_THREADS)
batch_residual_kernel(const BatchInst<typename Real<S>::type>* __restrict__ table,
                      const int* __restrict__ tile_owner, int total_tiles, int parity,
                      double* __restrict__ partial) {
    using R = typename Real<S>::type;
    __shared__ BatchInst<R> I;
    __shared__ R red[BATCH_THREADS / 32][9];
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        const int k = tile_owner[tile];
        __syncthreads();
        load_inst(table, k, I);
        __syncthreads();
        R dmax[4] = {0, 0, 0, 0}, amax[4] = {0, 0, 0, 0};
        int bad = 0;
        if (I.active && I.snap) {
            const int local = tile - I.tile_begin;
            const int ty = local / I.tiles_x, tx = local - ty * I.tiles_x;
            const int tw = 1 << I.tile_w_log2;
            const int x0 = tx << I.tile_w_log2, y0 = ty * I.tile_h;
            const int mode = batch_mode(I, parity, AA);
            const S* buf = (const S*)batch_cur(I, parity, AA);
            const Geom G = I.G;
            const size_t n = (size_t)G.nx * G.ny;
            for (int e = threadIdx.x; e < tw * I.tile_h; e += BATCH_THREADS) {
                const int i = x0 + (e & (tw - 1)), j = y0 + (e >> I.tile_w_log2);
                if (i >= G.nx || j >= G.ny) continue;
                // snapshot loads first, stores last, as in lbm_residual's pass
                const size_t kk = (size_t)j * G.nx + i;
                R old[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) old[q] = I.snap[q * n + kk];
                R f[9], g[5], h[5];
                gather<true>(mode, buf, G, i, j, I.c, f, g, h);
                Macro<R> M = macro(I.c, f, g, h);
                // differences in the compute precision on the deviations (exact for
                // close values), as lbm_residual does
                const R phi[4] = {M.ux, M.uy, M.Tp, M.Cp};
                const R absv[4] = {M.ux, M.uy, I.c.T0 + M.Tp, I.c.C0 + M.Cp};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (!finite_(phi[q])) bad = 1;
                    dmax[q] = max_(dmax[q], abs_(phi[q] - old[q]));
                    amax[q] = max_(amax[q], abs_(absv[q]));
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) I.snap[q * n + kk] = phi[q];
            }
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const R v[9] = {dmax[0], dmax[1], dmax[2], dmax[3], amax[0], amax[1], amax[2], amax[3],
                        (R)bad};
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const R r = warp_max(v[q]);
            if (lane == 0) red[warp][q] = r;
        }
        __syncthreads();
        if (threadIdx.x < 9) {
            R s = 0;
            for (int w = 0; w < BATCH_THREADS / 32; ++w) s = max_(s, red[w][threadIdx.x]);
            partial[(size_t)tile * 9 + threadIdx.x] = (double)s;
        }
    }
}

// Residual pass 2: block k folds the partials of cavity k's tiles into out[k][9].
template <typename R>
__global__ void __launch_bounds__(BATCH_THREADS)
batch_residual_fold_kernel(const BatchInst<R>* __restrict__ table, const int* __restrict__ ntiles,
                           const double* __restrict__ partial, double* __restrict__ out) {
    const int k = blockIdx.x;
    const int b0 = table[k].tile_begin, nt = ntiles[k];
    __shared__ double red[BATCH_THREADS / 32][9];
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < nt; t += blockDim.x)
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] = fmax(v[q], partial[(size_t)(b0 + t) * 9 + q]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const double r = warp_max(v[q]);
        if (lane == 0) red[warp][q] = r;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double s = 0;
        for (int w = 0; w < BATCH_THREADS / 32; ++w) s = fmax(s, red[w][threadIdx.x]);
        out[(size_t)k * 9 + threadIdx.x] = s;
    }
}

// Nu / Sh of every cavity (Eq. 38): block k reduces cavity k's wall columns.
template <typename S, bool AA>
__global__ void __launch_bounds__(BATCH_THREADS)
batch_nush_kernel(const BatchInst<typename Real<S>::type>* __restrict__ table,
                  const WallSpec* __restrict__ walls, int parity, double* __restrict__ out) {
    using R = typename Real<S>::type;
    const int k = blockIdx.x;
    __shared__ BatchInst<R> I;
    load_inst(table, k, I);
    __syncthreads();
    double acc[4] = {0, 0, 0, 0};
    const WallSpec W = walls[k];
    if (I.active) {
        const int mode = batch_mode(I, parity, AA);
        const S* buf = (const S*)batch_cur(I, parity, AA);
        const Geom G = I.G;
        if (W.nee) {
            // nodes on the walls: the node stencil and the trapezoidal mean of nush_kernel
            for (int j = threadIdx.x; j < G.ny; j += blockDim.x) {
                R f[9], g[5], h[5];
                double T[6], C[6];
                const int cols[6] = {0, 1, 2, G.nx - 3, G.nx - 2, G.nx - 1};
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    gather<false>(mode, buf, G, cols[q], j, I.c, f, g, h);
                    const R sg = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
                    const R sh = ((h[0] + h[1]) + (h[2] + h[3])) + h[4];
                    T[q] = W.T0 + (double)(sg * I.c.inv_sigma);
                    C[q] = W.C0 + (double)(sh * I.c.inv_eps);
                }
                const double wj = (j == 0 || j == G.ny - 1) ? 0.5 : 1.0;
                acc[0] += wj * -W.L * (-3.0 * T[0] + 4.0 * T[1] - T[2]) / 2.0 / W.dT;
                acc[1] += wj * -W.L * (-3.0 * C[0] + 4.0 * C[1] - C[2]) / 2.0 / W.dC;
                acc[2] += wj * -W.L * (3.0 * T[5] - 4.0 * T[4] + T[3]) / 2.0 / W.dT;
                acc[3] += wj * -W.L * (3.0 * C[5] - 4.0 * C[4] + C[3]) / 2.0 / W.dC;
            }
        }
        for (int j = threadIdx.x; j < G.ny && !W.nee; j += blockDim.x) {
            R f[9], g[5], h[5];
            double T[4], C[4];
            const int cols[4] = {0, 1, G.nx - 2, G.nx - 1};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                gather<false>(mode, buf, G, cols[q], j, I.c, f, g, h);
                const R sg = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
                const R sh = ((h[0] + h[1]) + (h[2] + h[3])) + h[4];
                T[q] = W.T0 + (double)(sg * I.c.inv_sigma);
                C[q] = W.C0 + (double)(sh * I.c.inv_eps);
            }
            acc[0] += -W.L * (-8.0 * W.Tw[0] + 9.0 * T[0] - T[1]) / 3.0 / W.dT;
            acc[1] += -W.L * (-8.0 * W.Cw[0] + 9.0 * C[0] - C[1]) / 3.0 / W.dC;
            acc[2] += -W.L * (8.0 * W.Tw[1] - 9.0 * T[3] + T[2]) / 3.0 / W.dT;
            acc[3] += -W.L * (8.0 * W.Cw[1] - 9.0 * C[3] + C[2]) / 3.0 / W.dC;
        }
    }
    __shared__ double red[BATCH_THREADS / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0;
        for (int w = 0; w < BATCH_THREADS / 32; ++w) s += red[w][threadIdx.x];
        out[(size_t)k * 4 + threadIdx.x] = I.active ? s / (W.nee ? I.G.ny - 1.0 : (double)I.G.ny) : 0.0;
    }
}

}  // namespace lbm
