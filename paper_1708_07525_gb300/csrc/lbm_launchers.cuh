// Definitions of the launchers declared in lbm_launch.h (included by the
// per-precision translation units, which instantiate them).
#pragma once
#include <algorithm>
#include <type_traits>

#include "lbm_kernels.cuh"
#include "lbm_pair.cuh"

namespace lbm {

inline dim3 grid_for(const Geom& G, int bx, int by) {
    return dim3((unsigned)((G.nx + bx - 1) / bx), (unsigned)((G.ny + by - 1) / by), 1);
}

template <typename S>
cudaError_t launch_init(void* buf, void* hist, const Geom& G, const Coef<typename Real<S>::type>& c,
                        const InitSpec& I, bool pull, cudaStream_t st) {
    using R = typename Real<S>::type;
    dim3 b(128, 1), gr = grid_for(G, 128, 1);
    if (pull)
        init_kernel<S, true><<<gr, b, 0, st>>>((S*)buf, (R*)hist, G, c, I);
    else
        init_kernel<S, false><<<gr, b, 0, st>>>((S*)buf, (R*)hist, G, c, I);
    if (c.nee && pull) {   // wall nodes: the t = 0 state obeys the wall rules too
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        nee_hist_kernel<S><<<gr, b, 0, st>>>((const S*)buf, (R*)hist, G, c);
    }
    return cudaGetLastError();
}

// Grids of the two-nodes-per-thread kernels (lbm_pair.cuh); false if the cavity does
// not take them (too small, or too many rows for one launch).
// The pull grid: erows block rows of edge nodes, then the rows of inner pairs.
inline bool pair_grid_ab(const Geom& G, dim3& gr, int& erows) {
    const int np = inner_pairs(G.nx), rows = G.ny - 2;
    if (G.nx < 8 || rows < 1 || np < 1) return false;
    const long long gx = (np + PAIR_BX) / PAIR_BX;
    const long long eb = (edge_count(G) + PAIR_BX * PAIR_BY - 1) / (PAIR_BX * PAIR_BY);
    const long long er = (eb + gx - 1) / gx;
    const long long gy = (rows + PAIR_BY - 1) / PAIR_BY + er;
    if (gy > 65535) return false;
    erows = (int)er;
    gr = dim3((unsigned)gx, (unsigned)gy, 1);
    return true;
}
inline bool pair_grid_aa_even(const Geom& G, dim3& gr) {
    if (G.nx & 1) return false;
    gr = dim3((unsigned)((G.nx / 2 + PAIR_BX - 1) / PAIR_BX), (unsigned)((G.ny + PAIR_BY - 1) / PAIR_BY), 1);
    return gr.y <= 65535u;
}

// With FP32 arithmetic the in-place odd step splits the inner nodes (no wall logic) from
// the ring of outermost nodes from this many nodes on, below it runs as one kernel with
// the wall logic for every node.  GB300, FP32, us per step over alternating odd and even
// steps, one kernel / split with the ring on a second stream / split in one launch (the
// ring's block rows first): 128^2 2.5 / 4.6 / 3.9, 256^2 2.9 / 4.9 / 4.6, 512^2 6.9 / 7.8 /
// 6.3, 1024^2 28.2 / 27.5 / 25.5, 2048^2 121.3 / 117.0 / 114.6, 4096^2 - / 460.5 / 458.8.
// FP64 splits at every size, the ring on a second stream (128^2 33.1 / 13.5 us, 1024^2
// 507.5 / 502.3).
#ifndef LBM_AA_SPLIT_MIN_NODES
#define LBM_AA_SPLIT_MIN_NODES (1LL << 17)
#endif
// With FP32 arithmetic the split odd step is one launch (step_aa_odd_fused_kernel: the
// ring's block rows, then the inner nodes), and so is the two-buffer step with wall nodes
// (Sec. 3.3; step_ab_nee_fused_kernel): no second stream, no fork / join, a programmatic
// dependent launch.  FP64 keeps the ring on a second stream beside the inner launch.  With
// wall nodes, FP32, us per step (second stream / one launch): 1024^2 33.3 / 30.5, 4096^2
// 459.2 / 456.7.
#ifndef LBM_AA_ODD_FUSED
#define LBM_AA_ODD_FUSED 1
#endif
#ifndef LBM_AB_NEE_FUSED
#define LBM_AB_NEE_FUSED 1
#endif

template <typename S>
cudaError_t launch_step_ab(const void* src, void* dst, void* hist, const Geom& G,
                           const Coef<typename Real<S>::type>& c, const LaunchCfg& L) {
    using R = typename Real<S>::type;
    dim3 b(L.bx, L.by), gr = grid_for(G, L.bx, L.by);
    if (G.jb != 0 || G.je != G.ny) {
        // a slab of a split cavity: the rows between its ghost rows, one launch with the
        // general pull (the ghost rows are ordinary neighbours, walls only where real)
        gr.y = (unsigned)((step_rows(G) + L.by - 1) / L.by);
        if (c.poro || c.moving)
            step_ab_kernel<S, true><<<gr, b, 0, L.stream>>>((const S*)src, (S*)dst, (R*)hist, G, c);
        else
            step_ab_kernel<S, false><<<gr, b, 0, L.stream>>>((const S*)src, (S*)dst, (R*)hist, G, c);
        return cudaGetLastError();
    }
    if constexpr (Store<S>::kLow) {
        dim3 gp;
        int erows = 0;
        if (L.pair && !c.nee && !c.poro && !c.moving && pair_grid_ab(G, gp, erows))
            // inner column pairs two nodes per thread, the edge set one node per thread,
            // in one programmatic dependent launch
            return launch_pdl(step_ab_pair_kernel<S>, gp, dim3(PAIR_BX, PAIR_BY), L.stream, (const S*)src,
                              (S*)dst, (float*)hist, G, *L.pair, c, erows);
    }
    if constexpr (std::is_same<R, float>::value && LBM_AB_NEE_FUSED) {
        if (c.nee) {
            // the ring of wall nodes (the rebuild, Sec. 3.3) in the first block rows, the
            // inner nodes (the plain pull) after them: one programmatic dependent launch
            const long long threads = (long long)b.x * b.y;
            const long long rrows = ((2LL * G.nx + 2LL * (G.ny - 2) + threads - 1) / threads + gr.x - 1) / gr.x;
            if (gr.y + rrows <= 65535) {
                const dim3 gf(gr.x, (unsigned)(gr.y + rrows), 1);
                if (c.poro)
                    return launch_pdl(step_ab_nee_fused_kernel<S, true>, gf, b, L.stream, (const S*)src, (S*)dst,
                                      (R*)hist, G, c, (int)rrows);
                return launch_pdl(step_ab_nee_fused_kernel<S, false>, gf, b, L.stream, (const S*)src, (S*)dst,
                                  (R*)hist, G, c, (int)rrows);
            }
        }
    }
    if (c.nee) {
        // the ring of wall nodes: the rebuild (Sec. 3.3); inner nodes: the plain pull
        cudaStream_t rs;
        cudaError_t e = ring_fork(L, &rs);
        if (e != cudaSuccess) return e;
        const long long nring = 2LL * G.nx + 2LL * (G.ny - 2);
        nee_ring_kernel<S><<<(unsigned)((nring + 127) / 128), 128, 0, rs>>>(
            (const S*)src, (S*)dst, (R*)hist, G, c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (c.poro)
            step_ab_kernel<S, true, true><<<gr, b, 0, L.stream>>>((const S*)src, (S*)dst, (R*)hist, G, c);
        else
            step_ab_kernel<S, false, true><<<gr, b, 0, L.stream>>>((const S*)src, (S*)dst, (R*)hist, G, c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return ring_join(L);
    } else if (!std::is_same<S, float>::value && G.nx >= 3 && G.ny >= 3) {
        // inner nodes with no wall logic, then the ring of outermost nodes.  GB300, 4096^2:
        // BF16 385 -> 377 us, FP16 442 -> 410 us, FP64 (2048^2) 2201 -> 2148 us; the
        // DRAM-bound FP32 step measured slower split (446 -> 460 us) and stays one kernel.
        const bool ext = c.poro || c.moving;
        cudaStream_t rs;
        cudaError_t e = ring_fork(L, &rs);
        if (e != cudaSuccess) return e;
        const long long nring = 2LL * G.nx + 2LL * (G.ny - 2);
        const unsigned nb = (unsigned)((nring + 127) / 128);
        if (ext)
            step_ab_ring_kernel<S, true><<<nb, 128, 0, rs>>>((const S*)src, (S*)dst, (R*)hist, G, c);
        else
            step_ab_ring_kernel<S, false><<<nb, 128, 0, rs>>>((const S*)src, (S*)dst, (R*)hist, G, c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (ext)
            step_ab_kernel<S, true, true><<<gr, b, 0, L.stream>>>((const S*)src, (S*)dst, (R*)hist, G, c);
        else
            step_ab_kernel<S, false, true><<<gr, b, 0, L.stream>>>((const S*)src, (S*)dst, (R*)hist, G, c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return ring_join(L);
    }
    // one kernel per step: a programmatic dependent launch, so that this step's CTAs are
    // placed while the step before drains
    if (c.poro || c.moving)
        return launch_pdl(step_ab_kernel<S, true>, gr, b, L.stream, (const S*)src, (S*)dst, (R*)hist, G, c);
    return launch_pdl(step_ab_kernel<S, false>, gr, b, L.stream, (const S*)src, (S*)dst, (R*)hist, G, c);
}


template <typename S>
cudaError_t launch_step_aa(void* buf, void* hist, const Geom& G,
                           const Coef<typename Real<S>::type>& c, bool odd, const LaunchCfg& L) {
    using R = typename Real<S>::type;
    dim3 b(L.bx, L.by), gr = grid_for(G, L.bx, L.by);
    const bool ext = c.poro || c.moving;
    if constexpr (Store<S>::kLow) {
        dim3 gp, ge;
        int erows = 0;
        if (L.pair && !ext && pair_grid_ab(G, gp, erows) && pair_grid_aa_even(G, ge)) {
            const dim3 pb(PAIR_BX, PAIR_BY);
            if (!odd)
                return launch_pdl(step_aa_even_pair_kernel<S>, ge, pb, L.stream, (S*)buf, (float*)hist, G,
                                  *L.pair);
            return launch_pdl(step_aa_odd_pair_kernel<S>, gp, pb, L.stream, (S*)buf, (float*)hist, G,
                              *L.pair, c, erows);
        }
    }
    const long long split_min = std::is_same<R, double>::value ? 0 : LBM_AA_SPLIT_MIN_NODES;
    if constexpr (std::is_same<R, float>::value && LBM_AA_ODD_FUSED) {
        if (odd && G.nx >= 3 && G.ny >= 3 && (long long)G.nx * G.ny >= split_min) {
            // ring and inner nodes in one programmatic dependent launch (the ring's block
            // rows first)
            const long long threads = (long long)b.x * b.y;
            const long long rrows = ((ring_count(G) + threads - 1) / threads + gr.x - 1) / gr.x;
            if (gr.y + rrows <= 65535) {
                const dim3 gf(gr.x, (unsigned)(gr.y + rrows), 1);
                if (ext)
                    return launch_pdl(step_aa_odd_fused_kernel<S, true>, gf, b, L.stream, (S*)buf, (R*)hist, G,
                                      c, (int)rrows);
                return launch_pdl(step_aa_odd_fused_kernel<S, false>, gf, b, L.stream, (S*)buf, (R*)hist, G, c,
                                  (int)rrows);
            }
        }
    }
    if (odd && G.nx >= 3 && G.ny >= 3 && (long long)G.nx * G.ny >= split_min) {
        // the ring of outermost nodes beside the inner nodes (no wall logic); the two
        // launches touch disjoint locations
        cudaStream_t rs;
        cudaError_t e = ring_fork(L, &rs);
        if (e != cudaSuccess) return e;
        const long long nring = 2LL * G.nx + 2LL * (G.ny - 2);
        const unsigned nb = (unsigned)((nring + 127) / 128);
        if (ext)
            step_aa_odd_ring_kernel<S, true><<<nb, 128, 0, rs>>>((S*)buf, (R*)hist, G, c);
        else
            step_aa_odd_ring_kernel<S, false><<<nb, 128, 0, rs>>>((S*)buf, (R*)hist, G, c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (ext)
            step_aa_odd_inner_kernel<S, true><<<gr, b, 0, L.stream>>>((S*)buf, (R*)hist, G, c);
        else
            step_aa_odd_inner_kernel<S, false><<<gr, b, 0, L.stream>>>((S*)buf, (R*)hist, G, c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return ring_join(L);
    }
    // one kernel per step: a programmatic dependent launch, as in launch_step_ab
    if (odd && ext) return launch_pdl(step_aa_kernel<S, true, true>, gr, b, L.stream, (S*)buf, (R*)hist, G, c);
    if (odd) return launch_pdl(step_aa_kernel<S, true, false>, gr, b, L.stream, (S*)buf, (R*)hist, G, c);
    if (ext) return launch_pdl(step_aa_kernel<S, false, true>, gr, b, L.stream, (S*)buf, (R*)hist, G, c);
    return launch_pdl(step_aa_kernel<S, false, false>, gr, b, L.stream, (S*)buf, (R*)hist, G, c);
}

template <typename S>
cudaError_t launch_fields(const void* buf, const Geom& G, const Coef<typename Real<S>::type>& c,
                          int mode, int x0, int y0, int w, int h, double* out, cudaStream_t st) {
    if (w <= 0 || h <= 0) return cudaSuccess;
    dim3 b(128, 1), gr((unsigned)((w + 127) / 128), (unsigned)h, 1);
    fields_kernel<S><<<gr, b, 0, st>>>((const S*)buf, G, c, mode, x0, y0, w, h, out);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_nush(const void* buf, const Geom& G, const Coef<typename Real<S>::type>& c,
                        int mode, const WallSpec& W, double* out, cudaStream_t st) {
    nush_kernel<S><<<1, NUSH_THREADS, 0, st>>>((const S*)buf, G, c, mode, W, out);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_nush_tb(const void* buf, const Geom& G, const Coef<typename Real<S>::type>& c,
                           int mode, const WallSpec& W, double* out, cudaStream_t st) {
    nush_tb_kernel<S><<<1, NUSH_THREADS, 0, st>>>((const S*)buf, G, c, mode, W, out);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_residual(const void* buf, const Geom& G, const Coef<typename Real<S>::type>& c,
                            int mode, void* snap, double* partial, double* out,
                            cudaStream_t st) {
    using R = typename Real<S>::type;
    cudaError_t e = launch_residual_pass1<S, R>((const S*)buf, G, c, mode, (R*)snap, partial,
                                                RES_SLOTS, st);
    if (e != cudaSuccess) return e;
    residual_final_kernel<<<1, RES_THREADS, 0, st>>>(partial, RES_SLOTS, out);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_halo(void* buf, const Geom& G, int row, int up, void* face, int pack,
                        cudaStream_t st) {
    const dim3 gr((unsigned)((G.nx + 127) / 128), 5, 1);
    halo_kernel<S><<<gr, 128, 0, st>>>((S*)buf, G, row, up, (S*)face, pack);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE(S)                                                                      \
    template cudaError_t launch_init<S>(void*, void*, const Geom&,                             \
                                        const Coef<Real<S>::type>&, const InitSpec&, bool,     \
                                        cudaStream_t);                                         \
    template cudaError_t launch_step_ab<S>(const void*, void*, void*, const Geom&,             \
                                           const Coef<Real<S>::type>&, const LaunchCfg&);      \
    template cudaError_t launch_step_aa<S>(void*, void*, const Geom&,                          \
                                           const Coef<Real<S>::type>&, bool,                   \
                                           const LaunchCfg&);                                  \
    template cudaError_t launch_fields<S>(const void*, const Geom&,                            \
                                          const Coef<Real<S>::type>&, int, int, int, int, int, \
                                          double*, cudaStream_t);                              \
    template cudaError_t launch_nush<S>(const void*, const Geom&, const Coef<Real<S>::type>&,  \
                                        int, const WallSpec&, double*, cudaStream_t);          \
    template cudaError_t launch_nush_tb<S>(const void*, const Geom&, const Coef<Real<S>::type>&,\
                                           int, const WallSpec&, double*, cudaStream_t);       \
    template cudaError_t launch_residual<S>(const void*, const Geom&,                          \
                                            const Coef<Real<S>::type>&, int, void*, double*,   \
                                            double*, cudaStream_t);                            \
    template cudaError_t launch_halo<S>(void*, const Geom&, int, int, void*, int, cudaStream_t);

}  // namespace lbm
