// The fused step for 16-bit storage with two x-adjacent nodes per thread.
//
// The 16-bit kernels with one node per thread are issue-bound, not DRAM-bound: every
// stored value costs a conversion, a few integer instructions of stochastic rounding
// and a 16-bit store, and the FP32 collision is a few hundred scalar instructions per
// node.  Here a thread takes the nodes (i, j) and (i + 1, j) with i even:
//   - populations whose source (pull) or target (push) lies in the same column pair
//     move as one 32-bit word (two 16-bit values); the others as two 16-bit values;
//   - the collision runs once for both nodes on f2 values (packed FP32x2 arithmetic,
//     the same change-only form as the one-node code: collide() with R = f2);
//   - two values are converted and stochastically rounded by one cvt.rs (sm_100a and
//     later), with 32 random bits per pair from the node pair's stream.
// Only nodes away from the walls run here (every neighbour in the cavity): the inner
// column pairs (2, 3), (4, 5), ... of the rows 1 .. ny - 2.  The other nodes (the rows
// 0 and ny - 1, and the columns 0, 1, nx - 1 and, for even nx, nx - 2) form the "edge"
// set, stepped by the one-node code with the wall rules in the first block rows of the
// same launch (its registers fit the pair code's budget), so that every 16-bit step is one
// kernel and goes out as a programmatic dependent launch.  The in-place even step has no
// wall logic and runs every column pair (even nx).
#pragma once
#include "lbm_kernels.cuh"

namespace lbm {

// Pair loads and conversions of 16-bit storage.  ld2 reads two consecutive values at an
// even element offset (one 4-byte aligned word), ld1 one value; widen / narrow convert a
// word of two 16-bit values to and from an f2 (the first node in the low half).
template <typename S> struct Pair;

template <> struct Pair<__nv_bfloat16> {
    using S = __nv_bfloat16;
    __device__ static f2 widen(uint32_t u) {          // low half: first node
        return f2(make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u)));
    }
    __device__ static f2 ld2(const S* p) { return widen(*reinterpret_cast<const uint32_t*>(p)); }
    __device__ static f2 ld2_nc(const S* p) { return widen(__ldg(reinterpret_cast<const unsigned int*>(p))); }
    __device__ static float ld1(const S* p) { return __bfloat162float(*p); }
    __device__ static float ld1_nc(const S* p) { return __bfloat162float(__ldg(p)); }
    // two values packed, first node in the low half; stochastic rounding with the
    // random bits r (one 16-bit field per value), or to nearest even
    __device__ static uint32_t narrow(f2 v, int sr, uint32_t r) {
        uint32_t d;
        if (sr)
            asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x), "r"(r));
        else
            asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x));
        return d;
    }
};

// FP16 holds the deviations scaled by 2^12, as the one-node code does (Store<__half>).
template <> struct Pair<__half> {
    using S = __half;
    __device__ static f2 widen(uint32_t u) {
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u));
        return f2(__fmul2_rn(a, make_float2(Store<__half>::kInvScale, Store<__half>::kInvScale)));
    }
    __device__ static f2 ld2(const S* p) { return widen(*reinterpret_cast<const uint32_t*>(p)); }
    __device__ static f2 ld2_nc(const S* p) { return widen(__ldg(reinterpret_cast<const unsigned int*>(p))); }
    __device__ static float ld1(const S* p) { return Store<__half>::ld(p); }
    __device__ static float ld1_nc(const S* p) { return Store<__half>::ld_nc(p); }
    __device__ static uint32_t narrow(f2 v, int sr, uint32_t r) {
        const float2 s = __fmul2_rn(v.v, make_float2(Store<__half>::kScale, Store<__half>::kScale));
        uint32_t d;
        if (sr)
            asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(s.y), "f"(s.x), "r"(r));
        else
            asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(s.y), "f"(s.x));
        return d;
    }
};

// 32 random bits for the next stored pair: a step of the pair's linear congruential
// stream (the 32-bit constants of Numerical Recipes) with its high half folded into the
// low half, whose own bits have short periods.
__device__ __forceinline__ uint32_t pair_bits(uint32_t& state) {
    state = state * 1664525u + 1013904223u;
    return state ^ (state >> 16);
}

// Stream seed of a node pair: a hash of the first node's index and of the bits of two
// of each node's pre-collision populations (as node_seed(), for two nodes).
__device__ __forceinline__ uint32_t pair_seed(size_t self, f2 a, f2 b) {
    const uint32_t x = __float_as_uint(a.v.x) ^ mix32(__float_as_uint(a.v.y));
    const uint32_t y = __float_as_uint(b.v.x) ^ mix32(__float_as_uint(b.v.y));
    return mix32(x ^ mix32(y ^ mix32((uint32_t)self ^ (uint32_t)(self >> 32) * 0x27D4EB2Fu)));
}

// The values at p and p + 1 (the first and the second node's); `aligned`: p is at an even
// element offset (the source or target column pair is the node pair itself), so that one
// 32-bit word holds both.
template <typename S, bool NC>
__device__ __forceinline__ f2 ld_pair(const S* p, bool aligned) {
    if (aligned) return NC ? Pair<S>::ld2_nc(p) : Pair<S>::ld2(p);
    return f2(make_float2(NC ? Pair<S>::ld1_nc(p) : Pair<S>::ld1(p),
                          NC ? Pair<S>::ld1_nc(p + 1) : Pair<S>::ld1(p + 1)));
}
// CS: a streaming store (evict-first): the two-buffer step writes a buffer that it does not
// read again (GB300, 4096^2 BF16 two-buffer step 322 -> 318 us; the in-place steps, whose
// lines are read again, were slower with it: 302 -> 322 us; evict-first loads of the
// two-buffer source: 318 -> 337 us; streaming stores in the FP32 two-buffer step: 446 ->
// 449 us).
template <bool CS = false, typename S>
__device__ __forceinline__ void st_pair(S* p, bool aligned, f2 v, int sr, uint32_t& state) {
    const uint32_t r = sr ? pair_bits(state) : 0u;
    const uint32_t d = Pair<S>::narrow(v, sr, r);
    if (aligned) {
        if (CS)
            __stcs(reinterpret_cast<unsigned int*>(p), (unsigned int)d);
        else
            *reinterpret_cast<uint32_t*>(p) = d;
    } else {
        reinterpret_cast<unsigned short*>(p)[0] = (unsigned short)(d & 0xFFFFu);
        reinterpret_cast<unsigned short*>(p)[1] = (unsigned short)(d >> 16);
    }
}

// Pre-collision populations of the pair at `self` (even offset, both nodes away from the
// walls), pulled from x - e_q: slot q (two-buffer layout) or slot opp(q) (in-place layout
// after an even step).  Directions with e_x = 0 read one 32-bit word.
template <bool SWAP, bool NC, typename S>
__device__ __forceinline__ void gather_pair_pull(const S* __restrict__ buf, const Geom& G, size_t self,
                                                 f2 f[9], f2 g[5], f2 h[5]) {
    const S* p = buf + self;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const long long off = (long long)(QF + (SWAP ? opp_of(q) : q)) * (long long)G.plane -
                              ex_of(q) - (long long)ey_of(q) * G.pitch;
        f[q] = ld_pair<S, NC>(p + off, ex_of(q) == 0);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const long long d = -(long long)ex_of(q) - (long long)ey_of(q) * G.pitch;
        const int slot = SWAP ? opp_of(q) : q;
        g[q] = ld_pair<S, NC>(p + ((long long)(QG + slot) * (long long)G.plane + d), ex_of(q) == 0);
        h[q] = ld_pair<S, NC>(p + ((long long)(QH + slot) * (long long)G.plane + d), ex_of(q) == 0);
    }
}

// Natural (in-place, even level) populations of the pair: all 32-bit words.
template <typename S>
__device__ __forceinline__ void gather_pair_local(const S* __restrict__ buf, const Geom& G, size_t self,
                                                  f2 f[9], f2 g[5], f2 h[5]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = Pair<S>::ld2_nc(buf + (size_t)(QF + q) * G.plane + self);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        g[q] = Pair<S>::ld2_nc(buf + (size_t)(QG + q) * G.plane + self);
        h[q] = Pair<S>::ld2_nc(buf + (size_t)(QH + q) * G.plane + self);
    }
}

__device__ __forceinline__ void load_hist_pair(const float* __restrict__ hist, const Geom& G, size_t self,
                                               f2 hv[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) hv[k] = f2(*reinterpret_cast<const float2*>(hist + (size_t)k * G.plane + self));
}
__device__ __forceinline__ void store_hist_pair(float* __restrict__ hist, const Geom& G, size_t self,
                                                const f2 hv[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) *reinterpret_cast<float2*>(hist + (size_t)k * G.plane + self) = hv[k].v;
}

// Stores of the pair's post-collision populations, the flow lattice (f) and the two
// scalar lattices (g, h) apart: slot q of the pair itself (two-buffer layout,
// DST_OPP = false, streaming stores) or slot opp(q) (in-place even step, DST_OPP = true).
template <bool DST_OPP, typename S>
__device__ __forceinline__ void store_pair_self_f(S* __restrict__ dst, const Geom& G, size_t self, int sr,
                                                  const f2 f[9], uint32_t& state) {
#pragma unroll
    for (int q = 0; q < 9; ++q)
        st_pair<!DST_OPP>(dst + (size_t)(QF + (DST_OPP ? opp_of(q) : q)) * G.plane + self, true, f[q],
                          sr, state);
}
template <bool DST_OPP, typename S>
__device__ __forceinline__ void store_pair_self_gh(S* __restrict__ dst, const Geom& G, size_t self, int sr,
                                                   const f2 g[5], const f2 h[5], uint32_t& state) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int slot = DST_OPP ? opp_of(q) : q;
        st_pair<!DST_OPP>(dst + (size_t)(QG + slot) * G.plane + self, true, g[q], sr, state);
        st_pair<!DST_OPP>(dst + (size_t)(QH + slot) * G.plane + self, true, h[q], sr, state);
    }
}

// In-place odd step: slot q of x + e_q (both nodes away from the walls).
template <typename S>
__device__ __forceinline__ void store_pair_push_f(S* __restrict__ buf, const Geom& G, size_t self, int sr,
                                                  const f2 f[9], uint32_t& state) {
    S* p = buf + self;
#pragma unroll
    for (int q = 0; q < 9; ++q)
        st_pair(p + ((long long)(QF + q) * (long long)G.plane + ex_of(q) + (long long)ey_of(q) * G.pitch),
                ex_of(q) == 0, f[q], sr, state);
}
template <typename S>
__device__ __forceinline__ void store_pair_push_gh(S* __restrict__ buf, const Geom& G, size_t self, int sr,
                                                   const f2 g[5], const f2 h[5], uint32_t& state) {
    S* p = buf + self;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const long long d = (long long)ex_of(q) + (long long)ey_of(q) * G.pitch;
        st_pair(p + ((long long)(QG + q) * (long long)G.plane + d), ex_of(q) == 0, g[q], sr, state);
        st_pair(p + ((long long)(QH + q) * (long long)G.plane + d), ex_of(q) == 0, h[q], sr, state);
    }
}

// Number of inner column pairs (2, 3), (4, 5), ... with both nodes in 1 .. nx - 2.
__host__ __device__ inline int inner_pairs(int nx) { return nx >= 5 ? (nx - 3) / 2 : 0; }

// Thread m of a row of the inner-pair kernels takes the column pair (2m, 2m + 1); m = 0
// (the edge columns 0 and 1) has no work.  With rows starting on 128-byte lines, a warp's
// 32 pairs then cover whole lines of every 16-bit plane (128 B) and of the FP32 history
// (256 B); numbered from column 2 instead, each warp's words started 4 bytes into a line,
// so the first sector of every line of the two-buffer destination was written by two
// warps in two parts.
__device__ __forceinline__ bool inner_pair_of(const Geom& G, int erows, int& m, int& j) {
    m = blockIdx.x * blockDim.x + threadIdx.x;
    j = 1 + ((int)blockIdx.y - erows) * blockDim.y + threadIdx.y;
    return m >= 1 && m <= inner_pairs(G.nx) && j <= G.ny - 2;
}

// The edge set of the pair kernels: rows 0 and ny - 1 (all columns), then for the rows
// 1 .. ny - 2 the columns 0, 1, nx - 1 and, for even nx, nx - 2.
__host__ __device__ inline int edge_cols(int nx) { return (nx & 1) ? 3 : 4; }
__host__ __device__ inline long long edge_count(const Geom& G) {
    return 2LL * G.nx + (long long)(G.ny - 2) * edge_cols(G.nx);
}
__device__ __forceinline__ void edge_node(const Geom& G, long long k, int& i, int& j) {
    if (k < 2LL * G.nx) {
        j = k < G.nx ? 0 : G.ny - 1;
        i = (int)(k < G.nx ? k : k - G.nx);
        return;
    }
    const int e = edge_cols(G.nx);
    const long long r = k - 2LL * G.nx;
    j = 1 + (int)(r / e);
    const int c = (int)(r - (long long)(j - 1) * e);
    i = c == 0 ? 0 : c == 1 ? 1 : c == 2 ? G.nx - 1 : G.nx - 2;
}

// The edge blocks of a pair launch: the first `erows` rows of its grid take the edge set,
// one node per thread with the wall rules (first, so that their slower nodes do not form
// the launch's tail); the pair rows follow.  Edge node k of block (bx, by) and thread t:
// k = (by gridDim.x + bx) * threads + t.
__device__ __forceinline__ long long edge_index() {
    return ((long long)blockIdx.y * gridDim.x + blockIdx.x) * (blockDim.x * blockDim.y) +
           threadIdx.y * blockDim.x + threadIdx.x;
}

// One-node steps of the edge set: the two-buffer pull and the in-place odd step.
template <typename S>
__device__ __forceinline__ void ab_edge_node(const S* __restrict__ src, S* __restrict__ dst,
                                             float* __restrict__ hist, const Geom& G,
                                             const Coef<float>& c, long long k) {
    int i, j;
    edge_node(G, k, i, j);
    float f[9], g[5], h[5], hv[4];
    const size_t self = (size_t)j * G.pitch + i;
    gather_pull<false, true, false>(src, G, i, j, c, f, g, h);
    load_hist(hist, G, self, hv);
    uint32_t seed = node_seed(self, f[0], g[0]);
    collide(c, f, g, h, hv);
    store_ab(dst, G, self, c, f, g, h, seed);
    store_hist(hist, G, self, hv);
}

template <typename S>
__device__ __forceinline__ void aa_odd_edge_node(S* __restrict__ buf, float* __restrict__ hist,
                                                 const Geom& G, const Coef<float>& c, long long k) {
    int i, j;
    edge_node(G, k, i, j);
    float f[9], g[5], h[5], hv[4];
    const size_t self = (size_t)j * G.pitch + i;
    gather_pull<true, true, false>(buf, G, i, j, c, f, g, h);
    load_hist(hist, G, self, hv);
    uint32_t seed = node_seed(self, f[0], g[0]);
    collide(c, f, g, h, hv);
    store_aa_odd<false>(buf, G, i, j, self, c, f, g, h, seed);
    store_hist(hist, G, self, hv);
}

// ---- kernels -------------------------------------------------------------------------
// Two-buffer pull step: block (PAIR_BX, PAIR_BY) over (1 + pairs, erows + rows 1 .. ny - 2):
// the edge blocks (edge_index), then the inner column pairs, the first thread of a row idle
// (inner_pair_of).
// Launch shape: 128 pairs per block, at least 5 blocks per SM (96 registers).  GB300,
// 4096^2 BF16, us per step (two-buffer / in-place): 64 x 2 threads unbounded (118
// registers) 342 / 317; 128 x 1 held to 5 blocks 324 / 302 (6 blocks spill: 336 / 315;
// 4 blocks: 333 / 324).  The two-buffer kernel reads its source through the
// non-coherent path (nothing writes it during the step): 324 -> 322.  A persistent form
// that asked L2 for each block's next tile (prefetch.global.L2, a line per thread) ran
// slower (408 us).  Those figures predate the line-aligned numbering of inner_pair_of(),
// which with the streaming stores took the two sides to 303.5 / 300.1 us.
#ifndef LBM_PAIR_BX
#define LBM_PAIR_BX 128
#endif
#ifndef LBM_PAIR_BY
#define LBM_PAIR_BY 1
#endif
#ifndef LBM_PAIR_MIN_BLOCKS
#define LBM_PAIR_MIN_BLOCKS 5
#endif
#ifndef LBM_PAIR_AB_NC
#define LBM_PAIR_AB_NC true
#endif

constexpr int PAIR_BX = LBM_PAIR_BX, PAIR_BY = LBM_PAIR_BY;

template <typename S>
__global__ void __launch_bounds__(PAIR_BX * PAIR_BY, LBM_PAIR_MIN_BLOCKS)
step_ab_pair_kernel(const S* __restrict__ src, S* __restrict__ dst, float* __restrict__ hist, Geom G,
                    Coef<f2> c, Coef<float> c1, int erows) {
    pdl_trigger();
    pdl_wait();                                // launched by launch_pdl()
    if ((int)blockIdx.y < erows) {
        const long long k = edge_index();
        if (k < edge_count(G)) ab_edge_node(src, dst, hist, G, c1, k);
        return;
    }
    int m, j;
    if (!inner_pair_of(G, erows, m, j)) return;
    const size_t self = (size_t)j * G.pitch + 2 * m;
    f2 f[9], g[5], h[5], hv[4];
    gather_pair_pull<false, LBM_PAIR_AB_NC>(src, G, self, f, g, h);
    load_hist_pair(hist, G, self, hv);
    uint32_t state = pair_seed(self, f[0], g[0]);
    const Macro<f2> M = macro(c, f, g, h);
    collide_flow(c, M, f);
    store_pair_self_f<false>(dst, G, self, c.sr, f, state);   // f's registers free early
    collide_scalars(c, M, g, h, hv);
    store_pair_self_gh<false>(dst, G, self, c.sr, g, h, state);
    store_hist_pair(hist, G, self, hv);
}

// In-place even step of every column pair (even nx): block (PAIR_BX, PAIR_BY) over
// (nx / 2, ny).
template <typename S>
__global__ void __launch_bounds__(PAIR_BX * PAIR_BY, LBM_PAIR_MIN_BLOCKS)
step_aa_even_pair_kernel(S* __restrict__ buf, float* __restrict__ hist, Geom G, Coef<f2> c) {
    pdl_trigger();
    pdl_wait();                                // launched by launch_pdl()
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (2 * m >= G.nx || j >= G.ny) return;
    const size_t self = (size_t)j * G.pitch + 2 * m;
    f2 f[9], g[5], h[5], hv[4];
    gather_pair_local(buf, G, self, f, g, h);
    load_hist_pair(hist, G, self, hv);
    uint32_t state = pair_seed(self, f[0], g[0]);
    const Macro<f2> M = macro(c, f, g, h);
    collide_flow(c, M, f);
    store_pair_self_f<true>(buf, G, self, c.sr, f, state);
    collide_scalars(c, M, g, h, hv);
    store_pair_self_gh<true>(buf, G, self, c.sr, g, h, state);
    store_hist_pair(hist, G, self, hv);
}

// In-place odd step: the edge blocks, then the inner column pairs (each thread reads and
// writes only its own node's or pair's locations, so the two parts touch disjoint memory).
template <typename S>
__global__ void __launch_bounds__(PAIR_BX * PAIR_BY, LBM_PAIR_MIN_BLOCKS)
step_aa_odd_pair_kernel(S* __restrict__ buf, float* __restrict__ hist, Geom G, Coef<f2> c,
                        Coef<float> c1, int erows) {
    pdl_trigger();
    pdl_wait();                                // launched by launch_pdl()
    if ((int)blockIdx.y < erows) {
        const long long k = edge_index();
        if (k < edge_count(G)) aa_odd_edge_node(buf, hist, G, c1, k);
        return;
    }
    int m, j;
    if (!inner_pair_of(G, erows, m, j)) return;
    const size_t self = (size_t)j * G.pitch + 2 * m;
    f2 f[9], g[5], h[5], hv[4];
    gather_pair_pull<true, true>(buf, G, self, f, g, h);
    load_hist_pair(hist, G, self, hv);
    uint32_t state = pair_seed(self, f[0], g[0]);
    const Macro<f2> M = macro(c, f, g, h);
    collide_flow(c, M, f);
    store_pair_push_f(buf, G, self, c.sr, f, state);
    collide_scalars(c, M, g, h, hv);
    store_pair_push_gh(buf, G, self, c.sr, g, h, state);
    store_hist_pair(hist, G, self, hv);
}

}  // namespace lbm
