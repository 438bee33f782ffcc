// Kernels of the fused three-lattice step and its read-outs.  Included by the
// per-precision translation units, which instantiate them.
#pragma once
#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace lbm {

// ---- programmatic dependent launch ----------------------------------------------------
// A kernel launched by launch_pdl() may be scheduled while the kernel before it on the
// same stream is still running.  pdl_trigger() at the start of every CTA lets the next
// launch begin once all CTAs of this one have started; pdl_wait() holds a CTA until the
// launch before it has completed and its writes are visible.  A kernel that waits before
// its first access to the state, in every thread, and reads before that only what no
// kernel writes, gives the results of ordinary stream order, and it completes only after
// the launch before it.  Under an ordinary launch (also what launch_pdl() makes on the
// legacy default stream, with its implicit synchronisation) both instructions return at
// once.
#ifndef LBM_PDL
#define LBM_PDL 1
#endif
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed =
        LBM_PDL && st != nullptr && st != cudaStreamLegacy ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Which wall a link crosses.  Sides: 0 left (x = 0), 1 right (x = nx),
// 2 bottom (y = 0), 3 top (y = ny).
// A population pulled along direction q from x - e_q crosses the wall behind it:
__host__ __device__ constexpr int pull_side(int q) {
    return q == 1 ? 0 : q == 3 ? 1 : q == 2 ? 2 : 3;
}
// A population pushed along direction q to x + e_q crosses the wall ahead of it:
__host__ __device__ constexpr int push_side(int q) {
    return q == 1 ? 1 : q == 3 ? 0 : q == 2 ? 3 : 2;
}

template <typename R>
__device__ __forceinline__ R wall_value(const Coef<R>& c, const R* wall, int side, R reflected) {
    // Dirichlet (anti-bounce-back, in deviations): -g*_opp + 2 w~ (Phi_w - Phi0);
    // adiabatic (bounce-back): g*_opp.
    return ((c.dirichlet_mask >> side) & 1) ? wall[side] - reflected : reflected;
}

// Wall side of a link whose far end (ti, tj) lies outside the cavity; a link
// through a corner takes the bottom / top wall.
__device__ __forceinline__ int link_side(int ti, int tj, const Geom& G) {
    return (unsigned)tj >= (unsigned)G.ny ? (tj < 0 ? 2 : 3) : (ti < 0 ? 0 : 1);
}

// Momentum a wall moving with u_w gives a population bounced back into direction q:
// 2 w_q rho0 (e_q . u_w) / c_s^2 (halfway bounce-back off a moving wall; the
// no-slip rule is u_w = 0).
template <typename R>
__device__ __forceinline__ R wall_momentum(const Coef<R>& c, int side, int q) {
    return R(w9_of(q)) * (R(ex_of(q)) * c.wmom[side][0] + R(ey_of(q)) * c.wmom[side][1]);
}

// Pre-collision populations of node (i, j) at level t from a buffer of level
// t-1 post-collision values (pull streaming, Eq. 11, with the halfway wall
// rules).  SWAP = false: two-buffer layout, slot q of the source node.
// SWAP = true: in-place AA layout after an even step, slot opp(q) of the source.
// EXT: the cavity may have moving walls (checked at run time); without it the
// moving-wall code is not compiled in (the fast path of the plain cavity).
// Nodes whose eight neighbours all lie in the cavity (every node but the outermost
// ring) can take a path with no wall rule, where each address is the node's own plus
// an offset that is the same for every thread (kept in uniform registers).  The
// single-cavity kernels for the inner nodes call it directly (with the ring in a
// launch of its own); inside gather_pull it is taken for 16-bit storage in the
// two-buffer layout (the batch kernels), whose kernels are issue-bound.  Compiled
// into the DRAM-bound FP32 kernels, either way, it measured slower (3-13 %).
// NC: load through the non-coherent path (the in-place odd step, whose threads each
// write only the locations they have read themselves).
template <bool SWAP, bool WITH_F, bool NC = false, typename S, typename R>
__device__ __forceinline__ void gather_pull_inner(const S* __restrict__ buf, const Geom& G,
                                                  size_t self, R f[9], R g[5], R h[5]) {
    const S* p = buf + self;
    if (WITH_F) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const long long off = (long long)(QF + (SWAP ? opp_of(q) : q)) * (long long)G.plane -
                                  ex_of(q) - (long long)ey_of(q) * G.pitch;
            f[q] = NC ? Store<S>::ld_nc(p + off) : Store<S>::ld(p + off);
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const long long d = -(long long)ex_of(q) - (long long)ey_of(q) * G.pitch;
        const int slot = SWAP ? opp_of(q) : q;
        const S* pg = p + ((long long)(QG + slot) * (long long)G.plane + d);
        const S* ph = p + ((long long)(QH + slot) * (long long)G.plane + d);
        g[q] = NC ? Store<S>::ld_nc(pg) : Store<S>::ld(pg);
        h[q] = NC ? Store<S>::ld_nc(ph) : Store<S>::ld(ph);
    }
}

template <bool SWAP, bool WITH_F, bool EXT = true, typename S, typename R>
__device__ __forceinline__ void gather_pull(const S* __restrict__ buf, const Geom& G, int i, int j,
                                            const Coef<R>& c, R f[9], R g[5], R h[5]) {
    const size_t self = (size_t)j * G.pitch + i;
    if (Store<S>::kLow && !SWAP && (unsigned)(i - 1) < (unsigned)(G.nx - 2) &&
        (unsigned)(j - 1) < (unsigned)(G.ny - 2)) {
        gather_pull_inner<SWAP, WITH_F>(buf, G, self, f, g, h);
        return;
    }
    if (WITH_F) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int si = i - ex_of(q), sj = j - ey_of(q);
            const bool in = (unsigned)si < (unsigned)G.nx && (unsigned)sj < (unsigned)G.ny;
            const int slot_src = SWAP ? opp_of(q) : q;
            const int slot_self = SWAP ? q : opp_of(q);
            const S* p = in ? buf + (size_t)(QF + slot_src) * G.plane + (size_t)sj * G.pitch + si
                            : buf + (size_t)(QF + slot_self) * G.plane + self;
            f[q] = Store<S>::ld(p);   // halfway bounce-back when !in
            if (EXT && !in && c.moving) f[q] += wall_momentum(c, link_side(si, sj, G), q);
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int si = i - ex_of(q), sj = j - ey_of(q);
        const bool in = (unsigned)si < (unsigned)G.nx && (unsigned)sj < (unsigned)G.ny;
        const int slot_src = SWAP ? opp_of(q) : q;
        const int slot_self = SWAP ? q : opp_of(q);
        const size_t off = in ? (size_t)sj * G.pitch + si : self;
        const int slot = in ? slot_src : slot_self;
        R vg = Store<S>::ld(buf + (size_t)(QG + slot) * G.plane + off);
        R vh = Store<S>::ld(buf + (size_t)(QH + slot) * G.plane + off);
        if (q > 0 && !in) {
            vg = wall_value(c, c.wallT, pull_side(q), vg);
            vh = wall_value(c, c.wallC, pull_side(q), vh);
        }
        g[q] = vg;
        h[q] = vh;
    }
}

// Natural (in-place) pre-collision populations of node (i, j).
template <bool WITH_F, typename S, typename R>
__device__ __forceinline__ void gather_local(const S* __restrict__ buf, const Geom& G, int i,
                                             int j, R f[9], R g[5], R h[5]) {
    const size_t self = (size_t)j * G.pitch + i;
    if (WITH_F) {
#pragma unroll
        for (int q = 0; q < 9; ++q) f[q] = Store<S>::ld_nc(buf + (size_t)(QF + q) * G.plane + self);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        g[q] = Store<S>::ld_nc(buf + (size_t)(QG + q) * G.plane + self);
        h[q] = Store<S>::ld_nc(buf + (size_t)(QH + q) * G.plane + self);
    }
}

// ---- walls with nodes on them (Sec. 3.3) --------------------------------------------
// Wall value (deviation) of a scalar at a wall node whose inward link is (di, dj):
// a Dirichlet side at the node gives its value (the left / right side first);
// otherwise Eq. 36 / 37 along the link, Phi_b = (4 Phi_f - Phi_ff - 2 dx . grad Phi_b) / 3,
// with dx . grad Phi_b = sum over the node's sides of b_s (Phi_b - Phi_w,s) (b_s = Bi / L
// of a convective side, Eq. 39; 0 for an adiabatic one), solved for Phi_b.
template <typename R>
__device__ __forceinline__ R nee_scalar(const Coef<R>& c, int di, int dj, const R Pw[4],
                                        const R b[4], R Pf, R Pff) {
    const int sv = di > 0 ? 0 : 1, sh = dj > 0 ? 2 : 3;
    if (di && b[sv] == R(0) && ((c.dirichlet_mask >> sv) & 1)) return Pw[sv];
    if (dj && b[sh] == R(0) && ((c.dirichlet_mask >> sh) & 1)) return Pw[sh];
    R a = R(0), w = R(0);
    if (di) { a += b[sv]; w += b[sv] * Pw[sv]; }
    if (dj) { a += b[sh]; w += b[sh] * Pw[sh]; }
    return (R(4) * Pf - Pff + R(2) * w) / (R(3) + R(2) * a);
}

// Pre-collision populations (deviations) of wall node (i, j) with inward link (di, dj)
// in the two-buffer pull layout, rebuilt by Eqs. 33-35 from the nearest interior node
// x_f = (i + di, j + dj) and, for the wall value, x_ff = (i + 2 di, j + 2 dj):
//   f'_b = f'_f + f^eq(rho_f, u_w; eps_b) - f^eq(rho_f, u_f; eps_f)
//        = f'_f + w_q [Q(u_w, eps_b) - Q(u_f, eps_f)],  Q = 3 e.u + 4.5 (e.u)^2 / eps - 1.5 u^2 / eps
//   g'_b = g'_f + a0/a1 (T'_b - T'_f) + (e_q . (u_w T_b - u_f T_f)) / 2           (Eq. 34)
//   h'_b = h'_f + a_b C'_b - a_f C'_f + (e_q . (u_w C_b - u_f C_f)) / 2           (Eq. 35)
// (the storage shifts of f, g, h cancel against those of x_f).  u_f from Eq. 18 with
// x_f's porous constants; u_w the velocity of the wall (the bottom / top wall's at a corner).
template <typename S, typename R>
__device__ __forceinline__ void nee_rebuild(const S* __restrict__ buf, const Geom& G, int i, int j,
                                            int di, int dj, const Coef<R>& c, R f[9], R g[5],
                                            R h[5]) {
    const int fi = i + di, fj = j + dj;
    gather_pull<false, true, false>(buf, G, fi, fj, c, f, g, h);   // x_f is interior
    R g2[5], h2[5], dummy[9];
    gather_pull<false, false, false>(buf, G, i + 2 * di, j + 2 * dj, c, dummy, g2, h2);
    Coef<R> cf = c, cb = c;
    R inv_eps_ff = c.inv_eps;
    if (c.poro) {
        porous_at(cf, (size_t)fj * G.pitch + fi, G.plane);
        porous_at(cb, (size_t)j * G.pitch + i, G.plane);
        inv_eps_ff = R(1) / c.poro[(size_t)(j + 2 * dj) * G.pitch + (i + 2 * di)];
    }
    const Macro<R> M = macro(cf, f, g, h);
    const R Tff = (((g2[0] + g2[1]) + (g2[2] + g2[3])) + g2[4]) * c.inv_sigma;   // Eq. 26
    const R Cff = (((h2[0] + h2[1]) + (h2[2] + h2[3])) + h2[4]) * inv_eps_ff;
    const R Tb = nee_scalar(c, di, dj, c.TwP, c.bT, M.Tp, Tff);
    const R Cb = nee_scalar(c, di, dj, c.CwP, c.bC, M.Cp, Cff);
    const int sv = dj ? (dj > 0 ? 2 : 3) : (di > 0 ? 0 : 1);
    const R ubx = c.uwall[sv][0], uby = c.uwall[sv][1];
    const R ub2 = ubx * ubx + uby * uby, uf2 = M.ux * M.ux + M.uy * M.uy;
    const R ieb = cb.inv_eps_f, ief = cf.inv_eps_f;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const R eb = R(ex_of(q)) * ubx + R(ey_of(q)) * uby;
        const R ef = R(ex_of(q)) * M.ux + R(ey_of(q)) * M.uy;
        const R Qb = R(3) * eb + (R(4.5) * eb * eb - R(1.5) * ub2) * ieb;
        const R Qf = R(3) * ef + (R(4.5) * ef * ef - R(1.5) * uf2) * ief;
        f[q] += R(w9_of(q)) * (Qb - Qf);
    }
    const R TB = c.T0 + Tb, TF = c.T0 + M.Tp, CB = c.C0 + Cb, CF = c.C0 + M.Cp;
    g[0] += c.aT0 * (Tb - M.Tp);
    h[0] += cb.aC0 * Cb - cf.aC0 * M.Cp;
#pragma unroll
    for (int q = 1; q < 5; ++q) {
        const R eb = R(ex_of(q)) * ubx + R(ey_of(q)) * uby;
        const R ef = R(ex_of(q)) * M.ux + R(ey_of(q)) * M.uy;
        g[q] += c.aT1 * (Tb - M.Tp) + R(0.5) * (eb * TB - ef * TF);
        h[q] += cb.aC1 * Cb - cf.aC1 * M.Cp + R(0.5) * (eb * CB - ef * CF);
    }
}

// Pre-collision populations of node (i, j) on a grid with wall nodes: the plain pull
// inside (every neighbour is a node), the rebuild of Eqs. 33-35 on the walls.
template <typename S, typename R>
__device__ __forceinline__ void gather_nee(const S* __restrict__ buf, const Geom& G, int i, int j,
                                           const Coef<R>& c, R f[9], R g[5], R h[5]) {
    const int di = i == 0 ? 1 : (i == G.nx - 1 ? -1 : 0);
    const int dj = j == 0 ? 1 : (j == G.ny - 1 ? -1 : 0);
    if (di | dj)
        nee_rebuild(buf, G, i, j, di, dj, c, f, g, h);
    else
        gather_pull<false, true, false>(buf, G, i, j, c, f, g, h);
}

// The same with the mode fixed at compile time (no code for the other two modes).
template <int MODE, typename S, typename R>
__device__ __forceinline__ void gather_m(const S* __restrict__ buf, const Geom& G, int i, int j,
                                         const Coef<R>& c, R f[9], R g[5], R h[5]) {
    if (MODE == GATHER_PULL_AB)
        gather_pull<false, true>(buf, G, i, j, c, f, g, h);
    else if (MODE == GATHER_PULL_AA)
        gather_pull<true, true>(buf, G, i, j, c, f, g, h);
    else if (MODE == GATHER_NEE_AB)
        gather_nee(buf, G, i, j, c, f, g, h);
    else
        gather_local<true>(buf, G, i, j, f, g, h);
}

template <bool WITH_F, typename S, typename R>
__device__ __forceinline__ void gather(int mode, const S* __restrict__ buf, const Geom& G, int i,
                                       int j, const Coef<R>& c, R f[9], R g[5], R h[5]) {
    if (mode == GATHER_PULL_AB)
        gather_pull<false, WITH_F>(buf, G, i, j, c, f, g, h);
    else if (mode == GATHER_PULL_AA)
        gather_pull<true, WITH_F>(buf, G, i, j, c, f, g, h);
    else if (mode == GATHER_NEE_AB)
        gather_nee(buf, G, i, j, c, f, g, h);
    else
        gather_local<WITH_F>(buf, G, i, j, f, g, h);
}

template <typename R>
__device__ __forceinline__ void load_hist(const R* __restrict__ hist, const Geom& G, size_t self,
                                          R hv[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) hv[k] = hist[(size_t)k * G.plane + self];
}
template <typename R>
__device__ __forceinline__ void store_hist(R* __restrict__ hist, const Geom& G, size_t self,
                                           const R hv[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) hist[(size_t)k * G.plane + self] = hv[k];
}

// ---- stores of a node's post-collision populations ----------------------------------
// Two-buffer layout: slot q of the node itself in the destination buffer.
template <typename S, typename R>
__device__ __forceinline__ void store_ab(S* __restrict__ dst, const Geom& G, size_t self,
                                         const Coef<R>& c, const R f[9], const R g[5],
                                         const R h[5], uint32_t& seed) {
    const int sr = sr_node<S>(c.sr, f, g, h);
#pragma unroll
    for (int q = 0; q < 9; ++q) put(dst + (size_t)(QF + q) * G.plane + self, f[q], sr, seed, q);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        put(dst + (size_t)(QG + q) * G.plane + self, g[q], sr, seed, QG + q);
        put(dst + (size_t)(QH + q) * G.plane + self, h[q], sr, seed, QH + q);
    }
}

// In-place layout, even step: slot opp(q) of the node itself.
template <typename S, typename R>
__device__ __forceinline__ void store_aa_even(S* __restrict__ buf, const Geom& G, size_t self,
                                              const Coef<R>& c, const R f[9], const R g[5],
                                              const R h[5], uint32_t& seed) {
    const int sr = sr_node<S>(c.sr, f, g, h);
#pragma unroll
    for (int q = 0; q < 9; ++q)
        put(buf + (size_t)(QF + opp_of(q)) * G.plane + self, f[q], sr, seed, q);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        put(buf + (size_t)(QG + opp_of(q)) * G.plane + self, g[q], sr, seed, QG + q);
        put(buf + (size_t)(QH + opp_of(q)) * G.plane + self, h[q], sr, seed, QH + q);
    }
}

// In-place layout, odd step: slot q of the neighbour x + e_q, or, where that link
// crosses a wall, the wall rule's value in slot opp(q) of the node itself.
template <bool EXT = true, typename S, typename R>
__device__ __forceinline__ void store_aa_odd(S* __restrict__ buf, const Geom& G, int i, int j,
                                             size_t self, const Coef<R>& c, const R f[9],
                                             const R g[5], const R h[5], uint32_t& seed) {
    const int sr = sr_node<S>(c.sr, f, g, h);   // the wall rules add finite constants
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int ti = i + ex_of(q), tj = j + ey_of(q);
        const bool in = (unsigned)ti < (unsigned)G.nx && (unsigned)tj < (unsigned)G.ny;
        S* p = in ? buf + (size_t)(QF + q) * G.plane + (size_t)tj * G.pitch + ti
                  : buf + (size_t)(QF + opp_of(q)) * G.plane + self;
        R v = f[q];
        if (EXT && !in && c.moving) v -= wall_momentum(c, link_side(ti, tj, G), q);
        put(p, v, sr, seed, q);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int ti = i + ex_of(q), tj = j + ey_of(q);
        const bool in = (unsigned)ti < (unsigned)G.nx && (unsigned)tj < (unsigned)G.ny;
        R vg = g[q], vh = h[q];
        size_t off = self;
        int slot = opp_of(q);
        if (in) {
            off = (size_t)tj * G.pitch + ti;
            slot = q;
        } else if (q > 0) {
            vg = wall_value(c, c.wallT, push_side(q), vg);
            vh = wall_value(c, c.wallC, push_side(q), vh);
        }
        put(buf + (size_t)(QG + slot) * G.plane + off, vg, sr, seed, QG + q);
        put(buf + (size_t)(QH + slot) * G.plane + off, vh, sr, seed, QH + q);
    }
}

// Collision with the node's own porous constants when the cavity has a porous field
// (EXT builds only; the plain cavity's kernel compiles one collision).
template <bool EXT, typename R>
__device__ __forceinline__ void collide_node(const Coef<R>& c, size_t self, size_t plane, R f[9],
                                             R g[5], R h[5], R hv[4]) {
    if (EXT && c.poro) {
        Coef<R> cl = c;
        porous_at(cl, self, plane);
        collide(cl, f, g, h, hv);
    } else {
        collide(c, f, g, h, hv);
    }
}

// ---- the fused step, two-buffer pull layout ---------------------------------------
// One node of the two-buffer step; INNER: all eight neighbours in the cavity, no wall
// logic compiled in.
template <typename S, bool EXT, bool INNER, typename R>
__device__ __forceinline__ void ab_node(const S* __restrict__ src, S* __restrict__ dst, R* __restrict__ hist,
                                        const Geom& G, const Coef<R>& c, int i, int j) {
    R f[9], g[5], h[5], hv[4];
    const size_t self = (size_t)j * G.pitch + i;
    if (INNER)
        gather_pull_inner<false, true>(src, G, self, f, g, h);
    else
        gather_pull<false, true, EXT>(src, G, i, j, c, f, g, h);
    load_hist(hist, G, self, hv);
    uint32_t seed = Store<S>::kLow ? node_seed(self + c.seed_off, f[0], g[0]) : 0u;
    collide_node<EXT>(c, self, G.plane, f, g, h, hv);
    store_ab(dst, G, self, c, f, g, h, seed);
    store_hist(hist, G, self, hv);
}

// EXT = true for cavities with moving walls or porous fields, false otherwise.
// INNER = true: the outermost ring of nodes is left to nee_ring_kernel (walls with
// nodes on them), so this kernel keeps the plain pull's registers and occupancy.
template <typename S, bool EXT, bool INNER = false>
__global__ void __launch_bounds__(256)
step_ab_kernel(const S* __restrict__ src, S* __restrict__ dst,
               typename Real<S>::type* __restrict__ hist, Geom G,
               Coef<typename Real<S>::type> c) {
    using R = typename Real<S>::type;
    pdl_trigger();
    pdl_wait();                                // launched by launch_pdl() in one-kernel steps
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = G.jb + blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.je) return;
    if (INNER && !((unsigned)(i - 1) < (unsigned)(G.nx - 2) && (unsigned)(j - 1) < (unsigned)(G.ny - 2)))
        return;
    ab_node<S, EXT, INNER>(src, dst, hist, G, c, i, j);
}

// Node k of the outermost ring, k = 0 .. 2 nx + 2 (ny - 2) - 1: bottom row, top row,
// left column, right column (rows 1 .. ny - 2).
__device__ __forceinline__ void ring_node(const Geom& G, long long k, int& i, int& j) {
    if (k < G.nx) {
        i = (int)k; j = 0;
    } else if (k < 2LL * G.nx) {
        i = (int)(k - G.nx); j = G.ny - 1;
    } else if (k < 2LL * G.nx + (G.ny - 2)) {
        i = 0; j = (int)(k - 2LL * G.nx) + 1;
    } else {
        i = G.nx - 1; j = (int)(k - 2LL * G.nx - (G.ny - 2)) + 1;
    }
}

// The outermost ring of nodes of the two-buffer step with halfway walls (the inner
// nodes run step_ab_kernel<S, EXT, true>): node k of the ring as in ring_node().
template <typename S, bool EXT>
__global__ void __launch_bounds__(128)
step_ab_ring_kernel(const S* __restrict__ src, S* __restrict__ dst,
                    typename Real<S>::type* __restrict__ hist, Geom G,
                    Coef<typename Real<S>::type> c) {
    using R = typename Real<S>::type;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2LL * G.nx + 2LL * (G.ny - 2)) return;
    int i, j;
    ring_node(G, k, i, j);
    R f[9], g[5], h[5], hv[4];
    const size_t self = (size_t)j * G.pitch + i;
    gather_pull<false, true, EXT>(src, G, i, j, c, f, g, h);
    load_hist(hist, G, self, hv);
    uint32_t seed = Store<S>::kLow ? node_seed(self, f[0], g[0]) : 0u;
    collide_node<EXT>(c, self, G.plane, f, g, h, hv);
    store_ab(dst, G, self, c, f, g, h, seed);
    store_hist(hist, G, self, hv);
}

// ---- the fused step with wall nodes (Sec. 3.3), two-buffer pull layout ---------------
// The inner nodes take step_ab_kernel<S, EXT, true> (the plain pull); nee_ring_node
// takes the ring of wall nodes, k = 0 .. 2 nx + 2 (ny - 2) - 1 (bottom row, top row,
// left column, right column): populations rebuilt by Eqs. 33-35 from the
// post-streaming populations of x_f and x_ff (both pulled from src, which no
// launch of this step writes), then the same collision as every node.
template <typename S, typename R>
__device__ __forceinline__ void nee_ring_node(const S* __restrict__ src, S* __restrict__ dst, R* __restrict__ hist,
                                              const Geom& G, const Coef<R>& c, long long k) {
    int i, j;
    if (k < G.nx) {
        i = (int)k; j = 0;
    } else if (k < 2LL * G.nx) {
        i = (int)(k - G.nx); j = G.ny - 1;
    } else if (k < 2LL * G.nx + (G.ny - 2)) {
        i = 0; j = (int)(k - 2LL * G.nx) + 1;
    } else {
        i = G.nx - 1; j = (int)(k - 2LL * G.nx - (G.ny - 2)) + 1;
    }
    R f[9], g[5], h[5], hv[4];
    const size_t self = (size_t)j * G.pitch + i;
    gather_nee(src, G, i, j, c, f, g, h);
    load_hist(hist, G, self, hv);
    uint32_t seed = Store<S>::kLow ? node_seed(self, f[0], g[0]) : 0u;
    collide_node<true>(c, self, G.plane, f, g, h, hv);
    store_ab(dst, G, self, c, f, g, h, seed);
    store_hist(hist, G, self, hv);
}

template <typename S>
__global__ void __launch_bounds__(256)
nee_ring_kernel(const S* __restrict__ src, S* __restrict__ dst,
                typename Real<S>::type* __restrict__ hist, Geom G,
                Coef<typename Real<S>::type> c) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2LL * G.nx + 2LL * (G.ny - 2)) return;
    nee_ring_node(src, dst, hist, G, c, k);
}

// The step with wall nodes as one launch: the first `rrows` block rows take the ring of
// wall nodes (node k = (by gridDim.x + bx) * threads + t), the others the inner nodes
// (row j = by - rrows) with the plain pull; held to the inner code's 64 registers.
template <typename S, bool EXT>
__global__ void __launch_bounds__(256, 4)
step_ab_nee_fused_kernel(const S* __restrict__ src, S* __restrict__ dst,
                         typename Real<S>::type* __restrict__ hist, Geom G,
                         Coef<typename Real<S>::type> c, int rrows) {
    pdl_trigger();
    pdl_wait();                                // launched by launch_pdl()
    if ((int)blockIdx.y < rrows) {
        const long long k = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * (blockDim.x * blockDim.y) +
                            threadIdx.y * blockDim.x + threadIdx.x;
        if (k < 2LL * G.nx + 2LL * (G.ny - 2)) nee_ring_node(src, dst, hist, G, c, k);
        return;
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = ((int)blockIdx.y - rrows) * blockDim.y + threadIdx.y;
    if (!((unsigned)(i - 1) < (unsigned)(G.nx - 2) && (unsigned)(j - 1) < (unsigned)(G.ny - 2)))
        return;
    ab_node<S, EXT, true>(src, dst, hist, G, c, i, j);
}

// History (T u, C u) at t = 0 of the wall nodes, from their rebuilt initial state
// (init_kernel wrote the interior's and the buffer the pull reads).
template <typename S>
__global__ void nee_hist_kernel(const S* __restrict__ buf, typename Real<S>::type* __restrict__ hist,
                                Geom G, Coef<typename Real<S>::type> c) {
    using R = typename Real<S>::type;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    if (i > 0 && i < G.nx - 1 && j > 0 && j < G.ny - 1) return;
    R f[9], g[5], h[5];
    gather_nee(buf, G, i, j, c, f, g, h);
    const size_t self = (size_t)j * G.pitch + i;
    Coef<R> cl = c;
    if (c.poro) porous_at(cl, self, G.plane);
    const Macro<R> M = macro(cl, f, g, h);
    const R T = c.T0 + M.Tp, C = c.C0 + M.Cp;
    const R hv[4] = {T * M.ux, T * M.uy, C * M.ux, C * M.uy};
    store_hist(hist, G, self, hv);
}

// ---- the fused step, in-place AA layout -------------------------------------------
// Even step (level t even): natural pre-collision values at x -> collide ->
// post-collision value of direction q stored in slot opp(q) of x.
// Odd step: pull from the swapped slots of the neighbours (with wall rules),
// collide, push post-collision value of direction q into slot q of x + e_q
// (or, where that link crosses a wall, the reflected value into slot opp(q)
// of x).  Each thread reads and writes the same set of locations, so the
// update is race-free in place.
template <typename S, bool ODD, bool EXT>
__global__ void __launch_bounds__(256)
step_aa_kernel(S* __restrict__ buf, typename Real<S>::type* __restrict__ hist, Geom G,
               Coef<typename Real<S>::type> c) {
    using R = typename Real<S>::type;
    pdl_trigger();
    pdl_wait();                                // launched by launch_pdl()
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    R f[9], g[5], h[5], hv[4];
    const size_t self = (size_t)j * G.pitch + i;
    if (ODD)
        gather_pull<true, true, EXT>(buf, G, i, j, c, f, g, h);
    else
        gather_local<true>(buf, G, i, j, f, g, h);
    load_hist(hist, G, self, hv);
    uint32_t seed = Store<S>::kLow ? node_seed(self, f[0], g[0]) : 0u;
    collide_node<EXT>(c, self, G.plane, f, g, h, hv);
    if (ODD)
        store_aa_odd<EXT>(buf, G, i, j, self, c, f, g, h, seed);
    else
        store_aa_even(buf, G, self, c, f, g, h, seed);
    store_hist(hist, G, self, hv);
}

// The odd step split in two launches: the inner nodes (all eight neighbours in the
// cavity) with no wall logic and uniform address offsets, and the ring of outermost
// nodes with the general code.  Each thread reads and writes only its own set of
// locations, so the two launches touch disjoint memory.  The odd step compiled as
// one kernel needed 78 registers and 1.6x the even step's instructions.
template <typename S, typename R>
__device__ __forceinline__ void store_aa_odd_inner(S* __restrict__ buf, const Geom& G, size_t self,
                                                   const Coef<R>& c, const R f[9], const R g[5],
                                                   const R h[5], uint32_t& seed) {
    const int sr = sr_node<S>(c.sr, f, g, h);
    S* p = buf + self;
#pragma unroll
    for (int q = 0; q < 9; ++q)
        put(p + ((long long)(QF + q) * (long long)G.plane + ex_of(q) + (long long)ey_of(q) * G.pitch),
            f[q], sr, seed, q);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const long long d = (long long)ex_of(q) + (long long)ey_of(q) * G.pitch;
        put(p + ((long long)(QG + q) * (long long)G.plane + d), g[q], sr, seed, QG + q);
        put(p + ((long long)(QH + q) * (long long)G.plane + d), h[q], sr, seed, QH + q);
    }
}

// One node of the odd step's inner part (all eight neighbours in the cavity) and of its
// ring of outermost nodes (ring_node(k), the general code with the wall rules).
template <typename S, bool EXT, typename R>
__device__ __forceinline__ void aa_odd_inner_node(S* __restrict__ buf, R* __restrict__ hist, const Geom& G,
                                                  const Coef<R>& c, int i, int j) {
    R f[9], g[5], h[5], hv[4];
    const size_t self = (size_t)j * G.pitch + i;
    gather_pull_inner<true, true, true>(buf, G, self, f, g, h);
    load_hist(hist, G, self, hv);
    uint32_t seed = Store<S>::kLow ? node_seed(self, f[0], g[0]) : 0u;
    collide_node<EXT>(c, self, G.plane, f, g, h, hv);
    store_aa_odd_inner(buf, G, self, c, f, g, h, seed);
    store_hist(hist, G, self, hv);
}
template <typename S, bool EXT, typename R>
__device__ __forceinline__ void aa_odd_ring_node(S* __restrict__ buf, R* __restrict__ hist, const Geom& G,
                                                 const Coef<R>& c, long long k) {
    int i, j;
    ring_node(G, k, i, j);
    R f[9], g[5], h[5], hv[4];
    const size_t self = (size_t)j * G.pitch + i;
    gather_pull<true, true, EXT>(buf, G, i, j, c, f, g, h);
    load_hist(hist, G, self, hv);
    uint32_t seed = Store<S>::kLow ? node_seed(self, f[0], g[0]) : 0u;
    collide_node<EXT>(c, self, G.plane, f, g, h, hv);
    store_aa_odd<EXT>(buf, G, i, j, self, c, f, g, h, seed);
    store_hist(hist, G, self, hv);
}
__host__ __device__ inline long long ring_count(const Geom& G) { return 2LL * G.nx + 2LL * (G.ny - 2); }

template <typename S, bool EXT>
__global__ void __launch_bounds__(256)
step_aa_odd_inner_kernel(S* __restrict__ buf, typename Real<S>::type* __restrict__ hist, Geom G,
                         Coef<typename Real<S>::type> c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (!((unsigned)(i - 1) < (unsigned)(G.nx - 2) && (unsigned)(j - 1) < (unsigned)(G.ny - 2)))
        return;
    aa_odd_inner_node<S, EXT>(buf, hist, G, c, i, j);
}

template <typename S, bool EXT>
__global__ void __launch_bounds__(128)
step_aa_odd_ring_kernel(S* __restrict__ buf, typename Real<S>::type* __restrict__ hist, Geom G,
                        Coef<typename Real<S>::type> c) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ring_count(G)) return;
    aa_odd_ring_node<S, EXT>(buf, hist, G, c, k);
}

// The odd step as one launch: the first `rrows` block rows take the ring (node k =
// (by gridDim.x + bx) * threads + t), the others the inner nodes (row j = by - rrows).
// Held to the inner code's 64 registers (256 threads x 4 blocks); the ring code, which
// alone takes 80, spills within that budget.
template <typename S, bool EXT>
__global__ void __launch_bounds__(256, 4)
step_aa_odd_fused_kernel(S* __restrict__ buf, typename Real<S>::type* __restrict__ hist, Geom G,
                         Coef<typename Real<S>::type> c, int rrows) {
    pdl_trigger();
    pdl_wait();                                // launched by launch_pdl()
    if ((int)blockIdx.y < rrows) {
        const long long k = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * (blockDim.x * blockDim.y) +
                            threadIdx.y * blockDim.x + threadIdx.x;
        if (k < ring_count(G)) aa_odd_ring_node<S, EXT>(buf, hist, G, c, k);
        return;
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = ((int)blockIdx.y - rrows) * blockDim.y + threadIdx.y;
    if (!((unsigned)(i - 1) < (unsigned)(G.nx - 2) && (unsigned)(j - 1) < (unsigned)(G.ny - 2)))
        return;
    aa_odd_inner_node<S, EXT>(buf, hist, G, c, i, j);
}

// ---- initial state ---------------------------------------------------------------
// T - T0 and C - C0 at t = 0 in the compute precision W: from caller arrays (FP64
// [ny][nx]) or from the SplitMix64 noise with key (field * ny + j) * nx + i (in FP32
// the uniform keeps the top 24 of its 53 bits, a change below 2^-24 of the noise).
template <typename W>
__device__ __forceinline__ W uniform_w(uint64_t seed, uint64_t k) {
    if (sizeof(W) == sizeof(double)) return (W)uniform01(seed, k);
    return (W)(uint32_t)(splitmix64_at(seed, k) >> 40) * W(1.0f / 16777216.0f);
}

template <typename W>
__device__ __forceinline__ void initial_TC(const InitSpec& I, const Geom& G, int i, int j, W& Tp,
                                           W& Cp) {
    if (I.T_init) {
        if (j < G.jb || j >= G.je) {          // ghost rows of a slab: never read at t = 0
            Tp = Cp = W(0);
            return;
        }
        const size_t k = (size_t)(j - G.jb) * G.nx + i;
        Tp = (W)I.T_init[k] - (W)I.T0;
        Cp = (W)I.C_init[k] - (W)I.C0;
    } else {
        const size_t k = (size_t)(I.key_j0 + j) * G.nx + i;
        const size_t n = (size_t)G.nx * I.key_ny;
        Tp = (W)I.noise * (W(2) * uniform_w<W>(I.seed, k) - W(1));
        Cp = (W)I.noise * (W(2) * uniform_w<W>(I.seed, n + k) - W(1));
    }
}

// Deviation of the D2Q5 rest equilibrium of Eq. 28 at u = 0 for Phi' = Phi - Phi0
// (model A: w~_q cap Phi', from the velocity-space form of Eqs. 30-31).
template <typename W>
__device__ __forceinline__ W eq5_dev(int q, W cap, W varpi, W Pp, int model_a) {
    if (model_a) return (q == 0 ? W(1) - varpi : W(0.25) * varpi) * cap * Pp;
    return q == 0 ? (cap - varpi) * Pp : W(0.25) * varpi * Pp;
}

// Writes the state at t = 0.  AB (PULL = true): the buffer must give the t = 0
// populations when pulled, so slot q of node y holds the t = 0 population of
// y + e_q (or, for a link that leaves the cavity, the value whose wall rule
// gives the t = 0 population of y).  AA (PULL = false): natural slots.
// The flow populations are at rest (f' = 0).  History = (T u, C u) of t = 0.
// Everything is computed in the compute precision R (FP64 or FP32).
template <typename S, bool PULL>
__global__ void init_kernel(S* __restrict__ buf, typename Real<S>::type* __restrict__ hist, Geom G,
                            Coef<typename Real<S>::type> c, InitSpec I) {
    using R = typename Real<S>::type;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const size_t self = (size_t)j * G.pitch + i;
    R Tp, Cp;
    initial_TC(I, G, i, j, Tp, Cp);
    const R sig = (R)I.sigma, vp = (R)I.varpi;
    // porosity of this node (the h rest equilibrium depends on it, Eq. 28)
    const R eps_n = c.poro ? c.poro[self] : (R)I.eps;
    // flow at rest: f' = 0; in the pull layout a slot whose link leaves the cavity holds
    // the value the moving-wall rule turns into 0 (wall_momentum of that wall).
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        R v = R(0);
        const int ti = i + ex_of(q), tj = j + ey_of(q);
        if (PULL && c.moving && !((unsigned)ti < (unsigned)G.nx && (unsigned)tj < (unsigned)G.ny))
            v = wall_momentum(c, link_side(ti, tj, G), q);
        Store<S>::st(buf + (size_t)(QF + q) * G.plane + self, v);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        R vg, vh;
        if (!PULL) {
            vg = eq5_dev(q, sig, vp, Tp, I.model_a);
            vh = eq5_dev(q, eps_n, vp, Cp, I.model_a);
        } else {
            const int ti = i + ex_of(q), tj = j + ey_of(q);
            if ((unsigned)ti < (unsigned)G.nx && (unsigned)tj < (unsigned)G.ny) {
                R Tn, Cn;
                initial_TC(I, G, ti, tj, Tn, Cn);
                const R eps_t = c.poro ? c.poro[(size_t)tj * G.pitch + ti] : (R)I.eps;
                vg = eq5_dev(q, sig, vp, Tn, I.model_a);
                vh = eq5_dev(q, eps_t, vp, Cn, I.model_a);
            } else {
                // pulled back at y along opp(q) through the wall ahead of q
                const int o = opp_of(q), side = pull_side(o);
                const R wg = eq5_dev(o, sig, vp, Tp, I.model_a);
                const R wh = eq5_dev(o, eps_n, vp, Cp, I.model_a);
                const bool dir = (c.dirichlet_mask >> side) & 1;
                vg = dir ? c.wallT[side] - wg : wg;
                vh = dir ? c.wallC[side] - wh : wh;
            }
        }
        Store<S>::st(buf + (size_t)(QG + q) * G.plane + self, vg);
        Store<S>::st(buf + (size_t)(QH + q) * G.plane + self, vh);
    }
    // history from the t = 0 macroscopic state (Eqs. 16-19, 26)
    R f[9], g[5], h[5];
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = R(0);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        g[q] = eq5_dev(q, sig, vp, Tp, I.model_a);
        h[q] = eq5_dev(q, eps_n, vp, Cp, I.model_a);
    }
    Coef<R> cl = c;
    if (c.poro) porous_at(cl, self, G.plane);
    Macro<R> M = macro(cl, f, g, h);
    R hv[4];
    const R T = c.T0 + M.Tp, C = c.C0 + M.Cp;
    hv[0] = T * M.ux;
    hv[1] = T * M.uy;
    hv[2] = C * M.ux;
    hv[3] = C * M.uy;
    store_hist(hist, G, self, hv);
}

// ---- slabs of a cavity split along y -------------------------------------------------
// Planes of the populations that cross a horizontal cut between two slabs (Eq. 11 pulls
// them across it): moving up (e_y = +1) f2, f5, f6, g2, h2; moving down (e_y = -1)
// f4, f7, f8, g4, h4.
__host__ __device__ constexpr int halo_plane(int up, int k) {
    return up ? (k == 0 ? QF + 2 : k == 1 ? QF + 5 : k == 2 ? QF + 6 : k == 3 ? QG + 2 : QH + 2)
              : (k == 0 ? QF + 4 : k == 1 ? QF + 7 : k == 2 ? QF + 8 : k == 3 ? QG + 4 : QH + 4);
}

// Copies the five crossing planes of one row between the state and a face buffer
// face[5][nx] (pack = 1: state -> face, 0: face -> state).  Grid (ceil(nx / 128), 5).
template <typename S>
__global__ void __launch_bounds__(128)
halo_kernel(S* __restrict__ buf, Geom G, int row, int up, S* __restrict__ face, int pack) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= G.nx || k >= 5) return;
    S* p = buf + (size_t)halo_plane(up, k) * G.plane + (size_t)row * G.pitch + i;
    S* q = face + (size_t)k * G.nx + i;
    if (pack)
        *q = *p;
    else
        *p = *q;
}

// ---- read-outs -----------------------------------------------------------------------
// Fields at the current level over the window [x0, x0 + w) x [y0, y0 + h):
// out planes [5][h][w] = ux, uy, T, C, rho (FP64).
template <typename S>
__global__ void fields_kernel(const S* __restrict__ buf, Geom G, Coef<typename Real<S>::type> c,
                              int mode, int x0, int y0, int w, int h, double* __restrict__ out) {
    using R = typename Real<S>::type;
    const int wi = blockIdx.x * blockDim.x + threadIdx.x;
    const int wj = blockIdx.y * blockDim.y + threadIdx.y;
    if (wi >= w || wj >= h) return;
    const int i = x0 + wi, j = y0 + wj;
    R f[9], g[5], hh[5];
    gather<true>(mode, buf, G, i, j, c, f, g, hh);
    Coef<R> cl = c;
    if (c.poro) porous_at(cl, (size_t)j * G.pitch + i, G.plane);
    Macro<R> M = macro(cl, f, g, hh);
    const size_t n = (size_t)w * h, k = (size_t)wj * w + wi;
    out[k] = (double)M.ux;
    out[n + k] = (double)M.uy;
    out[2 * n + k] = (double)c.T0 + (double)M.Tp;
    out[3 * n + k] = (double)c.C0 + (double)M.Cp;
    out[4 * n + k] = 1.0 + (double)M.rho;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// FP32 maxima stay in FP32: GB300's FP64 pipe is narrow, and a per-block max in
// FP64 (shuffle + fmax per step) made the residual pass FP64-bound.
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Mean Nu / Sh on the left and right walls (Eq. 38), one block, FP64 sums with a
// fixed reduction order (deterministic).  out = {Nu_L, Sh_L, Nu_R, Sh_R}.
template <typename S>
__global__ void __launch_bounds__(NUSH_THREADS)
nush_kernel(const S* __restrict__ buf, Geom G, Coef<typename Real<S>::type> c, int mode,
            WallSpec W, double* __restrict__ out) {
    using R = typename Real<S>::type;
    double acc[4] = {0, 0, 0, 0};
    if (W.nee) {
        // nodes on the walls: dPhi/dx|wall = (-3 Phi_0 + 4 Phi_1 - Phi_2) / 2, mirrored on
        // the right; trapezoidal mean over the ny - 1 spacings
        for (int j = threadIdx.x; j < G.ny; j += blockDim.x) {
            R f[9], g[5], h[5];
            double T[6], C[6];
            const int cols[6] = {0, 1, 2, G.nx - 3, G.nx - 2, G.nx - 1};
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                gather<false>(mode, buf, G, cols[k], j, c, f, g, h);
                const R sg = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
                const R sh = ((h[0] + h[1]) + (h[2] + h[3])) + h[4];
                const R ie = c.poro ? R(1) / c.poro[(size_t)j * G.pitch + cols[k]] : c.inv_eps;
                T[k] = W.T0 + (double)(sg * c.inv_sigma);
                C[k] = W.C0 + (double)(sh * ie);
            }
            const double wj = (j == 0 || j == G.ny - 1) ? 0.5 : 1.0;
            acc[0] += wj * -W.L * (-3.0 * T[0] + 4.0 * T[1] - T[2]) / 2.0 / W.dT;
            acc[1] += wj * -W.L * (-3.0 * C[0] + 4.0 * C[1] - C[2]) / 2.0 / W.dC;
            acc[2] += wj * -W.L * (3.0 * T[5] - 4.0 * T[4] + T[3]) / 2.0 / W.dT;
            acc[3] += wj * -W.L * (3.0 * C[5] - 4.0 * C[4] + C[3]) / 2.0 / W.dC;
        }
    }
    for (int j = G.jb + threadIdx.x; j < G.je && !W.nee; j += blockDim.x) {
        R f[9], g[5], h[5];
        double T[4], C[4];
        const int cols[4] = {0, 1, G.nx - 2, G.nx - 1};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            gather<false>(mode, buf, G, cols[k], j, c, f, g, h);
            const R sg = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
            const R sh = ((h[0] + h[1]) + (h[2] + h[3])) + h[4];
            const R ie = c.poro ? R(1) / c.poro[(size_t)j * G.pitch + cols[k]] : c.inv_eps;
            T[k] = W.T0 + (double)(sg * c.inv_sigma);
            C[k] = W.C0 + (double)(sh * ie);
        }
        // dPhi/dx at the wall: (-8 Phi_w + 9 Phi_0 - Phi_1) / 3, mirrored on the right
        acc[0] += -W.L * (-8.0 * W.Tw[0] + 9.0 * T[0] - T[1]) / 3.0 / W.dT;
        acc[1] += -W.L * (-8.0 * W.Cw[0] + 9.0 * C[0] - C[1]) / 3.0 / W.dC;
        acc[2] += -W.L * (8.0 * W.Tw[1] - 9.0 * T[3] + T[2]) / 3.0 / W.dT;
        acc[3] += -W.L * (8.0 * W.Cw[1] - 9.0 * C[3] + C[2]) / 3.0 / W.dC;
    }
    __shared__ double red[NUSH_THREADS / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s / (W.nee ? G.ny - 1.0 : (double)step_rows(G));
    }
}

// Mean Nu / Sh on the bottom and top walls, one block, FP64, fixed reduction order.
// W.Tw / W.Cw = {bottom, top}; out = {Nu_B, Sh_B, Nu_T, Sh_T}.
template <typename S>
__global__ void __launch_bounds__(NUSH_THREADS)
nush_tb_kernel(const S* __restrict__ buf, Geom G, Coef<typename Real<S>::type> c, int mode,
               WallSpec W, double* __restrict__ out) {
    using R = typename Real<S>::type;
    double acc[4] = {0, 0, 0, 0};
    if (W.nee) {
        // as on the left / right walls, transposed (node stencil, trapezoidal mean over x)
        for (int i = threadIdx.x; i < G.nx; i += blockDim.x) {
            R f[9], g[5], h[5];
            double T[6], C[6];
            const int rows[6] = {0, 1, 2, G.ny - 3, G.ny - 2, G.ny - 1};
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                gather<false>(mode, buf, G, i, rows[k], c, f, g, h);
                const R sg = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
                const R sh = ((h[0] + h[1]) + (h[2] + h[3])) + h[4];
                const R ie = c.poro ? R(1) / c.poro[(size_t)rows[k] * G.pitch + i] : c.inv_eps;
                T[k] = W.T0 + (double)(sg * c.inv_sigma);
                C[k] = W.C0 + (double)(sh * ie);
            }
            const double wi = (i == 0 || i == G.nx - 1) ? 0.5 : 1.0;
            acc[0] += wi * W.L * (-3.0 * T[0] + 4.0 * T[1] - T[2]) / 2.0 / W.dT;
            acc[1] += wi * W.L * (-3.0 * C[0] + 4.0 * C[1] - C[2]) / 2.0 / W.dC;
            acc[2] += wi * W.L * (3.0 * T[5] - 4.0 * T[4] + T[3]) / 2.0 / W.dT;
            acc[3] += wi * W.L * (3.0 * C[5] - 4.0 * C[4] + C[3]) / 2.0 / W.dC;
        }
    }
    for (int i = threadIdx.x; i < G.nx && !W.nee; i += blockDim.x) {
        R f[9], g[5], h[5];
        double T[4], C[4];
        const int rows[4] = {0, 1, G.ny - 2, G.ny - 1};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            gather<false>(mode, buf, G, i, rows[k], c, f, g, h);
            const R sg = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
            const R sh = ((h[0] + h[1]) + (h[2] + h[3])) + h[4];
            const R ie = c.poro ? R(1) / c.poro[(size_t)rows[k] * G.pitch + i] : c.inv_eps;
            T[k] = W.T0 + (double)(sg * c.inv_sigma);
            C[k] = W.C0 + (double)(sh * ie);
        }
        // dPhi/dy at the wall through the wall value and the first two rows
        acc[0] += W.L * (-8.0 * W.Tw[0] + 9.0 * T[0] - T[1]) / 3.0 / W.dT;
        acc[1] += W.L * (-8.0 * W.Cw[0] + 9.0 * C[0] - C[1]) / 3.0 / W.dC;
        acc[2] += W.L * (8.0 * W.Tw[1] - 9.0 * T[3] + T[2]) / 3.0 / W.dT;
        acc[3] += W.L * (8.0 * W.Cw[1] - 9.0 * C[3] + C[2]) / 3.0 / W.dC;
    }
    __shared__ double red[NUSH_THREADS / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s / (W.nee ? G.nx - 1.0 : (double)G.nx);
    }
}

// Residual pass 1: per node phi = (u_x, u_y, T - T0, C - C0) at the current level
// in the compute precision R (the deviations make the difference of two close
// values exact); snap (element type P) is replaced by phi.  Each block reduces the
// maxima of |phi - snap|, of |(u_x, u_y, T, C)| and a non-finite flag, and folds
// them into slot (block index mod nslots) of slots[nslots][9] with an integer
// atomicMax on the FP64 bit patterns (all values are >= 0, whose bit patterns
// order as the values do); the slots must be zero before the launch.  Block
// (bx, by) takes the 256-column tiles bx, bx + gridDim.x, ... of the rows by,
// by + gridDim.y, ...; with the grid of residual_grid() that is one node per thread.
// Blocks per SM the residual pass is compiled for: its general gather with the wall rules
// takes 90 registers left alone (2 blocks of 256 threads per SM, a quarter of the warp
// slots, for a pass that is all loads).  GB300, 4096^2 FP32 two-buffer, ms per residual
// call (at most 128 / 72 / 64 registers): 0.562 / 0.442 / 0.396.  The wall-node gather
// would spill 112 bytes at 64 and takes 3 blocks (80 registers); FP64 is left alone.
#ifndef LBM_RES_MIN_BLOCKS
#define LBM_RES_MIN_BLOCKS 4
#endif
template <typename S, int MODE>
constexpr int res_min_blocks() {
    return sizeof(typename Real<S>::type) == 8 ? 1 : (MODE == GATHER_NEE_AB ? 3 : LBM_RES_MIN_BLOCKS);
}

template <typename S, bool EXT, typename P, int MODE>
__global__ void __launch_bounds__(RES_THREADS, res_min_blocks<S, MODE>())
residual_kernel(const S* __restrict__ buf, Geom G, Coef<typename Real<S>::type> c,
                P* __restrict__ snap, unsigned long long* __restrict__ slots, int nslots) {
    using R = typename Real<S>::type;
    R dmax[4] = {0, 0, 0, 0}, amax[4] = {0, 0, 0, 0};
    int bad = 0;
    const size_t n = (size_t)G.nx * G.ny;
    const int ntx = (G.nx + RES_THREADS - 1) / RES_THREADS;
    for (int tx = blockIdx.x; tx < ntx; tx += gridDim.x) {
        const int i = tx * RES_THREADS + threadIdx.x;
        if (i >= G.nx) continue;
        for (int j = G.jb + blockIdx.y; j < G.je; j += gridDim.y) {
            // all loads first (the snapshot's with the populations), then the stores:
            // a load after a store to the same array waits for nothing, but the
            // compiler keeps them in program order, which would serialise four
            // round trips to memory per node
            const size_t k = (size_t)j * G.nx + i;
            R old[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) old[q] = (R)snap[q * n + k];
            R f[9], g[5], h[5];
            gather_m<MODE>(buf, G, i, j, c, f, g, h);
            Macro<R> M;
            if (EXT && c.poro) {
                Coef<R> cl = c;
                porous_at(cl, (size_t)j * G.pitch + i, G.plane);
                M = macro(cl, f, g, h);
            } else {
                M = macro(c, f, g, h);
            }
            const R phi[4] = {M.ux, M.uy, M.Tp, M.Cp};
            const R absv[4] = {M.ux, M.uy, c.T0 + M.Tp, c.C0 + M.Cp};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!finite_(phi[q])) bad = 1;
                dmax[q] = max_(dmax[q], abs_(phi[q] - old[q]));
                amax[q] = max_(amax[q], abs_(absv[q]));
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) snap[q * n + k] = (P)phi[q];
        }
    }
    // block maxima in R, one FP64 value per quantity for the slot
    __shared__ R red[RES_THREADS / 32][9];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const R v[9] = {dmax[0], dmax[1], dmax[2], dmax[3], amax[0], amax[1], amax[2], amax[3], (R)bad};
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const R r = warp_max(v[q]);
        if (lane == 0) red[warp][q] = r;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        R s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = max_(s, red[w][threadIdx.x]);
        const size_t b = ((size_t)blockIdx.y * gridDim.x + blockIdx.x) % (size_t)nslots;
        atomicMax(slots + b * 9 + threadIdx.x, (unsigned long long)__double_as_longlong((double)s));
    }
}

// Clears the slots and launches pass 1 with the gather mode and the porous-field
// code fixed at compile time.
template <typename S, typename P>
cudaError_t launch_residual_pass1(const S* buf, const Geom& G, const Coef<typename Real<S>::type>& c,
                                  int mode, P* snap, double* slots, int nslots, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(slots, 0, (size_t)nslots * 9 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const dim3 grid = residual_grid(G);
    unsigned long long* sl = reinterpret_cast<unsigned long long*>(slots);
#define LBM_RES_CASE(M)                                                                          \
    if (mode == M) {                                                                             \
        if (c.poro)                                                                              \
            residual_kernel<S, true, P, M><<<grid, RES_THREADS, 0, st>>>(buf, G, c, snap, sl,     \
                                                                        nslots);                 \
        else                                                                                     \
            residual_kernel<S, false, P, M><<<grid, RES_THREADS, 0, st>>>(buf, G, c, snap, sl,    \
                                                                         nslots);                \
        return cudaGetLastError();                                                               \
    }
    LBM_RES_CASE(GATHER_PULL_AB)
    LBM_RES_CASE(GATHER_PULL_AA)
    LBM_RES_CASE(GATHER_LOCAL)
    LBM_RES_CASE(GATHER_NEE_AB)
#undef LBM_RES_CASE
    return cudaErrorInvalidValue;
}

// Residual pass 2: one block folds partial[nblocks][9] into out[9].
__global__ void __launch_bounds__(RES_THREADS)
residual_final_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ out);

}  // namespace lbm
