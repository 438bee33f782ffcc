// C ABI of the batch (many cavities, one fused launch per step): device arena,
// slot table, tiles, CUDA-graph replay and the tile autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_batch.h"
#include "lbm_batch_kernels.cuh"

using namespace lbm;

namespace {

thread_local std::string g_err;

void gerr(const char* fmt, ...) {
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    g_err = b;
}

size_t esize(int prec) { return prec == LBM_F32 ? 4 : 2; }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

Geom geom_for(int nx, int ny, int prec) {
    Geom G;
    const int per128 = (int)(128 / esize(prec));
    G.nx = nx;
    G.ny = ny;
    G.pitch = (nx + per128 - 1) / per128 * per128;
    G.plane = (size_t)ny * G.pitch;
    G.jb = 0;
    G.je = ny;
    return G;
}

// Arena bytes of one cavity: state buffers, FP32 history, FP32 residual snapshot.
size_t inst_bytes(const Geom& G, int prec, int layout) {
    const size_t st = align_up((size_t)NQ * G.plane * esize(prec), 256);
    const size_t hi = align_up((size_t)4 * G.plane * sizeof(float), 256);
    const size_t sn = align_up((size_t)4 * G.nx * G.ny * sizeof(float), 256);
    return (layout == LBM_AA ? 1 : 2) * st + hi + sn;
}

// First-fit allocator over one device block; free blocks are coalesced.
struct Arena {
    char* base = nullptr;
    size_t size = 0, used = 0;
    std::map<size_t, size_t> free_;   // offset -> length
    void reset(char* b, size_t n) {
        base = b;
        size = n;
        used = 0;
        free_.clear();
        if (n) free_[0] = n;
    }
    bool alloc(size_t n, size_t* off) {
        n = align_up(n, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t roff = it->first + n;
                free_.erase(it);
                if (rest) free_[roff] = rest;
                used += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = align_up(n, 256);
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Slot {
    bool used = false;
    lbm_params P{};
    uint64_t seed = 0;
    double noise = 0;
    size_t off = 0, bytes = 0;
    Geom G{};
    int tw_log2 = 7, th = 4;
    int64_t t_added = 0;
    int phase = 0;
    bool snap_valid = false;
};

// Tile-shape cache shared by all batches of the process.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune;   // (nx,ny,prec,layout) -> (log2 w, h)

// Default tile: BATCH_THREADS nodes (one per thread), as wide as the cavity allows.
void default_tile(int nx, int* wlog2, int* th) {
    int w = 32;
    while (w < nx && w < BATCH_THREADS) w <<= 1;
    int l = 0;
    while ((1 << l) < w) ++l;
    *wlog2 = l;
    *th = std::max(1, BATCH_THREADS / w);
}

}  // namespace

namespace {
Coef<float> coef_from(const lbm_params& P, bool sr) {
    Coef<float> c = make_coef<float>(P);
    c.sr = sr ? 1 : 0;
    return c;
}

bool params_ok(const lbm_params& P, std::string* why) {
    auto bad = [&](const char* m) { *why = m; return false; };
    for (int s = 0; s < 4; ++s)
        if (P.uw[s][0] != 0.0 || P.uw[s][1] != 0.0)
            return bad("moving walls are not supported in batches (use a single cavity)");
    if (P.nee != 0 && P.nee != 1) return bad("nee must be 0 or 1");
    if (P.nee && (P.nx < 5 || P.ny < 5)) return bad("walls with nodes on them need nx, ny >= 5");
    for (int s = 0; s < 4; ++s) {
        if (!(P.BiT[s] >= 0.0) || !(P.BiC[s] >= 0.0) || !std::isfinite(P.BiT[s]) ||
            !std::isfinite(P.BiC[s]))
            return bad("Biot numbers must be finite and >= 0");
        if (!P.nee && (P.BiT[s] != 0.0 || P.BiC[s] != 0.0))
            return bad("convective (Robin) walls need walls with nodes on them (nee = 1)");
    }
    if (P.nx < 3 || P.ny < 3) return bad("nx and ny must be >= 3");
    if (!(P.eps > 0.0 && P.eps <= 1.0)) return bad("eps must lie in (0, 1]");
    if (!(P.sigma > 0.0) || !(P.K > 0.0)) return bad("sigma and K must be positive");
    if (!(P.varpi > 0.0 && P.varpi < 1.0)) return bad("varpi must lie in (0, 1)");
    for (int k = 0; k < 9; ++k)
        if (!(P.s[k] > 0.0 && P.s[k] < 2.0)) return bad("a flow relaxation rate lies outside (0, 2)");
    for (int k = 0; k < 5; ++k)
        if (!(P.zeta[k] > 0.0 && P.zeta[k] < 2.0) || !(P.eta[k] > 0.0 && P.eta[k] < 2.0))
            return bad("a scalar relaxation rate lies outside (0, 2)");
    return true;
}
}  // namespace

struct lbm_batch {
    int prec = LBM_F32, layout = LBM_AB_PULL;
    bool sr = true;
    int capacity = 0;
    std::vector<Slot> slots;
    Arena arena;
    void* arena_mem = nullptr;
    size_t arena_alloc_bytes = 0;
    // device tables
    BatchInst<float>* d_table = nullptr;
    WallSpec* d_walls = nullptr;
    int* d_ntiles = nullptr;
    double* d_out = nullptr;             // capacity * 9 (residual) + capacity * 4 (Nu/Sh)
    int* d_owner = nullptr;
    size_t owner_cap = 0;
    double* d_partial = nullptr;
    size_t partial_cap = 0;
    double* d_fields = nullptr;
    size_t fields_cap = 0;
    std::vector<BatchInst<float>> h_table;
    std::vector<int> h_owner, h_ntiles;
    int total_tiles = 0;
    bool one_node_tiles = false;         // every tile has BATCH_THREADS nodes
    bool has_nee = false;                // some cavity has wall nodes (Sec. 3.3)
    // L2 temporal blocking: groups of cavities whose working set fits in a share of
    // L2 are advanced `tblock` steps at a time.
    std::vector<std::pair<int, int>> groups;   // [tile_begin, tile_end)
    // Per group: the slot of its one cavity when that cavity alone exceeds its lane's L2
    // share (its state streams from HBM whatever the blocking), else -1.  Such a group
    // runs the single-cavity step kernels over that cavity, whose per-node arithmetic is
    // the tile kernel's (bit for bit) and which stream HBM faster than 128-node tiles.
    std::vector<int> group_direct;
    // Groups are independent, so they are dealt round-robin to kLanes streams (the
    // batch's own and kLanes - 1 more): one lane's launches fill the others' wave
    // tails and launch gaps.  The kLanes groups in flight share the L2 budget.
    static constexpr int kLanes = 2;
    cudaStream_t lane[kLanes - 1] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kLanes - 1] = {};
    size_t l2_budget = 48u << 20;
    int tblock = 64;
    bool dirty = true;
    int64_t t = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int sms = 152, bps = 4;
    int graph_chunk = 64;
    cudaGraphExec_t graph = nullptr;
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    std::string err;

    lbm_status fail(lbm_status s, const char* fmt, ...) {
        char b[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b, sizeof b, fmt, ap);
        va_end(ap);
        err = b;
        g_err = b;
        return s;
    }
    void* dalloc(size_t n) {
        void* p = nullptr;
        if (alloc) {
            p = alloc(n, alloc_user, (void*)stream);
            if (p && ((uintptr_t)p & 255u)) {
                free_fn(p, alloc_user, (void*)stream);
                p = nullptr;
            }
        } else if (cudaMalloc(&p, n) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return p;
    }
    void dfree(void* p) {
        if (!p) return;
        if (alloc)
            free_fn(p, alloc_user, (void*)stream);
        else
            cudaFree(p);
    }
    int used_slots() const {
        int n = 0;
        for (const Slot& s : slots) n += s.used;
        return n;
    }
    void* slot_buf(const Slot& s, int k) const {
        const size_t st = align_up((size_t)NQ * s.G.plane * esize(prec), 256);
        return arena.base + s.off + (size_t)k * st;
    }
    void* slot_hist(const Slot& s) const {
        const size_t st = align_up((size_t)NQ * s.G.plane * esize(prec), 256);
        return arena.base + s.off + (layout == LBM_AA ? 1 : 2) * st;
    }
    float* slot_snap(const Slot& s) const {
        const size_t st = align_up((size_t)NQ * s.G.plane * esize(prec), 256);
        const size_t hi = align_up((size_t)4 * s.G.plane * sizeof(float), 256);
        return (float*)(arena.base + s.off + (layout == LBM_AA ? 1 : 2) * st + hi);
    }
    int parity() const { return (int)(t & 1); }
    int mode_of(const Slot& s) const {
        const int odd = (int)((t + s.phase) & 1);
        if (layout == LBM_AB_PULL) return s.P.nee ? GATHER_NEE_AB : GATHER_PULL_AB;
        return odd ? GATHER_PULL_AA : GATHER_LOCAL;
    }
    const void* cur_of(const Slot& s) const {
        if (layout == LBM_AA) return slot_buf(s, 0);
        return slot_buf(s, (int)((t + s.phase) & 1));
    }
};

namespace {

void invalidate(lbm_batch* b) {
    b->dirty = true;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

// Rebuilds the descriptor table and the tile list, uploads them.
lbm_status sync_tables(lbm_batch* b) {
    if (!b->dirty) return LBM_OK;
    b->h_table.assign(b->capacity, BatchInst<float>{});
    b->h_ntiles.assign(b->capacity, 0);
    b->h_owner.clear();
    std::vector<WallSpec> walls(b->capacity);
    int tiles = 0;
    b->has_nee = false;
    for (int k = 0; k < b->capacity; ++k) {
        BatchInst<float>& I = b->h_table[k];
        std::memset(&I, 0, sizeof I);
        const Slot& s = b->slots[k];
        I.tile_begin = tiles;
        if (!s.used) continue;
        I.buf[0] = b->slot_buf(s, 0);
        I.buf[1] = b->layout == LBM_AA ? nullptr : b->slot_buf(s, 1);
        I.hist = b->slot_hist(s);
        I.snap = b->slot_snap(s);
        I.G = s.G;
        I.c = coef_from(s.P, b->sr);
        I.tile_w_log2 = s.tw_log2;
        I.tile_h = s.th;
        const int tw = 1 << s.tw_log2;
        I.tiles_x = (s.G.nx + tw - 1) / tw;
        const int tiles_y = (s.G.ny + s.th - 1) / s.th;
        I.phase = s.phase;
        I.active = 1;
        const int nt = I.tiles_x * tiles_y;
        b->h_ntiles[k] = nt;
        for (int q = 0; q < nt; ++q) b->h_owner.push_back(k);
        tiles += nt;
        WallSpec& W = walls[k];
        W.Tw[0] = s.P.Tw[0];
        W.Tw[1] = s.P.Tw[1];
        W.Cw[0] = s.P.Cw[0];
        W.Cw[1] = s.P.Cw[1];
        W.T0 = s.P.T0;
        W.C0 = s.P.C0;
        W.dT = s.P.Tw[0] - s.P.Tw[1];
        W.dC = s.P.Cw[0] - s.P.Cw[1];
        W.nee = s.P.nee;
        W.L = s.P.nee ? s.P.nx - 1.0 : (double)s.P.nx;
        if (s.P.nee) b->has_nee = true;
    }
    b->total_tiles = tiles;
    b->one_node_tiles = true;
    for (int k = 0; k < b->capacity; ++k)
        if (b->slots[k].used && (1 << b->slots[k].tw_log2) * b->slots[k].th != BATCH_THREADS)
            b->one_node_tiles = false;
    // groups: consecutive cavities while their per-step working set (buffers read
    // and written, history) stays within the L2 budget
    b->groups.clear();
    b->group_direct.clear();
    {
        size_t ws = 0;
        int gbeg = 0, members = 0, last = -1;
        const size_t share = b->l2_budget / lbm_batch::kLanes;
        auto close = [&](int t_end) {
            b->groups.push_back({gbeg, t_end});
            const bool alone_big = members == 1 && ws > share && !b->slots[last].P.nee;
            b->group_direct.push_back(alone_big ? last : -1);
        };
        for (int k = 0; k < b->capacity; ++k) {
            const Slot& s = b->slots[k];
            if (!s.used) continue;
            const size_t w = (b->layout == LBM_AA ? 1 : 2) * (size_t)NQ * s.G.plane * esize(b->prec) +
                             (size_t)4 * s.G.plane * sizeof(float);
            const int t0 = b->h_table[k].tile_begin;
            if (ws > 0 && ws + w > share) {
                close(t0);
                gbeg = t0;
                ws = 0;
                members = 0;
            }
            ws += w;
            members += 1;
            last = k;
        }
        if (tiles > gbeg) close(tiles);
    }
    if ((size_t)tiles > b->owner_cap) {
        b->dfree(b->d_owner);
        b->dfree(b->d_partial);
        size_t cap = std::max<size_t>(1024, (size_t)tiles * 2);
        b->d_owner = (int*)b->dalloc(cap * sizeof(int));
        b->d_partial = (double*)b->dalloc(cap * 9 * sizeof(double));
        if (!b->d_owner || !b->d_partial) {
            b->owner_cap = 0;
            return b->fail(LBM_ERR_NOMEM, "lbm_batch: no device memory for the tile list");
        }
        b->owner_cap = cap;
    }
    cudaError_t e = cudaSuccess;
    if (tiles)
        e = cudaMemcpyAsync(b->d_owner, b->h_owner.data(), tiles * sizeof(int), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_table, b->h_table.data(), b->capacity * sizeof(BatchInst<float>),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_ntiles, b->h_ntiles.data(), b->capacity * sizeof(int),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_walls, walls.data(), b->capacity * sizeof(WallSpec),
                            cudaMemcpyHostToDevice, b->stream);
    // the host vectors are pageable: make sure the copies have left them before they change
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch: table upload: %s", cudaGetErrorString(e));
    b->dirty = false;
    return LBM_OK;
}

// Reductions: a grid of resident CTAs striding over the tiles (the step kernel
// runs one CTA per tile).
int reduce_grid(const lbm_batch* b) {
    return std::max(1, std::min(b->sms * b->bps, std::max(1, b->total_tiles)));
}

cudaError_t launch_range(lbm_batch* b, int tile_begin, int tile_end, int parity, cudaStream_t st) {
    const bool aa = b->layout == LBM_AA;
    const bool one = b->one_node_tiles, nee = b->has_nee;
    switch (b->prec) {
        case LBM_F32: return launch_batch_step<float>(b->d_table, b->d_owner, tile_begin, tile_end, parity, aa, one, nee, st);
        case LBM_BF16: return launch_batch_step<__nv_bfloat16>(b->d_table, b->d_owner, tile_begin, tile_end, parity, aa, one, nee, st);
        default: return launch_batch_step<__half>(b->d_table, b->d_owner, tile_begin, tile_end, parity, aa, one, nee, st);
    }
}

// One step of the cavity in slot k with the single-cavity kernels (see group_direct).
cudaError_t launch_direct(lbm_batch* b, int k, int parity, cudaStream_t st) {
    const BatchInst<float>& I = b->h_table[k];
    const int odd = (parity + I.phase) & 1;
    LaunchCfg L;
    std::memset(&L, 0, sizeof L);
    L.bx = 128;
    L.by = 1;
    L.stream = st;                 // the ring of a split step runs on the same stream
    const bool aa = b->layout == LBM_AA;
    void* src = aa ? I.buf[0] : I.buf[odd];
    void* dst = aa ? I.buf[0] : I.buf[odd ^ 1];
    switch (b->prec) {
        case LBM_F32:
            return aa ? launch_step_aa<float>(src, I.hist, I.G, I.c, odd != 0, L)
                      : launch_step_ab<float>(src, dst, I.hist, I.G, I.c, L);
        case LBM_BF16:
            return aa ? launch_step_aa<__nv_bfloat16>(src, I.hist, I.G, I.c, odd != 0, L)
                      : launch_step_ab<__nv_bfloat16>(src, dst, I.hist, I.G, I.c, L);
        default:
            return aa ? launch_step_aa<__half>(src, I.hist, I.G, I.c, odd != 0, L)
                      : launch_step_ab<__half>(src, dst, I.hist, I.G, I.c, L);
    }
}

void destroy_lanes(lbm_batch* b) {
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    for (int l = 0; l + 1 < lbm_batch::kLanes; ++l) {
        if (b->ev_join[l]) cudaEventDestroy(b->ev_join[l]);
        if (b->lane[l]) cudaStreamDestroy(b->lane[l]);
    }
}

// One step of every cavity (one launch over all tiles).
cudaError_t launch_step(lbm_batch* b) {
    cudaError_t e = launch_range(b, 0, b->total_tiles, b->parity(), b->stream);
    b->t += 1;
    return e;
}

// k steps of every cavity, group by group: each group's k launches run back to
// back, so its state stays in L2 between them.  Group i runs on lane i mod kLanes
// (lane 0 is the batch's stream; the others are forked from it and joined back at
// the end, also inside a captured graph).  Every cavity sees the same sequence of
// steps as with launch_step.
cudaError_t launch_block(lbm_batch* b, int k) {
    const int lanes = (int)std::min<size_t>(lbm_batch::kLanes, b->groups.size());
    cudaError_t e = cudaSuccess;
    if (lanes > 1) e = cudaEventRecord(b->ev_fork, b->stream);
    for (int l = 1; l < lanes && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(b->lane[l - 1], b->ev_fork, 0);
    for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
        const auto& g = b->groups[gi];
        const int l = (int)(gi % (size_t)lanes);
        const cudaStream_t st = l == 0 ? b->stream : b->lane[l - 1];
        const int direct = b->group_direct[gi];
        for (int s = 0; s < k && e == cudaSuccess; ++s)
            e = direct >= 0 ? launch_direct(b, direct, (int)((b->t + s) & 1), st)
                            : launch_range(b, g.first, g.second, (int)((b->t + s) & 1), st);
    }
    // join even after a failed launch, so that a capture is never left forked
    for (int l = 1; l < lanes; ++l) {
        cudaError_t j = cudaEventRecord(b->ev_join[l - 1], b->lane[l - 1]);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(b->stream, b->ev_join[l - 1], 0);
        if (e == cudaSuccess) e = j;
    }
    b->t += k;
    return e;
}

lbm_status init_slot(lbm_batch* b, int k) {
    Slot& s = b->slots[k];
    InitSpec I;
    std::memset(&I, 0, sizeof I);
    I.seed = s.seed;
    I.noise = s.noise < 0 ? 0.0 : (s.noise == 0 ? 1e-3 : s.noise);
    I.T0 = s.P.T0;
    I.C0 = s.P.C0;
    I.sigma = s.P.sigma;
    I.eps = s.P.eps;
    I.varpi = s.P.varpi;
    I.model_a = s.P.model_a;
    I.key_ny = s.G.ny;
    I.key_j0 = 0;
    const Coef<float> c = coef_from(s.P, b->sr);
    const bool pull = b->layout == LBM_AB_PULL;
    void* buf0 = b->slot_buf(s, 0);
    cudaError_t e = cudaMemsetAsync(b->arena.base + s.off, 0, s.bytes, b->stream);
    if (e == cudaSuccess) {
        switch (b->prec) {
            case LBM_F32: e = launch_init<float>(buf0, b->slot_hist(s), s.G, c, I, pull, b->stream); break;
            case LBM_BF16: e = launch_init<__nv_bfloat16>(buf0, b->slot_hist(s), s.G, c, I, pull, b->stream); break;
            default: e = launch_init<__half>(buf0, b->slot_hist(s), s.G, c, I, pull, b->stream); break;
        }
    }
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch: init: %s", cudaGetErrorString(e));
    return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_batch_instance_bytes(lbm_grid grid, const lbm_options* opt) {
    const int prec = opt ? opt->precision : LBM_F32;
    const int layout = opt ? opt->layout : LBM_AB_PULL;
    if (grid.nx < 3 || grid.ny < 3) return 0;
    return inst_bytes(geom_for(grid.nx, grid.ny, prec), prec, layout);
}

lbm_status lbm_batch_create(const lbm_instance* inst, int count, int capacity, size_t arena_bytes,
                            const lbm_options* opt, lbm_batch** out) {
    if (!out || count < 0 || capacity < std::max(count, 1) || (count > 0 && !inst)) {
        gerr("lbm_batch_create: need out, 0 <= count <= capacity, capacity >= 1");
        return LBM_ERR_INVALID;
    }
    *out = nullptr;
    lbm_options O;
    std::memset(&O, 0, sizeof O);
    if (opt) O = *opt;
    if (O.precision != LBM_F32 && O.precision != LBM_BF16 && O.precision != LBM_F16) {
        gerr("lbm_batch_create: batches store FP32, BF16 or FP16 (got precision %d)", O.precision);
        return LBM_ERR_INVALID;
    }
    if (O.layout != LBM_AB_PULL && O.layout != LBM_AA) {
        gerr("lbm_batch_create: unknown layout %d", O.layout);
        return LBM_ERR_INVALID;
    }
    if ((O.alloc == nullptr) != (O.free == nullptr)) {
        gerr("lbm_batch_create: alloc and free hooks must be given together");
        return LBM_ERR_INVALID;
    }
    for (int k = 0; k < count; ++k) {
        std::string why;
        if (!params_ok(inst[k].params, &why)) {
            gerr("lbm_batch_create: cavity %d: %s", k, why.c_str());
            return LBM_ERR_INVALID;
        }
        if (inst[k].params.nee && O.layout != LBM_AB_PULL) {
            gerr("lbm_batch_create: cavity %d: walls with nodes on them need the two-buffer layout", k);
            return LBM_ERR_INVALID;
        }
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) {
        gerr("lbm_batch_create: out of host memory");
        return LBM_ERR_NOMEM;
    }
    b->prec = O.precision;
    b->layout = O.layout;
    b->sr = O.round_nearest == 0;
    b->capacity = capacity;
    b->slots.assign(capacity, Slot{});
    b->alloc = O.alloc;
    b->free_fn = O.free;
    b->alloc_user = O.alloc_user;
    b->graph_chunk = O.graph_chunk == 0 ? 64 : (O.graph_chunk < 0 ? 0 : O.graph_chunk + (O.graph_chunk & 1));
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->device);
    // 3/8 of L2 for the groups in flight, 64 steps per block.  GB300, 512 mixed cavities,
    // FP32 two-buffer / in place, GLUPS with programmatic dependent launches: 3/8 and 64
    // steps 40.6 / 35.2, 1/2 and 32 steps 40.2 / 34.8, 3/4 39.3 / 28.4; below 3/8 the 256^2
    // cavities exceed a lane's share and take the single-cavity kernels (1/4: 36.9 / 34.9).
    if (l2 > 0) b->l2_budget = (size_t)l2 / 8 * 3;
    if (O.stream) {
        b->stream = (cudaStream_t)O.stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            lbm_status s = b->fail(LBM_ERR_CUDA, "lbm_batch_create: cudaStreamCreate failed");
            delete b;
            return s;
        }
        b->own_stream = true;
    }
    bool lanes_ok = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int l = 0; l + 1 < lbm_batch::kLanes && lanes_ok; ++l)
        lanes_ok = cudaStreamCreateWithFlags(&b->lane[l], cudaStreamNonBlocking) == cudaSuccess &&
                   cudaEventCreateWithFlags(&b->ev_join[l], cudaEventDisableTiming) == cudaSuccess;
    if (!lanes_ok) {
        lbm_status s = b->fail(LBM_ERR_CUDA, "lbm_batch_create: lane streams / events failed");
        destroy_lanes(b);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return s;
    }
    if (b->stream == nullptr || b->stream == cudaStreamLegacy || b->stream == cudaStreamPerThread)
        b->graph_chunk = 0;
    switch (b->prec) {
        case LBM_F32: b->bps = batch_step_blocks_per_sm<float>(b->layout == LBM_AA); break;
        case LBM_BF16: b->bps = batch_step_blocks_per_sm<__nv_bfloat16>(b->layout == LBM_AA); break;
        default: b->bps = batch_step_blocks_per_sm<__half>(b->layout == LBM_AA); break;
    }
    size_t need = 0;
    for (int k = 0; k < count; ++k)
        need += align_up(inst_bytes(geom_for(inst[k].params.nx, inst[k].params.ny, b->prec), b->prec,
                                    b->layout), 256);
    if (arena_bytes == 0) arena_bytes = need;
    arena_bytes = align_up(std::max<size_t>(arena_bytes, 256), 256);
    b->arena_mem = b->dalloc(arena_bytes);
    b->d_table = (BatchInst<float>*)b->dalloc(capacity * sizeof(BatchInst<float>));
    b->d_walls = (WallSpec*)b->dalloc(capacity * sizeof(WallSpec));
    b->d_ntiles = (int*)b->dalloc(capacity * sizeof(int));
    b->d_out = (double*)b->dalloc((size_t)capacity * 13 * sizeof(double));
    if (!b->arena_mem || !b->d_table || !b->d_walls || !b->d_ntiles || !b->d_out) {
        lbm_status s = b->fail(LBM_ERR_NOMEM, "lbm_batch_create: device allocation (arena %.3f GB) failed",
                               arena_bytes / 1e9);
        g_err = b->err;
        lbm_batch_destroy(b);
        return s;
    }
    b->arena_alloc_bytes = arena_bytes;
    b->arena.reset((char*)b->arena_mem, arena_bytes);
    for (int k = 0; k < count; ++k) {
        int slot = -1;
        lbm_status s = lbm_batch_add(b, &inst[k], &slot);
        if (s != LBM_OK) {
            g_err = b->err;
            lbm_batch_destroy(b);
            return s;
        }
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        lbm_status s = b->fail(LBM_ERR_CUDA, "lbm_batch_create: %s", cudaGetErrorString(e));
        g_err = b->err;
        lbm_batch_destroy(b);
        return s;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_add(lbm_batch* b, const lbm_instance* inst, int* slot) {
    if (!b || !inst || !slot) {
        gerr("lbm_batch_add: NULL argument");
        return LBM_ERR_INVALID;
    }
    std::string why;
    if (!params_ok(inst->params, &why)) return b->fail(LBM_ERR_INVALID, "lbm_batch_add: %s", why.c_str());
    if (inst->params.nee && b->layout != LBM_AB_PULL)
        return b->fail(LBM_ERR_INVALID, "lbm_batch_add: walls with nodes on them need the two-buffer layout");
    int k = -1;
    for (int q = 0; q < b->capacity; ++q)
        if (!b->slots[q].used) {
            k = q;
            break;
        }
    if (k < 0) return b->fail(LBM_ERR_NOMEM, "lbm_batch_add: all %d slots in use", b->capacity);
    Slot s;
    s.P = inst->params;
    s.seed = inst->seed;
    s.noise = inst->noise;
    s.G = geom_for(s.P.nx, s.P.ny, b->prec);
    s.bytes = inst_bytes(s.G, b->prec, b->layout);
    if (!b->arena.alloc(s.bytes, &s.off))
        return b->fail(LBM_ERR_NOMEM, "lbm_batch_add: arena has no free block of %zu bytes (%zu of %zu used)",
                       s.bytes, b->arena.used, b->arena.size);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(std::make_tuple(s.P.nx, s.P.ny, b->prec, b->layout));
        if (it != g_tune.end()) {
            s.tw_log2 = it->second.first;
            s.th = it->second.second;
        } else {
            default_tile(s.P.nx, &s.tw_log2, &s.th);
        }
    }
    s.used = true;
    s.t_added = b->t;
    s.phase = (int)(b->t & 1);
    s.snap_valid = false;
    b->slots[k] = s;
    lbm_status st = init_slot(b, k);
    if (st != LBM_OK) {
        b->arena.release(s.off, s.bytes);
        b->slots[k] = Slot{};
        return st;
    }
    invalidate(b);
    *slot = k;
    return LBM_OK;
}

lbm_status lbm_batch_remove(lbm_batch* b, int slot) {
    if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) {
        if (b) return b->fail(LBM_ERR_INVALID, "lbm_batch_remove: slot %d is not in use", slot);
        gerr("lbm_batch_remove: NULL batch");
        return LBM_ERR_INVALID;
    }
    // work already queued on the stream may still read this block
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch_remove: %s", cudaGetErrorString(e));
    b->arena.release(b->slots[slot].off, b->slots[slot].bytes);
    b->slots[slot] = Slot{};
    invalidate(b);
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t n) {
    if (!b || n < 0) {
        gerr("lbm_batch_step: invalid arguments");
        return LBM_ERR_INVALID;
    }
    lbm_status s = sync_tables(b);
    if (s != LBM_OK) return s;
    if (b->total_tiles == 0) {
        b->t += n;
        return LBM_OK;
    }
    cudaError_t e = cudaSuccess;
    while (n > 0 && (b->t & 1) && e == cudaSuccess) {
        e = launch_step(b);
        --n;
    }
    // a chunk = whole temporal blocks, an even number of steps
    const int tb = b->groups.size() > 1 ? std::max(1, b->tblock) : 1;
    int chunk = b->graph_chunk > 0 ? std::max(b->graph_chunk / tb, 1) * tb : 0;
    if (chunk & 1) chunk *= 2;
    if (chunk > 0 && n >= chunk && e == cudaSuccess) {
        if (!b->graph) {
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const int64_t t0 = b->t;
                cudaError_t le = cudaSuccess;
                for (int k = 0; k < chunk && le == cudaSuccess; k += tb) le = launch_block(b, tb);
                b->t = t0;
                e = cudaStreamEndCapture(b->stream, &g);
                if (le != cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                b->graph = nullptr;
                return b->fail(LBM_ERR_CUDA, "lbm_batch_step: graph capture: %s", cudaGetErrorString(e));
            }
        }
        while (n >= chunk && e == cudaSuccess) {
            e = cudaGraphLaunch(b->graph, b->stream);
            b->t += chunk;
            n -= chunk;
        }
    }
    while (n >= tb && tb > 1 && e == cudaSuccess) {
        e = launch_block(b, tb);
        n -= tb;
    }
    if (n > 0 && tb > 1 && e == cudaSuccess) {   // the rest as one shorter block
        e = launch_block(b, n);
        n = 0;
    }
    while (n > 0 && e == cudaSuccess) {
        e = launch_step(b);
        --n;
    }
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch_step: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int64_t lbm_batch_time(const lbm_batch* b, int slot) {
    if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return -1;
    return b->t - b->slots[slot].t_added;
}

lbm_status lbm_batch_nusselt_sherwood(lbm_batch* b, double* out) {
    if (!b || !out) {
        gerr("lbm_batch_nusselt_sherwood: NULL argument");
        return LBM_ERR_INVALID;
    }
    lbm_status s = sync_tables(b);
    if (s != LBM_OK) return s;
    const bool aa = b->layout == LBM_AA;
    double* o = b->d_out + (size_t)b->capacity * 9;
    cudaError_t e;
    switch (b->prec) {
        case LBM_F32: e = launch_batch_nush<float>(b->d_table, b->d_walls, b->capacity, b->parity(), aa, o, b->stream); break;
        case LBM_BF16: e = launch_batch_nush<__nv_bfloat16>(b->d_table, b->d_walls, b->capacity, b->parity(), aa, o, b->stream); break;
        default: e = launch_batch_nush<__half>(b->d_table, b->d_walls, b->capacity, b->parity(), aa, o, b->stream); break;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, o, (size_t)b->capacity * 4 * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch_nusselt_sherwood: %s", cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status lbm_batch_residual(lbm_batch* b, double* r, int* diverged) {
    if (!b || !r) {
        gerr("lbm_batch_residual: NULL argument");
        return LBM_ERR_INVALID;
    }
    lbm_status s = sync_tables(b);
    if (s != LBM_OK) return s;
    const bool aa = b->layout == LBM_AA;
    const int grid = reduce_grid(b);
    cudaError_t e;
    switch (b->prec) {
        case LBM_F32: e = launch_batch_residual<float>(b->d_table, b->d_owner, b->d_ntiles, b->total_tiles, b->capacity, b->parity(), aa, grid, b->d_partial, b->d_out, b->stream); break;
        case LBM_BF16: e = launch_batch_residual<__nv_bfloat16>(b->d_table, b->d_owner, b->d_ntiles, b->total_tiles, b->capacity, b->parity(), aa, grid, b->d_partial, b->d_out, b->stream); break;
        default: e = launch_batch_residual<__half>(b->d_table, b->d_owner, b->d_ntiles, b->total_tiles, b->capacity, b->parity(), aa, grid, b->d_partial, b->d_out, b->stream); break;
    }
    std::vector<double> h((size_t)b->capacity * 9, 0.0);
    if (e == cudaSuccess && b->total_tiles > 0)
        e = cudaMemcpyAsync(h.data(), b->d_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch_residual: %s", cudaGetErrorString(e));
    for (int k = 0; k < b->capacity; ++k) {
        Slot& sl = b->slots[k];
        if (diverged) diverged[k] = 0;
        if (!sl.used) {
            r[k] = 0.0;
            continue;
        }
        const double* v = &h[(size_t)k * 9];
        double res = 0.0;
        for (int q = 0; q < 4; ++q) {
            const double rq = v[4 + q] > 0 ? v[q] / v[4 + q] : (v[q] > 0 ? INFINITY : 0.0);
            res = rq > res ? rq : res;
        }
        r[k] = sl.snap_valid ? res : INFINITY;
        sl.snap_valid = true;
        if (v[8] != 0.0 && diverged) diverged[k] = 1;
        if (v[8] != 0.0) r[k] = NAN;
    }
    return LBM_OK;
}

lbm_status lbm_batch_fields(lbm_batch* b, int slot, double* ux, double* uy, double* T, double* C,
                            double* rho) {
    if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) {
        if (b) return b->fail(LBM_ERR_INVALID, "lbm_batch_fields: slot %d is not in use", slot);
        gerr("lbm_batch_fields: NULL batch");
        return LBM_ERR_INVALID;
    }
    const Slot& s = b->slots[slot];
    const size_t n = (size_t)s.G.nx * s.G.ny;
    if (n * 5 > b->fields_cap) {
        b->dfree(b->d_fields);
        b->d_fields = (double*)b->dalloc(n * 5 * sizeof(double));
        b->fields_cap = b->d_fields ? n * 5 : 0;
        if (!b->d_fields) return b->fail(LBM_ERR_NOMEM, "lbm_batch_fields: no device memory for read-out");
    }
    const Coef<float> c = coef_from(s.P, b->sr);
    const int mode = b->mode_of(s);
    const void* cur = b->cur_of(s);
    cudaError_t e;
    switch (b->prec) {
        case LBM_F32: e = launch_fields<float>(cur, s.G, c, mode, 0, 0, s.G.nx, s.G.ny, b->d_fields, b->stream); break;
        case LBM_BF16: e = launch_fields<__nv_bfloat16>(cur, s.G, c, mode, 0, 0, s.G.nx, s.G.ny, b->d_fields, b->stream); break;
        default: e = launch_fields<__half>(cur, s.G, c, mode, 0, 0, s.G.nx, s.G.ny, b->d_fields, b->stream); break;
    }
    double* outs[5] = {ux, uy, T, C, rho};
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
        if (outs[k])
            e = cudaMemcpyAsync(outs[k], b->d_fields + k * n, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->fail(LBM_ERR_CUDA, "lbm_batch_fields: %s", cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int trial_steps, char* report, size_t cap) {
    if (!b) {
        gerr("lbm_batch_autotune: NULL batch");
        return LBM_ERR_INVALID;
    }
    if (trial_steps < 2) trial_steps = 2;
    trial_steps += trial_steps & 1;
    std::string rep;
    // distinct grid sizes and how many cavities of each the batch holds
    std::map<std::pair<int, int>, std::vector<int>> classes;
    for (int k = 0; k < b->capacity; ++k)
        if (b->slots[k].used) classes[{b->slots[k].P.nx, b->slots[k].P.ny}].push_back(k);
    for (auto& cl : classes) {
        const int nx = cl.first.first, ny = cl.first.second;
        const lbm_params& P0 = b->slots[cl.second[0]].P;
        // scratch cavities of this size: as many as the batch holds, capped at ~16M nodes
        const long cap_nodes = 1L << 24;
        int count = (int)std::min<long>((long)cl.second.size(), std::max<long>(1, cap_nodes / ((long)nx * ny)));
        std::vector<lbm_instance> tmp(count);
        for (int q = 0; q < count; ++q) {
            tmp[q].params = P0;
            tmp[q].seed = 1000 + q;
            tmp[q].noise = 1e-3;
        }
        lbm_options o;
        std::memset(&o, 0, sizeof o);
        o.precision = b->prec;
        o.layout = b->layout;
        o.stream = b->stream;
        o.alloc = b->alloc;
        o.free = b->free_fn;
        o.alloc_user = b->alloc_user;
        o.graph_chunk = -1;
        o.round_nearest = b->sr ? 0 : 1;
        lbm_batch* s = nullptr;
        lbm_status st = lbm_batch_create(tmp.data(), count, count, 0, &o, &s);
        if (st != LBM_OK) return b->fail(st, "lbm_batch_autotune: scratch batch: %s", g_err.c_str());
        int best_w = b->slots[cl.second[0]].tw_log2, best_h = b->slots[cl.second[0]].th;
        double best_us = 1e300;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        // candidates: tiles of one node per thread (the loop-free kernel), 32..128 wide
        for (int wl = 5; wl <= 7; ++wl) {
            const int w = 1 << wl;
            if (w > 2 * std::max(32, nx)) continue;       // more than half a tile would be idle
            for (int h = 1; h <= 16; h <<= 1) {
                const int nodes = w * h;
                if (nodes != BATCH_THREADS) continue;
                for (int q = 0; q < count; ++q) {
                    s->slots[q].tw_log2 = wl;
                    s->slots[q].th = h;
                }
                invalidate(s);
                st = lbm_batch_step(s, 2);                // upload + warm-up
                if (st != LBM_OK) break;
                cudaEventRecord(e0, s->stream);
                st = lbm_batch_step(s, trial_steps);
                cudaEventRecord(e1, s->stream);
                cudaEventSynchronize(e1);
                if (st != LBM_OK) break;
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                const double us = 1e3 * ms / trial_steps;
                if (us < best_us) {
                    best_us = us;
                    best_w = wl;
                    best_h = h;
                }
            }
            if (st != LBM_OK) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        lbm_batch_destroy(s);
        if (st != LBM_OK) return b->fail(st, "lbm_batch_autotune: trial failed: %s", g_err.c_str());
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[std::make_tuple(nx, ny, b->prec, b->layout)] = {best_w, best_h};
        }
        for (int k : cl.second) {
            b->slots[k].tw_log2 = best_w;
            b->slots[k].th = best_h;
        }
        char line[128];
        std::snprintf(line, sizeof line, "%d %d %d %d %.3f\n", nx, ny, 1 << best_w, best_h, best_us);
        rep += line;
    }
    invalidate(b);
    {
        lbm_status s2 = sync_tables(b);
        if (s2 != LBM_OK) return s2;
        char line[128];
        std::snprintf(line, sizeof line, "# groups %zu l2_budget %zu tiles %d\n", b->groups.size(),
                      b->l2_budget, b->total_tiles);
        rep += line;
    }
    if (report && cap) {
        std::strncpy(report, rep.c_str(), cap - 1);
        report[cap - 1] = 0;
    }
    return LBM_OK;
}

lbm_status lbm_batch_set_tile(lbm_batch* b, int slot, int tile_w, int tile_h) {
    if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) {
        if (b) return b->fail(LBM_ERR_INVALID, "lbm_batch_set_tile: slot %d is not in use", slot);
        gerr("lbm_batch_set_tile: NULL batch");
        return LBM_ERR_INVALID;
    }
    int l = 5;
    while ((1 << l) < tile_w && l < 8) ++l;
    if ((1 << l) != tile_w || tile_h < 1 || tile_w * tile_h > 4096)
        return b->fail(LBM_ERR_INVALID, "lbm_batch_set_tile: bad tile %d x %d", tile_w, tile_h);
    b->slots[slot].tw_log2 = l;
    b->slots[slot].th = tile_h;
    invalidate(b);
    return LBM_OK;
}

lbm_status lbm_batch_set_blocking(lbm_batch* b, int steps, size_t l2_bytes) {
    if (!b || steps < 1) {
        if (b) return b->fail(LBM_ERR_INVALID, "lbm_batch_set_blocking: steps must be >= 1");
        gerr("lbm_batch_set_blocking: NULL batch");
        return LBM_ERR_INVALID;
    }
    b->tblock = steps;
    if (l2_bytes) b->l2_budget = l2_bytes;
    invalidate(b);
    return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch* b, int* capacity, int* used, size_t* arena_bytes,
                          size_t* arena_used) {
    if (!b) {
        gerr("lbm_batch_info: NULL batch");
        return LBM_ERR_INVALID;
    }
    if (capacity) *capacity = b->capacity;
    if (used) *used = b->used_slots();
    if (arena_bytes) *arena_bytes = b->arena.size;
    if (arena_used) *arena_used = b->arena.used;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->dfree(b->arena_mem);
    b->dfree(b->d_table);
    b->dfree(b->d_walls);
    b->dfree(b->d_ntiles);
    b->dfree(b->d_out);
    b->dfree(b->d_owner);
    b->dfree(b->d_partial);
    b->dfree(b->d_fields);
    destroy_lanes(b);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : g_err.c_str(); }

}  // extern "C"
