// Host-side launch interface between the C ABI (lbm_api.cu) and the
// per-precision kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {

// Geometry of one state: planes of ny rows of `pitch` elements (x fastest).
// A step updates the rows jb .. je - 1: all rows of a cavity; for a slab of a cavity
// split along y (lbm_create_slab), the rows between its ghost rows, which hold the
// neighbouring slabs' boundary populations.
struct Geom {
    int nx, ny;
    int pitch;       // elements per row, rows start 128-byte aligned
    int jb;          // first row a step updates
    size_t plane;    // elements per plane = ny * pitch
    int je;          // one past the last row a step updates
};
__host__ __device__ inline int step_rows(const Geom& G) { return G.je - G.jb; }

// How the pre-collision populations of the current level are read.
enum { GATHER_LOCAL = 0, GATHER_PULL_AB = 1, GATHER_PULL_AA = 2, GATHER_NEE_AB = 3 };

struct InitSpec {
    const double* T_init;   // device [je - jb][nx] (the rows a step updates) or NULL (noise)
    const double* C_init;
    int key_ny, key_j0;     // noise keys (field * key_ny + key_j0 + j) * nx + i: the whole
                            // cavity's rows and the global row of row 0
    uint64_t seed;
    double noise;
    double T0, C0, sigma, eps, varpi;
    int model_a;            // equilibria of Eqs. 30-31 instead of Eqs. 24-25
};

struct WallSpec {
    double Tw[2], Cw[2];    // absolute wall values, left / right
    double T0, C0, dT, dC, L;
    int nee;                // 1: nodes on the walls (node stencil, trapezoidal mean)
};

constexpr int NUSH_THREADS = 512;
constexpr int RES_THREADS = 256;

struct LaunchCfg {
    int bx, by;
    cudaStream_t stream;
    // Optional second stream with two events: where a step is an inner-node launch plus
    // a small launch for the outermost ring, the ring runs on `aux` beside the inner
    // launch (the two write disjoint locations), joined back before the next step.
    // aux == nullptr: both launches go to `stream`.
    cudaStream_t aux;
    cudaEvent_t fork, join;
    // 16-bit storage: the cavity's constants as pairs for the two-nodes-per-thread
    // kernels (lbm_pair.cuh); nullptr -> the one-node kernels
    const Coef<f2>* pair;
};

// Stream for the ring launch of a split step (after forking from L.stream).
inline cudaError_t ring_fork(const LaunchCfg& L, cudaStream_t* rs) {
    *rs = L.stream;
    if (!L.aux) return cudaSuccess;
    cudaError_t e = cudaEventRecord(L.fork, L.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L.aux, L.fork, 0);
    if (e == cudaSuccess) *rs = L.aux;
    return e;
}
// Makes L.stream wait for the ring launch.
inline cudaError_t ring_join(const LaunchCfg& L) {
    if (!L.aux) return cudaSuccess;
    cudaError_t e = cudaEventRecord(L.join, L.aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L.stream, L.join, 0);
    return e;
}

// Launchers, explicitly instantiated for S = double, float, __nv_bfloat16, __half.
template <typename S>
cudaError_t launch_init(void* buf, void* hist, const Geom& G, const Coef<typename Real<S>::type>& c,
                        const InitSpec& I, bool pull, cudaStream_t st);
template <typename S>
cudaError_t launch_step_ab(const void* src, void* dst, void* hist, const Geom& G,
                           const Coef<typename Real<S>::type>& c, const LaunchCfg& L);
template <typename S>
cudaError_t launch_step_aa(void* buf, void* hist, const Geom& G,
                           const Coef<typename Real<S>::type>& c, bool odd, const LaunchCfg& L);
// Fields over the window [x0, x0 + w) x [y0, y0 + h) into out[5][h][w].
template <typename S>
cudaError_t launch_fields(const void* buf, const Geom& G, const Coef<typename Real<S>::type>& c,
                          int mode, int x0, int y0, int w, int h, double* out, cudaStream_t st);
template <typename S>
cudaError_t launch_nush(const void* buf, const Geom& G, const Coef<typename Real<S>::type>& c,
                        int mode, const WallSpec& W, double* out, cudaStream_t st);
// Nu / Sh on the bottom (Tw[0], Cw[0]) and top (Tw[1], Cw[1]) walls; out 4 doubles.
template <typename S>
cudaError_t launch_nush_tb(const void* buf, const Geom& G, const Coef<typename Real<S>::type>& c,
                           int mode, const WallSpec& W, double* out, cudaStream_t st);
// snap holds 4 * nx * ny values of the compute precision (FP64 for FP64 storage,
// else FP32); partial must hold RES_SLOTS * 9 doubles; out 9 doubles.
template <typename S>
cudaError_t launch_residual(const void* buf, const Geom& G, const Coef<typename Real<S>::type>& c,
                            int mode, void* snap, double* partial, double* out,
                            cudaStream_t st);
// Copies the five populations of `row` that cross a horizontal cut moving up (up = 1)
// or down between the state and face[5][nx] (pack = 1: state -> face).
template <typename S>
cudaError_t launch_halo(void* buf, const Geom& G, int row, int up, void* face, int pack,
                        cudaStream_t st);
// Grid of the residual's first pass: 256-column tiles along x, one row per block
// along y (each block loops when ny exceeds the grid's y limit).
inline dim3 residual_grid(const Geom& G) {
    const int ntx = (G.nx + RES_THREADS - 1) / RES_THREADS;
    const int rows = step_rows(G);
    const int gy = rows < 65535 ? rows : 65535;
    return dim3((unsigned)ntx, (unsigned)(gy > 0 ? gy : 1), 1);
}
// Slots the first pass folds its block maxima into (atomically); the second pass
// reduces the slots.
constexpr int RES_SLOTS = 4096;

// Makes `dev` the calling thread's current device for the guard's lifetime and
// restores the previous one afterwards (every entry point that touches a context's
// device state holds one).
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Kernel constants of a cavity from its lattice parameters (lbm_api.cu);
// stochastic rounding of 16-bit stores is enabled (Coef::sr = 1).
template <typename R>
Coef<R> make_coef(const lbm_params& P);

// Read-only view of a context's device state, for entry points defined in
// other translation units of the library.
struct CtxView {
    int prec;
    const void* buf;         // buffer holding the current state
    Geom G;
    const Coef<double>* cd;
    const Coef<float>* cf;
    int mode;                // GATHER_* for the current level
    cudaStream_t stream;
    int device;
};

}  // namespace lbm

struct lbm_ctx;
bool lbm_ctx_view(const lbm_ctx* ctx, lbm::CtxView* out);
// Records msg as the last error of ctx (or of the calling thread if ctx is NULL).
void lbm_set_error(lbm_ctx* ctx, const char* msg);
