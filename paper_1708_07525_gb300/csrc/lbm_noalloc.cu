// Steady-state residual without any device allocation.
//
// lbm_residual() allocates its snapshot and its per-block partial maxima on
// the first call.  Some callers cannot allocate device memory at that point:
// a host framework that has reserved the device memory for its own pool, or
// a loop that must not stall on cudaMalloc / cudaFree, which can synchronise
// the device.  lbm_residual_noalloc() computes the same residual with the
// caller's snapshot buffer and with its partial maxima in the file-scope
// array below.  There is no counterpart in the paper; this is plumbing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"

using namespace lbm;

namespace {

constexpr int NOALLOC_OUT = LBM_NOALLOC_MAX_BLOCKS * 9;   // offset of the 9 results

// Partial maxima of up to LBM_NOALLOC_MAX_BLOCKS blocks (9 doubles each) plus the
// 9 folded results.  Every GPU that loads the library holds this array (about
// 288 KiB) until the process exits.  In host code `noalloc_scratch` is only a
// host-side stand-in for the symbol; its device address comes from
// cudaGetSymbolAddress (see scratch_for_device).
__device__ __align__(256) double noalloc_scratch[LBM_NOALLOC_MAX_BLOCKS * 9 + 16];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on `dev`, looked up once per device; the caller
// has made `dev` current.  This happens on the first call on each device, so that first
// call must not come while a stream is being captured.  The address is kept for the
// life of the process: a device reset (which unloads the module) makes it stale.
cudaError_t scratch_for_device(int dev, double** out) {
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        double* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&p, noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

inline const Coef<double>& coef_of(const CtxView& v, double*) { return *v.cd; }
inline const Coef<float>& coef_of(const CtxView& v, float*) { return *v.cf; }

template <typename S>
cudaError_t launch(const CtxView& v, double* snap, double* scratch) {
    using R = typename Real<S>::type;
    const Coef<R>& c = coef_of(v, (R*)nullptr);
    cudaError_t e = launch_residual_pass1<S, double>((const S*)v.buf, v.G, c, v.mode, snap, scratch,
                                                     LBM_NOALLOC_MAX_BLOCKS, v.stream);
    if (e != cudaSuccess) return e;
    residual_final_kernel<<<1, RES_THREADS, 0, v.stream>>>(scratch, LBM_NOALLOC_MAX_BLOCKS,
                                                          scratch + NOALLOC_OUT);
    return cudaGetLastError();
}

lbm_status fail(lbm_ctx* ctx, lbm_status s, const char* m, const char* detail = "") {
    char msg[256];
    std::snprintf(msg, sizeof msg, "lbm_residual_noalloc: %s%s", m, detail);
    lbm_set_error(ctx, msg);
    return s;
}

}  // namespace

extern "C" {

lbm_status lbm_residual_noalloc(lbm_ctx* ctx, double* snapshot, int have_snapshot, double* r) {
    CtxView v;
    if (!ctx || !snapshot || !r || !lbm_ctx_view(ctx, &v))
        return fail(ctx, LBM_ERR_INVALID, "ctx, snapshot and r must be non-NULL");
    if (v.G.jb != 0 || v.G.je != v.G.ny)   // a slab: its snapshot would include ghost rows
        return fail(ctx, LBM_ERR_INVALID, "not defined on a slab (use lbm_residual_parts)");
    // the context's device for the whole call: the symbol lookup, the launches on the
    // context's stream and the copy all belong to it
    DeviceGuard dg(v.device);
    double* scratch = nullptr;
    cudaError_t e = scratch_for_device(v.device, &scratch);
    if (e != cudaSuccess) return fail(ctx, LBM_ERR_CUDA, "cudaGetSymbolAddress: ", cudaGetErrorString(e));
    // The call clears the slots of the shared array before its first pass folds into
    // them, and the fold writes all nine results.
    switch (v.prec) {
        case LBM_F64: e = launch<double>(v, snapshot, scratch); break;
        case LBM_F32: e = launch<float>(v, snapshot, scratch); break;
        case LBM_BF16: e = launch<__nv_bfloat16>(v, snapshot, scratch); break;
        default: e = launch<__half>(v, snapshot, scratch); break;
    }
    double h[9];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, scratch + NOALLOC_OUT, sizeof h, cudaMemcpyDeviceToHost, v.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
    if (e != cudaSuccess) return fail(ctx, LBM_ERR_CUDA, "", cudaGetErrorString(e));
    if (h[8] != 0.0) return fail(ctx, LBM_ERR_DIVERGED, "non-finite field value");
    double res = 0.0;
    for (int q = 0; q < 4; ++q) {
        const double rq = h[4 + q] > 0 ? h[q] / h[4 + q] : (h[q] > 0 ? INFINITY : 0.0);
        res = rq > res ? rq : res;
    }
    *r = have_snapshot ? res : INFINITY;
    return LBM_OK;
}

}  // extern "C"
