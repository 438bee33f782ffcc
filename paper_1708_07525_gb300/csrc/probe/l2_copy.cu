// Measurement utility, not part of the method: the copy bandwidth of a working set that
// stays in L2, the bound of the batched step (whose L2 blocking keeps a group of
// cavities' state in L2 for all but the first of its steps).  Loaded by the benchmark
// only (libprobe.so); nothing in liblbm calls it.
#include <cuda_runtime.h>
#include <stddef.h>

namespace {

// `passes` copies back and forth between a and b (a -> b, b -> a, ...), each a
// grid-stride loop of 16-byte loads and stores.  Element i is copied by the same thread in
// every pass, so a pass reads what the same thread wrote in the one before; the loads and
// stores are volatile so that none is merged or dropped.
__device__ __forceinline__ float4 ld16(const float4* p) {
    float4 v;
    asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st16(float4* p, float4 v) {
    asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};"
                 :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}

__global__ void __launch_bounds__(256) ping_pong(float4* a, float4* b, size_t n4, int passes) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p) {
        const float4* src = (p & 1) ? b : a;
        float4* dst = (p & 1) ? a : b;
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
            st16(dst + i, ld16(src + i));
    }
}

}  // namespace

extern "C" int probe_l2_copy(void* a, void* b, size_t bytes, int passes, int blocks,
                             void* stream) {
    if (!a || !b || bytes < 16 || (bytes & 15) || passes < 1 || blocks < 1) return 1;
    ping_pong<<<blocks, 256, 0, (cudaStream_t)stream>>>((float4*)a, (float4*)b, bytes / 16,
                                                          passes);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
