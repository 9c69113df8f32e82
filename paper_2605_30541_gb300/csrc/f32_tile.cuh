// Device helpers of the FP32 2D kernels that work on float4 lanes of a
// shared-memory tile: lane access, 16-byte loads/stores, cp.async staging,
// the 12-float stencil windows and the acquire/release step counters.
#pragma once

#include "stencil.cuh"

namespace gsim {
namespace f32 {

__device__ __forceinline__ float lane_of(const float4 &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// 16-byte global -> shared copy that bypasses L1 (.cg), so data another CTA
// published through L2 is never read from a stale L1 line.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// second difference of the 12-float window v[0..11] at v[4 + k]
__device__ __forceinline__ float d2w(const float *v, int k) {
    return d2c<float>(v[4 + k], v[3 + k], v[5 + k], v[2 + k], v[6 + k], v[1 + k], v[7 + k], v[k], v[8 + k]);
}
// first difference of the 12-float window at v[4 + k]
__device__ __forceinline__ float d1w(const float *v, int k) {
    return float(kD1) * (v[5 + k] - v[3 + k]) + float(kD2) * (v[6 + k] - v[2 + k]) +
           float(kD3) * (v[7 + k] - v[1 + k]) + float(kD4) * (v[8 + k] - v[k]);
}
__device__ __forceinline__ void unpack3(const float4 &a, const float4 &b, const float4 &c, float *v) {
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

}  // namespace f32
}  // namespace gsim
