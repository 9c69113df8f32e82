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
// Second differences of a lane's four cells (columns C.x .. C.w) in FP32
// pairs (d2c2: the bits of d2c cell by cell): along x from the row's float4s
// L, C, R, along z from the nine rows w[0..8] of the lane's columns (w[4] =
// C). The pairs straddling float4s, (v3, v4) (v5, v6) (v1, v2) (v7, v8)
// (v9, v10) of the 12-float window, are assembled once.
struct Pairs4 {
    float2 xa, xb, za, zb;  // cells (0, 1) and (2, 3)
};
__device__ __forceinline__ Pairs4 d2_pairs(const float4 &L, const float4 &C, const float4 &R, const float4 *w) {
    const float2 v34 = make_float2(L.w, C.x), v56 = make_float2(C.y, C.z), v12 = make_float2(L.y, L.z),
                 v78 = make_float2(C.w, R.x), v910 = make_float2(R.y, R.z);
    Pairs4 o;
    o.xa = d2c2(lo2(C), v34, v56, hi2(L), hi2(C), v12, v78, lo2(L), lo2(R));
    o.xb = d2c2(hi2(C), v56, v78, lo2(C), lo2(R), v34, v910, hi2(L), hi2(R));
    o.za = d2c2(lo2(C), lo2(w[3]), lo2(w[5]), lo2(w[2]), lo2(w[6]), lo2(w[1]), lo2(w[7]), lo2(w[0]), lo2(w[8]));
    o.zb = d2c2(hi2(C), hi2(w[3]), hi2(w[5]), hi2(w[2]), hi2(w[6]), hi2(w[1]), hi2(w[7]), hi2(w[0]), hi2(w[8]));
    return o;
}
// First differences of a lane's four cells in pairs (d1c2): along x from the
// row's float4s L, C, R, and along an axis from the float4s of the four
// positions below (m4 .. m1) and above (p1 .. p4).
__device__ __forceinline__ void d1x_pairs(const float4 &L, const float4 &C, const float4 &R, float2 &da, float2 &db) {
    const float2 v34 = make_float2(L.w, C.x), v56 = make_float2(C.y, C.z), v12 = make_float2(L.y, L.z),
                 v78 = make_float2(C.w, R.x), v910 = make_float2(R.y, R.z);
    da = d1c2(v34, v56, hi2(L), hi2(C), v12, v78, lo2(L), lo2(R));
    db = d1c2(v56, v78, lo2(C), lo2(R), v34, v910, hi2(L), hi2(R));
}
__device__ __forceinline__ void d1_pairs(const float4 &m4, const float4 &m3, const float4 &m2, const float4 &m1,
                                         const float4 &p1, const float4 &p2, const float4 &p3, const float4 &p4,
                                         float2 &da, float2 &db) {
    da = d1c2(lo2(m1), lo2(p1), lo2(m2), lo2(p2), lo2(m3), lo2(p3), lo2(m4), lo2(p4));
    db = d1c2(hi2(m1), hi2(p1), hi2(m2), hi2(p2), hi2(m3), hi2(p3), hi2(m4), hi2(p4));
}
// the CPML memory recursion b m + a d of a pair: fma(a, d, b m)
__device__ __forceinline__ float2 rec2(float2 a, float2 d, float2 b, float2 m) { return fma2(a, d, mul2(b, m)); }

// the plain leapfrog update p^{n+1} = fma(c, rhs, fma(2, p, -p^{n-1})) of
// four cells in pairs; the scalar form is plain1 (the same roundings)
__device__ __forceinline__ float4 plain4(const float4 &p, const float4 &pp, const float4 &c, float2 ra, float2 rb) {
    const float2 two = splat2(2.f);
    const float2 a = fma2(lo2(c), ra, fma2(two, lo2(p), neg2(lo2(pp))));
    const float2 b = fma2(hi2(c), rb, fma2(two, hi2(p), neg2(hi2(pp))));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float plain1(float p, float pp, float c, float rhs) {
    return __fmaf_rn(c, rhs, __fmaf_rn(2.f, p, -pp));
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
