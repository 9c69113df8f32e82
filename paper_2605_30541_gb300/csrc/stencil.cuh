// Device helpers shared by the stencil kernels: the 8th-order weights,
// strided stencil sums and the FP16 snapshot scale.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace gsim {

// Central second-derivative weights of order 8 (M = 4), without the 1/h^2
// (App. E.3; Fornberg's weights for the 9-point stencil).
constexpr double kC0 = -205.0 / 72.0, kC1 = 8.0 / 5.0, kC2 = -1.0 / 5.0, kC3 = 8.0 / 315.0,
                 kC4 = -1.0 / 560.0;
// Central first-derivative weights of order 8, without the 1/h (CPML memory terms).
constexpr double kD1 = 4.0 / 5.0, kD2 = -1.0 / 5.0, kD3 = 4.0 / 105.0, kD4 = -1.0 / 280.0;

// Centre weight of the outer pairs: w_0 = -2 (w_1 + w_2 + w_3 + w_4), so
// sum_m w_m (p_m + p_-m) + w_0 p_0 = sum_{m=1,2} w_m ((p_m - p_0) + (p_-m - p_0))
//                                   + sum_{m=3,4} w_m (p_m + p_-m) + kC34 p_0.
constexpr double kC34 = -2.0 * (kC3 + kC4);

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Second difference along one axis (without 1/h^2) from the nine values
// c = p_0 and m_k = p_-k, p_k = p_+k. The two inner pairs, whose weights are
// large, enter as differences from the centre: for a smooth field those are
// exact in floating point and small, so the result carries no rounding error
// of the size of w_0 p_0 (the plain form cancels terms 2.85 |p_0| large; over
// thousands of FP32 steps that error accumulates into the wavefield). Summed
// from the smallest term up, every product-sum one fused multiply-add; every
// kernel uses this one sequence of roundings (d2c2 below is the same sequence
// on two cells at once), so all paths give the same bits.
template <typename T>
__device__ __forceinline__ T d2c(T c, T m1, T p1, T m2, T p2, T m3, T p3, T m4, T p4) {
    T r = T(kC34) * c;
    r = fma_rn(T(kC4), p4 + m4, r);
    r = fma_rn(T(kC3), p3 + m3, r);
    r = fma_rn(T(kC2), (p2 - c) + (m2 - c), r);
    r = fma_rn(T(kC1), (p1 - c) + (m1 - c), r);
    return r;
}

// Two cells per instruction: the FP32 pair arithmetic of this architecture
// (one instruction rounds both lanes as the scalar one rounds each), so a
// pair of cells costs the instructions of one.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }

// First difference (without 1/h) of two cells from the eight neighbours
// m_k = p_-k, p_k = p_+k: d_1 (p_1 - m_1) + d_2 (p_2 - m_2) + d_3 (p_3 - m_3) +
// d_4 (p_4 - m_4), each further term one fused multiply-add
__device__ __forceinline__ float2 d1c2(float2 m1, float2 p1, float2 m2, float2 p2, float2 m3, float2 p3, float2 m4,
                                       float2 p4) {
    float2 r = mul2(splat2(float(kD1)), add2(p1, neg2(m1)));
    r = fma2(splat2(float(kD2)), add2(p2, neg2(m2)), r);
    r = fma2(splat2(float(kD3)), add2(p3, neg2(m3)), r);
    r = fma2(splat2(float(kD4)), add2(p4, neg2(m4)), r);
    return r;
}

// d2c on two cells: the same operations in the same order, lane by lane
__device__ __forceinline__ float2 d2c2(float2 c, float2 m1, float2 p1, float2 m2, float2 p2, float2 m3, float2 p3,
                                       float2 m4, float2 p4) {
    const float2 nc = neg2(c);
    float2 r = mul2(splat2(float(kC34)), c);
    r = fma2(splat2(float(kC4)), add2(p4, m4), r);
    r = fma2(splat2(float(kC3)), add2(p3, m3), r);
    r = fma2(splat2(float(kC2)), add2(add2(p2, nc), add2(m2, nc)), r);
    r = fma2(splat2(float(kC1)), add2(add2(p1, nc), add2(m1, nc)), r);
    return r;
}

// the second difference at p[0] along stride s
template <typename T>
__device__ __forceinline__ T d2_col(const T *p, int s) {
    return d2c<T>(p[0], p[-s], p[s], p[-2 * s], p[2 * s], p[-3 * s], p[3 * s], p[-4 * s], p[4 * s]);
}

// sum_m d_m (p[m s] - p[-m s])
template <typename T>
__device__ __forceinline__ T d1_row(const T *p, int s) {
    return T(kD1) * (p[s] - p[-s]) + T(kD2) * (p[2 * s] - p[-2 * s]) +
           T(kD3) * (p[3 * s] - p[-3 * s]) + T(kD4) * (p[4 * s] - p[-4 * s]);
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Power-of-two scale of an FP16 snapshot: s = 2^(floor(log2 m) - 14), so the
// largest magnitude maps into [2^14, 2^15) and x / s is exact; 1 for m = 0,
// clamped to the smallest normal float for m below 2^-112.
__host__ __device__ inline float pow2_scale(float m) {
    if (!(m > 0.f)) return 1.f;
#ifdef __CUDA_ARCH__
    const unsigned b = __float_as_uint(m);
#else
    unsigned b;
    memcpy(&b, &m, 4);
#endif
    int e = (int)((b >> 23) & 0xffu) - 127;  // floor(log2 m) for normal m
    if (e < -112) e = -112;
    const unsigned sb = (unsigned)(e - 14 + 127) << 23;
#ifdef __CUDA_ARCH__
    return __uint_as_float(sb);
#else
    float s;
    memcpy(&s, &sb, 4);
    return s;
#endif
}

}  // namespace gsim
