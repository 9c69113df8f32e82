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

// sum_m w_m (p[m s] + p[-m s]) + w_0 p[0]
template <typename T>
__device__ __forceinline__ T d2_col(const T *p, int s) {
    return T(kC0) * p[0] + T(kC1) * (p[s] + p[-s]) + T(kC2) * (p[2 * s] + p[-2 * s]) +
           T(kC3) * (p[3 * s] + p[-3 * s]) + T(kC4) * (p[4 * s] + p[-4 * s]);
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
